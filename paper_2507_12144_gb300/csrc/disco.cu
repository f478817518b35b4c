// Discrete-continuous (DISCO) convolution on the sphere, Eq.
// (disco_convolution) in its longitude-shift form Eq.
// (disco_convolution_formula) (Sec. B.5, Sec. G.2.3):
//   y[c][k][h][w] = sum_{h', w'} psi[k][h][h'][w'] x[c][h'][(w' + s w) mod nlon_in],
// psi[k][h][h'][w'] = kb_k(R_h^{-1} x_{h', w'}) omega_{h'} for the output
// point (theta_h, longitude 0), nlon_in = s nlon_out, and its transpose
//   gx[c][h'][(w' + s w) mod nlon_in] += psi[k][h][h'][w'] gy[c][k][h][w]
// (the backward of the contraction).  The basis kb_k (Sec. B.5.1) lives on
// the cap vartheta' = vartheta / theta_cutoff <= 1 around the output point:
// h(vartheta') = cos^2(pi vartheta' / 2) times cos or sin of
// pi (l vartheta' sin varphi + m vartheta' cos varphi), 0 <= l, m < n (the
// real and imaginary parts of the Morlet-type factor; the sine of l = m = 0
// vanishes and is left out: K = 2 n^2 - 1, cosines first).  vartheta,
// varphi are the colatitude and azimuth of the input point after the
// rotation R_h^{-1} that takes the output point to the north pole.
//
// psi is built once on the host in FP64 and kept sparse in two row
// layouts: by output latitude (forward) and by input latitude (backward),
// each entry (other latitude, w', K values).  The kernels take an output
// (input) latitude per block row and longitudes per thread, CB channels per
// thread, so that each entry's K values, read once, serve CB channels; the
// field loads of one entry are coalesced along the longitudes.  On equal
// longitude grids the backward runs by runs instead: for one input latitude
// and one channel, the entries of one output latitude h form runs of
// consecutive w' (the cap meets a latitude ring in one arc), whose K gradient
// rows are staged whole in shared memory by bulk copies (double-buffered),
// and every thread keeps R consecutive input longitudes with a register
// window that slides along the run, so that each staged value is read once
// per thread and used R times.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "sht_internal.cuh"
#include "tc_common.cuh"

struct sht_disco_s {
  int device = 0;
  int nlat_in = 0, nlon_in = 0, nlat_out = 0, nlon_out = 0, s = 1, n = 1, K = 1;
  double theta_cutoff = 0.0;
  int64_t nnz = 0;
  int *d_row_f = nullptr;   // [nlat_out + 1]
  int2 *d_idx_f = nullptr;  // (h', w')
  float *d_val_f = nullptr; // [nnz][2 ceil(K / 2)] (a zero after the last value for odd K)
  int *d_row_b = nullptr;   // [nlat_in + 1]
  int2 *d_idx_b = nullptr;  // (h, w')
  float *d_val_b = nullptr; // [nnz][K]
  // runs of the backward on equal longitude grids: per input latitude the
  // entries of one output latitude h whose w' run through a, a + 1, ...
  // (mod nlon) as (h, first entry, length, a); values in run order
  int win_R = 0;            // outputs per thread of the run kernel (0: not used)
  int *d_run_row = nullptr; // [nlat_in + 1]
  int4 *d_runs = nullptr;
  float *d_val_w = nullptr; // [nnz][2 ceil(K / 2)], entries in run order
  unsigned *d_err = nullptr; // error word of the run kernel's bounded waits
};

namespace shtgb {
namespace {

constexpr int kDiscoThreads = 128;

// The device keeps the K values of an entry in 2 KP floats (a zero after
// the last for odd K), so that the run backward reads (psi_k, psi_k+1) as
// one 8-byte load for one packed FP32x2 FMA (each lane rounds as the
// scalar FMA).
template <int K>
constexpr int kpairs() {
  return (K + 1) / 2;
}

template <int K, int CB>
__global__ void __launch_bounds__(kDiscoThreads)
    disco_fwd_kernel(const float *__restrict__ x, float *__restrict__ y, const int *__restrict__ row,
                     const int2 *__restrict__ idx, const float *__restrict__ val, int64_t C, int Hi, int Wi, int Ho,
                     int Wo, int s) {
  const int w = blockIdx.x * kDiscoThreads + threadIdx.x;
  const int h = blockIdx.y;
  const int64_t c0 = (int64_t)blockIdx.z * CB;
  if (w >= Wo) return;
  float acc[CB][K];
#pragma unroll
  for (int j = 0; j < CB; j++)
#pragma unroll
    for (int k = 0; k < K; k++) acc[j][k] = 0.f;
  const int sw = s * w;
  const int64_t plane = (int64_t)Hi * Wi;
  const int eb = row[h], ee = row[h + 1];
  // entry e + 1's inputs and entry e + 2's index load during entry e's FMAs
  auto xload = [&](int2 hw, float (&xv)[CB]) {
    int col = hw.y + sw;
    if (col >= Wi) col -= Wi;
    const float *xp = x + c0 * plane + (int64_t)hw.x * Wi + col;
#pragma unroll
    for (int j = 0; j < CB; j++) xv[j] = c0 + j < C ? __ldg(xp + j * plane) : 0.f;
  };
  float xn[CB];
  int2 hw2 = make_int2(0, 0);
  if (eb < ee) xload(__ldg(idx + eb), xn);
  if (eb + 1 < ee) hw2 = __ldg(idx + eb + 1);
  for (int e = eb; e < ee; e++) {
    float xv[CB];
#pragma unroll
    for (int j = 0; j < CB; j++) xv[j] = xn[j];
    if (e + 1 < ee) {
      xload(hw2, xn);
      if (e + 2 < ee) hw2 = __ldg(idx + e + 2);
    }
    const float *vp = val + (int64_t)e * (2 * kpairs<K>());
#pragma unroll
    for (int k = 0; k < K; k++) {
      const float v = __ldg(vp + k);
#pragma unroll
      for (int j = 0; j < CB; j++) acc[j][k] = fmaf(v, xv[j], acc[j][k]);
    }
  }
  const int64_t oplane = (int64_t)Ho * Wo;
#pragma unroll
  for (int j = 0; j < CB; j++) {
    if (c0 + j >= C) break;
    float *yp = y + (c0 + j) * K * oplane + (int64_t)h * Wo + w;
#pragma unroll
    for (int k = 0; k < K; k++) yp[k * oplane] = acc[j][k];
  }
}

template <int K, int CB>
__global__ void __launch_bounds__(kDiscoThreads)
    disco_bwd_kernel(const float *__restrict__ gy, float *__restrict__ gx, const int *__restrict__ row,
                     const int2 *__restrict__ idx, const float *__restrict__ val, int64_t C, int Hi, int Wi, int Ho,
                     int Wo, int s) {
  const int wi = blockIdx.x * kDiscoThreads + threadIdx.x;  // input longitude
  const int hi = blockIdx.y;                                // input latitude
  const int64_t c0 = (int64_t)blockIdx.z * CB;
  if (wi >= Wi) return;
  float acc[CB];
#pragma unroll
  for (int j = 0; j < CB; j++) acc[j] = 0.f;
  const int64_t oplane = (int64_t)Ho * Wo;
  for (int e = row[hi]; e < row[hi + 1]; e++) {
    const int2 hw = __ldg(idx + e);  // (output latitude, w')
    int d = wi - hw.y;
    if (d < 0) d += Wi;
    if (d % s) continue;
    const int w = d / s;
    const float *gp = gy + c0 * K * oplane + (int64_t)hw.x * Wo + w;
    const float *vp = val + (int64_t)e * K;
    // a few basis functions at a time: all K x CB loads at once would not
    // fit in registers
#pragma unroll 4
    for (int k = 0; k < K; k++) {
      const float v = __ldg(vp + k);
#pragma unroll
      for (int j = 0; j < CB; j++)
        if (c0 + j < C) acc[j] = fmaf(v, __ldg(gp + (j * K + k) * oplane), acc[j]);
    }
  }
  const int64_t plane = (int64_t)Hi * Wi;
#pragma unroll
  for (int j = 0; j < CB; j++)
    if (c0 + j < C) gx[(c0 + j) * plane + (int64_t)hi * Wi + wi] = acc[j];
}

// Backward by runs (nlon_in == nlon_out = W): block (input latitude hi,
// channel c), W / R threads, thread t owns input longitudes v0 = R t ..
// v0 + R - 1.  For a run (h, e0, n, a) entry j has w' = a + j (mod W) and
// adds sum_k psi[e0 + j][k] gy[c][k][h][(v - a - j) mod W] to gx[c][hi][v]
// (the even and odd k in the two lanes of packed FMAs, added at the end).
// Window slots: at step j, output r reads the value of index q = v0 + r -
// a - j, kept in slot (r - j) mod R; after the step the value q = v0 - a -
// j - 1 replaces the one output R - 1 no longer needs (slot (-j - 1) mod R).
// R odd: the lanes' shared-memory reads, R words apart, meet distinct banks.
constexpr int kRunThreadsMax = 256;

template <int K, int R>
__global__ void __launch_bounds__(kRunThreadsMax, 1)
    disco_bwd_run_kernel(const float *__restrict__ gy, float *__restrict__ gx, const int *__restrict__ run_row,
                         const int4 *__restrict__ runs, const float *__restrict__ val, int Hi, int W, int Ho,
                         unsigned *err) {
  extern __shared__ __align__(16) float disco_smem[];
  __shared__ uint64_t full[2];
  const int hi = blockIdx.x;
  const int64_t c = blockIdx.y;
  const int t = threadIdx.x;
  const int v0 = R * t;
  const int64_t oplane = (int64_t)Ho * W;
  const float *gc = gy + c * K * oplane;
  const int r0 = run_row[hi], nr = run_row[hi + 1] - r0;
  const uint32_t row_bytes = 4u * (uint32_t)W;
  if (t == 0) {
    tc::mbar_init(&full[0], 1);
    tc::mbar_init(&full[1], 1);
    tc::mbar_fence_init();
  }
  __syncthreads();
  // the K rows gy[c][k][h][.] of run i into buffer b
  auto issue = [&](int i, int b) {
    const int h = runs[r0 + i].x;
    float *dst = disco_smem + (size_t)b * K * W;
    tc::mbar_arrive_expect_tx(&full[b], (uint32_t)K * row_bytes);
    for (int k = 0; k < K; k++) tc::bulk_load(dst + (size_t)k * W, gc + k * oplane + (int64_t)h * W, row_bytes, &full[b]);
  };
  if (t == 0) {
    if (nr > 0) issue(0, 0);
    if (nr > 1) issue(1, 1);
  }
  constexpr int KP = kpairs<K>();
  float2 acc[R];  // (even k, odd k) partial sums of output r
#pragma unroll
  for (int r = 0; r < R; r++) acc[r] = make_float2(0.f, 0.f);
  for (int i = 0; i < nr; i++) {
    const int b = i & 1;
    const bool ok = tc::mbar_wait(&full[b], (i >> 1) & 1, err);
    if (!__syncthreads_and(ok)) {
      // a wait gave up: let the copies still in flight land (bounded), leave
      // gx unwritten (the error word reports it)
      if (t == 0) {
        tc::mbar_wait(&full[b], (i >> 1) & 1, nullptr, 100000000ull);
        if (i + 1 < nr) tc::mbar_wait(&full[b ^ 1], ((i + 1) >> 1) & 1, nullptr, 100000000ull);
      }
      return;
    }
    const int4 run = runs[r0 + i];
    const int e0 = run.y, n = run.z, a = run.w;
    const float *S = disco_smem + (size_t)b * K * W;
    // basis functions in pairs (2 kk, 2 kk + 1; the second zero for odd K)
    auto pair_at = [&](int kk, int d) {
      return make_float2(S[2 * kk * W + d], 2 * kk + 1 < K ? S[(2 * kk + 1) * W + d] : 0.f);
    };
    float2 win[KP][R];
    // step 0: slot r holds index v0 + r - a
    int q = v0 - a;
    if (q < 0) q += W;
#pragma unroll
    for (int r = 0; r < R; r++) {
      int d = q + r;
      if (d >= W) d -= W;
#pragma unroll
      for (int kk = 0; kk < KP; kk++) win[kk][r] = pair_at(kk, d);
    }
    // the index loaded after step j: v0 - a - j - 1 (mod W)
    int dn = q - 1;
    if (dn < 0) dn += W;
    // the basis values of the next entry load during this entry's FMAs
    float2 pn[KP];
    {
      const float2 *pv = reinterpret_cast<const float2 *>(val) + (int64_t)e0 * KP;
#pragma unroll
      for (int kk = 0; kk < KP; kk++) pn[kk] = n > 0 ? __ldg(pv + kk) : make_float2(0.f, 0.f);
    }
    for (int j0 = 0; j0 < n; j0 += R) {
#pragma unroll
      for (int u = 0; u < R; u++) {
        const int j = j0 + u;
        if (j < n) {
          float2 pc[KP];
#pragma unroll
          for (int kk = 0; kk < KP; kk++) pc[kk] = pn[kk];
          if (j + 1 < n) {
            const float2 *pv = reinterpret_cast<const float2 *>(val) + (int64_t)(e0 + j + 1) * KP;
#pragma unroll
            for (int kk = 0; kk < KP; kk++) pn[kk] = __ldg(pv + kk);
          }
#pragma unroll
          for (int kk = 0; kk < KP; kk++) {
            const float2 p = pc[kk];
#pragma unroll
            for (int r = 0; r < R; r++) acc[r] = __ffma2_rn(p, win[kk][(r - u + R) % R], acc[r]);
          }
#pragma unroll
          for (int kk = 0; kk < KP; kk++) win[kk][(R - 1 - u) % R] = pair_at(kk, dn);
          dn = dn == 0 ? W - 1 : dn - 1;
        }
      }
    }
    tc::fence_proxy_async_smem();
    __syncthreads();
    if (t == 0 && i + 2 < nr) issue(i + 2, b);
  }
  float *out = gx + (c * Hi + hi) * (int64_t)W + v0;
#pragma unroll
  for (int r = 0; r < R; r++) out[r] = acc[r].x + acc[r].y;
}

constexpr int kCB = 4;

template <int K>
cudaError_t launch_fwd_k(const sht_disco_s *d, const float *x, float *y, int64_t C, cudaStream_t st) {
  for (int64_t c = 0; c < C; c += (int64_t)65535 * kCB) {
    const int64_t nc = std::min<int64_t>(C - c, (int64_t)65535 * kCB);
    const dim3 grid((unsigned)((d->nlon_out + kDiscoThreads - 1) / kDiscoThreads), (unsigned)d->nlat_out,
                    (unsigned)((nc + kCB - 1) / kCB));
    disco_fwd_kernel<K, kCB><<<grid, kDiscoThreads, 0, st>>>(
        x + c * d->nlat_in * (int64_t)d->nlon_in, y + c * K * d->nlat_out * (int64_t)d->nlon_out, d->d_row_f,
        d->d_idx_f, d->d_val_f, nc, d->nlat_in, d->nlon_in, d->nlat_out, d->nlon_out, d->s);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int K>
cudaError_t launch_bwd_k(const sht_disco_s *d, const float *gy, float *gx, int64_t C, cudaStream_t st) {
  for (int64_t c = 0; c < C; c += (int64_t)65535 * kCB) {
    const int64_t nc = std::min<int64_t>(C - c, (int64_t)65535 * kCB);
    const dim3 grid((unsigned)((d->nlon_in + kDiscoThreads - 1) / kDiscoThreads), (unsigned)d->nlat_in,
                    (unsigned)((nc + kCB - 1) / kCB));
    disco_bwd_kernel<K, kCB><<<grid, kDiscoThreads, 0, st>>>(
        gy + c * K * d->nlat_out * (int64_t)d->nlon_out, gx + c * d->nlat_in * (int64_t)d->nlon_in, d->d_row_b,
        d->d_idx_b, d->d_val_b, nc, d->nlat_in, d->nlon_in, d->nlat_out, d->nlon_out, d->s);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int K, int R>
cudaError_t launch_bwd_run(const sht_disco_s *d, const float *gy, float *gx, int64_t C, cudaStream_t st) {
  const int W = d->nlon_in;
  const size_t smem = sizeof(float) * 2 * (size_t)K * W;
  cudaError_t e = cudaFuncSetAttribute((const void *)disco_bwd_run_kernel<K, R>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t per_c = (int64_t)K * d->nlat_out * W, per_x = (int64_t)d->nlat_in * W;
  for (int64_t c = 0; c < C; c += 65535) {
    const int64_t nc = std::min<int64_t>(C - c, 65535);
    disco_bwd_run_kernel<K, R><<<dim3((unsigned)d->nlat_in, (unsigned)nc), W / R, smem, st>>>(
        gy + c * per_c, gx + c * per_x, d->d_run_row, d->d_runs, d->d_val_w, d->nlat_in, W, d->nlat_out, d->d_err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int K>
cudaError_t launch_bwd_any(const sht_disco_s *d, const float *gy, float *gx, int64_t C, cudaStream_t st) {
  switch (d->win_R) {
    case 9: return launch_bwd_run<K, (K > 17 ? 5 : 9)>(d, gy, gx, C, st);
    case 5: return launch_bwd_run<K, 5>(d, gy, gx, C, st);
    case 3: return launch_bwd_run<K, 3>(d, gy, gx, C, st);
    default: return launch_bwd_k<K>(d, gy, gx, C, st);
  }
}

// Outputs per thread of the run kernel for W longitudes and K basis
// functions (odd, dividing W, at most kRunThreadsMax threads, a register
// window of K R values), or 0 when it does not apply.
int run_outputs_per_thread(int W, int K) {
  if (W % 4 != 0) return 0;  // 16-byte rows for the bulk copies
  if (sizeof(float) * 2 * (size_t)K * W > 227 * 1024) return 0;
  for (int R : {9, 5, 3}) {
    if (K > 17 && R == 9) continue;
    if (W % R == 0 && W / R <= kRunThreadsMax) return R;
  }
  return 0;
}

// basis values at local coordinates (vartheta, varphi); false outside the cap
bool basis_values(double vt, double vp, double tc, int n, double *out) {
  const double t = vt / tc;
  if (t >= 1.0) return false;  // h(1) = 0: nothing on the rim
  const double c = std::cos(0.5 * M_PI * t);
  const double h = c * c;
  const double xs = t * std::sin(vp), ys = t * std::cos(vp);
  int k = 0;
  for (int l = 0; l < n; l++)
    for (int m = 0; m < n; m++) out[k++] = h * std::cos(M_PI * (l * xs + m * ys));
  for (int l = 0; l < n; l++)
    for (int m = 0; m < n; m++)
      if (l || m) out[k++] = h * std::sin(M_PI * (l * xs + m * ys));
  return true;
}

void free_disco(sht_disco_s *d) {
  if (!d) return;
  int prev = -1;
  if (cudaGetDevice(&prev) == cudaSuccess && prev != d->device) cudaSetDevice(d->device);
  cudaFree(d->d_row_f);
  cudaFree(d->d_idx_f);
  cudaFree(d->d_val_f);
  cudaFree(d->d_row_b);
  cudaFree(d->d_idx_b);
  cudaFree(d->d_val_b);
  cudaFree(d->d_run_row);
  cudaFree(d->d_runs);
  cudaFree(d->d_val_w);
  cudaFree(d->d_err);
  if (prev >= 0 && prev != d->device) cudaSetDevice(prev);
  delete d;
}

template <class T>
cudaError_t upload_vec(T **dst, const std::vector<T> &v) {
  const size_t bytes = std::max<size_t>(sizeof(T), sizeof(T) * v.size());
  cudaError_t e = cudaMalloc((void **)dst, bytes);
  if (e != cudaSuccess) return e;
  if (!v.empty()) e = cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
  return e;
}

}  // namespace
}  // namespace shtgb

using namespace shtgb;

extern "C" {

sht_status_t sht_disco_create(sht_disco_t *out, int nlat_in, int nlon_in, int grid_in, int nlat_out, int nlon_out,
                              int grid_out, int basis_n, double theta_cutoff, int device) {
  NvtxRange nvtx_range("sht_disco_create");
  if (!out) return fail(SHT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nlat_in < 2 || nlat_out < 2 || nlon_in < 1 || nlon_out < 1)
    return fail(SHT_ERR_INVALID_ARG, "need nlat >= 2 and nlon >= 1 on both grids");
  if (nlon_in % nlon_out) return fail(SHT_ERR_INVALID_ARG, "nlon_in must be a multiple of nlon_out");
  for (int g : {grid_in, grid_out})
    if (g != SHT_GRID_GAUSS && g != SHT_GRID_EQUIANGULAR_CC && g != SHT_GRID_EQUIANGULAR_TRAPZ)
      return fail(SHT_ERR_INVALID_ARG, "unknown grid");
  if (basis_n < 1 || basis_n > 4) return fail(SHT_ERR_INVALID_ARG, "basis_n must be 1 .. 4");
  if (!(theta_cutoff > 0.0) || theta_cutoff > M_PI) return fail(SHT_ERR_INVALID_ARG, "need 0 < theta_cutoff <= pi");
  sht_disco_s *d = new (std::nothrow) sht_disco_s();
  if (!d) return fail(SHT_ERR_OOM, "host allocation failed");
  d->device = device;
  d->nlat_in = nlat_in;
  d->nlon_in = nlon_in;
  d->nlat_out = nlat_out;
  d->nlon_out = nlon_out;
  d->s = nlon_in / nlon_out;
  d->n = basis_n;
  d->K = 2 * basis_n * basis_n - 1;
  d->theta_cutoff = theta_cutoff;
  const int K = d->K;
  std::vector<double> xi, si, wi, xo, so, wo;
  grid_nodes(grid_in, nlat_in, xi, si, wi);
  grid_nodes(grid_out, nlat_out, xo, so, wo);
  // entries by output latitude, then input latitude, then w'
  std::vector<int> row_f(nlat_out + 1, 0);
  std::vector<int2> idx_f;
  std::vector<float> val_f;
  std::vector<double> bv(K);
  for (int h = 0; h < nlat_out; h++) {
    const double to = std::atan2(so[h], xo[h]);
    const double co = xo[h], sno = so[h];
    for (int hp = 0; hp < nlat_in; hp++) {
      const double ti = std::atan2(si[hp], xi[hp]);
      if (std::fabs(ti - to) >= theta_cutoff) continue;  // the distance is at least |dtheta|
      const double omega = wi[hp] * 2.0 * M_PI / nlon_in;
      for (int wp = 0; wp < nlon_in; wp++) {
        const double ph = 2.0 * M_PI * wp / nlon_in;
        const double vx = co * si[hp] * std::cos(ph) - sno * xi[hp];
        const double vy = si[hp] * std::sin(ph);
        const double vz = sno * si[hp] * std::cos(ph) + co * xi[hp];
        const double vt = std::atan2(std::hypot(vx, vy), vz);
        if (!basis_values(vt, std::atan2(vy, vx), theta_cutoff, basis_n, bv.data())) continue;
        idx_f.push_back(make_int2(hp, wp));
        for (int k = 0; k < K; k++) val_f.push_back((float)(bv[k] * omega));
      }
    }
    row_f[h + 1] = (int)idx_f.size();
  }
  d->nnz = (int64_t)idx_f.size();
  // the same entries by input latitude
  std::vector<int> row_b(nlat_in + 1, 0);
  for (int h = 0; h < nlat_out; h++)
    for (int e = row_f[h]; e < row_f[h + 1]; e++) row_b[idx_f[e].x + 1]++;
  for (int hp = 0; hp < nlat_in; hp++) row_b[hp + 1] += row_b[hp];
  std::vector<int2> idx_b(idx_f.size());
  std::vector<float> val_b(val_f.size());
  std::vector<int> fill(row_b.begin(), row_b.end() - 1);
  for (int h = 0; h < nlat_out; h++)
    for (int e = row_f[h]; e < row_f[h + 1]; e++) {
      const int dst = fill[idx_f[e].x]++;
      idx_b[dst] = make_int2(h, idx_f[e].y);
      for (int k = 0; k < K; k++) val_b[(size_t)dst * K + k] = val_f[(size_t)e * K + k];
    }
  // runs of consecutive w' (mod nlon) per (input latitude, output latitude)
  // for the backward on equal longitude grids
  std::vector<int> run_row(nlat_in + 1, 0);
  std::vector<int4> runs;
  std::vector<float> val_w;
  d->win_R = d->s == 1 ? run_outputs_per_thread(nlon_in, K) : 0;
  if (d->win_R) {
    const int W = nlon_in;
    val_w.reserve(val_b.size());
    for (int hp = 0; hp < nlat_in; hp++) {
      for (int e0 = row_b[hp]; e0 < row_b[hp + 1];) {
        const int h = idx_b[e0].x;
        int e1 = e0;
        while (e1 < row_b[hp + 1] && idx_b[e1].x == h) e1++;
        const int n = e1 - e0;
        auto wp = [&](int i) { return idx_b[e0 + i % n].y; };
        // start after a gap in the circular order (none: the whole ring)
        int start = 0;
        if (n < W)
          for (int i = 0; i < n; i++)
            if ((wp(i + n - 1) + 1) % W != wp(i)) {
              start = i;
              break;
            }
        for (int i = 0; i < n;) {
          int len = 1;
          while (i + len < n && (wp(start + i + len - 1) + 1) % W == wp(start + i + len)) len++;
          runs.push_back(make_int4(h, (int)(val_w.size() / K), len, wp(start + i)));
          for (int q = 0; q < len; q++) {
            const size_t src = (size_t)(e0 + (start + i + q) % n) * K;
            val_w.insert(val_w.end(), val_b.begin() + src, val_b.begin() + src + K);
          }
          i += len;
        }
        e0 = e1;
      }
      run_row[hp + 1] = (int)runs.size();
    }
  }
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (prev != device && cudaSetDevice(device) != cudaSuccess) {
    delete d;
    return fail(SHT_ERR_CUDA, "cannot select the device");
  }
  // the forward and run kernels read an entry's values in pairs: 2 ceil(K / 2) floats
  auto pad_pairs = [&](const std::vector<float> &v) {
    const int K2 = K + (K & 1);
    if (K2 == K) return v;
    std::vector<float> out(v.size() / K * K2, 0.f);
    for (size_t r = 0; r < v.size() / K; r++) std::copy(v.begin() + r * K, v.begin() + (r + 1) * K, out.begin() + r * K2);
    return out;
  };
  cudaError_t e = upload_vec(&d->d_row_f, row_f);
  if (e == cudaSuccess) e = upload_vec(&d->d_idx_f, idx_f);
  if (e == cudaSuccess) e = upload_vec(&d->d_val_f, pad_pairs(val_f));
  if (e == cudaSuccess) e = upload_vec(&d->d_row_b, row_b);
  if (e == cudaSuccess) e = upload_vec(&d->d_idx_b, idx_b);
  if (e == cudaSuccess) e = upload_vec(&d->d_val_b, val_b);
  if (e == cudaSuccess && d->win_R) e = upload_vec(&d->d_run_row, run_row);
  if (e == cudaSuccess && d->win_R) e = upload_vec(&d->d_runs, runs);
  if (e == cudaSuccess && d->win_R) e = upload_vec(&d->d_val_w, pad_pairs(val_w));
  if (e == cudaSuccess) e = cudaMalloc((void **)&d->d_err, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(d->d_err, 0, sizeof(unsigned));
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    free_disco(d);
    return e == cudaErrorMemoryAllocation ? fail(SHT_ERR_OOM, "device allocation failed")
                                          : cuda_fail(e, "DISCO tensor upload");
  }
  *out = d;
  return SHT_OK;
}

sht_status_t sht_disco_info(sht_disco_t d, int *nbasis, int64_t *nnz) {
  if (!d) return fail(SHT_ERR_INVALID_ARG, "DISCO handle is NULL");
  if (nbasis) *nbasis = d->K;
  if (nnz) *nnz = d->nnz;
  return SHT_OK;
}

static sht_status_t disco_run(sht_disco_t d, const float *in, float *out, int64_t C, void *stream, bool fwd) {
  if (!d) return fail(SHT_ERR_INVALID_ARG, "DISCO handle is NULL");
  if (C < 0) return fail(SHT_ERR_INVALID_ARG, "channel count must be >= 0");
  if (C == 0) return SHT_OK;
  if (!in || !out) return fail(SHT_ERR_INVALID_ARG, "input and output must not be NULL");
  if ((((uintptr_t)in) | ((uintptr_t)out)) & 15) return fail(SHT_ERR_INVALID_ARG, "pointers must be 16-byte aligned");
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (prev != d->device && cudaSetDevice(d->device) != cudaSuccess)
    return fail(SHT_ERR_CUDA, "cannot select the device");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  switch (d->K) {
    case 1: e = fwd ? launch_fwd_k<1>(d, in, out, C, st) : launch_bwd_any<1>(d, in, out, C, st); break;
    case 7: e = fwd ? launch_fwd_k<7>(d, in, out, C, st) : launch_bwd_any<7>(d, in, out, C, st); break;
    case 17: e = fwd ? launch_fwd_k<17>(d, in, out, C, st) : launch_bwd_any<17>(d, in, out, C, st); break;
    default: e = fwd ? launch_fwd_k<31>(d, in, out, C, st) : launch_bwd_any<31>(d, in, out, C, st); break;
  }
  if (prev >= 0 && prev != d->device) cudaSetDevice(prev);
  return e == cudaSuccess ? SHT_OK : cuda_fail(e, fwd ? "disco_fwd_kernel" : "disco_bwd_kernel");
}

sht_status_t sht_disco_forward(sht_disco_t d, const float *x, float *y, int64_t C, void *stream) {
  NvtxRange nvtx_range("sht_disco_forward");
  return disco_run(d, x, y, C, stream, true);
}

sht_status_t sht_disco_backward(sht_disco_t d, const float *gy, float *gx, int64_t C, void *stream) {
  NvtxRange nvtx_range("sht_disco_backward");
  return disco_run(d, gy, gx, C, stream, false);
}

sht_status_t sht_disco_check(sht_disco_t d) {
  NvtxRange nvtx_range("sht_disco_check");
  if (!d) return fail(SHT_ERR_INVALID_ARG, "DISCO handle is NULL");
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (prev != d->device && cudaSetDevice(d->device) != cudaSuccess)
    return fail(SHT_ERR_CUDA, "cannot select the device");
  unsigned word = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&word, d->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && word) e = cudaMemset(d->d_err, 0, sizeof(unsigned));
  if (prev >= 0 && prev != d->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_fail(e, "DISCO error word read");
  if (word) return fail(SHT_ERR_TIMEOUT, "a DISCO kernel's wait for its staged rows ran out of time");
  return SHT_OK;
}

sht_status_t sht_disco_destroy(sht_disco_t d) {
  free_disco(d);
  return SHT_OK;
}

}  // extern "C"
