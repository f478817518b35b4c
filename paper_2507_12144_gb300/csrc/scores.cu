// Ensemble scores of forecasts, on spherical harmonic coefficients and on the
// grid:
//   angular power spectrum, Eq. (psd) (Sec. F.7):
//     PSD(l) = sum_{|m| <= l} |u_l^m|^2 = |u_l^0|^2 + 2 sum_{m = 1}^{l} |u_l^m|^2
//     (only m >= 0 is stored; for a real field |u_l^{-m}| = |u_l^m|);
//   ensemble CRPS, Eq. (spread_skill_crps), and fair CRPS,
//   Eq. (fair_spread_skill_crps) (Sec. D.4), evaluated on the sorted ensemble:
//     CRPS = (1/E) sum_e |u_e - u*| - S / D,
//     S = sum_{i=0}^{E-1} (2 i + 1 - E) u_(i)   (u_(0) <= ... <= u_(E-1)),
//     so that sum_e sum_i |u_e - u_i| = 2 S, with D = E^2 (biased) or
//     E (E - 1) (fair);
//   spectral CRPS, Eq. (spectral_loss) (Sec. E.1): the CRPS of the real and
//   of the imaginary part of every coefficient, summed over |m| <= l (m = 0
//   once, m > 0 twice);
//   spatial CRPS, Eq. (spatial_loss): the point-wise CRPS averaged over the
//   sphere with the grid's quadrature weights.
//
// Every score is one pass over its inputs: each thread sorts one value's E
// members in registers (a bitonic network over the next power of two, the
// padding at +inf), the thread block sums its row in a fixed order, and a
// warp per channel sums the rows, so results are deterministic.  The spread
// sum is taken over the differences to the observation, which it does not
// change (the weights 2 i + 1 - E sum to zero), so that a common offset of
// the members does not cancel in FP32.
#include <algorithm>
#include <cmath>

#include "sht_internal.cuh"

namespace shtgb {
namespace {

constexpr int kScoreThreads = 128;
constexpr int kMaxMembers = 64;

// ascending bitonic sort of NP values held in registers (all indices are
// compile-time constants after unrolling)
template <int NP>
__device__ __forceinline__ void bitonic_sort(float (&v)[NP]) {
#pragma unroll
  for (int k = 2; k <= NP; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
      for (int i = 0; i < NP; i++) {
        const int p = i ^ j;
        if (p > i) {
          const float lo = fminf(v[i], v[p]), hi = fmaxf(v[i], v[p]);
          if ((i & k) == 0) {
            v[i] = lo;
            v[p] = hi;
          } else {
            v[i] = hi;
            v[p] = lo;
          }
        }
      }
    }
  }
}

// The E members p[0], p[stride], ..., p[(E - 1) stride] of one real value
// (zeros when !ok or past E).
template <int NP>
__device__ __forceinline__ void load_members(float (&v)[NP], const float *__restrict__ p, int64_t stride, int E,
                                             bool ok) {
#pragma unroll
  for (int i = 0; i < NP; i++) v[i] = (ok && i < E) ? __ldg(p + i * stride) : 0.f;
}

// CRPS of one real value whose E members are in v, against its observation
// ob; inv_e = 1 / E, inv_d = 1 / D.  v is overwritten.
template <int NP>
__device__ __forceinline__ float crps_of(float (&v)[NP], int E, float ob, float inv_e, float inv_d) {
  float skill = 0.f;
#pragma unroll
  for (int i = 0; i < NP; i++) {
    if (i < E) {
      v[i] -= ob;
      skill += fabsf(v[i]);
    } else {
      v[i] = INFINITY;
    }
  }
  bitonic_sort<NP>(v);
  const float Ef = (float)E;
  float S = 0.f;
#pragma unroll
  for (int i = 0; i < NP; i++) S = fmaf((float)(2 * i + 1) - Ef, i < E ? v[i] : 0.f, S);
  return skill * inv_e - S * inv_d;
}

template <int NP>
__device__ __forceinline__ float crps_one(const float *__restrict__ p, int64_t stride, int E, float ob, float inv_e,
                                          float inv_d) {
  float v[NP];
  load_members<NP>(v, p, stride, E, true);
  return crps_of<NP>(v, E, ob, inv_e, inv_d);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of the block's per-thread values in a fixed order; valid in thread 0.
__device__ __forceinline__ float block_sum(float v) {
  __shared__ float part[kScoreThreads / 32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  float s = 0.f;
  if (threadIdx.x == 0)
#pragma unroll
    for (int w = 0; w < kScoreThreads / 32; w++) s += part[w];
  return s;
}

// One block per row (c, l) of the coefficients: thread pairs take the real
// and imaginary part of one order m.
template <int NP>
__global__ void __launch_bounds__(kScoreThreads) spectral_crps_kernel(const float *__restrict__ ens,
                                                                      const float *__restrict__ obs,
                                                                      float *__restrict__ crps_l,
                                                                      float *__restrict__ crps_lm, int E, int64_t C,
                                                                      int L, int M, float inv_e, float inv_d) {
  const int64_t row = blockIdx.x;  // c * L + l
  const int l = (int)(row % L);
  const int mlim = min(l + 1, M);
  const int part = threadIdx.x & 1;
  const int64_t stride = 2 * C * (int64_t)L * M;  // floats from one member to the next
  const float *erow = ens + row * 2 * M;
  const float *orow = obs + row * 2 * M;
  float acc = 0.f;
  for (int m0 = 0; m0 < mlim; m0 += kScoreThreads / 2) {
    const int m = m0 + (threadIdx.x >> 1);
    float v = 0.f;
    if (m < mlim) v = crps_one<NP>(erow + 2 * m + part, stride, E, __ldg(orow + 2 * m + part), inv_e, inv_d);
    v += __shfl_xor_sync(0xffffffffu, v, 1);  // real + imaginary part
    if (m < mlim && part == 0) {
      if (crps_lm) crps_lm[row * M + m] = v;
      acc = fmaf(m == 0 ? 1.f : 2.f, v, acc);
    }
  }
  if (crps_lm)
    for (int m = mlim + threadIdx.x; m < M; m += kScoreThreads) crps_lm[row * M + m] = 0.f;
  const float s = block_sum(acc);
  if (threadIdx.x == 0) crps_l[row] = s;
}

// One block per latitude row (c, k): the row's contribution to Eq.
// (spatial_loss), (1 / (4 pi)) w_k (2 pi / nlon) sum_j CRPS(k, j).
template <int NP>
__global__ void __launch_bounds__(kScoreThreads) spatial_crps_kernel(const float *__restrict__ ens,
                                                                     const float *__restrict__ obs,
                                                                     const float *__restrict__ ring_w,
                                                                     float *__restrict__ crps_k, int E, int64_t C,
                                                                     int nlat, int nlon, float inv_e, float inv_d) {
  const int64_t row = blockIdx.x;  // c * nlat + k
  const int k = (int)(row % nlat);
  const int64_t stride = C * (int64_t)nlat * nlon;
  const float *erow = ens + row * nlon;
  const float *orow = obs + row * nlon;
  float acc = 0.f;
  for (int j = threadIdx.x; j < nlon; j += kScoreThreads)
    acc += crps_one<NP>(erow + j, stride, E, __ldg(orow + j), inv_e, inv_d);
  const float s = block_sum(acc);
  if (threadIdx.x == 0) crps_k[row] = s * ring_w[k] * (float)(0.25 / M_PI);
}

__device__ __forceinline__ float sgnf(float x) { return (float)((x > 0.f) - (x < 0.f)); }

// Gradient of loss[c] = sum_{l_lo <= l < l_hi} crps_l[c][l] weighted by
// gloss[c].  For one real value with members u_e and observation u*,
//   d CRPS / d u_e = sign(u_e - u*) / E - (1/D) sum_i sign(u_e - u_i),
//   d CRPS / d u*  = -(1/E) sum_e sign(u_e - u*),
// the derivative of the spread-skill form (u_e enters the double sum twice),
// with sign(0) = 0: at ties the subgradient that averages the tied ranks
// (without ties sum_i sign(u_e - u_i) = 2 r_e + 1 - E for the rank r_e).
// The pair signs are taken once per pair in registers, so that each
// member's gradient is stored in member order (coalesced).  Every entry of
// gens (and gobs) is written: zero outside the degree range and at l < m.
template <int NP>
__global__ void __launch_bounds__(kScoreThreads)
    spectral_crps_grad_kernel(const float *__restrict__ ens, const float *__restrict__ obs,
                              const float *__restrict__ gloss, float *__restrict__ gens, float *__restrict__ gobs,
                              int E, int64_t C, int L, int M, int l_lo, int l_hi, float inv_e, float inv_d) {
  const int64_t row = blockIdx.x;  // c * L + l
  const int l = (int)(row % L);
  const int64_t c = row / L;
  const bool live = l >= l_lo && l < l_hi;
  const int mlim = live ? min(l + 1, M) : 0;
  const float g = live ? __ldg(gloss + c) : 0.f;
  const int part = threadIdx.x & 1;
  const int64_t stride = 2 * C * (int64_t)L * M;
  const float *erow = ens + row * 2 * M;
  const float *orow = obs + row * 2 * M;
  float *grow = gens + row * 2 * M;
  for (int m = threadIdx.x >> 1; m < M; m += kScoreThreads / 2) {
    const int off = 2 * m + part;
    if (m >= mlim) {
      for (int e = 0; e < E; e++) grow[e * stride + off] = 0.f;
      if (gobs) gobs[row * 2 * M + off] = 0.f;
      continue;
    }
    const float w = (m == 0 ? 1.f : 2.f) * g;
    // signs from the members themselves: the sign of an FP32 difference is
    // exact, so every decision is the one exact arithmetic makes
    float u[NP];
    load_members<NP>(u, erow + off, stride, E, true);
    const float ob = __ldg(orow + off);
    float ssum = 0.f, ps[NP];  // ps[e] = sum_i sign(u_e - u_i)
#pragma unroll
    for (int e = 0; e < NP; e++) {
      ps[e] = 0.f;
      if (e < E) ssum += sgnf(u[e] - ob);
    }
#pragma unroll
    for (int e = 1; e < NP; e++) {
      if (e < E) {
#pragma unroll
        for (int i = 0; i < e; i++) {
          const float t = sgnf(u[e] - u[i]);
          ps[e] += t;
          ps[i] -= t;
        }
      }
    }
#pragma unroll
    for (int e = 0; e < NP; e++)
      if (e < E) grow[e * stride + off] = w * (sgnf(u[e] - ob) * inv_e - ps[e] * inv_d);
    if (gobs) gobs[row * 2 * M + off] = -w * inv_e * ssum;
  }
}

// loss[c] = sum_{r0 <= r < r1} rows[c][r], one warp per channel (lanes take
// strided rows, then a fixed butterfly).
__global__ void __launch_bounds__(256) row_sum_kernel(const float *__restrict__ rows, float *__restrict__ loss,
                                                      int64_t C, int R, int r0, int r1) {
  const int64_t c = blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32;
  if (c >= C) return;
  const int lane = threadIdx.x & 31;
  float s = 0.f;
  for (int r = r0 + lane; r < r1; r += 32) s += rows[c * R + r];
  s = warp_sum(s);
  if (lane == 0) loss[c] = s;
}

// One warp per row (b, l): PSD(l) of Eq. (psd).
__global__ void __launch_bounds__(256) angular_psd_kernel(const float2 *__restrict__ x, float *__restrict__ psd,
                                                          int64_t rows, int L, int M) {
  const int64_t row = blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32;
  if (row >= rows) return;
  const int l = (int)(row % L);
  const int mlim = min(l + 1, M);
  const int lane = threadIdx.x & 31;
  const float2 *r = x + row * M;
  float acc = 0.f;
  for (int m = lane; m < mlim; m += 32) {
    const float2 v = __ldg(r + m);
    acc = fmaf(m == 0 ? 1.f : 2.f, fmaf(v.x, v.x, v.y * v.y), acc);
  }
  acc = warp_sum(acc);
  if (lane == 0) psd[row] = acc;
}

// Zonal power spectrum, Eq. (zonal_psd), from the plan's longitude FFT of
// ring pairs (no weights, FP32): E = X_k + X_kbar, O = X_k - X_kbar with
// X_k(m) = sum_j u_kj e^{-i m phi_j} (the equator ring of odd nlat: E = X_k),
//   zpsd[b][k][m] = zc[k] |X_k(m)|^2,  zc[k] = 2 pi sin(theta_k) (2 pi / nlon)^2.
// A block takes 32 orders x 32 fields of one ring pair through shared memory,
// so that it reads the folded rows along the fields and writes the output
// rows along the orders.
__global__ void __launch_bounds__(256) zonal_psd_kernel(const float *__restrict__ F, float *__restrict__ zpsd,
                                                        const float *__restrict__ zc, int nlat, int M, int nb,
                                                        FoldLayout fl) {
  __shared__ float tn[32][33], ts[32][33];
  const int kq = blockIdx.y, ks = nlat - 1 - kq;
  const int m0 = blockIdx.x * 32, b0 = blockIdx.z * 32;
  const bool eq = kq == ks;
  const float cn = zc[kq], cs = zc[ks];
  {
    const int b = threadIdx.x & 31;
    for (int mi = threadIdx.x >> 5; mi < 32; mi += 8) {
      const int m = m0 + mi;
      float vn = 0.f, vs = 0.f;
      if (m < M && b0 + b < nb) {
        const float2 E = *reinterpret_cast<const float2 *>(F + fold_row(fl, m, 0, kq) + 2 * (b0 + b));
        if (eq) {
          vn = cn * (E.x * E.x + E.y * E.y);
        } else {
          const float2 O = *reinterpret_cast<const float2 *>(F + fold_row(fl, m, 1, kq) + 2 * (b0 + b));
          const float nr = 0.5f * (E.x + O.x), ni = 0.5f * (E.y + O.y);
          const float sr = 0.5f * (E.x - O.x), si = 0.5f * (E.y - O.y);
          vn = cn * (nr * nr + ni * ni);
          vs = cs * (sr * sr + si * si);
        }
      }
      tn[mi][b] = vn;
      ts[mi][b] = vs;
    }
  }
  __syncthreads();
  const int mi = threadIdx.x & 31;
  if (m0 + mi >= M) return;
  for (int b = threadIdx.x >> 5; b < 32 && b0 + b < nb; b += 8) {
    float *out = zpsd + (int64_t)(b0 + b) * nlat * M + m0 + mi;
    out[(int64_t)kq * M] = tn[mi][b];
    if (!eq) out[(int64_t)ks * M] = ts[mi][b];
  }
}

int members_bucket(int E) {
  int np = 1;
  while (np < E) np <<= 1;
  return np;
}

template <template <int> class K, class... Args>
cudaError_t launch_bucket(int np, dim3 grid, cudaStream_t st, Args... args) {
  switch (np) {
    case 1: K<1>::launch(grid, st, args...); break;
    case 2: K<2>::launch(grid, st, args...); break;
    case 4: K<4>::launch(grid, st, args...); break;
    case 8: K<8>::launch(grid, st, args...); break;
    case 16: K<16>::launch(grid, st, args...); break;
    case 32: K<32>::launch(grid, st, args...); break;
    default: K<64>::launch(grid, st, args...); break;
  }
  return cudaGetLastError();
}

template <int NP>
struct SpectralLaunch {
  template <class... Args>
  static void launch(dim3 grid, cudaStream_t st, Args... args) {
    spectral_crps_kernel<NP><<<grid, kScoreThreads, 0, st>>>(args...);
  }
};
template <int NP>
struct GradLaunch {
  template <class... Args>
  static void launch(dim3 grid, cudaStream_t st, Args... args) {
    spectral_crps_grad_kernel<NP><<<grid, kScoreThreads, 0, st>>>(args...);
  }
};
template <int NP>
struct SpatialLaunch {
  template <class... Args>
  static void launch(dim3 grid, cudaStream_t st, Args... args) {
    spatial_crps_kernel<NP><<<grid, kScoreThreads, 0, st>>>(args...);
  }
};

sht_status_t check_dev_ptr(const void *ptr, const char *name, bool nullable) {
  if (!ptr) return nullable ? SHT_OK : fail(SHT_ERR_INVALID_ARG, std::string(name) + " is NULL");
  if (((uintptr_t)ptr) & 15) return fail(SHT_ERR_INVALID_ARG, std::string(name) + " is not 16-byte aligned");
  return SHT_OK;
}

sht_status_t check_members(int E, int fair) {
  if (E < 1 || E > kMaxMembers) return fail(SHT_ERR_INVALID_ARG, "the member count must be 1 .. 64");
  if (fair && E < 2) return fail(SHT_ERR_INVALID_ARG, "the fair CRPS needs at least two members");
  return SHT_OK;
}

cudaError_t launch_row_sum(const float *rows, float *loss, int64_t C, int R, int r0, int r1, cudaStream_t st) {
  const int64_t blocks = (C + 7) / 8;
  row_sum_kernel<<<(unsigned)blocks, 256, 0, st>>>(rows, loss, C, R, r0, r1);
  return cudaGetLastError();
}

}  // namespace
}  // namespace shtgb

using namespace shtgb;

#define SCORE_TRY(expr)                  \
  do {                                   \
    const sht_status_t _s = (expr);      \
    if (_s != SHT_OK) return _s;         \
  } while (0)

extern "C" {

sht_status_t sht_angular_psd(const void *xhat, float *psd, int64_t B, int lmax, int mmax, void *stream) {
  NvtxRange nvtx_range("sht_angular_psd");
  if (B < 0) return fail(SHT_ERR_INVALID_ARG, "batch must be >= 0");
  if (lmax < 1 || mmax < 1 || mmax > lmax) return fail(SHT_ERR_INVALID_ARG, "need 1 <= mmax <= lmax");
  if (B == 0) return SHT_OK;
  SCORE_TRY(check_dev_ptr(xhat, "xhat", false));
  SCORE_TRY(check_dev_ptr(psd, "psd", false));
  const int64_t rows = B * lmax;
  const int64_t blocks = (rows + 7) / 8;
  if (blocks > 0x7fffffff) return fail(SHT_ERR_INVALID_ARG, "too many rows");
  angular_psd_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>((const float2 *)xhat, psd, rows, lmax,
                                                                         mmax);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SHT_OK : cuda_fail(e, "angular_psd_kernel");
}

sht_status_t sht_spectral_crps(const void *ens, const void *obs, float *crps_l, float *crps_lm, float *loss, int E,
                               int64_t C, int lmax, int mmax, int fair, int l_lo, int l_hi, void *stream) {
  NvtxRange nvtx_range("sht_spectral_crps");
  SCORE_TRY(check_members(E, fair));
  if (C < 0) return fail(SHT_ERR_INVALID_ARG, "channel count must be >= 0");
  if (lmax < 1 || mmax < 1 || mmax > lmax) return fail(SHT_ERR_INVALID_ARG, "need 1 <= mmax <= lmax");
  if (l_lo < 0 || l_lo > l_hi || l_hi > lmax) return fail(SHT_ERR_INVALID_ARG, "need 0 <= l_lo <= l_hi <= lmax");
  if (C == 0) return SHT_OK;
  SCORE_TRY(check_dev_ptr(ens, "ens", false));
  SCORE_TRY(check_dev_ptr(obs, "obs", false));
  SCORE_TRY(check_dev_ptr(crps_l, "crps_l", false));
  SCORE_TRY(check_dev_ptr(crps_lm, "crps_lm", true));
  SCORE_TRY(check_dev_ptr(loss, "loss", true));
  const int64_t rows = C * lmax;
  if (rows > 0x7fffffff) return fail(SHT_ERR_INVALID_ARG, "too many rows");
  cudaStream_t st = (cudaStream_t)stream;
  const float inv_e = 1.0f / (float)E;
  const float inv_d = (float)(fair ? 1.0 / ((double)E * (E - 1)) : 1.0 / ((double)E * E));
  cudaError_t e = launch_bucket<SpectralLaunch>(members_bucket(E), dim3((unsigned)rows), st, (const float *)ens,
                                                (const float *)obs, crps_l, crps_lm, E, C, lmax, mmax, inv_e, inv_d);
  if (e != cudaSuccess) return cuda_fail(e, "spectral_crps_kernel");
  if (loss) {
    e = launch_row_sum(crps_l, loss, C, lmax, l_lo, l_hi, st);
    if (e != cudaSuccess) return cuda_fail(e, "row_sum_kernel");
  }
  return SHT_OK;
}

sht_status_t sht_spectral_crps_backward(const void *ens, const void *obs, const float *gloss, void *gens,
                                        void *gobs, int E, int64_t C, int lmax, int mmax, int fair, int l_lo,
                                        int l_hi, void *stream) {
  NvtxRange nvtx_range("sht_spectral_crps_backward");
  SCORE_TRY(check_members(E, fair));
  if (C < 0) return fail(SHT_ERR_INVALID_ARG, "channel count must be >= 0");
  if (lmax < 1 || mmax < 1 || mmax > lmax) return fail(SHT_ERR_INVALID_ARG, "need 1 <= mmax <= lmax");
  if (l_lo < 0 || l_lo > l_hi || l_hi > lmax) return fail(SHT_ERR_INVALID_ARG, "need 0 <= l_lo <= l_hi <= lmax");
  if (C == 0) return SHT_OK;
  SCORE_TRY(check_dev_ptr(ens, "ens", false));
  SCORE_TRY(check_dev_ptr(obs, "obs", false));
  SCORE_TRY(check_dev_ptr(gloss, "gloss", false));
  SCORE_TRY(check_dev_ptr(gens, "gens", false));
  SCORE_TRY(check_dev_ptr(gobs, "gobs", true));
  const int64_t rows = C * lmax;
  if (rows > 0x7fffffff) return fail(SHT_ERR_INVALID_ARG, "too many rows");
  const float inv_e = 1.0f / (float)E;
  const float inv_d = (float)(fair ? 1.0 / ((double)E * (E - 1)) : 1.0 / ((double)E * E));
  const cudaError_t e =
      launch_bucket<GradLaunch>(members_bucket(E), dim3((unsigned)rows), (cudaStream_t)stream, (const float *)ens,
                                (const float *)obs, gloss, (float *)gens, (float *)gobs, E, C, lmax, mmax, l_lo, l_hi,
                                inv_e, inv_d);
  return e == cudaSuccess ? SHT_OK : cuda_fail(e, "spectral_crps_grad_kernel");
}

sht_status_t sht_zonal_psd(sht_plan_t plan, const float *x, float *zpsd, int64_t B, void *stream) {
  NvtxRange nvtx_range("sht_zonal_psd");
  if (!plan) return fail(SHT_ERR_INVALID_ARG, "plan is NULL");
  if (B < 0) return fail(SHT_ERR_INVALID_ARG, "batch must be >= 0");
  if (B == 0) return SHT_OK;
  SCORE_TRY(check_dev_ptr(x, "x", false));
  SCORE_TRY(check_dev_ptr(zpsd, "zpsd", false));
  sht_plan_s *p = plan;
  // The FP32 folded FFT of a chunk of fields needs M x 2 x Kh rows of ld
  // floats (ld = 2 for one field, else 2 n rounded up to 4).  FP32 plans
  // use their analysis workspace (FP32 in every call, sized for max_batch
  // fields); tensor-core plans use their FP32 spectral buffer, never the
  // bf16 workspace, and take as many fields per chunk as it holds.
  const bool fp32 = p->precision == SHT_PREC_FP32;
  const size_t scratch = fp32 ? sizeof(float) * (size_t)p->M * 2 * p->Kh * p->ldc
                              : std::max(sizeof(float2) * (size_t)p->max_batch * p->L * p->M,
                                         sizeof(float) * (size_t)p->L * p->M * p->ldr);
  const size_t row_bytes = sizeof(float) * (size_t)p->M * 2 * p->Kh;
  auto ld_of = [](int64_t n) { return n == 1 ? (int64_t)2 : (2 * n + 3) / 4 * 4; };
  int64_t nb = std::min<int64_t>(p->max_batch, B);
  while (nb > 1 && row_bytes * (size_t)ld_of(nb) > scratch) nb--;
  if (row_bytes * (size_t)ld_of(nb) > scratch)
    return fail(SHT_ERR_UNSUPPORTED, "the plan's FP32 buffer is too small for one field's longitude FFT (lmax < nlat / 2 "
                                     "on a tensor-core plan); use an FP32 plan");
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (prev != p->device && cudaSetDevice(p->device) != cudaSuccess)
    return fail(SHT_ERR_CUDA, "cannot select the plan's device");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  float *F = fp32 ? p->d_work : reinterpret_cast<float *>(p->d_spec_b);
  const int64_t npix = (int64_t)p->nlat * p->nlon;
  for (int64_t b0 = 0; b0 < B && e == cudaSuccess; b0 += nb) {
    const int n = (int)std::min<int64_t>(nb, B - b0);
    const FoldLayout fl = classic_layout(p->Kh, (int)ld_of(n));
    if (fft45_supported(p->nlon))
      e = launch_r2c45(x + b0 * npix, F, nullptr, nullptr, p->nlat, p->nlon, p->M, n, fl, p->d_twiddle, nullptr, 0,
                       st);
    else
      e = launch_r2c(x + b0 * npix, F, p->nlat, p->nlon, p->M, n, fl, p->d_twiddle, p->radix, nullptr, 0, st);
    if (e != cudaSuccess) break;
    const dim3 grid((unsigned)((p->M + 31) / 32), (unsigned)p->Kh, (unsigned)((n + 31) / 32));
    zonal_psd_kernel<<<grid, 256, 0, st>>>(F, zpsd + b0 * p->nlat * (int64_t)p->M, p->d_zonal_c, p->nlat, p->M, n,
                                           fl);
    e = cudaGetLastError();
  }
  if (prev >= 0 && prev != p->device) cudaSetDevice(prev);
  return e == cudaSuccess ? SHT_OK : cuda_fail(e, "zonal power spectrum");
}

sht_status_t sht_spatial_crps(sht_plan_t plan, const float *ens, const float *obs, float *crps_k, float *loss, int E,
                              int64_t C, int fair, void *stream) {
  NvtxRange nvtx_range("sht_spatial_crps");
  if (!plan) return fail(SHT_ERR_INVALID_ARG, "plan is NULL");
  SCORE_TRY(check_members(E, fair));
  if (C < 0) return fail(SHT_ERR_INVALID_ARG, "channel count must be >= 0");
  if (C == 0) return SHT_OK;
  SCORE_TRY(check_dev_ptr(ens, "ens", false));
  SCORE_TRY(check_dev_ptr(obs, "obs", false));
  SCORE_TRY(check_dev_ptr(crps_k, "crps_k", false));
  SCORE_TRY(check_dev_ptr(loss, "loss", true));
  const int64_t rows = C * plan->nlat;
  if (rows > 0x7fffffff) return fail(SHT_ERR_INVALID_ARG, "too many rows");
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (prev != plan->device && cudaSetDevice(plan->device) != cudaSuccess)
    return fail(SHT_ERR_CUDA, "cannot select the plan's device");
  cudaStream_t st = (cudaStream_t)stream;
  const float inv_e = 1.0f / (float)E;
  const float inv_d = (float)(fair ? 1.0 / ((double)E * (E - 1)) : 1.0 / ((double)E * E));
  cudaError_t e = launch_bucket<SpatialLaunch>(members_bucket(E), dim3((unsigned)rows), st, ens, obs,
                                               (const float *)plan->d_ring_w, crps_k, E, C, plan->nlat, plan->nlon,
                                               inv_e, inv_d);
  if (e == cudaSuccess && loss) e = launch_row_sum(crps_k, loss, C, plan->nlat, 0, plan->nlat, st);
  if (prev >= 0 && prev != plan->device) cudaSetDevice(prev);
  return e == cudaSuccess ? SHT_OK : cuda_fail(e, "spatial_crps_kernel");
}

}  // extern "C"
