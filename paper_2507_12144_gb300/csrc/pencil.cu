// Partial transforms for the distributed (pencil) SHT of Algorithm 1
// (appendix, "Distributed spherical Harmonic transforms"): a rank there
// holds a block of latitude rows for the longitude steps and a block of
// orders m over all latitudes for the Legendre steps.  These entry points
// run exactly those local steps on one GPU; the exchanges between them are
// the caller's (paper_2507_12144_gb300.pencil).
//
//   sht_analysis_rows     F = w_k (2 pi / nlon) FFT_R2C(x) truncated to mmax,
//                         for latitude rows k0 .. k0 + nrows - 1
//   sht_legendre_orders   forward: xhat_lm = sum_k Phat_l^m(x_k) F_k(m),
//                         inverse: G_k(m) = sum_l Phat_l^m(x_k) yhat_lm,
//                         for orders m0 .. m0 + mcount - 1 over all latitudes
//   sht_synthesis_rows    y = sum_m c_m Re(G_k(m) e^{i m phi})
//
// The Legendre sums reuse the FP32 plan's parity-folded table and its tile
// kernels: the order block is folded into the plan's workspace (E = F_k +
// F_kbar, O = F_k - F_kbar), contracted by the tiles of those orders only,
// and taken out of (or put into) the plan's spectral buffer.
#include <algorithm>

#include "sht_internal.cuh"

namespace shtgb {
namespace {

// Fw[(m0 + j)][p][k'][2b + {re, im}] (classic folded layout, stride ld) from
// F[b][k][j]: p = 0: F_k' + F_kbar', p = 1: F_k' - F_kbar' (equator row: F, 0).
__global__ void fold_orders_kernel(const float2 *__restrict__ F, float *__restrict__ Fw, int nb, int nlat, int Kh,
                                   int m0, int mc, FoldLayout fl) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = (int64_t)nb * Kh * mc;
  if (t >= n) return;
  const int j = (int)(t % mc);
  const int64_t r = t / mc;
  const int kp = (int)(r % Kh);
  const int b = (int)(r / Kh);
  const int ks = nlat - 1 - kp;
  const float2 fn = F[((int64_t)b * nlat + kp) * mc + j];
  const float2 fs = ks != kp ? F[((int64_t)b * nlat + ks) * mc + j] : make_float2(0.f, 0.f);
  const int m = m0 + j;
  const int64_t col = fold_col(fl, 2 * (int64_t)b);
  *reinterpret_cast<float2 *>(Fw + fold_row(fl, m, 0, kp) + col) = make_float2(fn.x + fs.x, fn.y + fs.y);
  *reinterpret_cast<float2 *>(Fw + fold_row(fl, m, 1, kp) + col) = make_float2(fn.x - fs.x, fn.y - fs.y);
}

// G[b][k][j] from the folded inverse output: north row k' = E + O, south
// row nlat - 1 - k' = E - O (equator: E).
__global__ void unfold_orders_kernel(const float *__restrict__ Gw, float2 *__restrict__ G, int nb, int nlat, int Kh,
                                     int m0, int mc, FoldLayout fl) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = (int64_t)nb * Kh * mc;
  if (t >= n) return;
  const int j = (int)(t % mc);
  const int64_t r = t / mc;
  const int kp = (int)(r % Kh);
  const int b = (int)(r / Kh);
  const int ks = nlat - 1 - kp;
  const int m = m0 + j;
  const int64_t col = fold_col(fl, 2 * (int64_t)b);
  const float2 e = *reinterpret_cast<const float2 *>(Gw + fold_row(fl, m, 0, kp) + col);
  const float2 o = *reinterpret_cast<const float2 *>(Gw + fold_row(fl, m, 1, kp) + col);
  if (ks == kp) {
    G[((int64_t)b * nlat + kp) * mc + j] = e;
  } else {
    G[((int64_t)b * nlat + kp) * mc + j] = make_float2(e.x + o.x, e.y + o.y);
    G[((int64_t)b * nlat + ks) * mc + j] = make_float2(e.x - o.x, e.y - o.y);
  }
}

// Columns m0 .. m0 + mc - 1 of spec[b][l][M] to out[b][l][mc] (zero for l < m),
// or (put) from in[b][l][mc] into spec (zero for l < m).
__global__ void order_columns_kernel(const float2 *__restrict__ src, float2 *__restrict__ dst, int nb, int L, int M,
                                     int m0, int mc, int put) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = (int64_t)nb * L * mc;
  if (t >= n) return;
  const int j = (int)(t % mc);
  const int64_t r = t / mc;  // b L + l
  const int l = (int)(r % L);
  const int m = m0 + j;
  const float2 z = make_float2(0.f, 0.f);
  if (put)
    dst[r * M + m] = l >= m ? src[r * mc + j] : z;
  else
    dst[r * mc + j] = l >= m ? src[r * M + m] : z;
}

unsigned blocks_for(int64_t n) { return (unsigned)((n + 255) / 256); }

sht_status_t check_rows(sht_plan_s *p, int64_t B, int k0, int nrows, const void *a, const void *b) {
  if (!p) return fail(SHT_ERR_INVALID_ARG, "plan is NULL");
  if (B < 0) return fail(SHT_ERR_INVALID_ARG, "batch must be >= 0");
  if (k0 < 0 || nrows < 0 || (int64_t)k0 + nrows > p->nlat)
    return fail(SHT_ERR_INVALID_ARG, "latitude rows k0 .. k0 + nrows - 1 must lie in 0 .. nlat - 1");
  if (B == 0 || nrows == 0) return SHT_OK;
  if (!a || !b) return fail(SHT_ERR_INVALID_ARG, "input or output is NULL");
  if ((((uintptr_t)a) | ((uintptr_t)b)) & 15) return fail(SHT_ERR_INVALID_ARG, "input or output not 16-byte aligned");
  if (B * (int64_t)nrows > (int64_t)0x3fffffff * 2) return fail(SHT_ERR_INVALID_ARG, "too many rows");
  return SHT_OK;
}

struct DevSwitch {
  int prev = -1;
  bool changed = false;
  explicit DevSwitch(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DevSwitch() {
    if (changed) cudaSetDevice(prev);
  }
};

}  // namespace
}  // namespace shtgb

using namespace shtgb;

extern "C" sht_status_t sht_analysis_rows(sht_plan_t p, const float *x, void *F, int64_t B, int k0, int nrows,
                                          void *stream) {
  NvtxRange nvtx_range("sht_analysis_rows");
  sht_status_t st = check_rows(p, B, k0, nrows, x, F);
  if (st != SHT_OK || B == 0 || nrows == 0) return st;
  DevSwitch g(p->device);
  cudaError_t e = launch_r2c_rows(x, (float2 *)F, B * nrows, nrows, k0, p->nlon, p->M, p->d_twiddle, p->radix,
                                  p->d_ring_w, (cudaStream_t)stream);
  return e == cudaSuccess ? SHT_OK : cuda_fail(e, "row analysis launch");
}

extern "C" sht_status_t sht_synthesis_rows(sht_plan_t p, const void *G, float *y, int64_t B, int k0, int nrows,
                                           void *stream) {
  NvtxRange nvtx_range("sht_synthesis_rows");
  sht_status_t st = check_rows(p, B, k0, nrows, G, y);
  if (st != SHT_OK || B == 0 || nrows == 0) return st;
  DevSwitch g(p->device);
  cudaError_t e =
      launch_c2r_rows((const float2 *)G, y, B * nrows, p->nlon, p->M, p->d_twiddle, p->radix, (cudaStream_t)stream);
  return e == cudaSuccess ? SHT_OK : cuda_fail(e, "row synthesis launch");
}

extern "C" sht_status_t sht_legendre_orders(sht_plan_t p, int inverse, const void *in, void *out, int64_t B, int m0,
                                            int mcount, void *stream) {
  NvtxRange nvtx_range("sht_legendre_orders");
  if (!p) return fail(SHT_ERR_INVALID_ARG, "plan is NULL");
  if (inverse != 0 && inverse != 1) return fail(SHT_ERR_INVALID_ARG, "inverse must be 0 or 1");
  if (B < 0) return fail(SHT_ERR_INVALID_ARG, "batch must be >= 0");
  if (m0 < 0 || mcount < 0 || (int64_t)m0 + mcount > p->M)
    return fail(SHT_ERR_INVALID_ARG, "orders m0 .. m0 + mcount - 1 must lie in 0 .. mmax - 1");
  if (p->precision != SHT_PREC_FP32)
    return fail(SHT_ERR_UNSUPPORTED, "order-range Legendre sums run on FP32 plans");
  if (B == 0 || mcount == 0) return SHT_OK;
  if (!in || !out) return fail(SHT_ERR_INVALID_ARG, "input or output is NULL");
  if ((((uintptr_t)in) | ((uintptr_t)out)) & 15) return fail(SHT_ERR_INVALID_ARG, "input or output not 16-byte aligned");
  DevSwitch g(p->device);
  cudaStream_t s = (cudaStream_t)stream;
  const TableF32 T{p->d_table, p->d_tab_off, p->Khp};
  const int ft0 = p->fwd_tile_m[m0], ft1 = p->fwd_tile_m[m0 + mcount];
  const int it0 = p->inv_tile_m[m0], it1 = p->inv_tile_m[m0 + mcount];
  const float2 *src = (const float2 *)in;
  float2 *dst = (float2 *)out;
  const int64_t in_stride = (int64_t)(inverse ? p->L : p->nlat) * mcount;
  const int64_t out_stride = (int64_t)(inverse ? p->nlat : p->L) * mcount;
  for (int64_t b0 = 0; b0 < B; b0 += p->max_batch) {
    const int nb = (int)std::min<int64_t>(p->max_batch, B - b0);
    const float2 *ib = src + b0 * in_stride;
    float2 *ob = dst + b0 * out_stride;
    cudaError_t e;
    if (!inverse) {
      const int64_t n = (int64_t)nb * p->Kh * mcount;
      fold_orders_kernel<<<blocks_for(n), 256, 0, s>>>(ib, p->d_work, nb, p->nlat, p->Kh, m0, mcount, p->lay_f);
      e = cudaGetLastError();
      if (e == cudaSuccess && ft1 > ft0)
        e = launch_leg_fwd_f32(T, p->d_fwd_tiles + ft0, ft1 - ft0, p->d_work, p->d_spec_b, p->L, p->M, p->Kh, p->ldc,
                               nb, s);
      if (e == cudaSuccess) {
        const int64_t c = (int64_t)nb * p->L * mcount;
        order_columns_kernel<<<blocks_for(c), 256, 0, s>>>(p->d_spec_b, ob, nb, p->L, p->M, m0, mcount, 0);
        e = cudaGetLastError();
      }
    } else {
      const int64_t c = (int64_t)nb * p->L * mcount;
      order_columns_kernel<<<blocks_for(c), 256, 0, s>>>(ib, p->d_spec_b, nb, p->L, p->M, m0, mcount, 1);
      e = cudaGetLastError();
      if (e == cudaSuccess && it1 > it0)
        e = launch_leg_inv_f32(T, p->d_inv_tiles + it0, it1 - it0, p->d_spec_b, p->d_work, p->L, p->M, p->Kh,
                               p->ldc, nb, s);
      if (e == cudaSuccess) {
        const int64_t n = (int64_t)nb * p->Kh * mcount;
        unfold_orders_kernel<<<blocks_for(n), 256, 0, s>>>(p->d_work, ob, nb, p->nlat, p->Kh, m0, mcount, p->lay_g);
        e = cudaGetLastError();
      }
    }
    if (e != cudaSuccess) return cuda_fail(e, "order-range Legendre launch");
  }
  return SHT_OK;
}
