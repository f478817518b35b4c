// Spherical diffusion process, Eq. (spherical_diffusion) (Sec. B.7): one
// AR(1) step per spherical harmonic coefficient of B noise fields,
//   z[b][l][m] = phi z[b][l][m] + sigma_l(b) xi[b][l][m],
//   phi = exp(-lambda), sigma_l = F0 exp(-(kT / 2) l (l + 1)),
//   F0 = sigma sqrt(2 pi (1 - phi^2) / sum_{l = 1}^{lmax - 1} (2 l + 1) exp(-kT l (l + 1))),
// for 1 <= l < lmax, m <= min(l, mmax - 1) (zero at l = 0: the process has
// no l = 0 term), with xi = eta for m > 0 and xi = sqrt(2) Re(eta) at m = 0,
// so that every degree adds sigma_l^2 (2 l + 1) / (2 pi) to the variance of
// the real field at every point and the stationary variance is sigma^2.
//
// The standard normals eta are given, or drawn here from Philox4x32-10
// (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2,
// 3", SC 2011) under key = the 64-bit seed: one generator call at counter
// (idx >> 1, step) serves the two coefficients of flat indices idx (even
// and odd), which take its words (wa, wb) = (w0, w1) and (w2, w3) through
// the Box-Muller transform
//   u1 = ((wa >> 8) + 1) 2^-24, u2 = (wb >> 8) 2^-24,
//   eta = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2).
// For even mmax a thread updates the two orders 2j, 2j + 1 of one degree
// (one generator call, one sigma_l, one 16-byte access), threads numbered
// over the pairs of the l >= m triangle row by row; for odd mmax one
// thread per coefficient (the pairs then straddle rows).  No block or lane
// falls above the diagonal, the state is read and written once, and
// entries with m > l are neither read nor written.
#include <cmath>

#include "sht_internal.cuh"

namespace shtgb {
namespace {

constexpr int kMaxScales = 16;

struct DiffusionParams {
  float phi;
  int nk;
  unsigned kbase;  // (first field of the launch) mod nk
  float F0[kMaxScales];
  float half_kT[kMaxScales];
};

// Philox4x32 with 10 rounds: multipliers 0xD2511F53, 0xCD9E8D57, key
// increments 0x9E3779B9, 0xBB67AE85 (the published constants).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

constexpr int kDiffThreads = 128;

__device__ __forceinline__ float2 box_muller(uint32_t wa, uint32_t wb) {
  const float u1 = (float)((wa >> 8) + 1u) * 0x1p-24f;
  const float u2 = (float)(wb >> 8) * 0x1p-24f;
  const float rad = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  return make_float2(rad * c, rad * s);
}

// the generator's words for the coefficient pair of flat index idx
__device__ __forceinline__ uint4 philox_pair(int64_t idx, uint2 step, uint2 key) {
  const uint64_t c = (uint64_t)idx >> 1;
  return philox4x32_10(make_uint4((uint32_t)c, (uint32_t)(c >> 32), step.x, step.y), key);
}

// (l, m) of triangle index t (row by row, rows l < M holding l + 1 orders,
// the rest M): l from the square root, corrected in integers.
__device__ __forceinline__ void tri_lm(int t, int M, int &l, int &m) {
  const int T0 = M * (M + 1) / 2;  // the rows l < M
  if (t >= T0) {
    const int r = (t - T0) / M;
    l = M + r;
    m = t - T0 - r * M;
    return;
  }
  int q = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while (q * (q + 1) / 2 > t) q--;
  while ((q + 1) * (q + 2) / 2 <= t) q++;
  l = q;
  m = t - q * (q + 1) / 2;
}

// (l, j) of pair index t for even M (pair j of degree l: orders 2j, 2j + 1):
// rows 2q and 2q + 1 hold q + 1 pairs each (q (q + 1) pairs before row 2q),
// rows l >= M hold M / 2.
__device__ __forceinline__ void tri_pair(int t, int M, int &l, int &j) {
  const int Q = M / 2;
  const int T0 = Q * (Q + 1);  // the rows l < M
  if (t >= T0) {
    const int r = (t - T0) / Q;
    l = M + r;
    j = t - T0 - r * Q;
    return;
  }
  int q = (int)((sqrtf(4.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while (q > 0 && q * (q + 1) > t) q--;
  while ((q + 1) * (q + 2) <= t) q++;
  const int r = t - q * (q + 1);
  if (r <= q) {
    l = 2 * q;
    j = r;
  } else {
    l = 2 * q + 1;
    j = r - q - 1;
  }
}

__device__ __forceinline__ float diffusion_sigma(const DiffusionParams &P, int64_t b, int l) {
  const int k = (int)((P.kbase + (unsigned)b) % (unsigned)P.nk);
  return P.F0[k] * expf(-P.half_kT[k] * (float)l * (float)(l + 1));
}

// even M, grid (pairs / 128, fields)
__global__ void __launch_bounds__(kDiffThreads) diffusion_pair_kernel(float2 *__restrict__ z,
                                                                      const float2 *__restrict__ eta, int64_t b0,
                                                                      int L, int M, int npair, DiffusionParams P,
                                                                      uint2 key, uint2 step) {
  const int t = blockIdx.x * kDiffThreads + threadIdx.x;
  if (t >= npair) return;
  int l, j;
  tri_pair(t, M, l, j);
  const int64_t b = b0 + blockIdx.y;
  const int m0 = 2 * j;
  const int64_t idx = (b * L + l) * M + m0;  // even: the pair's first coefficient
  if (l == 0) {
    z[idx] = make_float2(0.f, 0.f);  // the only coefficient of degree 0
    return;
  }
  const bool two = m0 + 1 <= min(l, M - 1);
  float2 e0, e1 = make_float2(0.f, 0.f);
  if (eta) {
    if (two) {
      const float4 q = __ldg(reinterpret_cast<const float4 *>(eta + idx));
      e0 = make_float2(q.x, q.y);
      e1 = make_float2(q.z, q.w);
    } else {
      e0 = __ldg(eta + idx);
    }
  } else {
    const uint4 w = philox_pair(idx, step, key);
    e0 = box_muller(w.x, w.y);
    if (two) e1 = box_muller(w.z, w.w);
  }
  const float sig = diffusion_sigma(P, blockIdx.y, l);
  const float2 xi0 = m0 == 0 ? make_float2(1.41421356237309515f * e0.x, 0.f) : e0;
  if (two) {
    float4 *zp = reinterpret_cast<float4 *>(z + idx);
    const float4 v = *zp;
    *zp = make_float4(fmaf(P.phi, v.x, sig * xi0.x), fmaf(P.phi, v.y, sig * xi0.y), fmaf(P.phi, v.z, sig * e1.x),
                      fmaf(P.phi, v.w, sig * e1.y));
  } else {
    const float2 v = z[idx];
    z[idx] = make_float2(fmaf(P.phi, v.x, sig * xi0.x), fmaf(P.phi, v.y, sig * xi0.y));
  }
}

// odd M, grid (triangle / 128, fields): one thread per coefficient
__global__ void __launch_bounds__(kDiffThreads) diffusion_step_kernel(float2 *__restrict__ z,
                                                                      const float2 *__restrict__ eta, int64_t b0,
                                                                      int L, int M, int ntri, DiffusionParams P,
                                                                      uint2 key, uint2 step) {
  const int t = blockIdx.x * kDiffThreads + threadIdx.x;
  if (t >= ntri) return;
  int l, m;
  tri_lm(t, M, l, m);
  const int64_t b = b0 + blockIdx.y;
  const int64_t idx = (b * L + l) * M + m;
  if (l == 0) {
    z[idx] = make_float2(0.f, 0.f);
    return;
  }
  float2 e;
  if (eta) {
    e = __ldg(eta + idx);
  } else {
    const uint4 w = philox_pair(idx, step, key);
    e = (idx & 1) ? box_muller(w.z, w.w) : box_muller(w.x, w.y);
  }
  const float sig = diffusion_sigma(P, blockIdx.y, l);
  const float2 xi = m == 0 ? make_float2(1.41421356237309515f * e.x, 0.f) : e;
  const float2 v = z[idx];
  z[idx] = make_float2(fmaf(P.phi, v.x, sig * xi.x), fmaf(P.phi, v.y, sig * xi.y));
}

}  // namespace
}  // namespace shtgb

using namespace shtgb;

extern "C" {

sht_status_t sht_diffusion_step(void *zhat, const void *eta, int64_t B, int lmax, int mmax, const double *kT, int nk,
                                double lambda, double sigma, uint64_t seed, uint64_t step, void *stream) {
  NvtxRange nvtx_range("sht_diffusion_step");
  if (B < 0) return fail(SHT_ERR_INVALID_ARG, "batch must be >= 0");
  if (lmax < 2 || mmax < 1 || mmax > lmax) return fail(SHT_ERR_INVALID_ARG, "need lmax >= 2 and 1 <= mmax <= lmax");
  if (!kT || nk < 1 || nk > kMaxScales) return fail(SHT_ERR_INVALID_ARG, "need 1 .. 16 length scales kT");
  if (!(lambda > 0.0) || !(sigma >= 0.0)) return fail(SHT_ERR_INVALID_ARG, "need lambda > 0 and sigma >= 0");
  for (int i = 0; i < nk; i++)
    if (!(kT[i] >= 0.0)) return fail(SHT_ERR_INVALID_ARG, "length scales kT must be >= 0");
  if (B == 0) return SHT_OK;
  if (!zhat) return fail(SHT_ERR_INVALID_ARG, "zhat is NULL");
  if ((((uintptr_t)zhat) | ((uintptr_t)eta)) & 15)
    return fail(SHT_ERR_INVALID_ARG, "zhat and eta must be 16-byte aligned");
  DiffusionParams P{};
  const double phi = std::exp(-lambda);
  P.phi = (float)phi;
  P.nk = nk;
  for (int i = 0; i < nk; i++) {
    double norm = 0.0;
    for (int l = 1; l < lmax; l++) norm += (2.0 * l + 1.0) * std::exp(-kT[i] * l * (l + 1.0));
    P.F0[i] = (float)(sigma * std::sqrt(2.0 * M_PI * (1.0 - phi * phi) / norm));
    P.half_kT[i] = (float)(0.5 * kT[i]);
  }
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  const uint2 st2 = make_uint2((uint32_t)step, (uint32_t)(step >> 32));
  const int ntri = mmax * (mmax + 1) / 2 + (lmax - mmax) * mmax;  // coefficients with m <= l
  const int npair = (mmax / 2) * (mmax / 2 + 1) + (lmax - mmax) * (mmax / 2);  // their pairs (even mmax)
  const bool pairs = mmax % 2 == 0;
  const int nthr = pairs ? npair : ntri;
  for (int64_t b0 = 0; b0 < B; b0 += 65535) {
    P.kbase = (unsigned)(b0 % nk);
    const dim3 grid((unsigned)((nthr + kDiffThreads - 1) / kDiffThreads), (unsigned)std::min<int64_t>(65535, B - b0));
    if (pairs)
      diffusion_pair_kernel<<<grid, kDiffThreads, 0, (cudaStream_t)stream>>>((float2 *)zhat, (const float2 *)eta, b0,
                                                                             lmax, mmax, npair, P, key, st2);
    else
      diffusion_step_kernel<<<grid, kDiffThreads, 0, (cudaStream_t)stream>>>((float2 *)zhat, (const float2 *)eta, b0,
                                                                             lmax, mmax, ntri, P, key, st2);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SHT_OK : cuda_fail(e, "diffusion_step_kernel");
}

}  // extern "C"
