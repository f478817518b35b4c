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
// 3", SC 2011): key = the 64-bit seed, counter = (coefficient index, step),
// and the Box-Muller transform of the first two output words,
//   u1 = ((w0 >> 8) + 1) 2^-24, u2 = (w1 >> 8) 2^-24,
//   eta = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2).
// One thread per coefficient of the l >= m triangle, numbered row by row
// (t = l (l + 1) / 2 + m for l < mmax, then mmax per row), so that no
// block or lane falls above the diagonal: the step reads and writes the
// state once; the generator adds about 130 instructions per coefficient.
// Entries with m > l are neither read nor written.
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

// grid (triangle / 128, fields)
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
    const uint4 w = philox4x32_10(make_uint4((uint32_t)idx, (uint32_t)((uint64_t)idx >> 32), step.x, step.y), key);
    const float u1 = (float)((w.x >> 8) + 1u) * 0x1p-24f;
    const float u2 = (float)(w.y >> 8) * 0x1p-24f;
    const float rad = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    e = make_float2(rad * c, rad * s);
  }
  const int k = (int)((P.kbase + blockIdx.y) % (unsigned)P.nk);
  const float sig = P.F0[k] * expf(-P.half_kT[k] * (float)l * (float)(l + 1));
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
  for (int64_t b0 = 0; b0 < B; b0 += 65535) {
    P.kbase = (unsigned)(b0 % nk);
    const dim3 grid((unsigned)((ntri + kDiffThreads - 1) / kDiffThreads), (unsigned)std::min<int64_t>(65535, B - b0));
    diffusion_step_kernel<<<grid, kDiffThreads, 0, (cudaStream_t)stream>>>((float2 *)zhat, (const float2 *)eta, b0,
                                                                           lmax, mmax, ntri, P, key, st2);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SHT_OK : cuda_fail(e, "diffusion_step_kernel");
}

}  // extern "C"
