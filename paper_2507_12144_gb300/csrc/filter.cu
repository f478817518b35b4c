// Spectral filter of the global block: the convolution theorem on the
// sphere (Eq. s2_spectral_conv) multiplies each degree l by one filter
// value; with channel mixing the filter becomes a complex matrix per degree,
//   y[b][o][l][m] = sum_i W[l][o][i] x[b][i][l][m],   m <= l,
// and its adjoints
//   gx[b][i][l][m] = sum_o conj(W[l][o][i]) gy[b][o][l][m]
//   gW[l][o][i]    = sum_{b, m <= l} gy[b][o][l][m] conj(x[b][i][l][m]).
// FP32 complex arithmetic on the CUDA cores.
#include "sht_internal.cuh"

namespace shtgb {
namespace {

constexpr int kTO = 32;   // output channels per CTA
constexpr int kTM = 64;   // orders m per CTA
constexpr int kTK = 16;   // reduction chunk (input channels)
constexpr int kThreads = 256;
constexpr int kFThreads = 128;  // filter: 4 outputs x 4 orders per thread

// c + a b (complex) on packed two-lane FMAs, with a given as its broadcast
// pairs ar = (Re a, Re a), ai = (-Im a, Im a) and b as b, bs = (Im b, Re b).
__device__ __forceinline__ float2 cfma2(float2 ar, float2 ai, float2 b, float2 bs, float2 c) {
  return __ffma2_rn(ai, bs, __ffma2_rn(ar, b, c));
}

// grid: x = l * mtiles + mt, y = output-channel tile, z = member b
template <bool kAdjoint>
__global__ void __launch_bounds__(kFThreads)
filter_kernel(const float2 *__restrict__ x, const float2 *__restrict__ W, float2 *__restrict__ y, int L, int M,
              int Cin, int Cout) {
  __shared__ __align__(16) float2 Ws[kTK][kTO];
  __shared__ __align__(16) float2 Xs[kTK][kTM];
  const int mtiles = (M + kTM - 1) / kTM;
  const int l = blockIdx.x / mtiles;
  const int m0 = (blockIdx.x - l * mtiles) * kTM;
  const int o0 = blockIdx.y * kTO;
  const int64_t b = blockIdx.z;
  // roles: kAdjoint swaps which channel count is the output
  const int Cout_ = kAdjoint ? Cin : Cout;
  const int Cred = kAdjoint ? Cout : Cin;
  const int64_t LM = (int64_t)L * M;
  const float2 *xb = x + b * Cred * LM + (int64_t)l * M;
  float2 *yb = y + b * Cout_ * LM + (int64_t)l * M;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // ty: 4 outputs, tx: 4 orders
  if (m0 > l) {
    // whole tile above the diagonal: zeros
    for (int e = threadIdx.x; e < kTO * kTM; e += kFThreads) {
      const int oo = e / kTM, mm = e - oo * kTM;
      if (o0 + oo < Cout_ && m0 + mm < M) yb[(int64_t)(o0 + oo) * LM + m0 + mm] = make_float2(0.f, 0.f);
    }
    return;
  }
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = make_float2(0.f, 0.f);
  const int mlim = min(M, l + 1);
  for (int k0 = 0; k0 < Cred; k0 += kTK) {
    // W tile: Ws[kk][oo] = Wmat(o0 + oo, k0 + kk)
    for (int e = threadIdx.x; e < kTK * kTO; e += kFThreads) {
      int kk, oo;
      float2 w = make_float2(0.f, 0.f);
      if (!kAdjoint) {
        oo = e / kTK;
        kk = e - oo * kTK;  // consecutive threads read consecutive input channels
        if (o0 + oo < Cout_ && k0 + kk < Cred) w = W[((int64_t)l * Cout + o0 + oo) * Cin + k0 + kk];
      } else {
        kk = e / kTO;
        oo = e - kk * kTO;  // consecutive threads read consecutive "output" (= input channel) index
        if (o0 + oo < Cout_ && k0 + kk < Cred) {
          w = W[((int64_t)l * Cout + k0 + kk) * Cin + o0 + oo];
          w.y = -w.y;
        }
      }
      Ws[kk][oo] = w;
    }
    for (int e = threadIdx.x; e < kTK * kTM; e += kFThreads) {
      const int kk = e / kTM, mm = e - kk * kTM;
      float2 v = make_float2(0.f, 0.f);
      if (k0 + kk < Cred && m0 + mm < mlim) v = xb[(int64_t)(k0 + kk) * LM + m0 + mm];
      Xs[kk][mm] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTK; kk++) {
      float2 wr[4], wi[4], xv[4], xs[4];
#pragma unroll
      for (int i = 0; i < 4; i++) {
        const float2 w = Ws[kk][ty * 4 + i];
        wr[i] = make_float2(w.x, w.x);
        wi[i] = make_float2(-w.y, w.y);
      }
#pragma unroll
      for (int j = 0; j < 4; j++) {
        xv[j] = Xs[kk][tx + 16 * j];
        xs[j] = make_float2(xv[j].y, xv[j].x);
      }
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = cfma2(wr[i], wi[i], xv[j], xs[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int o = o0 + ty * 4 + i;
    if (o >= Cout_) continue;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int m = m0 + tx + 16 * j;
      if (m < M) yb[(int64_t)o * LM + m] = (m <= l) ? acc[i][j] : make_float2(0.f, 0.f);
    }
  }
}

// gW[l][o][i] = sum_{b, m <= l} gy[b][o][l][m] conj(x[b][i][l][m])
// grid: x = l, y = o tile (32), z = i tile (32).  Each thread owns 2 x 2
// outputs; the reduction runs over (b, m) in chunks of 32.
constexpr int kDW = 32;
constexpr int kDK = 32;
__global__ void __launch_bounds__(kThreads)
filter_dw_kernel(const float2 *__restrict__ gy, const float2 *__restrict__ x, float2 *__restrict__ gW, int L, int M,
                 int64_t Bm, int Cin, int Cout, int accumulate) {
  __shared__ float2 Gs[kDW][kDK + 1];
  __shared__ float2 Xs[kDW][kDK + 1];
  const int l = blockIdx.x;
  const int o0 = blockIdx.y * kDW, i0 = blockIdx.z * kDW;
  const int64_t LM = (int64_t)L * M;
  const int mlim = min(M, l + 1);
  const int64_t K = Bm * mlim;
  const int to = threadIdx.x >> 4, ti = threadIdx.x & 15;
  float2 acc[2][2];
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int c = 0; c < 2; c++) acc[a][c] = make_float2(0.f, 0.f);
  for (int64_t k0 = 0; k0 < K; k0 += kDK) {
    for (int e = threadIdx.x; e < kDW * kDK; e += kThreads) {
      const int rr = e / kDK, kk = e - rr * kDK;
      const int64_t kg = k0 + kk;
      float2 g = make_float2(0.f, 0.f), v = make_float2(0.f, 0.f);
      if (kg < K) {
        const int64_t b = kg / mlim;
        const int m = (int)(kg - b * mlim);
        if (o0 + rr < Cout) g = gy[(b * Cout + o0 + rr) * LM + (int64_t)l * M + m];
        if (i0 + rr < Cin) v = x[(b * Cin + i0 + rr) * LM + (int64_t)l * M + m];
      }
      Gs[rr][kk] = g;
      Xs[rr][kk] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kDK; kk++) {
      const float2 g0 = Gs[to * 2 + 0][kk], g1 = Gs[to * 2 + 1][kk];
      const float2 v0 = Xs[ti * 2 + 0][kk], v1 = Xs[ti * 2 + 1][kk];
      // g * conj(v)
      acc[0][0].x += g0.x * v0.x + g0.y * v0.y;
      acc[0][0].y += g0.y * v0.x - g0.x * v0.y;
      acc[0][1].x += g0.x * v1.x + g0.y * v1.y;
      acc[0][1].y += g0.y * v1.x - g0.x * v1.y;
      acc[1][0].x += g1.x * v0.x + g1.y * v0.y;
      acc[1][0].y += g1.y * v0.x - g1.x * v0.y;
      acc[1][1].x += g1.x * v1.x + g1.y * v1.y;
      acc[1][1].y += g1.y * v1.x - g1.x * v1.y;
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int c = 0; c < 2; c++) {
      const int o = o0 + to * 2 + a, i = i0 + ti * 2 + c;
      if (o < Cout && i < Cin) {
        float2 *w = gW + ((int64_t)l * Cout + o) * Cin + i;
        *w = accumulate ? make_float2(w->x + acc[a][c].x, w->y + acc[a][c].y) : acc[a][c];
      }
    }
}

// Wt[l][i][o] = conj(W[l][o][i]) through 32 x 32 shared-memory tiles
// (coalesced reads and writes); grid (Cin / 32, Cout / 32, L).
__global__ void __launch_bounds__(256) transpose_conj_kernel(const float2 *__restrict__ W, float2 *__restrict__ Wt,
                                                             int Cout, int Cin) {
  __shared__ float2 T[32][33];
  const int i0 = blockIdx.x * 32, o0 = blockIdx.y * 32;
  const int64_t base = (int64_t)blockIdx.z * Cout * Cin;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int o = o0 + r, i = i0 + tx;
    if (o < Cout && i < Cin) T[r][tx] = W[base + (int64_t)o * Cin + i];
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r, o = o0 + tx;
    if (o < Cout && i < Cin) {
      const float2 w = T[tx][r];
      Wt[base + (int64_t)i * Cout + o] = make_float2(w.x, -w.y);
    }
  }
}

}  // namespace

cudaError_t launch_transpose_conj(const float2 *W, float2 *Wt, int L, int Cout, int Cin, cudaStream_t st) {
  if (L <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((Cin + 31) / 32), (unsigned)((Cout + 31) / 32), (unsigned)L);
  transpose_conj_kernel<<<grid, 256, 0, st>>>(W, Wt, Cout, Cin);
  return cudaGetLastError();
}

cudaError_t launch_filter(const float2 *x, const float2 *W, float2 *y, int L, int M, int64_t Bm, int Cin, int Cout,
                          int adjoint, cudaStream_t st) {
  if (Bm <= 0) return cudaSuccess;
  const int mtiles = (M + kTM - 1) / kTM;
  const int cout = adjoint ? Cin : Cout;
  dim3 grid(L * mtiles, (cout + kTO - 1) / kTO, (unsigned)Bm);
  if (adjoint)
    filter_kernel<true><<<grid, kFThreads, 0, st>>>(x, W, y, L, M, Cin, Cout);
  else
    filter_kernel<false><<<grid, kFThreads, 0, st>>>(x, W, y, L, M, Cin, Cout);
  return cudaGetLastError();
}

cudaError_t launch_filter_dw(const float2 *gy, const float2 *x, float2 *gW, int L, int M, int64_t Bm, int Cin,
                             int Cout, cudaStream_t st, int accumulate) {
  dim3 grid(L, (Cout + kDW - 1) / kDW, (Cin + kDW - 1) / kDW);
  filter_dw_kernel<<<grid, kThreads, 0, st>>>(gy, x, gW, L, M, Bm, Cin, Cout, accumulate);
  return cudaGetLastError();
}

}  // namespace shtgb
