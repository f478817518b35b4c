// Legendre contractions of the SHT on the CUDA cores in FP32, and the FP64
// generation of the normalised Legendre table.
//
// Forward (Algorithm 1, "Legendre-Gauss quadrature via tensor contraction",
// with the quadrature weight applied in the longitude step):
//   xhat[b][l][m] = sum_k Phat_l^m(x_k) F_k(m)
// Inverse (Eq. isht):
//   G_k(m) = sum_l Phat_l^m(x_k) yhat[b][l][m]
// Both are folded by parity: Phat_l^m(-x) = (-1)^{l+m} Phat_l^m(x) and the
// grids are symmetric about the equator, so for parity p = (l + m) mod 2 only
// the northern half-rows k' < Kh enter, against E = F_k + F_kbar (p = 0) or
// O = F_k - F_kbar (p = 1).  This halves the work of the dominant O(nlat L M)
// term (Sec. B.3).
//
// Each (m, p) block is an independent GEMM of rows i (l = m + p + 2 i) by the
// 2B real columns (re, im of each field); tiles of the ragged triangle are
// enumerated on the host in a tile list.
#include "sht_internal.cuh"

namespace shtgb {
namespace {

constexpr int kTileR = 64;   // rows (l in the forward, k' in the inverse)
constexpr int kTileC = 64;   // real columns (2 per field)
constexpr int kTileK = 16;   // reduction chunk
constexpr int kThreads = 256;

// Forward: C[i][c] = sum_k' T[i][k'] F[k'][c]   (i rows of block (m, p))
// CTA bid of the forward contraction of one problem.
__device__ __forceinline__ void leg_fwd_f32_body(int bid, const TableF32 &T, const LegTile *__restrict__ tiles,
                                                 const float *__restrict__ Fw, float2 *__restrict__ xhat, int L,
                                                 int M, int Kh, int ldc, int B, int nct) {
  __shared__ __align__(16) float As[kTileK][kTileR];
  __shared__ __align__(16) float Bs[kTileK][kTileC];
  // column tiles vary fastest so that the CTAs sharing one table tile run
  // back to back and find it in L2
  const LegTile tile = tiles[bid / nct];
  const int m = tile.m, p = tile.p, r0 = tile.r0;
  const int nrows = leg_rows(L, m, p);
  const int c0 = (bid % nct) * kTileC;
  const float *A = T.data + T.off[2 * m + p];
  const float *Bm = Fw + ((int64_t)m * 2 + p) * Kh * (int64_t)ldc;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = 0.f;

  // loader coordinates
  const int ar = threadIdx.x >> 2, ak = (threadIdx.x & 3) * 4;    // A: 64 rows x 16 k
  const int bk = threadIdx.x >> 4, bc = (threadIdx.x & 15) * 4;   // B: 16 k x 64 c
  for (int k0 = 0; k0 < Kh; k0 += kTileK) {
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r0 + ar < nrows) a = *reinterpret_cast<const float4 *>(A + (int64_t)(r0 + ar) * T.Khp + k0 + ak);
    As[ak + 0][ar] = a.x;
    As[ak + 1][ar] = a.y;
    As[ak + 2][ar] = a.z;
    As[ak + 3][ar] = a.w;
    float4 bv = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k0 + bk < Kh && c0 + bc < ldc) bv = *reinterpret_cast<const float4 *>(Bm + (int64_t)(k0 + bk) * ldc + c0 + bc);
    *reinterpret_cast<float4 *>(&Bs[bk][bc]) = bv;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTileK; kk++) {
      const float4 av = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
      const float4 bw = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
      const float ar4[4] = {av.x, av.y, av.z, av.w};
      const float br4[4] = {bw.x, bw.y, bw.z, bw.w};
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = fmaf(ar4[i], br4[j], acc[i][j]);
    }
    __syncthreads();
  }
  // write: columns (c, c+1) are (re, im) of field c / 2
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int r = r0 + ty * 4 + i;
    if (r >= nrows) continue;
    const int l = m + p + 2 * r;
#pragma unroll
    for (int j = 0; j < 4; j += 2) {
      const int c = c0 + tx * 4 + j;
      const int b = c >> 1;
      if (b < B) xhat[((int64_t)b * L + l) * M + m] = make_float2(acc[i][j], acc[i][j + 1]);
    }
  }
}

// Inverse: C[k'][c] = sum_i T[i][k'] Y[i][c],  Y[i][2b + {0,1}] = yhat[b][l_i][m]
__device__ __forceinline__ void leg_inv_f32_body(int bid, const TableF32 &T, const LegTile *__restrict__ tiles,
                                                 const float2 *__restrict__ yhat, float *__restrict__ Gw, int L,
                                                 int M, int Kh, int ldc, int B, int nct) {
  __shared__ __align__(16) float As[kTileK][kTileR];
  __shared__ __align__(16) float Bs[kTileK][kTileC];
  const LegTile tile = tiles[bid / nct];
  const int m = tile.m, p = tile.p, k0r = tile.r0;  // r0 = first k'
  const int nrows = leg_rows(L, m, p);              // reduction length
  const int c0 = (bid % nct) * kTileC;
  const float *A = T.data + T.off[2 * m + p];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = 0.f;

  const int ai = threadIdx.x >> 4, ak = (threadIdx.x & 15) * 4;   // A: 16 i x 64 k'
  for (int i0 = 0; i0 < nrows; i0 += kTileK) {
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i0 + ai < nrows && k0r + ak < T.Khp)
      a = *reinterpret_cast<const float4 *>(A + (int64_t)(i0 + ai) * T.Khp + k0r + ak);
    *reinterpret_cast<float4 *>(&As[ai][ak]) = a;
    // B: 16 i x 32 fields, two float2 per thread
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int e = threadIdx.x + h * kThreads;  // 0 .. 511
      const int ii = e >> 5, f = e & 31;
      const int b = (c0 >> 1) + f;
      float2 v = make_float2(0.f, 0.f);
      if (i0 + ii < nrows && b < B) {
        const int l = m + p + 2 * (i0 + ii);
        v = yhat[((int64_t)b * L + l) * M + m];
      }
      *reinterpret_cast<float2 *>(&Bs[ii][2 * f]) = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTileK; kk++) {
      const float4 av = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
      const float4 bw = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
      const float ar4[4] = {av.x, av.y, av.z, av.w};
      const float br4[4] = {bw.x, bw.y, bw.z, bw.w};
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = fmaf(ar4[i], br4[j], acc[i][j]);
    }
    __syncthreads();
  }
  float *G = Gw + ((int64_t)m * 2 + p) * Kh * (int64_t)ldc;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int k = k0r + ty * 4 + i;
    if (k >= Kh) continue;
    const int c = c0 + tx * 4;
    if (c < ldc) *reinterpret_cast<float4 *>(G + (int64_t)k * ldc + c) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
  }
}

// One problem of a grouped FP32 launch; CTA j belongs to the problem s with
// blk0[s] <= j < blk0[s + 1].
struct F32Seg {
  TableF32 T;
  const LegTile *tiles;
  const float *Fw;
  float2 *xhat;
  const float2 *yhat;
  float *Gw;
  int L, M, Kh, ldc, B, nct, blk0;
};
struct F32Group {
  F32Seg seg[kMaxLegGroup];
  int nseg;
};

__device__ __forceinline__ int f32_segment(const F32Group &g, int blk) {
  int s = 0;
  while (s + 1 < g.nseg && blk >= g.seg[s + 1].blk0) s++;
  return s;
}

__global__ void __launch_bounds__(kThreads)
leg_fwd_f32_kernel(TableF32 T, const LegTile *__restrict__ tiles, const float *__restrict__ Fw,
                   float2 *__restrict__ xhat, int L, int M, int Kh, int ldc, int B, int nct) {
  leg_fwd_f32_body(blockIdx.x, T, tiles, Fw, xhat, L, M, Kh, ldc, B, nct);
}

__global__ void __launch_bounds__(kThreads)
leg_inv_f32_kernel(TableF32 T, const LegTile *__restrict__ tiles, const float2 *__restrict__ yhat,
                   float *__restrict__ Gw, int L, int M, int Kh, int ldc, int B, int nct) {
  leg_inv_f32_body(blockIdx.x, T, tiles, yhat, Gw, L, M, Kh, ldc, B, nct);
}

__global__ void __launch_bounds__(kThreads) leg_fwd_f32_grouped(const __grid_constant__ F32Group g) {
  const F32Seg &q = g.seg[f32_segment(g, blockIdx.x)];
  leg_fwd_f32_body(blockIdx.x - q.blk0, q.T, q.tiles, q.Fw, q.xhat, q.L, q.M, q.Kh, q.ldc, q.B, q.nct);
}

__global__ void __launch_bounds__(kThreads) leg_inv_f32_grouped(const __grid_constant__ F32Group g) {
  const F32Seg &q = g.seg[f32_segment(g, blockIdx.x)];
  leg_inv_f32_body(blockIdx.x - q.blk0, q.T, q.tiles, q.yhat, q.Gw, q.L, q.M, q.Kh, q.ldc, q.B, q.nct);
}

// Zero fill of the l < m entries of several problems: one warp per (b, l)
// row, rows of problem s from row0[s].
struct ZeroGroup {
  float2 *xhat[kMaxLegGroup];
  int64_t row0[kMaxLegGroup + 1];
  int L[kMaxLegGroup], M[kMaxLegGroup];
  int nseg;
};

__global__ void zero_upper_grouped(const __grid_constant__ ZeroGroup g) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (row >= g.row0[g.nseg]) return;
  int s = 0;
  while (s + 1 < g.nseg && row >= g.row0[s + 1]) s++;
  const int64_t r = row - g.row0[s];
  const int L = g.L[s], M = g.M[s];
  const int l = (int)(r % L);
  float2 *out = g.xhat[s] + r * M;
  for (int m = l + 1 + (threadIdx.x & 31); m < M; m += 32) out[m] = make_float2(0.f, 0.f);
}

__global__ void zero_upper_kernel(float2 *__restrict__ xhat, int L, int M, int64_t rows) {
  // one warp per (b, l) row; zero m in (l, M)
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (row >= rows) return;
  const int l = (int)(row % L);
  float2 *r = xhat + row * M;
  for (int m = l + 1 + (threadIdx.x & 31); m < M; m += 32) r[m] = make_float2(0.f, 0.f);
}

// One thread per (m, k'): FP64 recurrence in l for the normalised functions
//   Phat_m^m = -sqrt((2m+1)/(2m)) s Phat_{m-1}^{m-1},  Phat_0^0 = 1/sqrt(4 pi)
//   Phat_{m+1}^m = sqrt(2m+3) x Phat_m^m
//   Phat_l^m = a_lm (x Phat_{l-1}^m - b_lm Phat_{l-2}^m)
// seed[i] = -sqrt((2i+1)/(2i)) (i >= 1), a/b indexed [l * M + m].
__global__ void table_gen_f32_kernel(float *__restrict__ table, const int64_t *__restrict__ off, int Khp,
                                     const double *__restrict__ xk, const double *__restrict__ sk,
                                     const double *__restrict__ a, const double *__restrict__ bcoef,
                                     const double *__restrict__ seed, int L, int M, int Kh) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (k >= Kh || m >= M) return;
  const double x = xk[k], s = sk[k];
  double pmm = 0.28209479177387814347;  // 1 / sqrt(4 pi)
  for (int i = 1; i <= m; i++) pmm *= seed[i] * s;
  float *t0 = table + off[2 * m + 0];
  float *t1 = table + off[2 * m + 1];
  if (m < L) t0[k] = (float)pmm;
  if (m + 1 >= L) return;
  double p0 = pmm;
  double p1 = sqrt(2.0 * m + 3.0) * x * pmm;
  t1[k] = (float)p1;
  for (int l = m + 2; l < L; l++) {
    const int64_t ci = (int64_t)l * M + m;
    const double p2 = a[ci] * (x * p1 - bcoef[ci] * p0);
    const int d = l - m;
    float *t = (d & 1) ? t1 : t0;
    t[(int64_t)(d >> 1) * Khp + k] = (float)p2;
    p0 = p1;
    p1 = p2;
  }
}

}  // namespace

cudaError_t launch_leg_fwd_f32(const TableF32 &T, const LegTile *tiles, int ntiles, const float *Fw, float2 *xhat,
                               int L, int M, int Kh, int ldc, int B, cudaStream_t st) {
  if (ntiles == 0 || B <= 0) return cudaSuccess;
  const int nct = (2 * B + kTileC - 1) / kTileC;
  leg_fwd_f32_kernel<<<(unsigned)ntiles * nct, kThreads, 0, st>>>(T, tiles, Fw, xhat, L, M, Kh, ldc, B, nct);
  return cudaGetLastError();
}

cudaError_t launch_leg_inv_f32(const TableF32 &T, const LegTile *tiles, int ntiles, const float2 *yhat, float *Gw,
                               int L, int M, int Kh, int ldc, int B, cudaStream_t st) {
  if (ntiles == 0 || B <= 0) return cudaSuccess;
  const int nct = (2 * B + kTileC - 1) / kTileC;
  leg_inv_f32_kernel<<<(unsigned)ntiles * nct, kThreads, 0, st>>>(T, tiles, yhat, Gw, L, M, Kh, ldc, B, nct);
  return cudaGetLastError();
}

cudaError_t launch_leg_f32_group(int inverse, const F32LegItem *items, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (n > kMaxLegGroup) return cudaErrorInvalidValue;
  F32Group g{};
  int64_t blk = 0;
  for (int i = 0; i < n; i++) {
    const F32LegItem &it = items[i];
    if (it.ntiles <= 0 || it.B <= 0) continue;
    F32Seg &q = g.seg[g.nseg++];
    q.T = it.T;
    q.tiles = it.tiles;
    q.Fw = it.Fw;
    q.xhat = it.xhat;
    q.yhat = it.yhat;
    q.Gw = it.Gw;
    q.L = it.L;
    q.M = it.M;
    q.Kh = it.Kh;
    q.ldc = it.ldc;
    q.B = it.B;
    q.nct = (2 * it.B + kTileC - 1) / kTileC;
    q.blk0 = (int)blk;
    blk += (int64_t)it.ntiles * q.nct;
  }
  if (g.nseg == 0) return cudaSuccess;
  if (blk > 0x7fffffff) return cudaErrorInvalidValue;
  if (inverse)
    leg_inv_f32_grouped<<<(unsigned)blk, kThreads, 0, st>>>(g);
  else
    leg_fwd_f32_grouped<<<(unsigned)blk, kThreads, 0, st>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_zero_upper_group(float2 *const *xhat, const int *L, const int *M, const int64_t *B, int n,
                                    cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (n > kMaxLegGroup) return cudaErrorInvalidValue;
  ZeroGroup g{};
  int64_t rows = 0;
  for (int i = 0; i < n; i++) {
    if (B[i] <= 0 || M[i] <= 1) continue;
    const int s = g.nseg++;
    g.xhat[s] = xhat[i];
    g.L[s] = L[i];
    g.M[s] = M[i];
    g.row0[s] = rows;
    rows += B[i] * L[i];
  }
  g.row0[g.nseg] = rows;
  if (rows == 0) return cudaSuccess;
  const int wpb = 8;
  zero_upper_grouped<<<(unsigned)((rows + wpb - 1) / wpb), wpb * 32, 0, st>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_zero_upper(float2 *xhat, int L, int M, int64_t B, cudaStream_t st) {
  const int64_t rows = B * L;
  if (rows == 0 || M <= 1) return cudaSuccess;
  const int wpb = 8;
  zero_upper_kernel<<<(unsigned)((rows + wpb - 1) / wpb), wpb * 32, 0, st>>>(xhat, L, M, rows);
  return cudaGetLastError();
}

cudaError_t launch_table_gen_f32(float *table, const int64_t *off, int Khp, const double *xk, const double *sk,
                                 const double *a, const double *b, const double *seed, int L, int M, int Kh,
                                 cudaStream_t st) {
  dim3 grid((Kh + 127) / 128, M);
  table_gen_f32_kernel<<<grid, 128, 0, st>>>(table, off, Khp, xk, sk, a, b, seed, L, M, Kh);
  return cudaGetLastError();
}

}  // namespace shtgb
