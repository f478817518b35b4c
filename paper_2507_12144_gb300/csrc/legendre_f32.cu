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
// Legendre GEMMs: 64 threads per 64 x 64 tile, 8 x 8 outputs per thread
// (thread (ty, tx) owns rows 8 ty .. 8 ty + 7 and columns 8 tx .. 8 tx + 7),
// so that each K step reads 16 values from shared memory for 64 FMAs; the
// products run as packed two-lane FMAs along the columns; shared memory is
// double-buffered with the next K chunk loaded into registers meanwhile.
constexpr int kLegThreads = 64;
constexpr int kApad = kTileR + 4;  // A rows padded against bank conflicts of the transposed stores

__device__ __forceinline__ void mma8x8(float2 (&acc)[8][4], const float *a8, const float *b8) {
  const float4 a0 = *reinterpret_cast<const float4 *>(a8), a1 = *reinterpret_cast<const float4 *>(a8 + 4);
  const float4 b0 = *reinterpret_cast<const float4 *>(b8), b1 = *reinterpret_cast<const float4 *>(b8 + 4);
  const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
  const float2 bv[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w), make_float2(b1.x, b1.y),
                        make_float2(b1.z, b1.w)};
#pragma unroll
  for (int i = 0; i < 8; i++) {
    const float2 ai = make_float2(av[i], av[i]);
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = __ffma2_rn(ai, bv[j], acc[i][j]);
  }
}

// Forward: C[i][c] = sum_k' T[i][k'] F[k'][c]   (i rows of block (m, p))
// CTA bid of the forward contraction of one problem.
__device__ __forceinline__ void leg_fwd_f32_body(int bid, const TableF32 &T, const LegTile *__restrict__ tiles,
                                                 const float *__restrict__ Fw, float2 *__restrict__ xhat, int L,
                                                 int M, int Kh, int ldc, int B, int nct) {
  __shared__ __align__(16) float As[2][kTileK][kApad];
  __shared__ __align__(16) float Bs[2][kTileK][kTileC];
  // column tiles vary fastest so that the CTAs sharing one table tile run
  // back to back and find it in L2
  const LegTile tile = tiles[bid / nct];
  const int m = tile.m, p = tile.p, r0 = tile.r0;
  const int nrows = leg_rows(L, m, p);
  const int c0 = (bid % nct) * kTileC;
  const float *A = T.data + T.off[2 * m + p];
  const float *Bm = Fw + ((int64_t)m * 2 + p) * Kh * (int64_t)ldc;
  const int t = threadIdx.x, tx = t & 7, ty = t >> 3;
  float2 acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = make_float2(0.f, 0.f);

  // loaders: A rows (t >> 2) + 16 q, k (t & 3) 4 .. + 3; B k (t >> 4) + 4 q,
  // columns (t & 15) 4 .. + 3
  const int ar = t >> 2, ak = (t & 3) * 4, bk = t >> 4, bc = (t & 15) * 4;
  float4 an[4], bn[4];
  auto gload = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int r = ar + 16 * q, k = bk + 4 * q;
      an[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r0 + r < nrows) an[q] = *reinterpret_cast<const float4 *>(A + (int64_t)(r0 + r) * T.Khp + k0 + ak);
      bn[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k0 + k < Kh && c0 + bc < ldc) bn[q] = *reinterpret_cast<const float4 *>(Bm + (int64_t)(k0 + k) * ldc + c0 + bc);
    }
  };
  auto sstore = [&](int u) {
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int r = ar + 16 * q;
      As[u][ak + 0][r] = an[q].x;
      As[u][ak + 1][r] = an[q].y;
      As[u][ak + 2][r] = an[q].z;
      As[u][ak + 3][r] = an[q].w;
      *reinterpret_cast<float4 *>(&Bs[u][bk + 4 * q][bc]) = bn[q];
    }
  };
  gload(0);
  sstore(0);
  __syncthreads();
  int u = 0;
  for (int k0 = 0; k0 < Kh; k0 += kTileK) {
    const bool more = k0 + kTileK < Kh;
    if (more) gload(k0 + kTileK);
#pragma unroll
    for (int kk = 0; kk < kTileK; kk++) mma8x8(acc, &As[u][kk][ty * 8], &Bs[u][kk][tx * 8]);
    if (more) sstore(u ^ 1);
    __syncthreads();
    u ^= 1;
  }
  // write: columns (c, c+1) are (re, im) of field c / 2
#pragma unroll
  for (int i = 0; i < 8; i++) {
    const int r = r0 + ty * 8 + i;
    if (r >= nrows) continue;
    const int l = m + p + 2 * r;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int b = (c0 + tx * 8 + 2 * j) >> 1;
      if (b < B) xhat[((int64_t)b * L + l) * M + m] = acc[i][j];
    }
  }
}

// Inverse: C[k'][c] = sum_i T[i][k'] Y[i][c],  Y[i][2b + {0,1}] = yhat[b][l_i][m]
__device__ __forceinline__ void leg_inv_f32_body(int bid, const TableF32 &T, const LegTile *__restrict__ tiles,
                                                 const float2 *__restrict__ yhat, float *__restrict__ Gw, int L,
                                                 int M, int Kh, int ldc, int B, int nct) {
  __shared__ __align__(16) float As[2][kTileK][kApad];
  __shared__ __align__(16) float Bs[2][kTileK][kTileC];
  const LegTile tile = tiles[bid / nct];
  const int m = tile.m, p = tile.p, k0r = tile.r0;  // r0 = first k'
  const int nrows = leg_rows(L, m, p);              // reduction length
  const int c0 = (bid % nct) * kTileC;
  const float *A = T.data + T.off[2 * m + p];
  const int t = threadIdx.x, tx = t & 7, ty = t >> 3;
  float2 acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = make_float2(0.f, 0.f);

  // loaders: A rows i (t >> 4) + 4 q, k' (t & 15) 4 .. + 3; B: 16 i x 32
  // fields, element e = t + 64 q: row e >> 5, field e & 31
  const int ai = t >> 4, ak = (t & 15) * 4;
  float4 an[4];
  float2 bn[8];
  auto gload = [&](int i0) {
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int i = ai + 4 * q;
      an[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i0 + i < nrows && k0r + ak < T.Khp)
        an[q] = *reinterpret_cast<const float4 *>(A + (int64_t)(i0 + i) * T.Khp + k0r + ak);
    }
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const int e = t + kLegThreads * q;  // 0 .. 511
      const int ii = e >> 5, f = e & 31;
      const int b = (c0 >> 1) + f;
      bn[q] = make_float2(0.f, 0.f);
      if (i0 + ii < nrows && b < B) {
        const int l = m + p + 2 * (i0 + ii);
        bn[q] = yhat[((int64_t)b * L + l) * M + m];
      }
    }
  };
  auto sstore = [&](int u) {
#pragma unroll
    for (int q = 0; q < 4; q++) *reinterpret_cast<float4 *>(&As[u][ai + 4 * q][ak]) = an[q];
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const int e = t + kLegThreads * q;
      *reinterpret_cast<float2 *>(&Bs[u][e >> 5][2 * (e & 31)]) = bn[q];
    }
  };
  gload(0);
  sstore(0);
  __syncthreads();
  int u = 0;
  for (int i0 = 0; i0 < nrows; i0 += kTileK) {
    const bool more = i0 + kTileK < nrows;
    if (more) gload(i0 + kTileK);
#pragma unroll
    for (int kk = 0; kk < kTileK; kk++) mma8x8(acc, &As[u][kk][ty * 8], &Bs[u][kk][tx * 8]);
    if (more) sstore(u ^ 1);
    __syncthreads();
    u ^= 1;
  }
  float *G = Gw + ((int64_t)m * 2 + p) * Kh * (int64_t)ldc;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    const int k = k0r + ty * 8 + i;
    if (k >= Kh) continue;
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int c = c0 + tx * 8 + 4 * h;
      if (c < ldc)
        *reinterpret_cast<float4 *>(G + (int64_t)k * ldc + c) =
            make_float4(acc[i][2 * h].x, acc[i][2 * h].y, acc[i][2 * h + 1].x, acc[i][2 * h + 1].y);
    }
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

__global__ void __launch_bounds__(kLegThreads)
leg_fwd_f32_kernel(TableF32 T, const LegTile *__restrict__ tiles, const float *__restrict__ Fw,
                   float2 *__restrict__ xhat, int L, int M, int Kh, int ldc, int B, int nct) {
  leg_fwd_f32_body(blockIdx.x, T, tiles, Fw, xhat, L, M, Kh, ldc, B, nct);
}

__global__ void __launch_bounds__(kLegThreads)
leg_inv_f32_kernel(TableF32 T, const LegTile *__restrict__ tiles, const float2 *__restrict__ yhat,
                   float *__restrict__ Gw, int L, int M, int Kh, int ldc, int B, int nct) {
  leg_inv_f32_body(blockIdx.x, T, tiles, yhat, Gw, L, M, Kh, ldc, B, nct);
}

__global__ void __launch_bounds__(kLegThreads) leg_fwd_f32_grouped(const __grid_constant__ F32Group g) {
  const F32Seg &q = g.seg[f32_segment(g, blockIdx.x)];
  leg_fwd_f32_body(blockIdx.x - q.blk0, q.T, q.tiles, q.Fw, q.xhat, q.L, q.M, q.Kh, q.ldc, q.B, q.nct);
}

__global__ void __launch_bounds__(kLegThreads) leg_inv_f32_grouped(const __grid_constant__ F32Group g) {
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
  leg_fwd_f32_kernel<<<(unsigned)ntiles * nct, kLegThreads, 0, st>>>(T, tiles, Fw, xhat, L, M, Kh, ldc, B, nct);
  return cudaGetLastError();
}

cudaError_t launch_leg_inv_f32(const TableF32 &T, const LegTile *tiles, int ntiles, const float2 *yhat, float *Gw,
                               int L, int M, int Kh, int ldc, int B, cudaStream_t st) {
  if (ntiles == 0 || B <= 0) return cudaSuccess;
  const int nct = (2 * B + kTileC - 1) / kTileC;
  leg_inv_f32_kernel<<<(unsigned)ntiles * nct, kLegThreads, 0, st>>>(T, tiles, yhat, Gw, L, M, Kh, ldc, B, nct);
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
    leg_inv_f32_grouped<<<(unsigned)blk, kLegThreads, 0, st>>>(g);
  else
    leg_fwd_f32_grouped<<<(unsigned)blk, kLegThreads, 0, st>>>(g);
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
