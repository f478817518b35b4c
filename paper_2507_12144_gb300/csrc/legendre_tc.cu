// Legendre contractions of the SHT on the 5th-generation tensor cores
// (tcgen05), BF16 operands with FP32 accumulation in tensor memory.
//
// The contraction of Algorithm 1 ("Legendre-Gauss quadrature via tensor
// contraction") is, for each order m and parity p of l + m, a GEMM of the
// rows of the folded table by the 2B real columns of the data.  Precision
// forms, with x = x_hi + x_lo, x_hi = bf16(x), x_lo = bf16(x - x_hi):
//   split BF16: table and data split, T_hi D_hi + T_hi D_lo + T_lo D_hi (the
//               lo*lo term is below the FP32 accumulation error);
//   BF16:       data rounded to bf16, table split, T_hi D_hi + T_lo D_hi.
// The table keeps its lo part in both: a bf16-rounded table carries one
// systematic error per (l, m, k) shared by every field (up to the bf16 unit
// roundoff 2^-8), whereas rounding errors of the data are independent and
// average out in the sum over latitudes.  The paper trains in bf16 mixed
// precision (Sec. E.3); the split form recovers FP32-level accuracy.
//
// CTA layout (256 threads):
//   warp 0      TMA producer of the table tiles (A operand)
//   warp 1      MMA issuer (one thread)
//   warp 2      tensor-memory allocation
//   warps 4..7  converters of the data tiles (B operand: FP32 -> bf16 hi/lo
//               written in the K-major 128-byte-swizzled layout) and, after
//               the K loop, the epilogue (tensor memory -> registers ->
//               global), one 32-lane quarter of the accumulator each.
// Stages are guarded by mbarriers; every wait is bounded and records a
// timeout in the plan's error word instead of hanging.
#include <cudaTypedefs.h>

#include <algorithm>

#include "sht_internal.cuh"
#include "tc_common.cuh"

namespace shtgb {
namespace {

using namespace tc;

constexpr int kRows = 128;    // UMMA M
constexpr int kKc = 64;       // K per stage (one 128-byte bf16 row)
constexpr int kThreads = 256;
constexpr int kMaxStages = 6;
constexpr uint32_t kABytes = kRows * 128;  // one A tile (hi or lo)

__host__ __device__ inline int tmem_cols_for(int n) { return n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : 256; }

__device__ __forceinline__ unsigned char *align1024(unsigned char *p) {
  return reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// Stage buffers: A hi, A lo (split only), B hi, B lo; every buffer starts on
// a 1024-byte boundary.  A tiles are 128 rows x 64 k (K-major, 16 KB); B
// tiles are 64 k-rows x nbox column blocks of 64 (MN-major, nbox x 8 KB).
struct Stage {
  unsigned char *a_hi, *a_lo, *b_hi, *b_lo;
};

__host__ __device__ inline uint32_t b_tile_bytes(int nbox) { return (uint32_t)nbox * 8192u; }

__host__ __device__ inline uint32_t stage_bytes(int nbox, bool split) {
  return 2u * kABytes + (split ? 2u : 1u) * b_tile_bytes(nbox);
}

template <bool kSplit>
__device__ __forceinline__ Stage stage_ptr(unsigned char *base, int s, int nbox) {
  unsigned char *p = base + (size_t)s * stage_bytes(nbox, kSplit);
  Stage S;
  S.a_hi = p;
  S.a_lo = p + kABytes;
  S.b_hi = p + 2u * kABytes;
  S.b_lo = kSplit ? S.b_hi + b_tile_bytes(nbox) : S.b_hi;
  return S;
}

// One stage of MMAs: 4 k-steps of 16 rows.
template <bool kSplit>
__device__ __forceinline__ void issue_stage(const Stage &S, uint32_t tmem, uint32_t idesc, bool first) {
#pragma unroll
  for (int ks = 0; ks < kKc / 16; ks++) {
    const uint64_t ah = desc_advance(desc_kmajor_sw128(S.a_hi), ks * 32);
    const uint64_t al = desc_advance(desc_kmajor_sw128(S.a_lo), ks * 32);
    const uint64_t bh = desc_mnmajor_sw128(S.b_hi + ks * 2048, 8192, 1024);
    mma_bf16(tmem, ah, bh, idesc, (first && ks == 0) ? 0u : 1u);
    mma_bf16(tmem, al, bh, idesc, 1u);
    if (kSplit) {
      const uint64_t bl = desc_mnmajor_sw128(S.b_lo + ks * 2048, 8192, 1024);
      mma_bf16(tmem, ah, bl, idesc, 1u);
    }
  }
}

// Shared TMA -> MMA pipeline of both contractions.  A rows start at a_row
// (K chunk kc at column 64 kc), B k-rows start at b_row + 64 kc, B columns at
// c0 + 64 j.  Returns after the MMA thread committed the accumulator (or the
// loop was empty); the epilogue warps then wait on done_bar.
template <bool kSplit>
__device__ __forceinline__ void run_pipeline(const CUtensorMap *ta_hi, const CUtensorMap *ta_lo,
                                             const CUtensorMap *tb_hi, const CUtensorMap *tb_lo, int a_row,
                                             int b_row, int c0, int nk, int nbox, int Nt, int stages,
                                             unsigned char *base, uint64_t *full_bar, uint64_t *empty_bar,
                                             uint64_t *done_bar, uint32_t tmem, unsigned *err) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0 && lane == 0) {
    tma_prefetch_desc(ta_hi);
    tma_prefetch_desc(ta_lo);
    tma_prefetch_desc(tb_hi);
    if (kSplit) tma_prefetch_desc(tb_lo);
    const uint32_t tx = 2u * kABytes + (kSplit ? 2u : 1u) * b_tile_bytes(nbox);
    for (int kc = 0; kc < nk; kc++) {
      const int s = kc % stages, it = kc / stages;
      if (it > 0) mbar_wait(&empty_bar[s], (it - 1) & 1, err);
      const Stage S = stage_ptr<kSplit>(base, s, nbox);
      mbar_arrive_expect_tx(&full_bar[s], tx);
      tma_load_2d(S.a_hi, ta_hi, &full_bar[s], kc * kKc, a_row);
      tma_load_2d(S.a_lo, ta_lo, &full_bar[s], kc * kKc, a_row);
      for (int j = 0; j < nbox; j++) {
        tma_load_2d(S.b_hi + j * 8192, tb_hi, &full_bar[s], c0 + 64 * j, b_row + kc * kKc);
        if (kSplit) tma_load_2d(S.b_lo + j * 8192, tb_lo, &full_bar[s], c0 + 64 * j, b_row + kc * kKc);
      }
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = idesc_bf16_f32(kRows, Nt, true);
    for (int kc = 0; kc < nk; kc++) {
      const int s = kc % stages, it = kc / stages;
      mbar_wait(&full_bar[s], it & 1, err);
      tc_fence_after();
      issue_stage<kSplit>(stage_ptr<kSplit>(base, s, nbox), tmem, idesc, kc == 0);
      mma_commit(&empty_bar[s]);
    }
    if (nk > 0) mma_commit(done_bar);
  }
}

// ---------------------------------------------------------------------------
// Forward: D[i][c] = sum_k' T[m][p][i][k'] F[m][p][k'][c]
// A = table rows i (TMA, K-major), B = Fourier workspace rows k' (TMA,
// MN-major), D in TMEM.  Epilogue: to the API layout xhat[b][l][m]
// (out_rows == nullptr) or to the internal rows out_rows[soff + i][c].
// ---------------------------------------------------------------------------
template <bool kSplit>
__global__ void __launch_bounds__(kThreads, 1)
leg_fwd_tc_kernel(const __grid_constant__ CUtensorMap ta_hi, const __grid_constant__ CUtensorMap ta_lo,
                  const __grid_constant__ CUtensorMap tb_hi, const __grid_constant__ CUtensorMap tb_lo,
                  const int *__restrict__ roff, const int *__restrict__ soff, const LegTile *__restrict__ tiles,
                  float2 *__restrict__ xhat, float *__restrict__ out_rows, int ldo, int L, int M, int Kh, int B,
                  int Nt, int nct, int stages, unsigned *err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = align1024(smem_raw);
  __shared__ uint64_t full_bar[kMaxStages], empty_bar[kMaxStages], done_bar;
  __shared__ uint32_t tmem_slot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const LegTile tile = tiles[blockIdx.x / nct];
  const int m = tile.m, p = tile.p, r0 = tile.r0;
  const int nrows = leg_rows(L, m, p);
  const int c0 = (blockIdx.x % nct) * Nt;
  const int nk = (Kh + kKc - 1) / kKc;
  const int nbox = (Nt + 63) / 64;
  const uint32_t ncols = (uint32_t)tmem_cols_for(Nt);

  if (warp == 2) tmem_alloc(&tmem_slot, ncols);
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; s++) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    mbar_fence_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  run_pipeline<kSplit>(&ta_hi, &ta_lo, &tb_hi, &tb_lo, roff[2 * m + p] + r0, (m * 2 + p) * Kh, c0, nk, nbox, Nt,
                       stages, base, full_bar, empty_bar, &done_bar, tmem, err);
  if (warp >= 4) {
    const int q4 = warp - 4;
    mbar_wait(&done_bar, 0, err);
    tc_fence_after();
    const int r = r0 + q4 * 32 + lane;
    const bool row_ok = r < nrows;
    const int l = m + p + 2 * r;
    float *orow = out_rows ? out_rows + (int64_t)(soff[2 * m + p] + r) * ldo : nullptr;
    for (int j = 0; j < Nt / 16; j++) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(j * 16), v);
      if (!row_ok) continue;
      const int cb = c0 + j * 16;
      if (orow) {
#pragma unroll
        for (int u = 0; u < 4; u++)
          if (cb + 4 * u < 2 * B)
            *reinterpret_cast<float4 *>(orow + cb + 4 * u) =
                make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
      } else {
#pragma unroll
        for (int t = 0; t < 8; t++) {
          const int b = cb / 2 + t;
          if (b < B) xhat[((int64_t)b * L + l) * M + m] = make_float2(v[2 * t], v[2 * t + 1]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

// ---------------------------------------------------------------------------
// Inverse: G[m][p][k'][c] = sum_i T[m][p][i][k'] S[soff + i][c]
// A = transposed table rows k' (TMA, K-major), B = coefficient rows i of the
// internal layout (TMA, MN-major).  Blocks without rows write zeros.
// ---------------------------------------------------------------------------
template <bool kSplit>
__global__ void __launch_bounds__(kThreads, 1)
leg_inv_tc_kernel(const __grid_constant__ CUtensorMap ta_hi, const __grid_constant__ CUtensorMap ta_lo,
                  const __grid_constant__ CUtensorMap tb_hi, const __grid_constant__ CUtensorMap tb_lo,
                  const int *__restrict__ soff, const LegTile *__restrict__ tiles, float *__restrict__ Gw, int L,
                  int Kh, int ldc, int B, int Nt, int nct, int stages, unsigned *err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = align1024(smem_raw);
  __shared__ uint64_t full_bar[kMaxStages], empty_bar[kMaxStages], done_bar;
  __shared__ uint32_t tmem_slot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const LegTile tile = tiles[blockIdx.x / nct];
  const int m = tile.m, p = tile.p, k0 = tile.r0;
  const int nrows = leg_rows(L, m, p);
  const int c0 = (blockIdx.x % nct) * Nt;
  const int nk = (nrows + kKc - 1) / kKc;
  const int nbox = (Nt + 63) / 64;
  const uint32_t ncols = (uint32_t)tmem_cols_for(Nt);

  if (warp == 2) tmem_alloc(&tmem_slot, ncols);
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; s++) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    mbar_fence_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  run_pipeline<kSplit>(&ta_hi, &ta_lo, &tb_hi, &tb_lo, (m * 2 + p) * Kh + k0, soff[2 * m + p], c0, nk, nbox, Nt,
                       stages, base, full_bar, empty_bar, &done_bar, tmem, err);
  if (warp >= 4) {
    const int q4 = warp - 4;
    if (nk > 0) mbar_wait(&done_bar, 0, err);
    tc_fence_after();
    const int k = k0 + q4 * 32 + lane;
    float *G = Gw + (((int64_t)m * 2 + p) * Kh + k) * ldc;
    for (int j = 0; j < Nt / 16; j++) {
      float v[16];
      if (nk > 0) {
        tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(j * 16), v);
      } else {
#pragma unroll
        for (int t = 0; t < 16; t++) v[t] = 0.f;
      }
      if (k < Kh) {
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const int c = c0 + j * 16 + 4 * u;
          if (c < ldc)
            *reinterpret_cast<float4 *>(G + c) = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

// Repack API-layout coefficients yhat[b][l][m] (complex64) into the internal
// split rows S[soff(m, p) + i][2b + {re, im}] (bf16 hi and lo), l = m + p + 2i.
// One thread per (row, field).
__global__ void pack_rows_kernel(const float2 *__restrict__ yhat, __nv_bfloat16 *__restrict__ shi,
                                 __nv_bfloat16 *__restrict__ slo, const int *__restrict__ soff, int L, int M, int ldb,
                                 int B) {
  const int m = blockIdx.y >> 1, p = blockIdx.y & 1;
  const int nrows = leg_rows(L, m, p);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)nrows * B) return;
  const int i = (int)(e / B), b = (int)(e - (int64_t)i * B);
  const float2 v = yhat[((int64_t)b * L + m + p + 2 * i) * M + m];
  __nv_bfloat16 hr, lr, hi_, li;
  split_bf16(v.x, hr, lr);
  split_bf16(v.y, hi_, li);
  const int64_t o = (int64_t)(soff[2 * m + p] + i) * ldb + 2 * b;
  *reinterpret_cast<uint32_t *>(shi + o) = pack_bf16x2(hr, hi_);
  if (slo) *reinterpret_cast<uint32_t *>(slo + o) = pack_bf16x2(lr, li);
}

// FP64 generation of the bf16 hi/lo tables (forward layout [rows][Kp64] and
// transposed layout [(m, p, k')][Ip64]); same recurrence as the FP32 table.
__global__ void table_gen_bf16_kernel(__nv_bfloat16 *__restrict__ fhi, __nv_bfloat16 *__restrict__ flo,
                                      __nv_bfloat16 *__restrict__ ihi, __nv_bfloat16 *__restrict__ ilo,
                                      const int *__restrict__ roff, int Kp64, int Ip64, const double *__restrict__ xk,
                                      const double *__restrict__ sk, const double *__restrict__ a,
                                      const double *__restrict__ bcoef, const double *__restrict__ seed, int L, int M,
                                      int Kh) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (k >= Kh || m >= M) return;
  const double x = xk[k], s = sk[k];
  auto put = [&](int l, double v) {
    const int d = l - m, p = d & 1, i = d >> 1;
    const __nv_bfloat16 h = __double2bfloat16(v);
    const __nv_bfloat16 lo = __double2bfloat16(v - (double)__bfloat162float(h));
    const int64_t fo = (int64_t)(roff[2 * m + p] + i) * Kp64 + k;
    const int64_t io = ((int64_t)(m * 2 + p) * Kh + k) * Ip64 + i;
    fhi[fo] = h;
    ihi[io] = h;
    if (flo) {
      flo[fo] = lo;
      ilo[io] = lo;
    }
  };
  double pmm = 0.28209479177387814347;  // 1 / sqrt(4 pi)
  for (int i = 1; i <= m; i++) pmm *= seed[i] * s;
  if (m >= L) return;
  put(m, pmm);
  if (m + 1 >= L) return;
  double p0 = pmm, p1 = sqrt(2.0 * m + 3.0) * x * pmm;
  put(m + 1, p1);
  for (int l = m + 2; l < L; l++) {
    const int64_t ci = (int64_t)l * M + m;
    const double p2 = a[ci] * (x * p1 - bcoef[ci] * p0);
    put(l, p2);
    p0 = p1;
    p1 = p2;
  }
}

int choose_stages(int nbox, bool split) {
  const int budget = 220 * 1024 - 1024;
  return std::max(2, std::min(kMaxStages, budget / (int)stage_bytes(nbox, split)));
}

size_t smem_bytes(int nbox, bool split, int stages) { return 1024 + (size_t)stages * stage_bytes(nbox, split); }

// Column tiling of the 2B real columns: tiles of at most 256, multiple of 16.
void column_tiles(int B, int &Nt, int &nct) {
  const int C2 = 2 * B;
  nct = (C2 + 255) / 256;
  Nt = ((C2 + nct - 1) / nct + 15) / 16 * 16;
}

}  // namespace

bool tc_encode_2d(CUtensorMap *tm, const void *ptr, int64_t cols, int64_t rows, int box_cols, int box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void **)&enc, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !enc)
      return false;
  }
  if (!ptr) {
    *tm = CUtensorMap{};
    return true;
  }
  cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t gstr[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), gdim, gstr, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_table_gen_bf16(__nv_bfloat16 *fhi, __nv_bfloat16 *flo, __nv_bfloat16 *ihi, __nv_bfloat16 *ilo,
                                  const int *roff, int Kp64, int Ip64, const double *xk, const double *sk,
                                  const double *a, const double *b, const double *seed, int L, int M, int Kh,
                                  cudaStream_t st) {
  dim3 grid((Kh + 127) / 128, M);
  table_gen_bf16_kernel<<<grid, 128, 0, st>>>(fhi, flo, ihi, ilo, roff, Kp64, Ip64, xk, sk, a, b, seed, L, M, Kh);
  return cudaGetLastError();
}

cudaError_t launch_leg_fwd_tc(const TcPlanView &T, const LegTile *tiles, int ntiles, float2 *xhat, float *out_rows,
                              int ldo, int B, cudaStream_t st) {
  if (ntiles == 0 || B <= 0) return cudaSuccess;
  int Nt, nct;
  column_tiles(B, Nt, nct);
  const int nbox = (Nt + 63) / 64;
  const int stages = choose_stages(nbox, T.split);
  const size_t smem = smem_bytes(nbox, T.split, stages);
  const void *fn = T.split ? (const void *)leg_fwd_tc_kernel<true> : (const void *)leg_fwd_tc_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)ntiles * (unsigned)nct;
  if (T.split)
    leg_fwd_tc_kernel<true><<<grid, kThreads, smem, st>>>(T.tab_fwd_hi, T.tab_fwd_lo, T.f_hi, T.f_lo, T.roff, T.soff,
                                                           tiles, xhat, out_rows, ldo, T.L, T.M, T.Kh, B, Nt, nct,
                                                           stages, T.err);
  else
    leg_fwd_tc_kernel<false><<<grid, kThreads, smem, st>>>(T.tab_fwd_hi, T.tab_fwd_lo, T.f_hi, T.f_hi, T.roff,
                                                            T.soff, tiles, xhat, out_rows, ldo, T.L, T.M, T.Kh, B,
                                                            Nt, nct, stages, T.err);
  return cudaGetLastError();
}

cudaError_t launch_leg_inv_tc(const TcPlanView &T, const LegTile *tiles, int ntiles, float *Gw, int ldc, int B,
                              cudaStream_t st) {
  if (ntiles == 0 || B <= 0) return cudaSuccess;
  int Nt, nct;
  column_tiles(B, Nt, nct);
  const int nbox = (Nt + 63) / 64;
  const int stages = choose_stages(nbox, T.split);
  const size_t smem = smem_bytes(nbox, T.split, stages);
  const void *fn = T.split ? (const void *)leg_inv_tc_kernel<true> : (const void *)leg_inv_tc_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)ntiles * (unsigned)nct;
  if (T.split)
    leg_inv_tc_kernel<true><<<grid, kThreads, smem, st>>>(T.tab_inv_hi, T.tab_inv_lo, T.s_hi, T.s_lo, T.soff, tiles,
                                                           Gw, T.L, T.Kh, ldc, B, Nt, nct, stages, T.err);
  else
    leg_inv_tc_kernel<false><<<grid, kThreads, smem, st>>>(T.tab_inv_hi, T.tab_inv_lo, T.s_hi, T.s_hi, T.soff,
                                                            tiles, Gw, T.L, T.Kh, ldc, B, Nt, nct, stages, T.err);
  return cudaGetLastError();
}

cudaError_t launch_pack_rows(const float2 *yhat, __nv_bfloat16 *shi, __nv_bfloat16 *slo, const int *soff, int L,
                             int M, int ldb, int B, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  const int64_t maxrows = (int64_t)leg_rows(L, 0, 0) * B;
  dim3 grid((unsigned)((maxrows + 255) / 256), 2 * M);
  pack_rows_kernel<<<grid, 256, 0, st>>>(yhat, shi, slo, soff, L, M, ldb, B);
  return cudaGetLastError();
}

}  // namespace shtgb
