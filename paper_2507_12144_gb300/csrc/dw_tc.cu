// Weight gradient of the spectral filter on the tensor cores:
//   gW[l][o][i] = sum_{b, m <= l} g[b][o][l][m] conj(x[b][i][l][m]),
// g = ISHT^T(gy) and x = SHT(x) (the adjoint of the per-degree channel
// mixing of Eq. s2_spectral_conv with respect to W).  Both operands are
// the split bf16 l-major rows that the tensor-core forward writes, row
// (l, m) of member b holding channel c's real and imaginary part in
// columns b kx + 2 c and b kx + 2 c + 1.  Per degree l this is one real GEMM
//   D[o'][i'] = sum_{k = (b, m)} G[k][o'] X[k][i'],   o' = 2 o + s, i' = 2 i + t,
// whose 2 x 2 blocks give the complex result:
//   Re gW = D[2o][2i] + D[2o+1][2i+1],  Im gW = D[2o+1][2i] - D[2o][2i+1].
// Tiles of 128 rows o' by up to 256 columns i' per degree; K in stages of
// 32 rows m of one member (rows m > l of a degree are zero in the rows
// buffers), both operands MN-major (64-column boxes of 32 rows, 128-byte
// swizzle).  Split: G_hi X_hi + G_hi X_lo + G_lo X_hi.  Warp roles: TMA
// producer (warp 0), MMA issuer (warp 1, which also owns the 512 tensor-
// memory columns: two accumulators), epilogue (warps 2-5).
#include <algorithm>

#include "sht_internal.cuh"
#include "tc_common.cuh"

namespace shtgb {
namespace {

using namespace tc;

constexpr int kKr = 32;           // K rows (orders m of one member) per stage
constexpr int kBoxBytes = 64 * kKr * 2;
constexpr int kStages = 4;
constexpr int kTileM = 128;       // rows o' per tile
constexpr int kTileN = 256;       // columns i' per tile (at most)
constexpr int kAccCols = 256;
constexpr int kThreadsDw = 192;

struct DwParams {
  CUtensorMap a_hi, a_lo, b_hi, b_lo;
  float2 *gW;
  unsigned *err;
  int L, M, nb, Cin, Cout, kxa, kxb;
  int n_ot, n_it, ntiles;
  int accumulate;
};

struct DwTile {
  int l, ot, it, Nt, nk, nkm;
};

__device__ __forceinline__ DwTile dw_tile(const DwParams &P, int t) {
  DwTile d;
  const int per_l = P.n_ot * P.n_it;
  d.l = P.L - 1 - t / per_l;  // the longest K first
  const int r = t - (P.L - 1 - d.l) * per_l;
  d.ot = r / P.n_it;
  d.it = r - d.ot * P.n_it;
  const int c2 = (2 * P.Cin + 15) / 16 * 16;
  d.Nt = min(kTileN, c2 - kTileN * d.it);
  d.nkm = (min(d.l + 1, P.M) + kKr - 1) / kKr;
  d.nk = P.nb * d.nkm;
  return d;
}

__device__ __forceinline__ unsigned char *align1024(unsigned char *p) {
  return reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

template <bool kSplit>
__host__ __device__ constexpr uint32_t dw_stage_bytes() {
  return (kSplit ? 2u : 1u) * (2u + 4u) * kBoxBytes;  // A: 2 boxes, B: up to 4 boxes, per part
}

template <bool kSplit>
__global__ void __launch_bounds__(kThreadsDw, 1) dw_tc_kernel(const __grid_constant__ DwParams P) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = align1024(smem_raw);
  __shared__ uint64_t full_bar[kStages], empty_bar[kStages], tfull[2], tempty[2], done_bar;
  __shared__ uint32_t tmem_slot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr uint32_t sbytes = dw_stage_bytes<kSplit>();
  constexpr uint32_t kA = 2u * kBoxBytes;  // one part of A
  constexpr uint32_t kB = 4u * kBoxBytes;  // one part of B

  if (warp == 1) tmem_alloc(&tmem_slot, 2 * kAccCols);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; s++) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int i = 0; i < 2; i++) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 4);
    }
    mbar_init(&done_bar, 1);
    mbar_fence_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    // TMA producer: stage = (member b, rows m0 .. m0 + 31) of the tile's
    // degree; A: 128 columns o' of member b, B: Nt columns i'
    tma_prefetch_desc(&P.a_hi);
    tma_prefetch_desc(&P.b_hi);
    uint32_t g = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < P.ntiles && ok; t += gridDim.x) {
      const DwTile d = dw_tile(P, t);
      const int nbb = (d.Nt + 63) / 64;
      const uint32_t tx = (kSplit ? 2u : 1u) * (uint32_t)(2 + nbb) * kBoxBytes;
      for (int kc = 0; kc < d.nk; kc++, g++) {
        const int s = (int)(g % kStages);
        const uint32_t use = g / kStages;
        if (use > 0 && !mbar_wait(&empty_bar[s], (use - 1) & 1, P.err)) {
          ok = false;
          break;
        }
        const int b = kc / d.nkm, m0 = (kc - b * d.nkm) * kKr;
        unsigned char *st = base + (size_t)s * sbytes;
        mbar_arrive_expect_tx(&full_bar[s], tx);
        const int xa = b * P.kxa + kTileM * d.ot, xb = b * P.kxb + kTileN * d.it;
        for (int j = 0; j < 2; j++) {
          tma_load_3d(st + j * kBoxBytes, &P.a_hi, &full_bar[s], xa + 64 * j, m0, d.l);
          if (kSplit) tma_load_3d(st + kA + j * kBoxBytes, &P.a_lo, &full_bar[s], xa + 64 * j, m0, d.l);
        }
        unsigned char *sb = st + (kSplit ? 2 : 1) * kA;
        for (int j = 0; j < nbb; j++) {
          tma_load_3d(sb + j * kBoxBytes, &P.b_hi, &full_bar[s], xb + 64 * j, m0, d.l);
          if (kSplit) tma_load_3d(sb + kB + j * kBoxBytes, &P.b_lo, &full_bar[s], xb + 64 * j, m0, d.l);
        }
      }
    }
    // copies still in flight when a wait gave up: let the last stages'
    // copies land (bounded) before the CTA leaves
    if (!ok)
      for (uint32_t j = 0; j < kStages && j < g; j++) {
        const uint32_t c = g - 1 - j;
        mbar_wait(&full_bar[c % kStages], (c / kStages) & 1, nullptr, 100000000ull);
      }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      uint32_t g = 0, it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < P.ntiles && ok; t += gridDim.x, it++) {
        const DwTile d = dw_tile(P, t);
        uint32_t idesc = idesc_bf16_f32(kTileM, d.Nt, true) | (1u << 15);  // A and B MN-major
        const int acc = (int)(it & 1);
        const uint32_t use_a = it >> 1;
        if (use_a > 0 && !mbar_wait(&tempty[acc], (use_a - 1) & 1, P.err)) break;
        tc_fence_after();
        const uint32_t tacc = tmem + (uint32_t)acc * kAccCols;
        for (int kc = 0; kc < d.nk; kc++, g++) {
          const int s = (int)(g % kStages);
          const uint32_t use = g / kStages;
          if (!mbar_wait(&full_bar[s], use & 1, P.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          unsigned char *st = base + (size_t)s * sbytes;
          unsigned char *a_hi = st, *a_lo = st + kA;
          unsigned char *b_hi = st + (kSplit ? 2 : 1) * kA, *b_lo = b_hi + kB;
#pragma unroll
          for (int ks = 0; ks < kKr / 16; ks++) {
            const uint32_t acc0 = (kc == 0 && ks == 0) ? 0u : 1u;
            const uint64_t ah = desc_mnmajor_sw128(a_hi + ks * 2048, kBoxBytes, 1024);
            const uint64_t bh = desc_mnmajor_sw128(b_hi + ks * 2048, kBoxBytes, 1024);
            mma_bf16(tacc, ah, bh, idesc, acc0);
            if (kSplit) {
              mma_bf16(tacc, ah, desc_mnmajor_sw128(b_lo + ks * 2048, kBoxBytes, 1024), idesc, 1u);
              mma_bf16(tacc, desc_mnmajor_sw128(a_lo + ks * 2048, kBoxBytes, 1024), bh, idesc, 1u);
            }
          }
          mma_commit(&empty_bar[s]);
        }
        if (!ok) break;
        if (d.nk > 0)
          mma_commit(&tfull[acc]);
        else
          mbar_arrive(&tfull[acc]);
      }
      // every MMA of this CTA done before the tensor memory is released
      mma_commit(&done_bar);
      mbar_wait(&done_bar, 0, P.err, 100000000ull);
    }
    __syncwarp();
  } else if (warp >= 2) {
    // epilogue: warp q reads tensor-memory lanes 32 q .. 32 q + 31 (rows o'
    // of the tile); adjacent lanes hold the real and imaginary rows of one
    // o and trade half of their columns, so that every lane writes four
    // complex values: the even lane the first four i of each 16 columns,
    // the odd lane the last four
    const int q = warp & 3;
    uint32_t it = 0;
    for (int t = blockIdx.x; t < P.ntiles; t += gridDim.x, it++) {
      const DwTile d = dw_tile(P, t);
      const int acc = (int)(it & 1);
      // the warp leaves together: its tensor-memory loads are warp-wide
      if (!__all_sync(0xffffffffu, mbar_wait(&tfull[acc], (it >> 1) & 1, P.err))) break;
      tc_fence_after();
      const int orow = kTileM * d.ot + 32 * q + lane;  // o'
      const int o = orow >> 1;
      const bool odd = orow & 1;
      const bool o_ok = o < P.Cout;
      float2 *row = P.gW + ((int64_t)d.l * P.Cout + o) * P.Cin;
      const uint32_t tbase = tmem + (uint32_t)acc * kAccCols + ((uint32_t)(32 * q) << 16);
      for (int c0 = 0; c0 < d.Nt; c0 += 16) {
        float v[16];
        if (d.nk > 0) {
          tmem_ld16(tbase + (uint32_t)c0, v);
        } else {
#pragma unroll
          for (int j = 0; j < 16; j++) v[j] = 0.f;
        }
        float p[8];
#pragma unroll
        for (int j = 0; j < 8; j++) p[j] = __shfl_xor_sync(0xffffffffu, odd ? v[j] : v[8 + j], 1);
        // the partner's columns 0..7 (even lane) or 8..15 (odd lane) sit in p
        const int ib = (kTileN * d.it + c0) / 2 + (odd ? 4 : 0);
        float2 r[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
          if (!odd) {
            r[j] = make_float2(v[2 * j] + p[2 * j + 1], p[2 * j] - v[2 * j + 1]);
          } else {
            r[j] = make_float2(p[2 * j] + v[8 + 2 * j + 1], v[8 + 2 * j] - p[2 * j + 1]);
          }
        }
        if (!o_ok) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const int i = ib + j;
          if (i >= P.Cin) break;
          float2 w = r[j];
          if (P.accumulate) {
            const float2 old = row[i];
            w = make_float2(w.x + old.x, w.y + old.y);
          }
          row[i] = w;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[acc]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 2 * kAccCols);
  }
}

}  // namespace

cudaError_t launch_dw_tc(const __nv_bfloat16 *g_hi, const __nv_bfloat16 *g_lo, const __nv_bfloat16 *x_hi,
                         const __nv_bfloat16 *x_lo, int ldx, float2 *gW, int L, int M, int nb, int Cin, int Cout,
                         int kxa, int kxb, int accumulate, unsigned *err, cudaStream_t st) {
  if (nb <= 0 || L <= 0) return cudaSuccess;
  const bool split = g_lo && x_lo;
  DwParams P{};
  if (!(tc_encode_rows_mn_bf16(&P.a_hi, g_hi, ldx, M, L, kKr) && tc_encode_rows_mn_bf16(&P.b_hi, x_hi, ldx, M, L, kKr)))
    return cudaErrorInvalidValue;
  if (split && !(tc_encode_rows_mn_bf16(&P.a_lo, g_lo, ldx, M, L, kKr) &&
                 tc_encode_rows_mn_bf16(&P.b_lo, x_lo, ldx, M, L, kKr)))
    return cudaErrorInvalidValue;
  P.gW = gW;
  P.err = err;
  P.L = L;
  P.M = M;
  P.nb = nb;
  P.Cin = Cin;
  P.Cout = Cout;
  P.kxa = kxa;
  P.kxb = kxb;
  P.n_ot = (2 * Cout + kTileM - 1) / kTileM;
  P.n_it = (2 * Cin + kTileN - 1) / kTileN;
  P.ntiles = L * P.n_ot * P.n_it;
  P.accumulate = accumulate;
  const size_t smem = (size_t)kStages * (split ? dw_stage_bytes<true>() : dw_stage_bytes<false>()) + 1024;
  const void *fn = split ? (const void *)dw_tc_kernel<true> : (const void *)dw_tc_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)std::min(P.ntiles, sm_count());
  if (split)
    dw_tc_kernel<true><<<grid, kThreadsDw, smem, st>>>(P);
  else
    dw_tc_kernel<false><<<grid, kThreadsDw, smem, st>>>(P);
  return cudaGetLastError();
}

}  // namespace shtgb
