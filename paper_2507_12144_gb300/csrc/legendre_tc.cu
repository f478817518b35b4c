// Legendre contractions of the SHT on the 5th-generation tensor cores
// (tcgen05), BF16 operands with FP32 accumulation in tensor memory.
//
// The contraction of Algorithm 1 ("Legendre-Gauss quadrature via tensor
// contraction") is, for each order m and parity p of l + m, a GEMM of the
// rows of the folded table by the 2B real columns of the data.  Precision
// forms, with x = x_hi + x_lo, x_hi = bf16(x), x_lo = bf16(x - x_hi):
//   split BF16: table and data split, T_hi D_hi + T_hi D_lo + T_lo D_hi (the
//               lo*lo term is below the FP32 accumulation error); the table
//               generated in tensor memory for the inverse is split in three
//               (T = T_hi + T_lo + T_lo2, x_lo2 = bf16(x - x_hi - x_lo)) and
//               adds T_lo2 D_hi;
//   BF16:       data rounded to bf16, table split in two, T_hi D_hi + T_lo D_hi.
// The table keeps its lo part in both: its representation error is one
// systematic error per (l, m, k) shared by every field, and the sum over
// latitudes of oscillating Phat against smooth data cancels (the terms are
// about 8x the result at l^-3 spectra), which amplifies it; with two terms
// the table's error is 2.5x the data's, with three it is negligible.  The paper trains in bf16 mixed
// precision (Sec. E.3); the split form recovers FP32-level accuracy.
//
// Persistent kernels, one CTA per SM:
//   tc_persistent_kernel  streamed Legendre table (TMA) or the filter
//     (256 threads; the filter's weights are built on chip by 8 more warps):
//     warp 0 TMA producer, warp 1 MMA issuer (one thread), warp 2 tensor
//     memory allocation, warps 4..7 epilogue (tensor memory -> registers ->
//     swizzled shared staging -> TMA stores), warps 8..15 weight builders.
//   tc_gen_kernel  Legendre table generated on chip by the recurrence
//     (512 threads): the same roles, warps 8..15 generate the table chunks.
//     The generated table (A) and the TMA-loaded data (B) have separate
//     rings: two table slots of 64 K, and data stages of 32 K, as many as
//     fit.  The inverse writes its table slots into tensor memory, from
//     where the MMAs read A: the tcgen05 MMAs of 128 x 144 tiles are bound
//     by the shared-memory bandwidth of their operands (A 4 KB + B 4.6 KB
//     per K step of 16), so A out of shared memory is A off that bound.
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
constexpr int kThreads = 256;     // filter: TMA, MMA, TMEM, -, 4 epilogue warps
constexpr int kThreadsGen = 512;  // Legendre: the same + 8 table-generator warps
constexpr int kSeedRows = 32;     // rows between recurrence seeds
constexpr int kCoefPerThread = 3; // coefficient slice per generator thread (<= 768 per tile)
constexpr int kMaxStages = 6;
constexpr uint32_t kABytes = kRows * 128;  // one A tile (hi or lo)
// generated-table kernel: K rows per data stage (a divisor of kKc), table
// slots, data stages
constexpr int kKb = 32;
constexpr int kBPerA = kKc / kKb;  // data stages per table chunk
constexpr int kASlots = 2;
constexpr int kMaxBStages = 8;
// one shared-memory table slot of the generated-table forward: 128 rows x
// 64 K as hi and lo
constexpr uint32_t kASlotBytes = 2 * kABytes;
// the inverse's table slots in tensor memory (accumulators at columns 0 and
// 256, at most 160 wide): slot s at column 160 + 256 s, parts hi, lo, lo2
// 32 columns apart (64 K as bf16 pairs)
constexpr uint32_t kTmemAccStride = 256;
constexpr int kTmemMaxN = 160;
__host__ __device__ constexpr uint32_t a_tmem_col(int slot) { return 160u + 256u * (uint32_t)slot; }

__host__ __device__ inline int tmem_cols_for(int n) { return n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : 256; }

__device__ __forceinline__ unsigned char *align1024(unsigned char *p) {
  return reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

__device__ __forceinline__ void put_bf16_pair(__nv_bfloat16 *hi, __nv_bfloat16 *lo, int64_t idx, float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  *reinterpret_cast<__nv_bfloat162 *>(hi + idx) = h;
  if (lo) {
    const float2 hf = __bfloat1622float2(h);
    *reinterpret_cast<__nv_bfloat162 *>(lo + idx) = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  }
}

// Round 8 consecutive FP32 values to bf16 (and the remainder to bf16 when lo
// is set) and store them as 16-byte chunks at hi + idx / lo + idx.
__device__ __forceinline__ void put_bf16x8(__nv_bfloat16 *hi, __nv_bfloat16 *lo, int64_t idx, const float *v) {
  uint32_t h[4], r[4];
#pragma unroll
  for (int u = 0; u < 4; u++) {
    const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * u], v[2 * u + 1]);
    const float2 hf = __bfloat1622float2(hh);
    const __nv_bfloat162 ll = __floats2bfloat162_rn(v[2 * u] - hf.x, v[2 * u + 1] - hf.y);
    h[u] = *reinterpret_cast<const uint32_t *>(&hh);
    r[u] = *reinterpret_cast<const uint32_t *>(&ll);
  }
  *reinterpret_cast<uint4 *>(hi + idx) = make_uint4(h[0], h[1], h[2], h[3]);
  if (lo) *reinterpret_cast<uint4 *>(lo + idx) = make_uint4(r[0], r[1], r[2], r[3]);
}

// ---------------------------------------------------------------------------
// Persistent tensor-core kernel for the three contractions.  One CTA per SM
// walks its tiles (round i: tile i gridDim.x + blockIdx.x, or + gridDim.x
// - 1 - blockIdx.x on odd rounds).  A ring of `stages`
// shared-memory stages carries TMA loads to the MMA thread continuously
// across tiles; the accumulator is double-buffered in tensor memory so that
// the epilogue warps drain tile i while the MMAs of tile i + 1 run.
//   kFwd:  D[i][c]  = sum_k' T[m][p][i][k'] F[m][p][k'][c]   (A = table, B = data, MN-major)
//   kInv:  D[k'][c] = sum_i  T[m][p][i][k'] S[(m + p + 2i) M + m][c]   (A = table, B = data, MN-major;
//          A read from the forward table's rows i, k' contiguous: MN-major too)
//   kFilt: D[m][n]  = sum_k  X[l M + m][b kx + k] WR[l][n][k] (A = data, B = weights, K-major)
// Table and weights always enter split (hi + lo); data enters split for
// split BF16 and rounded (hi only) for BF16.  Here the Legendre table of
// kFwd / kInv streams from a precomputed bf16 table by TMA (kGen = false;
// the table generated on chip is tc_gen_kernel's); the filter's real-form
// weights WR are built on chip by 8 extra warps from the complex W (kFilt
// with kGen = true).  With the streamed table a tile runs only the nk
// chunks from K row k0 that cover its non-negligible table entries
// (tile_krange_kernel: near the poles the high orders' Phat are zero to
// working precision).
// ---------------------------------------------------------------------------
enum Mode { kFwd = 0, kInv = 1, kFilt = 2 };

struct FiltTile {
  int l, m0;
};

// Destination of the forward contraction: l-major bf16 rows (row l M + m,
// member b's channel ch at column b kx + 2 ch + {re, im}) for the
// tensor-core filter, or FP32 l-major rows (row l M + m, field f at columns
// 2 f + {re, im}, row stride ldr floats), which a transpose kernel turns
// into the API layout xhat[b][l][m].
struct FwdOut {
  __nv_bfloat16 *rows_hi, *rows_lo;
  int ldo, cin, kx;
  float *rowsf;
  int ldr;
};

// Recurrence seeds of the on-chip Legendre table: for order m, parity p,
// 32-row block j (rows i = 32 j .. 32 j + 31, l = m + p + 2 i) and latitude
// k', Phat at l0 = m + p + 64 j and l0 + 2 (the block's first two rows) in
// FP32, as float2 at [((2m + p) NB + j) Kh + k'].  Values below the FP32
// normal range are stored as zero: inside one block a row grows by at most
// about 10^32 over the previous 32 rows (the evanescent region just above
// l = m), so what such a seed would have grown into stays below 10^-6 and
// contributes nothing the FP32 accumulation keeps.

// One problem (a plan and its batch) of a Legendre launch.  A launch walks
// the tiles of up to kMaxSeg problems (grids of different sizes in one
// batched call); global tile t belongs to problem s with tile0[s] <= t <
// tile0[s + 1] and splits into row tile (t - tile0) / nct and column tile
// (t - tile0) % nct.
constexpr int kMaxSeg = 8;

struct SegArgs {
  int L, M, Kh, B;        // degrees, orders, ceil(nlat / 2), fields
  int Nt, nct, tile0;     // column tile width and count, first global tile
  int xoff;               // offset of this problem's x^2 in shared memory
  const LegTile *tiles;   // (m, p, first row, TMA row) of the row tiles
  FwdOut fout;            // forward destination
  float *Gw;              // inverse destination (folded FP32 workspace)
  int ldc;
  int gpair;              // its layout: parity-paired (1) or (m, p)-major (0)
  // on-chip table: seeds [((2m + p) NB + j) Kh + k'], two-step
  // coefficients coef[(2m + p) ldC + i] = (alpha, beta, gamma, 0) of row i,
  // squared latitudes x^2 = x2h + x2l
  const float2 *seeds;
  const float4 *coef;
  const float *x2h, *x2l;
  int NB, ldC;
  const int *roff;        // first forward-table row of block (m, p) at [2m + p]
  const int2 *krange;     // streamed table: K rows [x, y) of each row tile (nullptr: all)
};

// TMA maps of one problem: A (table hi/lo, or filter data), B (data, or
// filter weights), and store maps of the output with 32- and 16-column
// boxes of 32 rows: for the inverse the FP32 rows viewed as [2M][Kh][ldc]
// (o32_hi, o16_hi); for the forward into l-major bf16 rows those rows
// viewed as [L][M][ldx] with every second l (hi and lo); for the filter the
// internal rows S viewed as [L][M][ldcb], boxes of 32 m of one l.
struct SegMaps {
  CUtensorMap a_hi, a_lo, b_hi, b_lo, o32_hi, o32_lo, o16_hi, o16_lo;
};

struct TcParams {
  SegMaps maps[kMaxSeg];
  SegArgs seg[kMaxSeg];
  int nseg, ntiles, stages;
  int Nmax;               // widest column tile: stage layout and TMEM columns
  int ncmax, xtot;        // generator shared memory: coefficients, x^2 entries
  int epi_off;            // byte offset of the epilogue staging
  int epi_nbuf;           // its buffers per warp (generated-table kernel)
  // filter (one problem)
  const FiltTile *ftiles;
  int L, M, Nt, Bm, ntn, kx, nwr, cin, cout, lds;
  const float2 *W;        // complex weights [L][cout][cin] (B generated on chip)
  int wadj;               // 1: the weights of (output o, input i) are conj(W[l][i][o]), W [L][cin][cout]
                          // (selects the kernel instance; read on the host)
  __nv_bfloat16 *s_hi, *s_lo;
  unsigned *err;
};

// A tiles per stage: filter data (hi, lo when split); Legendre table (hi, lo)
__host__ __device__ inline int a_count(int mode, bool split) { return mode == kFilt ? (split ? 2 : 1) : 2; }
__host__ __device__ inline int threads_of(bool gen) { return gen ? kThreadsGen : kThreads; }
__host__ __device__ inline int b_count(int mode, bool split) { return (mode == kFilt || split) ? 2 : 1; }
__host__ __device__ inline uint32_t b_bytes_of(int mode, int Nt) {
  return mode == kFilt ? (uint32_t)Nt * 128u : (uint32_t)((Nt + 63) / 64) * 8192u;
}
__host__ __device__ inline uint32_t stage_bytes(int mode, bool split, int Nt) {
  return (uint32_t)a_count(mode, split) * kABytes + (uint32_t)b_count(mode, split) * b_bytes_of(mode, Nt);
}

struct TileInfo {
  int s, Nt;             // problem, its column tile width
  int nk;                // K chunks
  int k0;                // first K row of chunk 0 (the rows before meet only negligible table entries)
  int a_col0, a_row;     // A: K column of chunk 0, row
  int b_col0, b_row0;    // B: for MN-major (col of box 0, K row of chunk 0); for K-major (K col 0, row)
  // epilogue selectors
  int m, p, r0, c0, l, b, n0;
};

// A tile as fetched: its problem, index inside the problem and the row
// tile's descriptor (a pending load until decoded), so that every role can
// request the next tile one tile ahead.
struct RawTile {
  int s, local;
  int4 d;
};

template <int kMode>
__device__ __forceinline__ RawTile tile_fetch(const TcParams &P, int t) {
  RawTile r{0, t, make_int4(0, 0, 0, 0)};
  if (t >= P.ntiles) return r;
  if (kMode == kFilt) {
    const int per = P.Bm * P.ntn;
    const int2 ft = __ldg(reinterpret_cast<const int2 *>(P.ftiles) + t / per);
    r.d = make_int4(ft.x, ft.y, 0, 0);
  } else {
    int s = 0;
    while (s + 1 < P.nseg && t >= P.seg[s + 1].tile0) s++;
    r.s = s;
    r.local = t - P.seg[s].tile0;
    r.d = __ldg(reinterpret_cast<const int4 *>(P.seg[s].tiles) + r.local / P.seg[s].nct);
  }
  return r;
}

template <int kMode>
__device__ __forceinline__ TileInfo tile_decode(const TcParams &P, const RawTile &r) {
  TileInfo ti{};
  if (kMode == kFilt) {
    const int per = P.Bm * P.ntn;
    const int rem = r.local - (r.local / per) * per;
    ti.s = 0;
    ti.Nt = P.Nt;
    ti.l = r.d.x;
    ti.m = r.d.y;
    ti.b = rem / P.ntn;
    ti.n0 = (rem - ti.b * P.ntn) * P.Nt;
    ti.nk = (2 * P.cin + kKc - 1) / kKc;
    ti.a_col0 = ti.b * P.kx;
    ti.a_row = ti.l * P.M + ti.m;
    ti.b_col0 = 0;
    ti.b_row0 = ti.l * P.nwr + ti.n0;
  } else {
    const SegArgs &g = P.seg[r.s];
    ti.s = r.s;
    ti.Nt = g.Nt;
    ti.m = r.d.x;
    ti.p = r.d.y;
    ti.r0 = r.d.z;
    ti.c0 = (r.local % g.nct) * g.Nt;
    ti.b_col0 = ti.c0;
    ti.a_col0 = 0;
    if (kMode == kFwd) {
      ti.nk = (g.Kh + kKc - 1) / kKc;
      ti.a_row = r.d.w;         // table row of the tile
      ti.b_row0 = 2 * ti.m + ti.p;  // (2m + p) coordinate of the folded data map
    } else {
      ti.nk = (leg_rows(g.L, ti.m, ti.p) + kKc - 1) / kKc;
      // A: rows i of the block in the forward table, columns k' from r0
      ti.a_row = g.roff ? __ldg(g.roff + 2 * ti.m + ti.p) : 0;
      ti.a_col0 = ti.r0;
      ti.b_row0 = r.d.w;  // first degree m + p of the (m, p) block
    }
    if (g.krange) {
      const int2 kr = __ldg(g.krange + r.local / g.nct);
      ti.k0 = kr.x;
      ti.nk = (kr.y - kr.x + kKc - 1) / kKc;
    }
  }
  return ti;
}

// Tiles of this CTA in order, the next one fetched a tile ahead.  Round w
// of the walk covers tiles w G .. w G + G - 1 (G CTAs), in reverse CTA order
// on odd rounds: tile costs fall along the list (higher orders have fewer
// rows and K chunks), and the alternation evens out each CTA's total.
template <int kMode>
struct TileWalk {
  int w, t;
  RawTile nxt;
  __device__ __forceinline__ static int tile_of(int w) {
    return w * (int)gridDim.x + ((w & 1) ? (int)gridDim.x - 1 - (int)blockIdx.x : (int)blockIdx.x);
  }
  __device__ __forceinline__ TileWalk(const TcParams &P) : w(0), t(blockIdx.x) { nxt = tile_fetch<kMode>(P, t); }
  __device__ __forceinline__ bool more(const TcParams &P) const { return t < P.ntiles; }
  // the current tile's info; requests the one after it
  __device__ __forceinline__ TileInfo take(const TcParams &P) {
    const TileInfo ti = tile_decode<kMode>(P, nxt);
    t = tile_of(++w);
    nxt = tile_fetch<kMode>(P, t);
    return ti;
  }
};

// Bytes that the TMA loads of one chunk of the tile deliver.
template <int kMode, bool kSplit, bool kGen>
__device__ __forceinline__ uint32_t chunk_tx_bytes(const TileInfo &ti) {
  const uint32_t abytes = (uint32_t)a_count(kMode, kSplit) * kABytes;
  if (kMode == kFilt) return abytes + (kGen ? 0u : 2u * (uint32_t)ti.Nt * 128u);
  return abytes + (uint32_t)b_count(kMode, kSplit) * (uint32_t)((ti.Nt + 63) / 64) * 8192u;
}

// MMAs of one K chunk (kKc = 64) of a tile, N = the tile's column width;
// only the first nks K steps of 16 (the filter's last chunk ends at 2 Cin).
// Stage layout (for the launch's widest tile Nmax): A hi, A lo, B hi, B lo.
template <int kMode, bool kSplit, bool kGen>
__device__ __forceinline__ void issue_chunk(unsigned char *st, int Nmax, uint32_t tmem, uint32_t idesc, bool first,
                                            int nks = kKc / 16) {
  const int na = a_count(kMode, kSplit);
  const uint32_t bb = b_bytes_of(kMode, Nmax);
  unsigned char *a_hi = st, *a_lo = st + kABytes;
  unsigned char *b_hi = st + na * kABytes, *b_lo = b_hi + bb;
#pragma unroll
  for (int ks = 0; ks < kKc / 16; ks++) {
    if (ks >= nks) break;
    const uint32_t acc0 = (first && ks == 0) ? 0u : 1u;
    const uint64_t ah = desc_advance(desc_kmajor_sw128(a_hi), ks * 32);
    if (kMode == kFilt) {
      const uint64_t bh = desc_advance(desc_kmajor_sw128(b_hi), ks * 32);
      const uint64_t bl = desc_advance(desc_kmajor_sw128(b_lo), ks * 32);
      mma_bf16(tmem, ah, bh, idesc, acc0);
      mma_bf16(tmem, ah, bl, idesc, 1u);
      if (kSplit) mma_bf16(tmem, desc_advance(desc_kmajor_sw128(a_lo), ks * 32), bh, idesc, 1u);
    } else if (kMode == kFwd) {
      // A = table, K-major from TMA
      const uint64_t al = desc_advance(desc_kmajor_sw128(a_lo), ks * 32);
      const uint64_t bh = desc_mnmajor_sw128(b_hi + ks * 2048, 8192, 1024);
      mma_bf16(tmem, ah, bh, idesc, acc0);
      mma_bf16(tmem, al, bh, idesc, 1u);
      if (kSplit) mma_bf16(tmem, ah, desc_mnmajor_sw128(b_lo + ks * 2048, 8192, 1024), idesc, 1u);
    } else {
      // A = table, MN-major from TMA: two 64-column boxes (k') of 64 rows (i)
      const uint64_t ahm = desc_mnmajor_sw128(a_hi + ks * 2048, 8192, 1024);
      const uint64_t alm = desc_mnmajor_sw128(a_lo + ks * 2048, 8192, 1024);
      const uint64_t bh = desc_mnmajor_sw128(b_hi + ks * 2048, 8192, 1024);
      mma_bf16(tmem, ahm, bh, idesc, acc0);
      mma_bf16(tmem, alm, bh, idesc, 1u);
      if (kSplit) mma_bf16(tmem, ahm, desc_mnmajor_sw128(b_lo + ks * 2048, 8192, 1024), idesc, 1u);
    }
  }
}

template <int kMode, bool kSplit, bool kGen>
__device__ __forceinline__ void load_chunk(unsigned char *st, const TileInfo &ti, int kc, int Nmax, const SegMaps &mp,
                                           uint64_t *bar) {
  const int na = a_count(kMode, kSplit);
  const uint32_t bb = b_bytes_of(kMode, Nmax);
  unsigned char *a_hi = st, *a_lo = st + kABytes;
  unsigned char *b_hi = st + na * kABytes, *b_lo = b_hi + bb;
  const int kb = ti.k0 + kc * kKc;  // first K row of the chunk (k0: zero for the filter)
  if (kMode == kInv) {
    // the forward table's rows i = kb .. kb + 63 of the block, k'
    // columns r0 .. r0 + 127 as two 64-column boxes (rows past the block
    // belong to the next block and meet degrees past lmax: zero data)
    for (int j = 0; j < 2; j++) {
      tma_load_2d(a_hi + j * 8192, &mp.a_hi, bar, ti.a_col0 + 64 * j, ti.a_row + kb);
      tma_load_2d(a_lo + j * 8192, &mp.a_lo, bar, ti.a_col0 + 64 * j, ti.a_row + kb);
    }
  } else {
    tma_load_2d(a_hi, &mp.a_hi, bar, ti.a_col0 + kb, ti.a_row);
    if (na == 2) tma_load_2d(a_lo, &mp.a_lo, bar, ti.a_col0 + kb, ti.a_row);
  }
  if (kMode == kFilt) {
    if (!kGen) {
      tma_load_2d(b_hi, &mp.b_hi, bar, kb, ti.b_row0);
      tma_load_2d(b_lo, &mp.b_lo, bar, kb, ti.b_row0);
    }
  } else if (kMode == kFwd) {
    // the folded data as (column, 2m + p, k'): 64 rows k' of one (m, p)
    const int nbox = (ti.Nt + 63) / 64;
    for (int j = 0; j < nbox; j++) {
      tma_load_3d(b_hi + j * 8192, &mp.b_hi, bar, ti.b_col0 + 64 * j, ti.b_row0, kb);
      if (kSplit) tma_load_3d(b_lo + j * 8192, &mp.b_lo, bar, ti.b_col0 + 64 * j, ti.b_row0, kb);
    }
  } else {
    // the internal rows as (column, m, l) with every second l: 64 rows
    // l = m + p + 2 i of one (m, p) block per box
    const int nbox = (ti.Nt + 63) / 64;
    for (int j = 0; j < nbox; j++) {
      tma_load_3d(b_hi + j * 8192, &mp.b_hi, bar, ti.b_col0 + 64 * j, ti.m, ti.b_row0 + 2 * kb);
      if (kSplit) tma_load_3d(b_lo + j * 8192, &mp.b_lo, bar, ti.b_col0 + 64 * j, ti.m, ti.b_row0 + 2 * kb);
    }
  }
}

// Write accumulator columns [0, ncols) (a multiple of 16) of this warp's 32
// TMEM lanes as bf16 hi (and lo) through TMA stores: the 32-column chunk
// at j0 goes to (x + j0, y, z) of the 32-column maps, a 16-column tail to
// the 16-column maps.  nbuf (1 or 2) staging buffers of 4 KB (hi 2 KB, lo
// 2 KB) at stg; 64-byte rows swizzled for the 32-column box, 32-byte rows
// for the tail.  With one 4 KB buffer all chunks are 16 columns wide, two
// 2 KB buffers (hi 1 KB, lo 1 KB) in it, so that a chunk waits only for
// the store of the chunk before the previous one to have read its buffer.
__device__ __forceinline__ void store_rows_bf16_tma(uint32_t tl, int ncols, const CUtensorMap *m32h,
                                                    const CUtensorMap *m32l, const CUtensorMap *m16h,
                                                    const CUtensorMap *m16l, bool lo, int x, int y, int z,
                                                    unsigned char *stg, int nbuf, int lane) {
  if (nbuf == 1) {
    for (int j0 = 0, c = 0; j0 < ncols; j0 += 16, c++) {
      unsigned char *bh = stg + (c & 1) * 2048, *bl = bh + 1024;
      if (c >= 2) {
        if (lane == 0) bulk_wait_read<1>();
        __syncwarp();
      }
      float v[16];
      tmem_ld16(tl + (uint32_t)j0, v);
#pragma unroll
      for (int u = 0; u < 2; u++) {
        uint32_t h[4], r4[4];
#pragma unroll
        for (int w = 0; w < 4; w++) {
          const __nv_bfloat162 hh = __floats2bfloat162_rn(v[8 * u + 2 * w], v[8 * u + 2 * w + 1]);
          const float2 hf = __bfloat1622float2(hh);
          const __nv_bfloat162 ll = __floats2bfloat162_rn(v[8 * u + 2 * w] - hf.x, v[8 * u + 2 * w + 1] - hf.y);
          h[w] = *reinterpret_cast<const uint32_t *>(&hh);
          r4[w] = *reinterpret_cast<const uint32_t *>(&ll);
        }
        const uint32_t off = lane * 32 + u * 16;
        *reinterpret_cast<uint4 *>(bh + off) = make_uint4(h[0], h[1], h[2], h[3]);
        if (lo) *reinterpret_cast<uint4 *>(bl + off) = make_uint4(r4[0], r4[1], r4[2], r4[3]);
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        tma_store_3d(m16h, bh, x + j0, y, z);
        if (lo) tma_store_3d(m16l, bl, x + j0, y, z);
        bulk_commit();
      }
    }
    if (lane == 0) bulk_wait_read<0>();
    __syncwarp();
    return;
  }
  for (int j0 = 0, c = 0; j0 < ncols; j0 += 32, c++) {
    const bool half = ncols - j0 == 16;
    unsigned char *bh = stg + (c % nbuf) * 4096, *bl = bh + 2048;
    if (c >= nbuf) {
      if (lane == 0) {
        if (nbuf == 2)
          bulk_wait_read<1>();
        else
          bulk_wait_read<0>();
      }
      __syncwarp();
    }
    float v[32];
    tmem_ld16(tl + (uint32_t)j0, *reinterpret_cast<float(*)[16]>(v));
    if (!half) tmem_ld16(tl + (uint32_t)(j0 + 16), *reinterpret_cast<float(*)[16]>(v + 16));
    const int nchunk = half ? 2 : 4;  // 16-byte chunks of 8 values
    for (int u = 0; u < nchunk; u++) {
      uint32_t h[4], r4[4];
#pragma unroll
      for (int w = 0; w < 4; w++) {
        const __nv_bfloat162 hh = __floats2bfloat162_rn(v[8 * u + 2 * w], v[8 * u + 2 * w + 1]);
        const float2 hf = __bfloat1622float2(hh);
        const __nv_bfloat162 ll = __floats2bfloat162_rn(v[8 * u + 2 * w] - hf.x, v[8 * u + 2 * w + 1] - hf.y);
        h[w] = *reinterpret_cast<const uint32_t *>(&hh);
        r4[w] = *reinterpret_cast<const uint32_t *>(&ll);
      }
      const uint32_t off = half ? lane * 32 + u * 16 : lane * 64 + ((u ^ ((lane >> 1) & 3)) << 4);
      *reinterpret_cast<uint4 *>(bh + off) = make_uint4(h[0], h[1], h[2], h[3]);
      if (lo) *reinterpret_cast<uint4 *>(bl + off) = make_uint4(r4[0], r4[1], r4[2], r4[3]);
    }
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) {
      tma_store_3d(half ? m16h : m32h, bh, x + j0, y, z);
      if (lo) tma_store_3d(half ? m16l : m32l, bl, x + j0, y, z);
      bulk_commit();
    }
  }
  if (lane == 0) bulk_wait_read<0>();
  __syncwarp();
}

// Wait until at most nbuf - 1 of this warp's bulk stores still read their
// staging buffer (lane 0 issues them), before the next buffer is written.
__device__ __forceinline__ void staging_wait(int nbuf, int lane) {
  if (lane == 0) {
    if (nbuf == 2)
      bulk_wait_read<1>();
    else
      bulk_wait_read<0>();
  }
  __syncwarp();
}

// Epilogue of one tile for the accumulator at tacc (zero: write zeros),
// through nbuf (1 or 2) staging buffers of 4 KB per warp at stg.
template <int kMode>
__device__ __forceinline__ void epilogue(const TcParams &P, const TileInfo &ti, uint32_t tacc, int q4, int lane,
                                         bool zero, unsigned char *stg, int nbuf) {
  const int Nt = ti.Nt;
  const uint32_t tl = tacc + ((uint32_t)(q4 * 32) << 16);
  if (kMode == kFwd) {
    const SegArgs &g = P.seg[ti.s];
    // l-major bf16 rows of one member through TMA stores: the tile's
    // columns must lie in one member and start on a 16-byte boundary
    {
      const FwdOut &out = g.fout;
      const int mb = (ti.c0 / 2) / out.cin;
      const bool one_member = out.rows_hi && (out.cin & 3) == 0 && ((ti.c0 + Nt) / 2 - 1) / out.cin == mb;
      if (one_member) {
        const SegMaps &mp = P.maps[ti.s];
        const int x0 = mb * out.kx + (ti.c0 - 2 * mb * out.cin);  // output column of accumulator column c0
        const int l0 = ti.m + ti.p + 2 * (ti.r0 + q4 * 32);
        store_rows_bf16_tma(tl, Nt, &mp.o32_hi, &mp.o32_lo, &mp.o16_hi, &mp.o16_lo, out.rows_lo != nullptr, x0,
                            ti.m, l0, stg, nbuf, lane);
        return;
      }
    }
    if (g.fout.rowsf) {
      // FP32 l-major rows [L][M][ldr]: 32 x 32 boxes of every second l
      // through the warp's two swizzled staging buffers; rows past lmax and
      // columns past ldr fall outside the map
      const SegMaps &mp = P.maps[ti.s];
      const int l0 = ti.m + ti.p + 2 * (ti.r0 + q4 * 32);
      for (int j0 = 0, c = 0; j0 < Nt; j0 += 32, c++) {
        const bool half = Nt - j0 == 16;
        unsigned char *buf = stg + (c % nbuf) * 4096;
        if (c >= nbuf) staging_wait(nbuf, lane);
        float v[32];
        tmem_ld16(tl + (uint32_t)j0, *reinterpret_cast<float(*)[16]>(v));
        if (!half) tmem_ld16(tl + (uint32_t)(j0 + 16), *reinterpret_cast<float(*)[16]>(v + 16));
        if (!half) {
          // 128-byte rows, 16-byte chunk u at u ^ (row mod 8)
#pragma unroll
          for (int u = 0; u < 8; u++)
            *reinterpret_cast<float4 *>(buf + lane * 128 + ((u ^ (lane & 7)) << 4)) =
                make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
        } else {
          // 64-byte rows, 16-byte chunk u at u ^ ((row / 2) mod 4)
#pragma unroll
          for (int u = 0; u < 4; u++)
            *reinterpret_cast<float4 *>(buf + lane * 64 + ((u ^ ((lane >> 1) & 3)) << 4)) =
                make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          tma_store_3d(half ? &mp.o16_hi : &mp.o32_hi, buf, ti.c0 + j0, ti.m, l0);
          bulk_commit();
        }
      }
      if (lane == 0) bulk_wait_read<0>();
      __syncwarp();
      return;
    }
    const int r = ti.r0 + q4 * 32 + lane;
    const bool row_ok = r < leg_rows(g.L, ti.m, ti.p);
    const int l = ti.m + ti.p + 2 * r;
    const FwdOut out = g.fout;
    const int B = g.B, M = g.M;
    const int64_t orow = ((int64_t)l * M + ti.m) * out.ldo;
    for (int j = 0; j < Nt / 16; j++) {
      float v[16];
      tmem_ld16(tl + (uint32_t)(j * 16), v);
      if (!row_ok) continue;
      {
#pragma unroll
        for (int h = 0; h < 2; h++) {
          const int f = (ti.c0 + j * 16) / 2 + 4 * h;  // first of 4 fields
          if (f >= B) continue;
          const int mb = f / out.cin, ch = f - mb * out.cin;
          if ((ch & 3) == 0 && ch + 4 <= out.cin && f + 4 <= B) {
            put_bf16x8(out.rows_hi, out.rows_lo, orow + (int64_t)mb * out.kx + 2 * ch, v + 8 * h);
          } else {
            for (int u = 0; u < 4 && f + u < B; u++) {
              const int fu = f + u, mu = fu / out.cin, cu = fu - mu * out.cin;
              put_bf16_pair(out.rows_hi, out.rows_lo, orow + (int64_t)mu * out.kx + 2 * cu, v[8 * h + 2 * u],
                            v[8 * h + 2 * u + 1]);
            }
          }
        }
      }
    }
  } else if (kMode == kInv) {
    // FP32 folded rows through the warp's two swizzled 32 x 32 staging
    // buffers and TMA stores of whole 16-column groups (the 5-D map of the
    // workspace's layout); rows k' >= Kh fall outside the map's extents and
    // are not written
    const SegMaps &mp = P.maps[ti.s];
    const int k0 = ti.r0 + q4 * 32;
    for (int j0 = 0, c = 0; j0 < Nt; j0 += 32, c++) {
      const bool half = Nt - j0 == 16;
      unsigned char *buf = stg + (c % nbuf) * 4096;
      if (c >= nbuf) staging_wait(nbuf, lane);
      float v[32];
      if (!zero) {
        tmem_ld16(tl + (uint32_t)j0, *reinterpret_cast<float(*)[16]>(v));
        if (!half) tmem_ld16(tl + (uint32_t)(j0 + 16), *reinterpret_cast<float(*)[16]>(v + 16));
      } else {
#pragma unroll
        for (int u = 0; u < 32; u++) v[u] = 0.f;
      }
      if (!half) {
        // two 64-byte rows (one per 16-column group) per k', 16-byte chunk
        // q of a row at q ^ (k' mod 4) (the 64-byte swizzle of row 2 k' + g)
#pragma unroll
        for (int u = 0; u < 8; u++)
          *reinterpret_cast<float4 *>(buf + lane * 128 + (u >> 2) * 64 + (((u & 3) ^ (lane & 3)) << 4)) =
              make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
      } else {
        // 64-byte rows, 16-byte chunk u at u ^ ((row / 2) mod 4)
#pragma unroll
        for (int u = 0; u < 4; u++)
          *reinterpret_cast<float4 *>(buf + lane * 64 + ((u ^ ((lane >> 1) & 3)) << 4)) =
              make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        const int g = (ti.c0 + j0) >> 4;
        if (P.seg[ti.s].gpair)
          tma_store_5d(half ? &mp.o16_hi : &mp.o32_hi, buf, 0, ti.p, g, k0, ti.m);
        else
          tma_store_5d(half ? &mp.o16_hi : &mp.o32_hi, buf, 0, g, k0, ti.p, ti.m);
        bulk_commit();
      }
    }
    if (lane == 0) bulk_wait_read<0>();
    __syncwarp();
  } else {
    // internal rows S, l-major (row l M + m), member b's outputs at columns
    // 2 b cout + n; through TMA stores when the tile's columns are whole
    // 16-column chunks of one member (rows m > l receive values nothing
    // reads, rows m >= M are outside the map)
    const int ncol = min(Nt, 2 * P.cout - ti.n0);
    if (ti.m + 32 * q4 > ti.l) return;  // this warp's 32 orders are all above l: nothing reads them
    if ((P.cout & 3) == 0 && (ncol & 15) == 0) {
      const SegMaps &mp = P.maps[0];
      store_rows_bf16_tma(tl, ncol, &mp.o32_hi, &mp.o32_lo, &mp.o16_hi, &mp.o16_lo, P.s_lo != nullptr,
                          2 * ti.b * P.cout + ti.n0, ti.m + 32 * q4, ti.l, stg, 1, lane);
      return;
    }
    const int m = ti.m + q4 * 32 + lane;
    const bool ok = (m < P.M) && (m <= ti.l);
    const int64_t srow = ok ? ((int64_t)ti.l * P.M + m) * P.lds + 2 * (int64_t)ti.b * P.cout : 0;
    for (int j = 0; j < Nt / 16; j++) {
      float v[16];
      tmem_ld16(tl + (uint32_t)(j * 16), v);
      if (!ok) continue;
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int n = ti.n0 + j * 16 + 8 * h;  // 4 output channels
        if (n + 8 <= 2 * P.cout && ((srow + n) & 7) == 0) {
          put_bf16x8(P.s_hi, P.s_lo, srow + n, v + 8 * h);
        } else {
          for (int u = 0; u < 4; u++)
            if (n + 2 * u < 2 * P.cout)
              put_bf16_pair(P.s_hi, P.s_lo, srow + n + 2 * u, v[8 * h + 2 * u], v[8 * h + 2 * u + 1]);
        }
      }
    }
  }
}

// Table generator (warps 8..15 of tc_gen_kernel).  Two steps of the
// three-term recurrence of Eq. sht_legendre_recursion, composed so that
// only rows of one parity appear,
//   Phat_{l+2} = (alpha_l x^2 + beta_l) Phat_l + gamma_l Phat_{l-2},
//   alpha_l = a_{l+2} a_{l+1},
//   beta_l  = -a_{l+2} (b_{l+2} + a_{l+1} b_{l+1} / a_l),   (beta_m = -a_{m+2} b_{m+2})
//   gamma_l = -a_{l+2} a_{l+1} b_{l+1} b_l,                  (gamma_m = 0)
// give one FMA per stored row on the dependency chain.  One thread runs one
// latitude through one 32-row block of one parity from the block's FP32
// seeds, with x^2 = x2h + x2l.  The 32 values go to shared memory as bf16
// hi/lo in 16-byte chunks of 8 consecutive rows:
//   forward: A[i][k'] MN-major (rows i contiguous): thread (k' = 64 kc + g mod
//            64, block r0/32 + g/64) of tile rows r0 .. r0 + 127;
//   inverse: A[k'][i] K-major (i contiguous): thread (k' = r0 + g mod 128,
//            block 2 kc + g/128).
// Latitude k' and seed block j of table chunk kc (64 K) for thread g.
template <int kMode>
__device__ __forceinline__ void gen_coords(const TileInfo &ti, int kc, int g, int &kp, int &j) {
  if (kMode == kFwd) {
    kp = kc * kKc + (g & 63);
    j = ti.r0 / kSeedRows + (g >> 6);
  } else {
    kp = ti.r0 + (g & 127);
    j = 2 * kc + (g >> 7);
  }
}

// The seed of that chunk (zero where the latitude or the block does not exist).
template <int kMode>
__device__ __forceinline__ float2 gen_seed(const SegArgs &sg, const TileInfo &ti, int kc, int g) {
  int kp, j;
  gen_coords<kMode>(ti, kc, g, kp, j);
  if (kp >= sg.Kh || j >= sg.NB) return make_float2(0.f, 0.f);
  return __ldg(sg.seeds + ((int64_t)(ti.m * 2 + ti.p) * sg.NB + j) * sg.Kh + kp);
}

// The 32 rows of one thread's block, from its seeds sd and x^2 = (x2h,
// x2l), as bf16 pairs (row 2q in the lower half): h = hi, lw = lo and, when
// kLo2, l2 = lo2 (v - hi and (v - hi) - lo are exact in FP32).  cf: the
// coefficients of the block's second row onwards (the step to row i + 2
// uses those of row i + 1).  Blocks past the last row run the same steps
// over zero seeds and zero coefficients (the coefficient array is zero past
// lmax and the index stays inside the tile's slice), so the loop has no
// per-step selects.
// NQ row pairs per call; (pa, pb) carry rows i, i + 1 from call to call.
template <bool kLo2, int NQ>
__device__ __forceinline__ void recur_rows(float &pa, float &pb, float2 x2, const float4 *cf, uint32_t (&h)[NQ],
                                           uint32_t (&lw)[NQ], uint32_t (&l2)[NQ]) {
  const float x2h = x2.x, x2l = x2.y;
#pragma unroll
  for (int q = 0; q < NQ; q++) {
    const float v0 = pa, v1 = pb;
    const float4 c0 = cf[2 * q], c1 = cf[2 * q + 1];
    const float pc = fmaf(fmaf(c0.x, x2h, fmaf(c0.x, x2l, c0.y)), pb, c0.z * pa);
    const float pd = fmaf(fmaf(c1.x, x2h, fmaf(c1.x, x2l, c1.y)), pc, c1.z * pb);
    pa = pc;
    pb = pd;
    const __nv_bfloat162 hh = __floats2bfloat162_rn(v0, v1);
    const float2 hf = __bfloat1622float2(hh);
    const float r0 = v0 - hf.x, r1 = v1 - hf.y;
    const __nv_bfloat162 ll = __floats2bfloat162_rn(r0, r1);
    h[q] = *reinterpret_cast<const uint32_t *>(&hh);
    lw[q] = *reinterpret_cast<const uint32_t *>(&ll);
    if (kLo2) {
      const float2 lf = __bfloat1622float2(ll);
      const __nv_bfloat162 l22 = __floats2bfloat162_rn(r0 - lf.x, r1 - lf.y);
      l2[q] = *reinterpret_cast<const uint32_t *>(&l22);
    }
  }
}

// Forward table rows into a shared-memory slot (MN-major, 128-byte
// swizzle): thread g writes 16 rows (half hf of its 32) of latitude k' =
// 64 kc + g mod 64 as two 16-byte chunks of 8 rows per part.
__device__ __forceinline__ void store_rows_smem(int g, int hf, unsigned char *a_hi, unsigned char *a_lo,
                                                const uint32_t (&h)[8], const uint32_t (&lw)[8]) {
  const int row = g & 63;                         // column k' inside the chunk
  const int cbase = 4 * ((g >> 6) & 1) + 2 * hf;  // 8-row chunk index inside the 64-row M block
  const int hb = (g >> 6) >> 1;                   // 64-row M block of the 128-row tile
#pragma unroll
  for (int q = 0; q < 2; q++) {
    const uint32_t off = (uint32_t)hb * 8192u + (uint32_t)(row >> 3) * 1024u + (uint32_t)(row & 7) * 128u +
                         ((uint32_t)((cbase + q) ^ (row & 7)) << 4);
    *reinterpret_cast<uint4 *>(a_hi + off) = make_uint4(h[4 * q], h[4 * q + 1], h[4 * q + 2], h[4 * q + 3]);
    *reinterpret_cast<uint4 *>(a_lo + off) = make_uint4(lw[4 * q], lw[4 * q + 1], lw[4 * q + 2], lw[4 * q + 3]);
  }
}

template <int kMode, bool kSplit, bool kGen, bool kWAdj = false>
__global__ void __launch_bounds__(kGen ? kThreadsGen : kThreads, 1)
tc_persistent_kernel(const __grid_constant__ TcParams P) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = align1024(smem_raw);
  __shared__ uint64_t full_bar[kMaxStages], empty_bar[kMaxStages], tfull[2], tempty[2];
  __shared__ uint32_t tmem_slot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t acc_cols = (uint32_t)tmem_cols_for(P.Nmax);
  const uint32_t ncols = 2 * acc_cols;
  const uint32_t sbytes = stage_bytes(kMode, kSplit, P.Nmax);
  const int S = P.stages;

  if (warp == 2) tmem_alloc(&tmem_slot, ncols);
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; s++) {
      mbar_init(&full_bar[s], kGen ? 1 + 8 : 1);  // + the 8 generator warps
      mbar_init(&empty_bar[s], 1);
    }
    for (int i = 0; i < 2; i++) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 4);
    }
    mbar_fence_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    // TMA producer
    for (int s = 0; s < P.nseg; s++) {
      tma_prefetch_desc(&P.maps[s].a_hi);
      tma_prefetch_desc(&P.maps[s].b_hi);
    }
    uint32_t g = 0;
    for (TileWalk<kMode> w(P); w.more(P);) {
      const TileInfo ti = w.take(P);
      const uint32_t tx = chunk_tx_bytes<kMode, kSplit, kGen>(ti);
      for (int kc = 0; kc < ti.nk; kc++, g++) {
        const int s = (int)(g % (uint32_t)S);
        const uint32_t use = g / (uint32_t)S;
        if (use > 0) mbar_wait(&empty_bar[s], (use - 1) & 1, P.err);
        unsigned char *st = base + (size_t)s * sbytes;
        mbar_arrive_expect_tx(&full_bar[s], tx);
        load_chunk<kMode, kSplit, kGen>(st, ti, kc, P.Nmax, P.maps[ti.s], &full_bar[s]);
      }
    }
  } else if (kMode == kFilt && kGen && warp >= 8) {
    // filter weights in their real form, generated per K chunk from the
    // complex W[l][o][i]: row n = 2 o + a of the B operand multiplies
    // (Re x_i, Im x_i) by (Re W, -Im W) (a = 0) or (Im W, Re W) (a = 1);
    // zero past Cout and Cin.  bf16 hi/lo in the TMA SWIZZLE_128B K-major
    // layout (row n at 128 n bytes, 16-byte chunk q at q ^ (n mod 8)).
    // Thread item (o, q): 4 input channels of output channel o, both rows.
    // Two chunks' weights are in flight in two register sets: the loads of
    // chunk g + 2 are issued once chunk g is built, so they have the build
    // of chunk g + 1 to land (the stages are usually free by the time the
    // builders reach them, so one set would leave the load latency exposed).
    constexpr int kItems = 4;  // (Nt / 2) x 8 items <= 1024 over 256 threads
    const int gtid = threadIdx.x - 256;
    const int na = a_count(kMode, kSplit);
    const uint32_t bb = b_bytes_of(kMode, P.Nmax);
    TileWalk<kMode> w(P);
    TileInfo ti{};  // the walker's chunk (ti, kc): the last one fetched
    ti.nk = 0;
    int kc = -1;
    auto next = [&]() {
      kc++;
      while (kc >= ti.nk) {
        if (!w.more(P)) return false;
        ti = w.take(P);
        kc = 0;
      }
      return true;
    };
    auto fetch = [&](float4 (&wv)[kItems][2]) {
      const float2 *Wl = P.W + (int64_t)ti.l * P.cout * P.cin;
#pragma unroll
      for (int u = 0; u < kItems; u++) {
        const int e = gtid + 256 * u;
        const int o = (ti.n0 >> 1) + (e >> 3), i0 = kc * (kKc / 2) + 4 * (e & 7);
        wv[u][0] = wv[u][1] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (kWAdj) {
          // the adjoint filter: conj(W[l][i][o]), input channels i0 .. i0 + 3
          if (e < ti.Nt * 4 && o < P.cout) {
            float2 t4[4];
#pragma unroll
            for (int c = 0; c < 4; c++) {
              const float2 w = i0 + c < P.cin ? __ldg(Wl + (int64_t)(i0 + c) * P.cout + o) : make_float2(0.f, 0.f);
              t4[c] = make_float2(w.x, -w.y);
            }
            wv[u][0] = make_float4(t4[0].x, t4[0].y, t4[1].x, t4[1].y);
            wv[u][1] = make_float4(t4[2].x, t4[2].y, t4[3].x, t4[3].y);
          }
          continue;
        }
        if (e < ti.Nt * 4 && o < P.cout) {
          const float2 *src = Wl + (int64_t)o * P.cin + i0;
          if (i0 + 4 <= P.cin && (P.cin & 1) == 0) {
            wv[u][0] = __ldg(reinterpret_cast<const float4 *>(src));
            wv[u][1] = __ldg(reinterpret_cast<const float4 *>(src) + 1);
          } else {
            float2 t4[4];
#pragma unroll
            for (int c = 0; c < 4; c++) t4[c] = i0 + c < P.cin ? __ldg(src + c) : make_float2(0.f, 0.f);
            wv[u][0] = make_float4(t4[0].x, t4[0].y, t4[1].x, t4[1].y);
            wv[u][1] = make_float4(t4[2].x, t4[2].y, t4[3].x, t4[3].y);
          }
        }
      }
    };
    // builds chunk g (tile tb, chunk kb) from wv into its stage
    auto build = [&](const float4 (&wv)[kItems][2], const TileInfo &tb, int kb, uint32_t g) {
      const int s = (int)(g % (uint32_t)S);
      const uint32_t use = g / (uint32_t)S;
      if (use > 0) mbar_wait(&empty_bar[s], (use - 1) & 1, P.err);
      unsigned char *bh = base + (size_t)s * sbytes + na * kABytes, *bl = bh + bb;
      const int kcov = min(kKc, (2 * P.cin - kb * kKc + 15) / 16 * 16);  // real K the chunk's MMAs read
#pragma unroll
      for (int u = 0; u < kItems; u++) {
        const int e = gtid + 256 * u;
        // items past the last K step the MMAs issue (16-column steps up to
        // 2 Cin) would build zero weights that nothing reads
        if (e >= tb.Nt * 4 || 8 * (e & 7) >= kcov) continue;
        const int q = e & 7;
        const float wr[4] = {wv[u][0].x, wv[u][0].z, wv[u][1].x, wv[u][1].z};
        const float wi[4] = {wv[u][0].y, wv[u][0].w, wv[u][1].y, wv[u][1].w};
#pragma unroll
        for (int a = 0; a < 2; a++) {
          const int n = 2 * (e >> 3) + a;
          uint32_t h[4], r[4];
#pragma unroll
          for (int c = 0; c < 4; c++) {
            const float v0 = a ? wi[c] : wr[c];   // multiplies Re x_i
            const float v1 = a ? wr[c] : -wi[c];  // multiplies Im x_i
            const __nv_bfloat162 hh = __floats2bfloat162_rn(v0, v1);
            const float2 hf = __bfloat1622float2(hh);
            const __nv_bfloat162 ll = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
            h[c] = *reinterpret_cast<const uint32_t *>(&hh);
            r[c] = *reinterpret_cast<const uint32_t *>(&ll);
          }
          const uint32_t off = (uint32_t)n * 128u + ((uint32_t)(q ^ (n & 7)) << 4);
          *reinterpret_cast<uint4 *>(bh + off) = make_uint4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<uint4 *>(bl + off) = make_uint4(r[0], r[1], r[2], r[3]);
        }
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&full_bar[s]);
    };
    float4 wa[kItems][2], wb[kItems][2];
    // chunk g in the current set (cur tile tc / chunk kcur), chunk g + 1 in
    // the other (tile tn / chunk kn) while have_n
    bool have = next();
    TileInfo tc = ti, tn{};
    int kcur = kc, kn = 0;
    if (have) fetch(wa);
    bool have_n = have && next();
    if (have_n) {
      tn = ti;
      kn = kc;
      fetch(wb);
    }
    // one step: build chunk g from cur, then load chunk g + 2 into cur
    auto step = [&](float4 (&cur)[kItems][2], uint32_t g) {
      build(cur, tc, kcur, g);
      have = have_n;
      tc = tn;
      kcur = kn;
      have_n = have && next();
      if (have_n) {
        tn = ti;
        kn = kc;
        fetch(cur);
      }
    };
    for (uint32_t g = 0; have; g += 2) {
      step(wa, g);
      if (!have) break;
      step(wb, g + 1);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    uint32_t g = 0, it = 0;
    for (TileWalk<kMode> w(P); w.more(P); it++) {
      const TileInfo ti = w.take(P);
      // B MN-major for the Legendre modes; A MN-major for the inverse
      const uint32_t idesc = idesc_bf16_f32(kRows, ti.Nt, kMode != kFilt) | (kMode == kInv ? 1u << 15 : 0u);
      const int acc = (int)(it & 1);
      const uint32_t use_a = it >> 1;
      if (use_a > 0) mbar_wait(&tempty[acc], (use_a - 1) & 1, P.err);
      tc_fence_after();
      const uint32_t tacc = tmem + (uint32_t)acc * acc_cols;
      for (int kc = 0; kc < ti.nk; kc++, g++) {
        const int s = (int)(g % (uint32_t)S);
        const uint32_t use = g / (uint32_t)S;
        mbar_wait(&full_bar[s], use & 1, P.err);
        tc_fence_after();
        // filter: K steps past 2 Cin meet zero weights (and another member's columns)
        const int nks = kMode == kFilt ? min(kKc / 16, (2 * P.cin - kc * kKc + 15) / 16) : kKc / 16;
        issue_chunk<kMode, kSplit, kGen>(base + (size_t)s * sbytes, P.Nmax, tacc, idesc, kc == 0, nks);
        mma_commit(&empty_bar[s]);
      }
      if (ti.nk > 0)
        mma_commit(&tfull[acc]);
      else
        mbar_arrive(&tfull[acc]);
    }
  } else if (warp >= 4 && warp < 8) {
    // epilogue (the inverse's staging buffers: 8 KB per warp, 1024-aligned)
    const int q4 = warp - 4;
    unsigned char *stg = base + P.epi_off + q4 * (kMode == kFilt ? 4096 : 8192);
    uint32_t it = 0;
    for (TileWalk<kMode> w(P); w.more(P); it++) {
      const TileInfo ti = w.take(P);
      const int acc = (int)(it & 1);
      mbar_wait(&tfull[acc], (it >> 1) & 1, P.err);
      tc_fence_after();
      epilogue<kMode>(P, ti, tmem + (uint32_t)acc * acc_cols, q4, lane, ti.nk == 0, stg, 2);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[acc]);
    }
    if (lane == 0) bulk_wait<0>();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

// ---------------------------------------------------------------------------
// Legendre contractions with the table generated on chip.  The K dimension
// of a tile (latitudes k' for the forward, rows i of the (m, p) block for
// the inverse) runs in table chunks of 64 (A, built by the generator warps
// into one of two slots) and data stages of 32 (B, loaded by TMA into a
// ring of as many stages as shared memory holds); each table chunk meets
// the two data stages of its K range (one when the range ends inside it).
//   kFwd:  D[i][c]  = sum_k' T[m][p][i][k'] F[m][p][k'][c]   (A MN-major)
//   kInv:  D[k'][c] = sum_i  T[m][p][i][k'] S[(m + p + 2i) M + m][c]   (A K-major)
// B is MN-major (64-column boxes of 32 K rows, 128-byte swizzle).
// ---------------------------------------------------------------------------

// Data stages (32 K rows each) of a tile: those that hold rows of its K range.
template <int kMode>
__device__ __forceinline__ int gen_halves(const TcParams &P, const TileInfo &ti) {
  const int kext = kMode == kFwd ? P.seg[ti.s].Kh : leg_rows(P.seg[ti.s].L, ti.m, ti.p);
  return (kext + kKb - 1) / kKb;
}

__host__ __device__ inline uint32_t gen_box_bytes() { return 64u * kKb * 2u; }  // 64 columns x kKb rows, bf16
__host__ __device__ inline uint32_t gen_stage_bytes(bool split, int Nt) {
  return (uint32_t)(split ? 2 : 1) * (uint32_t)((Nt + 63) / 64) * gen_box_bytes();
}

// TMA loads of data stage h (K rows kKb h .. kKb h + kKb - 1) of a tile.
template <int kMode, bool kSplit>
__device__ __forceinline__ void gen_load_half(unsigned char *st, const TileInfo &ti, int h, int Nmax,
                                              const SegMaps &mp, uint64_t *bar) {
  const uint32_t bx = gen_box_bytes();
  const uint32_t half_b = (uint32_t)((Nmax + 63) / 64) * bx;
  unsigned char *b_hi = st, *b_lo = st + half_b;
  const int nbox = (ti.Nt + 63) / 64;
  for (int j = 0; j < nbox; j++) {
    if (kMode == kFwd) {
      // folded data as (column, 2m + p, k'): kKb rows k' of one (m, p)
      tma_load_3d(b_hi + j * bx, &mp.b_hi, bar, ti.b_col0 + 64 * j, ti.b_row0, h * kKb);
      if (kSplit) tma_load_3d(b_lo + j * bx, &mp.b_lo, bar, ti.b_col0 + 64 * j, ti.b_row0, h * kKb);
    } else {
      // internal rows as (column, m, l) with every second l: rows
      // l = m + p + 2 i, i = kKb h .. kKb h + kKb - 1, of one (m, p) block
      tma_load_3d(b_hi + j * bx, &mp.b_hi, bar, ti.b_col0 + 64 * j, ti.m, ti.b_row0 + 2 * h * kKb);
      if (kSplit) tma_load_3d(b_lo + j * bx, &mp.b_lo, bar, ti.b_col0 + 64 * j, ti.m, ti.b_row0 + 2 * h * kKb);
    }
  }
}

// MMAs of one data stage against part hh (K kKb hh .. kKb hh + kKb - 1) of
// the table slot, K steps of 16.  Forward: A from the shared-memory slot a
// (MN-major), T_hi D_hi + T_lo D_hi (+ T_hi D_lo when split).  Inverse: A
// from tensor memory at column a_col, T_hi D_hi + T_lo D_hi (+ T_lo2 D_hi +
// T_hi D_lo when split).
template <int kMode, bool kSplit>
__device__ __forceinline__ void gen_issue_half(const unsigned char *a, uint32_t a_col, int hh, const unsigned char *b,
                                               int Nmax, uint32_t tmem, uint32_t idesc, bool first) {
  const uint32_t half_b = (uint32_t)((Nmax + 63) / 64) * gen_box_bytes();
  const unsigned char *b_hi = b, *b_lo = b + half_b;
#pragma unroll
  for (int s = 0; s < kKb / 16; s++) {
    const int ks = (kKb / 16) * hh + s;  // K step of 16 inside the 64-K table chunk
    const uint32_t acc = (first && s == 0) ? 0u : 1u;
    const uint64_t bh = desc_mnmajor_sw128(b_hi + s * 2048, gen_box_bytes(), 1024);
    if (kMode == kFwd) {
      const uint64_t ah = desc_mnmajor_sw128(a + ks * 2048, 8192, 1024);
      const uint64_t al = desc_mnmajor_sw128(a + kABytes + ks * 2048, 8192, 1024);
      mma_bf16(tmem, ah, bh, idesc, acc);
      mma_bf16(tmem, al, bh, idesc, 1u);
      if (kSplit) mma_bf16(tmem, ah, desc_mnmajor_sw128(b_lo + s * 2048, gen_box_bytes(), 1024), idesc, 1u);
    } else {
      // 8 columns (16 bf16 of K) per step; parts 32 columns apart
      const uint32_t ah = a_col + (uint32_t)ks * 8u;
      mma_bf16_ta(tmem, ah, bh, idesc, acc);
      mma_bf16_ta(tmem, ah + 32u, bh, idesc, 1u);
      if (kSplit) {
        mma_bf16_ta(tmem, ah + 64u, bh, idesc, 1u);
        mma_bf16_ta(tmem, ah, desc_mnmajor_sw128(b_lo + s * 2048, gen_box_bytes(), 1024), idesc, 1u);
      }
    }
  }
}

template <int kMode, bool kSplit>
__global__ void __launch_bounds__(kThreadsGen, 1) tc_gen_kernel(const __grid_constant__ TcParams P) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = align1024(smem_raw);
  __shared__ uint64_t a_full[kASlots], a_empty[kASlots], b_full[kMaxBStages], b_empty[kMaxBStages], tfull[2],
      tempty[2];
  __shared__ uint32_t tmem_slot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the inverse holds its table slots in tensor memory beside the two
  // accumulators; the forward's slots are in shared memory
  constexpr bool kTA = kMode == kInv;
  const uint32_t acc_cols = kTA ? kTmemAccStride : (uint32_t)tmem_cols_for(P.Nmax);
  const uint32_t ncols = kTA ? 512u : 2 * acc_cols;
  const uint32_t bsb = gen_stage_bytes(kSplit, P.Nmax);
  const int SB = P.stages;
  unsigned char *abase = base;
  unsigned char *bbase = base + (kTA ? 0u : kASlots * kASlotBytes);

  if (warp == 2) tmem_alloc(&tmem_slot, ncols);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kASlots; s++) {
      mbar_init(&a_full[s], 8);  // the 8 generator warps
      mbar_init(&a_empty[s], 1);
    }
    for (int s = 0; s < SB; s++) {
      mbar_init(&b_full[s], 1);
      mbar_init(&b_empty[s], 1);
    }
    for (int i = 0; i < 2; i++) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 4);
    }
    mbar_fence_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    // TMA producer of the data stages
    for (int s = 0; s < P.nseg; s++) tma_prefetch_desc(&P.maps[s].b_hi);
    uint32_t g = 0;
    for (TileWalk<kMode> w(P); w.more(P);) {
      const TileInfo ti = w.take(P);
      const int nh = gen_halves<kMode>(P, ti);
      const uint32_t tx = gen_stage_bytes(kSplit, ti.Nt);
      for (int h = 0; h < nh; h++, g++) {
        const int s = (int)(g % (uint32_t)SB);
        const uint32_t use = g / (uint32_t)SB;
        if (use > 0) mbar_wait(&b_empty[s], (use - 1) & 1, P.err);
        mbar_arrive_expect_tx(&b_full[s], tx);
        gen_load_half<kMode, kSplit>(bbase + (size_t)s * bsb, ti, h, P.Nmax, P.maps[ti.s], &b_full[s]);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    uint32_t ga = 0, gb = 0, it = 0;
    for (TileWalk<kMode> w(P); w.more(P); it++) {
      const TileInfo ti = w.take(P);
      uint32_t idesc = idesc_bf16_f32(kRows, ti.Nt, true);
      if (kMode == kFwd) idesc |= 1u << 15;  // the generated forward table enters MN-major
      const int acc = (int)(it & 1);
      const uint32_t use_a = it >> 1;
      if (use_a > 0) mbar_wait(&tempty[acc], (use_a - 1) & 1, P.err);
      tc_fence_after();
      const uint32_t tacc = tmem + (uint32_t)acc * acc_cols;
      const int nh = gen_halves<kMode>(P, ti);
      for (int c = 0; c < (nh + kBPerA - 1) / kBPerA; c++, ga++) {
        const int sa = (int)(ga % kASlots);
        mbar_wait(&a_full[sa], (ga / kASlots) & 1, P.err);
        tc_fence_after();
        for (int hh = 0; hh < kBPerA && kBPerA * c + hh < nh; hh++, gb++) {
          const int sb = (int)(gb % (uint32_t)SB);
          mbar_wait(&b_full[sb], (gb / (uint32_t)SB) & 1, P.err);
          tc_fence_after();
          gen_issue_half<kMode, kSplit>(abase + (size_t)sa * kASlotBytes, tmem + a_tmem_col(sa), hh,
                                        bbase + (size_t)sb * bsb, P.Nmax, tacc, idesc, c == 0 && hh == 0);
          mma_commit(&b_empty[sb]);
        }
        mma_commit(&a_empty[sa]);
      }
      if (nh > 0)
        mma_commit(&tfull[acc]);
      else
        mbar_arrive(&tfull[acc]);
    }
  } else if (warp >= 4 && warp < 8) {
    // epilogue (4 KB of staging per buffer and warp, 1024-aligned)
    const int q4 = warp - 4;
    unsigned char *stg = base + P.epi_off + q4 * 4096 * P.epi_nbuf;
    uint32_t it = 0;
    for (TileWalk<kMode> w(P); w.more(P); it++) {
      const TileInfo ti = w.take(P);
      const int acc = (int)(it & 1);
      mbar_wait(&tfull[acc], (it >> 1) & 1, P.err);
      tc_fence_after();
      epilogue<kMode>(P, ti, tmem + (uint32_t)acc * acc_cols, q4, lane, gen_halves<kMode>(P, ti) == 0, stg,
                      P.epi_nbuf);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[acc]);
    }
    if (lane == 0) bulk_wait<0>();
  } else if (warp >= 8) {
    // table generators.  Shared memory after the data ring: the current
    // tile's two-step coefficients (the next tile's are loaded into
    // registers meanwhile) and x^2 of every problem's latitudes.  Each
    // thread's seeds are loaded two table chunks ahead.
    const int gtid = threadIdx.x - 256;
    float4 *cs = reinterpret_cast<float4 *>(bbase + (size_t)SB * bsb);
    float2 *xs = reinterpret_cast<float2 *>(cs + P.ncmax);
    for (int s = 0; s < P.nseg; s++)
      for (int k = gtid; k < P.seg[s].Kh; k += 256)
        xs[P.seg[s].xoff + k] = make_float2(__ldg(P.seg[s].x2h + k), __ldg(P.seg[s].x2l + k));
    // seed cursor over the same chunk sequence
    TileWalk<kMode> pw(P);
    TileInfo pti{};
    int pkc = 0, pnk = 0;
    auto next_seed = [&]() {
      while (pkc >= pnk && pw.more(P)) {
        pti = pw.take(P);
        pkc = 0;
        pnk = (gen_halves<kMode>(P, pti) + kBPerA - 1) / kBPerA;
      }
      if (pkc >= pnk) return make_float2(0.f, 0.f);
      return gen_seed<kMode>(P.seg[pti.s], pti, pkc++, gtid);
    };
    float2 sd0 = next_seed(), sd1 = next_seed();
    auto coef_range = [&](const TileInfo &ti, int &ibase, int &ncoef) {
      // forward: the tile's 128 rows (+ 4 past its end), inverse: every row
      ibase = kMode == kFwd ? ti.r0 : 0;
      ncoef = kMode == kFwd ? 2 * kKc + 4 : kKc * ((gen_halves<kMode>(P, ti) + kBPerA - 1) / kBPerA) + 4;
    };
    // coefficients of the next tile with chunks (cursor cw) into registers
    TileWalk<kMode> cw(P);
    auto coef_load = [&](float4 (&cr)[kCoefPerThread]) {
#pragma unroll
      for (int u = 0; u < kCoefPerThread; u++) cr[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      TileInfo ti{};
      bool got = false;
      while (!got && cw.more(P)) {
        ti = cw.take(P);
        got = gen_halves<kMode>(P, ti) > 0;
      }
      if (!got) return;
      const SegArgs &sg = P.seg[ti.s];
      int ibase, ncoef;
      coef_range(ti, ibase, ncoef);
      const float4 *src = sg.coef + (int64_t)(ti.m * 2 + ti.p) * sg.ldC;
#pragma unroll
      for (int u = 0; u < kCoefPerThread; u++) {
        const int e = gtid + 256 * u;
        if (e < ncoef && ibase + e < sg.ldC) cr[u] = __ldg(src + ibase + e);
      }
    };
    float4 creg[kCoefPerThread];
    coef_load(creg);
    uint32_t ga = 0;
    for (TileWalk<kMode> w(P); w.more(P);) {
      const TileInfo ti = w.take(P);
      const int nka = (gen_halves<kMode>(P, ti) + kBPerA - 1) / kBPerA;
      if (nka == 0) continue;
      const SegArgs &sg = P.seg[ti.s];
      int ibase, ncoef;
      coef_range(ti, ibase, ncoef);
      asm volatile("bar.sync 2, 256;" ::: "memory");  // previous tile's coefficients no longer read
#pragma unroll
      for (int u = 0; u < kCoefPerThread; u++) {
        const int e = gtid + 256 * u;
        if (e < ncoef) cs[e] = creg[u];
      }
      asm volatile("bar.sync 2, 256;" ::: "memory");  // also orders the x^2 stores of the first tile
      coef_load(creg);
      for (int kc = 0; kc < nka; kc++, ga++) {
        const int sa = (int)(ga % kASlots);
        const uint32_t use = ga / kASlots;
        const float2 sd = sd0;
        sd0 = sd1;
        sd1 = next_seed();
        int kp, j;
        gen_coords<kMode>(ti, kc, gtid, kp, j);
        const float2 x2 = kp < sg.Kh ? xs[sg.xoff + kp] : make_float2(0.f, 0.f);
        if (use > 0) mbar_wait(&a_empty[sa], (use - 1) & 1, P.err);
        if (kTA) tc_fence_after();
        // the thread's 32 rows in two halves of 16
        float pa = sd.x, pb = sd.y;
        const float4 *cf = cs + (kSeedRows * j + 1 - ibase);
#pragma unroll 1
        for (int hf = 0; hf < 2; hf++) {
          uint32_t h[8], lw[8], l2[8];
          recur_rows<kTA && kSplit, 8>(pa, pb, x2, cf + 16 * hf, h, lw, l2);
          if constexpr (kTA) {
            // rows i = 64 kc + 32 (g / 128) + 16 hf + 0 .. 15 of lane
            // k' - r0 (this warp's quarter of the 128 lanes): 8 columns per part
            const uint32_t t = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + a_tmem_col(sa) +
                               16u * (uint32_t)(gtid >> 7) + 8u * (uint32_t)hf;
            tmem_st8(t, h);
            tmem_st8(t + 32u, lw);
            if (kSplit) tmem_st8(t + 64u, l2);
          } else {
            unsigned char *st = abase + (size_t)sa * kASlotBytes;
            store_rows_smem(gtid, hf, st, st + kABytes, h, lw);
          }
        }
        if constexpr (kTA) {
          tmem_wait_st();
          tc_fence_before();
        } else {
          fence_proxy_async_smem();
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&a_full[sa]);
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

// Transposes between the API layout xhat[b][l][m] (complex64) and the
// l-major forms of the tensor-core path, through 32 x 32 shared tiles so
// that both sides are read and written in contiguous runs.  One CTA (32 x 8
// threads) per (32 orders m, degree l, 32 fields b).
struct RowsT {
  const float *rows;   // finalize: FP32 rows [l M + m][ldr]
  float2 *xhat;        // finalize: destination; pack: source
  __nv_bfloat16 *shi, *slo;  // pack: split rows [l M + m][ldb]
  int L, M, B, ld;     // ld = ldr (finalize) or ldb (pack)
};

// A CTA moves kRowsL consecutive degrees of one (32 orders, 32 fields)
// tile, so that each thread has 16 loads in flight before the exchange.
constexpr int kRowsL = 4;
using RowsTile = float2[kRowsL][32][33];

// xhat[b][l][m] = rows[l M + m][2b, 2b + 1] for m <= l, zero for m > l.
__device__ __forceinline__ void finalize_tile(const RowsT &a, int mt, int lg, int bt, RowsTile &T) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int m0 = mt * 32, b0 = bt * 32;
  float2 v[kRowsL][4];
#pragma unroll
  for (int q = 0; q < kRowsL; q++) {
    const int l = lg * kRowsL + q;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const int m = m0 + ty + 8 * k, b = b0 + tx;
      v[q][k] = make_float2(0.f, 0.f);
      if (l < a.L && m <= l && m < a.M && b < a.B)
        v[q][k] = *reinterpret_cast<const float2 *>(a.rows + ((int64_t)l * a.M + m) * a.ld + 2 * b);
    }
  }
#pragma unroll
  for (int q = 0; q < kRowsL; q++)
#pragma unroll
    for (int k = 0; k < 4; k++) T[q][ty + 8 * k][tx] = v[q][k];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kRowsL; q++) {
    const int l = lg * kRowsL + q;
    if (l >= a.L) break;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const int b = b0 + ty + 8 * k, m = m0 + tx;
      if (b < a.B && m < a.M) a.xhat[((int64_t)b * a.L + l) * a.M + m] = T[q][tx][ty + 8 * k];
    }
  }
}

// split rows S[l M + m][2b, 2b + 1] = hi/lo of xhat[b][l][m], m <= l.
__device__ __forceinline__ void pack_tile(const RowsT &a, int mt, int lg, int bt, RowsTile &T) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int m0 = mt * 32, b0 = bt * 32;
  float2 v[kRowsL][4];
#pragma unroll
  for (int q = 0; q < kRowsL; q++) {
    const int l = lg * kRowsL + q;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const int b = b0 + ty + 8 * k, m = m0 + tx;
      v[q][k] = make_float2(0.f, 0.f);
      if (l < a.L && b < a.B && m < a.M && m <= l) v[q][k] = a.xhat[((int64_t)b * a.L + l) * a.M + m];
    }
  }
#pragma unroll
  for (int q = 0; q < kRowsL; q++)
#pragma unroll
    for (int k = 0; k < 4; k++) T[q][tx][ty + 8 * k] = v[q][k];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kRowsL; q++) {
    const int l = lg * kRowsL + q;
    if (l >= a.L) break;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const int m = m0 + ty + 8 * k, b = b0 + tx;
      if (m > l || m >= a.M || b >= a.B) continue;
      const int64_t o = ((int64_t)l * a.M + m) * a.ld + 2 * b;
      const float2 w = T[q][ty + 8 * k][tx];
      __nv_bfloat16 hr, lr, hi_, li;
      split_bf16(w.x, hr, lr);
      split_bf16(w.y, hi_, li);
      *reinterpret_cast<uint32_t *>(a.shi + o) = pack_bf16x2(hr, hi_);
      if (a.slo) *reinterpret_cast<uint32_t *>(a.slo + o) = pack_bf16x2(lr, li);
    }
  }
}

// Several problems per launch: CTA j belongs to problem s with blk0[s] <= j
// < blk0[s + 1]; mt, then the degree group, then bt vary slowest.
struct RowsTGroup {
  RowsT seg[kMaxSeg];
  int blk0[kMaxSeg + 1];
  int nseg;
};

template <bool kPack>
__global__ void __launch_bounds__(256) rows_transpose_kernel(const __grid_constant__ RowsTGroup g) {
  __shared__ RowsTile T;
  int s = 0;
  while (s + 1 < g.nseg && (int)blockIdx.x >= g.blk0[s + 1]) s++;
  const RowsT &a = g.seg[s];
  const int mtiles = (a.M + 31) / 32, lgroups = (a.L + kRowsL - 1) / kRowsL;
  int local = blockIdx.x - g.blk0[s];
  const int mt = local % mtiles;
  local /= mtiles;
  const int lg = local % lgroups;
  const int bt = local / lgroups;
  if (kPack)
    pack_tile(a, mt, lg, bt, T);
  else
    finalize_tile(a, mt, lg, bt, T);
}

// FP64 generation of the bf16 hi/lo table (layout [rows][Kp64], block (m, p)
// from row roff[2m + p]); same recurrence as the FP32 table.
__global__ void table_gen_bf16_kernel(__nv_bfloat16 *__restrict__ fhi, __nv_bfloat16 *__restrict__ flo,
                                      const int *__restrict__ roff, int Kp64, const double *__restrict__ xk,
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
    fhi[fo] = h;
    flo[fo] = lo;
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

// K ranges of the streamed-table tiles.  Phat_lm(cos theta) is evanescent
// for sin(theta) < m / (l + 1/2): it decays exponentially towards the
// poles, so for large m the table entries at polar latitudes are zero to
// working precision (the "polar optimisation" of Schaeffer, Efficient
// spherical harmonic transforms aimed at pseudospectral numerical
// simulations, G-cubed 2013).  A forward tile (128 rows i of one (m, p)
// block, K = latitudes k') starts its 64-wide K chunks at the first
// latitude with a table entry of magnitude >= 2^-40, rounded down to a
// multiple of 8 (TMA boxes start on 16-byte boundaries along k'); an
// inverse tile (128 latitudes, K = rows i) at the first such row, rounded
// the same way.  Near the equator every order oscillates, so the live range
// runs to the end of K.  The orthonormal Phat is of order one where it
// oscillates, so a coefficient loses at most 2^-40 times the sum of |data|
// over the rows left out: far below the split form's rounding (2^-17 per
// product).  A last chunk past K meets zeros (the data past K reads zero).
// One block per tile; out = [first, end) of the live K rows, or the last
// 8-row group of K when none is live (sums that are zero to working
// precision), or (0, 0) for a block without rows.
constexpr float kNegligible = 9.094947017729282e-13f;  // 2^-40

__global__ void tile_krange_kernel(const __nv_bfloat16 *__restrict__ thi, int Kp64, const int *__restrict__ roff,
                                   const LegTile *__restrict__ tiles, int inverse, int L, int Kh,
                                   int2 *__restrict__ out) {
  __shared__ int first, last;
  const LegTile t = tiles[blockIdx.x];
  const int nrows = leg_rows(L, t.m, t.p);
  int r_lo, r_hi, c_lo, c_hi, nK;
  if (!inverse) {
    // rows of the tile (the rows past its block are discarded), all latitudes
    r_lo = t.row;
    r_hi = t.row + min(128, nrows - t.r0);
    c_lo = 0;
    c_hi = Kh;
    nK = Kh;
  } else {
    // every row of the block, the tile's latitudes
    r_lo = roff[2 * t.m + t.p];
    r_hi = r_lo + nrows;
    c_lo = t.r0;
    c_hi = min(t.r0 + 128, Kh);
    nK = nrows;
  }
  if (threadIdx.x == 0) {
    first = 0x7fffffff;
    last = -1;
  }
  __syncthreads();
  const int w = c_hi - c_lo;
  const int64_t n = (int64_t)max(r_hi - r_lo, 0) * max(w, 0);
  int f = 0x7fffffff, l = -1;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    const int r = (int)(e / w), c = c_lo + (int)(e - (int64_t)r * w);
    const float v = fabsf(__bfloat162float(thi[(int64_t)(r_lo + r) * Kp64 + c]));
    if (v >= kNegligible) {
      const int k = inverse ? r : c;  // the K index of the entry
      f = min(f, k);
      l = max(l, k);
    }
  }
  if (f != 0x7fffffff) atomicMin(&first, f);
  if (l >= 0) atomicMax(&last, l);
  __syncthreads();
  if (threadIdx.x == 0) {
    int2 kr = make_int2(0, 0);
    if (nK > 0) {
      kr = last >= 0 ? make_int2(first / 8 * 8, last + 1) : make_int2((nK - 1) / 8 * 8, nK);
    }
    out[blockIdx.x] = kr;
  }
}

// FP64 recurrence seeds (one thread per (m, k')): at the first row l0 of
// every 32-row block of both parities, Phat_{l0} and Phat_{l0+2} rounded to
// FP32 (zero below the FP32 normal range).
__device__ __forceinline__ float seed_f32(double v) {
  return fabs(v) < 1.1754943508222875e-38 ? 0.f : (float)v;
}

__global__ void seed_gen_kernel(float2 *__restrict__ seeds, int NB, const double *__restrict__ xk,
                                const double *__restrict__ sk, const double *__restrict__ a,
                                const double *__restrict__ bcoef, const double *__restrict__ seedf, int L, int M,
                                int Kh) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (k >= Kh || m >= M) return;
  const double x = xk[k], s = sk[k];
  double pmm = 0.28209479177387814347;  // 1 / sqrt(4 pi)
  for (int i = 1; i <= m; i++) pmm *= seedf[i] * s;
  // window of Phat_l, Phat_{l+1}, Phat_{l+2}, Phat_{l+3}
  double w[4];
  w[0] = pmm;
  w[1] = (m + 1 < L) ? sqrt(2.0 * m + 3.0) * x * pmm : 0.0;
  for (int q = 2; q < 4; q++) {
    const int l = m + q;
    w[q] = 0.0;
    if (l < L) {
      const int64_t ci = (int64_t)l * M + m;
      w[q] = a[ci] * (x * w[q - 1] - bcoef[ci] * w[q - 2]);
    }
  }
  for (int l = m; l < L; l++) {
    const int d = l - m, p = d & 1, i = d >> 1;
    if ((i % kSeedRows) == 0)
      seeds[((int64_t)(m * 2 + p) * NB + i / kSeedRows) * Kh + k] = make_float2(seed_f32(w[0]), seed_f32(w[2]));
    double nn = 0.0;
    if (l + 4 < L) {
      const int64_t ci = (int64_t)(l + 4) * M + m;
      nn = a[ci] * (x * w[3] - bcoef[ci] * w[2]);
    }
    w[0] = w[1];
    w[1] = w[2];
    w[2] = w[3];
    w[3] = nn;
  }
}

}  // namespace

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
  }
  return n;
}

namespace {

// Column tiling of the 2B real columns: balanced tiles of at most `cap`
// (a multiple of 16) columns, each a multiple of 16.
void column_tiles(int B, int cap, int &Nt, int &nct) {
  const int C2 = 2 * B;
  nct = (C2 + cap - 1) / cap;
  Nt = ((C2 + nct - 1) / nct + 15) / 16 * 16;
}

template <int kMode, bool kSplit, bool kGen, bool kWAdj = false>
cudaError_t start_persistent(unsigned grid, size_t smem, const TcParams &P, cudaStream_t st) {
  auto fn = tc_persistent_kernel<kMode, kSplit, kGen, kWAdj>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fn<<<grid, threads_of(kGen), smem, st>>>(P);
  return cudaSuccess;
}

// Shared memory of one CTA: 1024 B of alignment slack, the stage ring and
// the generators' area; at most 227 KB with the static barriers.
constexpr size_t kSmemLimit = 227 * 1024 - 256;

// Shared memory of tc_persistent_kernel beyond its stage ring: the
// epilogue staging.
template <int kMode>
size_t extra_smem() {
  return kMode != kFilt ? 4 * 8192 : 4 * 4096;
}

// Shared memory of tc_gen_kernel beyond the table slots and the data ring,
// without the epilogue staging: the coefficients of one tile and x^2 of
// every problem's latitudes (whole KB); fills the generators' layout fields
// of P.  SIZE_MAX when the problems cannot be served.
size_t gen_extra_smem(TcParams &P) {
  int rows_max = 0;
  P.xtot = 0;
  for (int s = 0; s < P.nseg; s++) {
    rows_max = std::max(rows_max, leg_rows(P.seg[s].L, 0, 0));
    P.seg[s].xoff = P.xtot;
    P.xtot += P.seg[s].Kh;
  }
  P.ncmax = std::max(2 * kKc + 4, kKc * ((rows_max + kKc - 1) / kKc) + 4);
  if (P.ncmax > 256 * kCoefPerThread) return SIZE_MAX;
  size_t cbytes = sizeof(float4) * (size_t)P.ncmax + sizeof(float2) * (size_t)((P.xtot + 1) & ~1);
  return (cbytes + 1023) / 1024 * 1024;
}

// Whether the launch fits one CTA: two pipeline stages and the extra areas
// (streamed table and filter), or the two table slots, two data stages and
// the generators' areas (generated table).
template <int kMode>
bool persistent_fits(bool split, bool gen, TcParams &P) {
  if (gen && kMode != kFilt) {
    const size_t extra = gen_extra_smem(P);
    const size_t aslots = kMode == kInv ? 0 : kASlots * (size_t)kASlotBytes;
    if (kMode == kInv && P.Nmax > kTmemMaxN) return false;
    return extra != SIZE_MAX &&
           1024 + aslots + 2 * (size_t)gen_stage_bytes(split, P.Nmax) + extra + 4 * 4096 <= kSmemLimit;
  }
  return 1024 + 2 * (size_t)stage_bytes(kMode, split, P.Nmax) + extra_smem<kMode>() <= kSmemLimit;
}

template <bool kSplit>
cudaError_t start_gen(int mode, unsigned grid, size_t smem, const TcParams &P, cudaStream_t st) {
  auto fn = mode == kFwd ? tc_gen_kernel<kFwd, kSplit> : tc_gen_kernel<kInv, kSplit>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fn<<<grid, kThreadsGen, smem, st>>>(P);
  return cudaSuccess;
}

template <int kMode>
cudaError_t launch_persistent(bool split, bool gen, TcParams &P, const TcLaunch &cfg, cudaStream_t st) {
  if (P.ntiles <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min(P.ntiles, cfg.grid > 0 ? cfg.grid : sm_count());
  cudaError_t e;
  if (gen && kMode != kFilt) {
    const size_t sb = gen_stage_bytes(split, P.Nmax);
    const size_t extra = gen_extra_smem(P);
    if (extra == SIZE_MAX || (kMode == kInv && P.Nmax > kTmemMaxN)) return cudaErrorInvalidValue;
    // the forward's table slots are in shared memory, the inverse's in
    // tensor memory; two staging buffers per epilogue warp unless that
    // leaves fewer than four data stages, then one
    const size_t aslots = kMode == kInv ? 0 : kASlots * (size_t)kASlotBytes;
    size_t fixed = 1024 + aslots + extra;
    P.epi_nbuf = fixed + 4 * 8192 + 4 * sb <= kSmemLimit ? 2 : 1;
    fixed += 4 * 4096 * (size_t)P.epi_nbuf;
    if (fixed + 2 * sb > kSmemLimit) return cudaErrorInvalidValue;
    int stages = (int)std::min<size_t>(kMaxBStages, (kSmemLimit - fixed) / sb);
    if (cfg.stages >= 2) stages = std::min(stages, cfg.stages);
    P.stages = stages;
    // the epilogue staging follows the generators' area (all parts are whole KB)
    P.epi_off = (int)(aslots + (size_t)stages * sb + extra);
    const size_t smem = fixed + (size_t)stages * sb;
    e = split ? start_gen<true>(kMode, grid, smem, P, st) : start_gen<false>(kMode, grid, smem, P, st);
  } else {
    const size_t sb = stage_bytes(kMode, split, P.Nmax);
    const size_t extra = extra_smem<kMode>();
    if (1024 + 2 * sb + extra > kSmemLimit) return cudaErrorInvalidValue;
    int stages = (int)std::min<size_t>(kMaxStages, (kSmemLimit - 1024 - extra) / sb);
    if (cfg.stages >= 2) stages = std::min(stages, cfg.stages);
    P.stages = stages;
    // the epilogue staging follows the stage ring (stages are whole KB)
    P.epi_off = (int)((size_t)stages * sb);
    const size_t smem = 1024 + (size_t)stages * sb + extra;
    if constexpr (kMode == kFilt) {
      if (gen && P.wadj)
        e = split ? start_persistent<kFilt, true, true, true>(grid, smem, P, st)
                  : start_persistent<kFilt, false, true, true>(grid, smem, P, st);
      else if (gen)
        e = split ? start_persistent<kFilt, true, true>(grid, smem, P, st)
                  : start_persistent<kFilt, false, true>(grid, smem, P, st);
      else
        e = split ? start_persistent<kFilt, true, false>(grid, smem, P, st)
                  : start_persistent<kFilt, false, false>(grid, smem, P, st);
    } else {
      e = split ? start_persistent<kMode, true, false>(grid, smem, P, st)
                : start_persistent<kMode, false, false>(grid, smem, P, st);
    }
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

bool tc_encode_2d(CUtensorMap *tm, const void *ptr, int64_t cols, int64_t rows, int box_cols, int box_rows,
                  int64_t ld) {
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
  cuuint64_t gstr[1] = {(cuuint64_t)(ld > 0 ? ld : cols) * 2};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), gdim, gstr, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void **)&enc, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      enc = nullptr;
  }
  return enc;
}
}  // namespace

bool tc_encode_fold_f32(CUtensorMap *tm, const float *ptr, const FoldLayout &fl, int ld, int nmp, int Kh,
                        int box_cols) {
  auto enc = encoder();
  if (!enc || (box_cols != 32 && box_cols != 16) || ld % 16 != 0 || nmp % 2 != 0) return false;
  // 5-D view, strides increasing: (column in group, group, k', p, m) for
  // the (m, p)-major layouts, (column in group, p, group, k', m) for the
  // parity-paired one; a box is box_cols / 16 groups x 32 rows k' of one
  // (m, p), laid out in shared memory as 64-byte rows (k', group) with the
  // 64-byte swizzle (the box's inner extent equals the swizzle span)
  const cuuint64_t ng = (cuuint64_t)ld / 16, M = (cuuint64_t)nmp / 2;
  cuuint64_t gdim[5], gstr[4];
  cuuint32_t box[5];
  if (fl.cg) {
    if (fl.sp != 16 || fl.sk != 2 * (int64_t)ld || fl.sm != fl.sk * Kh) return false;
    const cuuint64_t d[5] = {16, 2, ng, (cuuint64_t)Kh, M};
    const cuuint64_t st[4] = {16 * 4, 32 * 4, (cuuint64_t)fl.sk * 4, (cuuint64_t)fl.sm * 4};
    const cuuint32_t b[5] = {16, 1, (cuuint32_t)box_cols / 16, 32, 1};
    std::copy(d, d + 5, gdim);
    std::copy(st, st + 4, gstr);
    std::copy(b, b + 5, box);
  } else {
    if (fl.sk != ld || fl.sp != fl.sk * Kh || fl.sm != 2 * fl.sp) return false;  // (m, p)-major
    const cuuint64_t d[5] = {16, ng, (cuuint64_t)Kh, 2, M};
    const cuuint64_t st[4] = {16 * 4, (cuuint64_t)fl.sk * 4, (cuuint64_t)fl.sp * 4, (cuuint64_t)fl.sm * 4};
    const cuuint32_t b[5] = {16, (cuuint32_t)box_cols / 16, 32, 1, 1};
    std::copy(d, d + 5, gdim);
    std::copy(st, st + 4, gstr);
    std::copy(b, b + 5, box);
  }
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<float *>(ptr), gdim, gstr, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tc_encode_rows_mn_bf16(CUtensorMap *tm, const __nv_bfloat16 *ptr, int ldx, int M, int L, int box_rows) {
  auto enc = encoder();
  if (!enc || !ptr || ldx % 64 != 0 || box_rows < 8 || box_rows > 256) return false;
  const cuuint64_t gdim[3] = {(cuuint64_t)ldx, (cuuint64_t)M, (cuuint64_t)L};
  const cuuint64_t gstr[2] = {(cuuint64_t)ldx * 2, (cuuint64_t)M * ldx * 2};
  const cuuint32_t box[3] = {64, (cuuint32_t)box_rows, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16 *>(ptr),
             const_cast<cuuint64_t *>(gdim), const_cast<cuuint64_t *>(gstr), const_cast<cuuint32_t *>(box),
             const_cast<cuuint32_t *>(es), CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tc_encode_pair_rows_f32(CUtensorMap *tm, const float *ptr, const FoldLayout &fl, int Kh, int M, int box_rows) {
  auto enc = encoder();
  if (!enc || !fl.cg || fl.sp != 16 || fl.sk % 4 != 0 || fl.sm != fl.sk * Kh || box_rows < 1 || box_rows > 256)
    return false;
  const cuuint64_t gdim[3] = {(cuuint64_t)fl.sk, (cuuint64_t)Kh, (cuuint64_t)M};
  const cuuint64_t gstr[2] = {(cuuint64_t)fl.sk * 4, (cuuint64_t)fl.sm * 4};
  const cuuint32_t box[3] = {32, 1, (cuuint32_t)box_rows};
  const cuuint32_t es[3] = {1, 1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(ptr), const_cast<cuuint64_t *>(gdim),
             const_cast<cuuint64_t *>(gstr), const_cast<cuuint32_t *>(box), const_cast<cuuint32_t *>(es),
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tc_encode_fold_bf16(CUtensorMap *tm, const __nv_bfloat16 *ptr, const FoldLayout &fl, int ld, int nmp, int Kh,
                         int box_rows) {
  auto enc = encoder();
  if (!enc) return false;
  if (!ptr) {
    *tm = CUtensorMap{};
    return true;
  }
  if (fl.cg || fl.sm != 2 * fl.sp) return false;  // rows (2m + p) at stride sp
  cuuint64_t gdim[3] = {(cuuint64_t)ld, (cuuint64_t)nmp, (cuuint64_t)Kh};
  cuuint64_t gstr[2] = {(cuuint64_t)fl.sp * 2, (cuuint64_t)fl.sk * 2};
  if (box_rows != 64 && box_rows != 32) return false;
  cuuint32_t box[3] = {64, 1, (cuuint32_t)box_rows};
  cuuint32_t es[3] = {1, 1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16 *>(ptr), gdim, gstr, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tc_encode_srows_bf16(CUtensorMap *tm, const __nv_bfloat16 *ptr, int ld, int M, int L, bool load,
                          int box_cols, int load_rows) {
  auto enc = encoder();
  if (!enc) return false;
  if (!load && box_cols != 32 && box_cols != 16) return false;
  if (load && load_rows != 64 && load_rows != 32) return false;
  if (!ptr) {
    *tm = CUtensorMap{};
    return true;
  }
  // dims (column, m, l); loads: 64 columns x every second l (load_rows of
  // them), stores: box_cols columns x 32 m of one l
  cuuint64_t gdim[3] = {(cuuint64_t)ld, (cuuint64_t)M, (cuuint64_t)L};
  cuuint64_t gstr[2] = {(cuuint64_t)ld * 2, (cuuint64_t)ld * 2 * M};
  cuuint32_t box_l[3] = {64, 1, 2 * (cuuint32_t)load_rows}, box_s[3] = {(cuuint32_t)box_cols, 32, 1};
  cuuint32_t es_l[3] = {1, 1, 2}, es_s[3] = {1, 1, 1};
  const CUtensorMapSwizzle sw = load ? CU_TENSOR_MAP_SWIZZLE_128B
                                     : (box_cols == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE);
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16 *>(ptr), gdim, gstr,
             load ? box_l : box_s, load ? es_l : es_s, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tc_encode_lrows_f32(CUtensorMap *tm, const float *ptr, int ldr, int M, int L, int box_cols) {
  auto enc = encoder();
  if (!enc || (box_cols != 32 && box_cols != 16) || ldr % 4 != 0) return false;
  if (!ptr) {
    *tm = CUtensorMap{};
    return true;
  }
  // dims (column, m, l); every second l, 32 of them per box; the box's
  // inner extent (128 or 64 bytes) equals its swizzle span
  cuuint64_t gdim[3] = {(cuuint64_t)ldr, (cuuint64_t)M, (cuuint64_t)L};
  cuuint64_t gstr[2] = {(cuuint64_t)ldr * 4, (cuuint64_t)ldr * 4 * M};
  cuuint32_t box[3] = {(cuuint32_t)box_cols, 1, 64};
  cuuint32_t es[3] = {1, 1, 2};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(ptr), gdim, gstr, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, box_cols == 32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tc_encode_lrows_bf16(CUtensorMap *tm, const __nv_bfloat16 *ptr, int ldx, int M, int L, int box_cols) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void **)&enc, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !enc)
      return false;
  }
  if (box_cols != 32 && box_cols != 16) return false;
  if (!ptr) {
    *tm = CUtensorMap{};
    return true;
  }
  // dims (column, m, l); every second l, 32 of them per box
  cuuint64_t gdim[3] = {(cuuint64_t)ldx, (cuuint64_t)M, (cuuint64_t)L};
  cuuint64_t gstr[2] = {(cuuint64_t)ldx * 2, (cuuint64_t)ldx * 2 * M};
  cuuint32_t box[3] = {(cuuint32_t)box_cols, 1, 64};
  cuuint32_t es[3] = {1, 1, 2};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16 *>(ptr), gdim, gstr, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, box_cols == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_table_gen_bf16(__nv_bfloat16 *fhi, __nv_bfloat16 *flo, const int *roff, int Kp64, const double *xk,
                                  const double *sk, const double *a, const double *b, const double *seed, int L, int M,
                                  int Kh, cudaStream_t st) {
  dim3 grid((Kh + 127) / 128, M);
  table_gen_bf16_kernel<<<grid, 128, 0, st>>>(fhi, flo, roff, Kp64, xk, sk, a, b, seed, L, M, Kh);
  return cudaGetLastError();
}

cudaError_t launch_tile_krange(const __nv_bfloat16 *thi, int Kp64, const int *roff, const LegTile *tiles, int ntiles,
                               int inverse, int L, int Kh, int2 *out, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  tile_krange_kernel<<<ntiles, 256, 0, st>>>(thi, Kp64, roff, tiles, inverse, L, Kh, out);
  return cudaGetLastError();
}

cudaError_t launch_seed_gen(void *seeds, int NB, const double *xk, const double *sk, const double *a,
                            const double *b, const double *seedf, int L, int M, int Kh, cudaStream_t st) {
  dim3 grid((Kh + 127) / 128, M);
  seed_gen_kernel<<<grid, 128, 0, st>>>(reinterpret_cast<float2 *>(seeds), NB, xk, sk, a, b, seedf, L, M, Kh);
  return cudaGetLastError();
}

cudaError_t launch_leg_tc_group(int inverse, const TcLegItem *items, int n, const TcLaunch &cfg, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (n > kMaxSeg) return cudaErrorInvalidValue;
  const bool split = items[0].T->split;
  const bool gen = inverse ? items[0].T->gen_inv : items[0].T->gen_fwd;
  for (int i = 0; i < n; i++) {
    if (items[i].T->split != split || (inverse ? items[i].T->gen_inv : items[i].T->gen_fwd) != gen)
      return cudaErrorInvalidValue;
    if (items[i].Nt < 0 || items[i].Nt % 16 != 0 || items[i].Nt > 256) return cudaErrorInvalidValue;
  }
  // column tiles: the requested widths (or 256), narrowed until two
  // pipeline stages fit in shared memory
  const int caps[4] = {256, 192, 128, 64};
  for (int cap0 : caps) {
    const int cap = (gen && inverse) ? std::min(cap0, kTmemMaxN / 16 * 16) : cap0;
    TcParams P{};
    P.err = items[0].T->err;
    int nseg = 0, ntiles = 0;
    for (int i = 0; i < n; i++) {
      const TcLegItem &it = items[i];
      const TcPlanView &T = *it.T;
      if (it.ntiles <= 0 || it.B <= 0) continue;
      SegArgs &g = P.seg[nseg];
      g.L = T.L;
      g.M = T.M;
      g.Kh = T.Kh;
      g.B = it.B;
      column_tiles(it.B, std::min(it.Nt > 0 ? it.Nt : 256, cap), g.Nt, g.nct);
      g.tile0 = ntiles;
      g.tiles = it.tiles;
      g.fout = FwdOut{it.rows_hi, it.rows_lo, it.ldo, it.cin > 0 ? it.cin : 1, it.kx, it.rowsf, it.ldr};
      g.Gw = it.Gw;
      g.ldc = it.ldc;
      g.gpair = T.gpair;
      g.seeds = reinterpret_cast<const float2 *>(T.seeds);
      g.coef = T.coef;
      g.x2h = T.x2h;
      g.x2l = T.x2l;
      g.NB = T.NB;
      g.ldC = T.ldC;
      g.roff = T.roff;
      g.krange = gen ? nullptr : it.krange;
      SegMaps &mp = P.maps[nseg];
      if (!inverse) {
        mp.a_hi = T.tab_fwd_hi;
        mp.a_lo = T.tab_fwd_lo;
        // data: 64-row boxes for the streamed table's stages, 32-row boxes
        // for the generated table's data stages
        const bool box32 = gen && kKb == 32;
        mp.b_hi = box32 ? T.fh_hi : T.f_hi;
        mp.b_lo = split ? (box32 ? T.fh_lo : T.f_lo) : mp.b_hi;
        // store maps of the plan's l-major rows (used when the destination
        // is those rows)
        if (!it.rows_hi == !it.rowsf) return cudaErrorInvalidValue;  // exactly one destination
        if (it.rows_hi && (it.rows_hi != T.xrows_hi || it.ldo != T.ldx)) return cudaErrorInvalidValue;
        if (it.rowsf && (it.rowsf != T.frows || it.ldr != T.ldr)) return cudaErrorInvalidValue;
        mp.o32_hi = it.rowsf ? T.ro32 : T.xo32_hi;
        mp.o32_lo = T.xo32_lo;
        mp.o16_hi = it.rowsf ? T.ro16 : T.xo16_hi;
        mp.o16_lo = T.xo16_lo;
      } else {
        mp.a_hi = T.tab_inv_hi;
        mp.a_lo = T.tab_inv_lo;
        const bool box32 = gen && kKb == 32;
        mp.b_hi = box32 ? T.sh_hi : T.s_hi;
        mp.b_lo = split ? (box32 ? T.sh_lo : T.s_lo) : mp.b_hi;
        // the output maps describe the plan's FP32 workspace
        if (it.Gw != T.gw || it.ldc != T.gw_ldc) return cudaErrorInvalidValue;
        mp.o32_hi = T.g32;
        mp.o16_hi = T.g16;
      }
      P.Nmax = std::max(P.Nmax, g.Nt);
      ntiles += it.ntiles * g.nct;
      nseg++;
    }
    if (nseg == 0) return cudaSuccess;
    P.nseg = nseg;
    P.ntiles = ntiles;
    const bool fits = inverse ? persistent_fits<kInv>(split, gen, P) : persistent_fits<kFwd>(split, gen, P);
    if (!fits) continue;
    return inverse ? launch_persistent<kInv>(split, gen, P, cfg, st)
                   : launch_persistent<kFwd>(split, gen, P, cfg, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_leg_inv_tc(const TcPlanView &T, const LegTile *tiles, const int2 *krange, int ntiles, float *Gw,
                              int ldc, int B, cudaStream_t st) {
  TcLegItem it{};
  it.T = &T;
  it.tiles = tiles;
  it.krange = krange;
  it.ntiles = ntiles;
  it.B = B;
  it.Gw = Gw;
  it.ldc = ldc;
  return launch_leg_tc_group(1, &it, 1, TcLaunch{}, st);
}

cudaError_t launch_filter_tc(const TcPlanView &T, const void *ftiles, int nftiles, const CUtensorMap &ta_hi,
                             const CUtensorMap &ta_lo, const float2 *W, __nv_bfloat16 *s_hi, __nv_bfloat16 *s_lo,
                             int lds, int kx, int nwr, int Bm, int Cin, int Cout, int wadj, cudaStream_t st) {
  if (s_hi != T.srows_hi || lds != T.lds) return cudaErrorInvalidValue;  // the store maps describe these rows
  if (nftiles == 0 || Bm <= 0) return cudaSuccess;
  TcParams P{};
  P.nseg = 1;
  P.L = T.L;
  P.M = T.M;
  P.ntn = (2 * Cout + 255) / 256;
  P.Nt = ((2 * Cout + P.ntn - 1) / P.ntn + 15) / 16 * 16;
  P.Nmax = P.Nt;
  P.Bm = Bm;
  P.ntiles = nftiles * Bm * P.ntn;
  P.ftiles = reinterpret_cast<const FiltTile *>(ftiles);
  P.kx = kx;
  P.nwr = nwr;
  P.cin = Cin;
  P.cout = Cout;
  P.lds = lds;
  P.s_hi = s_hi;
  P.s_lo = s_lo;
  P.err = T.err;
  P.maps[0].a_hi = ta_hi;
  P.maps[0].a_lo = ta_lo;
  P.maps[0].o32_hi = T.so32_hi;
  P.maps[0].o32_lo = T.so32_lo;
  P.maps[0].o16_hi = T.so16_hi;
  P.maps[0].o16_lo = T.so16_lo;
  P.W = W;
  P.wadj = wadj;
  return launch_persistent<kFilt>(T.split, true, P, TcLaunch{}, st);
}

// A wait that nothing satisfies: one thread initialises a barrier for one
// arrival that never comes and waits on it with the given limit.
__global__ void stall_kernel(unsigned *err, uint64_t timeout_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  mbar_fence_init();
  mbar_wait(&bar, 0, err, timeout_ns);
}

cudaError_t launch_debug_stall(unsigned *err, int64_t timeout_ns, cudaStream_t st) {
  if (timeout_ns < 1 || timeout_ns > 2000000000ll) return cudaErrorInvalidValue;
  stall_kernel<<<1, 32, 0, st>>>(err, (uint64_t)timeout_ns);
  return cudaGetLastError();
}

cudaError_t launch_rows_transpose(bool pack, const RowsItem *items, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (n > kMaxSeg) return cudaErrorInvalidValue;
  RowsTGroup g{};
  int64_t blk = 0;
  for (int i = 0; i < n; i++) {
    const RowsItem &it = items[i];
    if (it.B <= 0) continue;
    const int s = g.nseg++;
    g.seg[s] = RowsT{it.rows, it.xhat, it.shi, it.slo, it.L, it.M, it.B, it.ld};
    g.blk0[s] = (int)blk;
    blk += (int64_t)((it.M + 31) / 32) * ((it.L + kRowsL - 1) / kRowsL) * ((it.B + 31) / 32);
  }
  g.blk0[g.nseg] = (int)blk;
  if (blk == 0) return cudaSuccess;
  if (blk > 0x7fffffff) return cudaErrorInvalidValue;
  if (pack)
    rows_transpose_kernel<true><<<(unsigned)blk, 256, 0, st>>>(g);
  else
    rows_transpose_kernel<false><<<(unsigned)blk, 256, 0, st>>>(g);
  return cudaGetLastError();
}

}  // namespace shtgb
