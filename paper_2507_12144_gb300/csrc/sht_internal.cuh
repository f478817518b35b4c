// Internal declarations of the shtgb CUDA library (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/sht.h"

namespace shtgb {

// NVTX range around a public entry point (host timeline of the enqueue;
// free when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

constexpr int kMaxRadices = 16;
constexpr int kMaxNlon = 8192;

// Factorisation of nlon into radix-2/3/4/5 Stockham stages.
struct RadixPlan {
  int n;
  int nstages;
  int r[kMaxRadices];
};

// One tile of a Legendre contraction: order m, parity p of l + m, first row
// (or latitude), and for the tensor-core kernels the row of its first
// operand (forward: table row roff[2m+p] + r0; inverse: the first degree
// m + p of the block).
struct __align__(16) LegTile {
  int m;
  int p;
  int r0;
  int row;
};

// Layout of a folded Fourier workspace (longitude coefficients E / O of
// ring pair k' for order m, parity p, fields as columns): row (m, p, k')
// starts at m sm + p sp + k' sk elements, and column n of a row sits at
// n + cg (n & ~15).
//   (m, p)-major ("classic"): sm = 2 Kh ld, sp = Kh ld, sk = ld, cg = 0;
//   ring-major: sm = 2 ld, sp = ld, sk = 2 mmax ld, cg = 0;
//   parity-paired: rows (m, k') of 2 ld elements in which 16-column groups
//     of the two parities alternate (sm = 2 Kh ld, sp = 16, sk = 2 ld,
//     cg = 1), so that E and O of 16 columns share one 128-byte line
//     (FP32).
// The longitude kernels take any layout whose 16-column groups hold the
// columns they access together; the tensor-core contractions address it
// through TMA maps built from the same strides.
struct FoldLayout {
  int64_t sm, sp, sk;
  int cg;
};
__host__ __device__ inline int64_t fold_row(const FoldLayout &fl, int m, int p, int k) {
  return (int64_t)m * fl.sm + p * fl.sp + (int64_t)k * fl.sk;
}
__host__ __device__ inline int64_t fold_col(const FoldLayout &fl, int64_t n) { return fl.cg ? n + (n & ~15) : n; }
inline FoldLayout classic_layout(int Kh, int ld) {
  return FoldLayout{2 * (int64_t)Kh * ld, (int64_t)Kh * ld, (int64_t)ld, 0};
}
inline FoldLayout ring_layout(int M, int ld) { return FoldLayout{2 * (int64_t)ld, (int64_t)ld, 2 * (int64_t)M * ld, 0}; }
// ld a multiple of 16
inline FoldLayout pair_layout(int Kh, int ld) { return FoldLayout{2 * (int64_t)Kh * ld, 16, 2 * (int64_t)ld, 1}; }

// Device-side view of the folded FP32 Legendre table.  For order m and
// parity p the rows are l = m + p + 2 i (i < nrows(m, p)), the columns are
// the northern half-rows k' = 0 .. Kh-1 (Kh = ceil(nlat / 2)), padded to Khp.
struct TableF32 {
  const float *data;
  const int64_t *off;  // [2 M] float offset of block (m, p)
  int Khp;
};

// Everything the tensor-core contractions of one plan need: TMA descriptors
// of the bf16 hi/lo Legendre table (layout [rows][Kp64] with block (m, p)
// at row roff[2m+p], read K-major by the forward and MN-major by the
// inverse), of the
// Fourier workspace F[(2m+p) Kh + k'][ldcb] (hi, lo) and of the internal
// coefficient rows S[l M + m][ldcb] (hi, lo, l-major), plus the error word.
struct TcPlanView {
  CUtensorMap tab_fwd_hi, tab_fwd_lo, tab_inv_hi, tab_inv_lo;  // bf16 table (streamed)
  CUtensorMap f_hi, f_lo, s_hi, s_lo;  // s: 3-D (column, m, l) loads of every second l
  CUtensorMap fh_hi, fh_lo, sh_hi, sh_lo;  // the same with 32-row boxes (generated-table kernel)
  CUtensorMap x_hi, x_lo;  // l-major forward output rows [L M][ldx] (bf16)
  CUtensorMap g32, g16;    // FP32 inverse output (folded workspace), store boxes 32 x 32, 16 x 32
  const float *gw;         // their base (the FP32 workspace), row stride and layout
  int gw_ldc;
  int gpair;               // 1: parity-paired layout (else (m, p)-major)
  CUtensorMap xo32_hi, xo32_lo, xo16_hi, xo16_lo;  // l-major rows [L][M][ldx], every second l, store boxes
  CUtensorMap so32_hi, so32_lo, so16_hi, so16_lo;  // internal rows S [L][M][ldcb], store boxes of 32 m
  CUtensorMap ro32, ro16;  // FP32 l-major rows of the API forward [L][M][ldr], every second l, store boxes
  const float *frows;      // their base and row stride (floats)
  int ldr;
  const __nv_bfloat16 *srows_hi;                    // their base and row stride
  int lds;
  const __nv_bfloat16 *xrows_hi;                    // their base and row stride
  int ldx;
  const int *roff;
  // on-chip Legendre table: FP32 seed pairs (float2) every 32 rows
  const void *seeds;
  const float4 *coef;        // two-step coefficients [(2m + p) ldC + i]
  const float *x2h, *x2l;    // x^2 = x2h + x2l per latitude
  int NB, ldC;
  int L, M, Kh;
  bool split;
  bool gen_fwd, gen_inv;  // generate the table on chip (per direction) instead of streaming it
  unsigned *err;
};

// 2-D bf16 map of rows x cols (row stride ld elements, default cols) with
// SWIZZLE_128B boxes box_cols x box_rows; columns past `cols` read as zero.
bool tc_encode_2d(CUtensorMap *tm, const void *ptr, int64_t cols, int64_t rows, int box_cols, int box_rows,
                  int64_t ld = 0);
// FP32 rows [nblocks][Kh][ldc] as a 3-D map with store boxes box_cols x 32
// (box_cols 32: 128-byte swizzle; 16: 64-byte swizzle).
// FP32 folded rows (layout fl, row length ld) as a 3-D map (column, 2m + p,
// k') with store boxes box_cols x 1 x 32 (box_cols 32: 128-byte swizzle;
// 16: 64-byte swizzle).
bool tc_encode_fold_f32(CUtensorMap *tm, const float *ptr, const FoldLayout &fl, int ld, int nmp, int Kh,
                        int box_cols);
// bf16 folded rows (layout fl, row length ld) as a 3-D map (column, 2m + p,
// k') with load boxes 64 x 1 x box_rows (box_rows 64 or 32; 128-byte swizzle).
bool tc_encode_fold_bf16(CUtensorMap *tm, const __nv_bfloat16 *ptr, const FoldLayout &fl, int ld, int nmp, int Kh,
                         int box_rows);
// bf16 l-major rows [L][M][ldx] as a 3-D map whose store boxes take box_cols
// columns of 32 rows l, l + 2, ..., l + 62 (element stride 2 along l).
bool tc_encode_lrows_bf16(CUtensorMap *tm, const __nv_bfloat16 *ptr, int ldx, int M, int L, int box_cols);
// FP32 l-major rows [L][M][ldr] as the same 3-D store view (32- or
// 16-column boxes, 128- or 64-byte swizzle).
bool tc_encode_lrows_f32(CUtensorMap *tm, const float *ptr, int ldr, int M, int L, int box_cols);
// The internal coefficient rows S [L][M][ld] (bf16, l-major) as a 3-D map
// (column, m, l): load = true: boxes of 64 columns x every second l
// (load_rows = 64 or 32 of them, 128-byte swizzle) for the inverse
// contraction; load = false: store boxes of box_cols columns x 32 m of one
// l (the filter's epilogue).
bool tc_encode_srows_bf16(CUtensorMap *tm, const __nv_bfloat16 *ptr, int ld, int M, int L, bool load,
                          int box_cols, int load_rows = 64);
// FP64 generation of the bf16 hi/lo table, layout [rows][Kp64] with block
// (m, p) from row roff[2m + p].
cudaError_t launch_table_gen_bf16(__nv_bfloat16 *fhi, __nv_bfloat16 *flo, const int *roff, int Kp64, const double *xk,
                                  const double *sk, const double *a, const double *b, const double *seed, int L, int M,
                                  int Kh, cudaStream_t st);
// K ranges of the streamed-table contractions, one int2 [first, end) per
// tile (inverse = 0: forward tiles, K = latitudes; 1: inverse tiles, K =
// rows i): from the first K row with a table entry of magnitude >= 2^-40
// (rounded down to a multiple of 8) to the end of K, read from the hi
// table at rows roff[2m + p] + i, pitch Kp64; (0, 0) for a block without rows.
cudaError_t launch_tile_krange(const __nv_bfloat16 *thi, int Kp64, const int *roff, const LegTile *tiles, int ntiles,
                               int inverse, int L, int Kh, int2 *out, cudaStream_t st);
// Seeds of the on-chip Legendre table (every 32 rows of every (m, p)),
// computed in FP64 and stored as FP32 pairs.
cudaError_t launch_seed_gen(void *seeds, int NB, const double *xk, const double *sk, const double *a,
                            const double *b, const double *seedf, int L, int M, int Kh, cudaStream_t st);
// Tensor-core filter from the l-major rows to the inverse's split rows.
// ftiles: (l, m0) pairs covering m <= l, m < M in steps of 128.
// ta: the forward rows (width = members x kx, row stride ldx); W: the
// complex weights [L][Cout][Cin] (device), turned into the real bf16 hi/lo
// form of each K chunk on chip; nwr = 2 Cout rounded to 16.  wadj = 1: the
// adjoint filter, output o from input i by conj(W[l][i][o]) with W
// [L][Cin][Cout].
cudaError_t launch_filter_tc(const TcPlanView &T, const void *ftiles, int nftiles, const CUtensorMap &ta_hi,
                             const CUtensorMap &ta_lo, const float2 *W, __nv_bfloat16 *s_hi, __nv_bfloat16 *s_lo,
                             int lds, int kx, int nwr, int Bm, int Cin, int Cout, int wadj, cudaStream_t st);
// Inverse contraction on the tensor cores from the bf16 internal rows to the
// FP32 folded workspace Gw[(2m+p) Kh + k'][ldc].
cudaError_t launch_leg_inv_tc(const TcPlanView &T, const LegTile *tiles, const int2 *krange, int ntiles, float *Gw,
                              int ldc, int B,
                              cudaStream_t st);
// One problem of a grouped tensor-core Legendre launch: a plan's view, its
// tiles, its batch, and the destination of the forward (the plan's l-major
// bf16 rows, rows[l M + m][ldo] with member b = f / cin at columns
// b kx + 2 (f mod cin), or its FP32 l-major rows rowsf) or of the inverse
// (Gw, ldc).  Nt = column tile width (multiple of 16, <= 256; 0 = balanced
// tiles of at most 256).
struct TcLegItem {
  const TcPlanView *T;
  const LegTile *tiles;
  int ntiles;
  // per tile of `tiles`: the K rows [x, y) that meet non-negligible
  // streamed-table entries (launch_tile_krange); nullptr: all of K
  const int2 *krange;
  int B, Nt;
  __nv_bfloat16 *rows_hi, *rows_lo;
  int ldo, cin, kx;
  float *rowsf;  // FP32 l-major rows (row l M + m, field f at 2f), stride ldr
  int ldr;
  float *Gw;
  int ldc;
};
// Launch shape of a persistent kernel: CTAs (0 = one per SM) and pipeline
// stages (0 = as many as fit).
struct TcLaunch {
  int grid;
  int stages;
};
// Up to 8 problems of equal precision and table source in one persistent
// launch (inverse = 0: forward contraction, 1: inverse).
cudaError_t launch_leg_tc_group(int inverse, const TcLegItem *items, int n, const TcLaunch &cfg, cudaStream_t st);
// Coalesced transposes of up to 8 problems per launch.
//   pack = false: xhat[b][l][m] = rows[l M + m][2b + {re, im}] (m <= l; zero
//                 for m > l), rows FP32 with row stride ld floats;
//   pack = true:  split bf16 rows S[l M + m][2b + {re, im}] (row stride ld)
//                 from xhat, m <= l.
struct RowsItem {
  const float *rows;
  float2 *xhat;
  __nv_bfloat16 *shi, *slo;
  int L, M, B, ld;
};
cudaError_t launch_rows_transpose(bool pack, const RowsItem *items, int n, cudaStream_t st);
// One kernel whose bounded barrier wait runs out (test hook).
cudaError_t launch_debug_stall(unsigned *err, int64_t timeout_ns, cudaStream_t st);
// Longitude analysis writing the folded Fourier workspace as bf16 hi/lo
// (same contract as launch_r2c).
cudaError_t launch_r2c_bf16(const float *x, __nv_bfloat16 *Fhi, __nv_bfloat16 *Flo, int nlat, int nlon, int M, int B,
                            FoldLayout fl, const float2 *twiddle, const RadixPlan &rp, const float *ring_scale,
                            int inverse_weights, cudaStream_t st);


// Record a failure message for sht_last_error_message() and return status.
sht_status_t fail(sht_status_t st, const std::string &msg);
// latitude nodes x = cos(theta_k), sin(theta_k) and weights w_k of a grid
// (the plan's grids; k = 0 is the northernmost row)
void grid_nodes(int grid, int nlat, std::vector<double> &x, std::vector<double> &s, std::vector<double> &w);
sht_status_t cuda_fail(cudaError_t err, const char *what);

// Number of l in parity class p at order m for lmax L.
__host__ __device__ inline int leg_rows(int L, int m, int p) {
  int n = L - m - p;
  return n > 0 ? (n + 1) / 2 : 0;
}

// ---------------------------------------------------------------------------
// Kernel launchers (each returns the launch status, nothing synchronises).
// ---------------------------------------------------------------------------

// Longitude analysis of pairs of rings (k, nlat-1-k):
//   F_k(m) = ring_scale[k] * c_m * sum_j x_kj e^{-2 pi i j m / nlon}
// folded by parity into Fw[m][p][k'][ldc] (p = 0: F_k + F_kbar, p = 1:
// F_k - F_kbar; the equator row of odd nlat goes to p = 0 alone).  c_m = 1
// when inverse_weights == 0, else the weight of the real inverse (1 for
// m = 0 and the Nyquist mode, 2 otherwise).  ring_scale may be NULL (= 1).
cudaError_t launch_r2c(const float *x, float *Fw, int nlat, int nlon, int M,
                       int B, FoldLayout fl, const float2 *twiddle,
                       const RadixPlan &rp, const float *ring_scale,
                       int inverse_weights, cudaStream_t st);

// Four-step register FFT versions of launch_r2c / launch_c2r for nlon = 45 P,
// P in {4, 8, 16, 32}.  The analysis writes FP32 (Fw != NULL) or bf16 hi
// (and lo when Flo != NULL) with row stride ldc elements.
bool fft45_supported(int nlon);
// SMs of the current device (queried once).
int sm_count();
// Both run as persistent kernels with bulk-copy staging when the input is
// 16-byte aligned (and, for the synthesis, in the parity-paired layout);
// err (may be NULL) receives the timeout code of their bounded waits.
cudaError_t launch_r2c45(const float *x, float *Fw, __nv_bfloat16 *Fhi, __nv_bfloat16 *Flo, int nlat, int nlon,
                         int M, int B, FoldLayout fl, const float2 *twiddle, const float *ring_scale, int inverse_weights,
                         cudaStream_t st, unsigned *err = nullptr);
cudaError_t launch_c2r45(const float *Gw, float *y, int nlat, int nlon, int M, int B, FoldLayout fl,
                         const float2 *twiddle, const float *ring_scale, int inverse_weights, cudaStream_t st,
                         unsigned *err = nullptr);
// FP32 parity-paired folded rows (layout fl, fl.cg set) as a 3-D map
// (column, k', m) whose load boxes take 32 columns (one 8-field group's E
// and O) of box_rows orders m of one ring pair, unswizzled.
bool tc_encode_pair_rows_f32(CUtensorMap *tm, const float *ptr, const FoldLayout &fl, int Kh, int M, int box_rows);
// bf16 l-major rows [L][M][ldx] as a 3-D map (column, m, l) whose load
// boxes take 64 columns of box_rows consecutive orders m of one degree l
// (128-byte swizzle; orders past M read as zero).
bool tc_encode_rows_mn_bf16(CUtensorMap *tm, const __nv_bfloat16 *ptr, int ldx, int M, int L, int box_rows);
// Weight gradient of the filter from the split bf16 l-major rows of
// g = ISHT^T(gy) (Cout channels per member, member blocks of kxa columns)
// and x = SHT(x) (Cin channels, blocks of kxb), both with row stride ldx:
// gW[l][o][i] (+)= sum_{b < nb, m <= l} g[b][o][l][m] conj(x[b][i][l][m]),
// FP32 complex [L][Cout][Cin]; accumulate = 0 overwrites.  g_lo / x_lo NULL:
// the single-part (BF16) operands.  Rows m > l of the buffers must be zero.
cudaError_t launch_dw_tc(const __nv_bfloat16 *g_hi, const __nv_bfloat16 *g_lo, const __nv_bfloat16 *x_hi,
                         const __nv_bfloat16 *x_lo, int ldx, float2 *gW, int L, int M, int nb, int Cin, int Cout,
                         int kxa, int kxb, int accumulate, unsigned *err, cudaStream_t st);

// One problem of a grouped longitude launch: the arguments of launch_r2c45
// (in = x; outf = Fw or hi/lo) or launch_c2r45 (in = Gw, outf = y).
struct Fft45Item {
  const float *in;
  float *outf;
  __nv_bfloat16 *hi, *lo;
  const float2 *twiddle;
  const float *ring_scale;
  FoldLayout fl;
  int nlat, nlon, M, B, inverse_weights;
};
constexpr int kMaxFftGroup = 8;
// Grouped launches of up to kMaxFftGroup problems (every nlon = 45 P, B >= 1)
// in one grid; bf16 selects the bf16 hi/lo output of the analysis.
cudaError_t launch_r2c45_grouped(const Fft45Item *items, int n, bool bf16, cudaStream_t st);
cudaError_t launch_c2r45_grouped(const Fft45Item *items, int n, cudaStream_t st);

// Longitude transforms of arbitrary latitude rows (distributed transform):
// F[r][m] = ring_scale[k0 + r mod nrows] sum_j x[r][j] e^{-2 pi i j m / nlon}
// for rows r < R, m < M; and y[r][j] = sum_m c_m Re(G[r][m] e^{2 pi i j m /
// nlon}).  Generic mixed-radix FFT (nlon factoring into 2, 3, 5).
cudaError_t launch_r2c_rows(const float *x, float2 *F, int64_t R, int nrows, int k0, int nlon, int M,
                            const float2 *twiddle, const RadixPlan &rp, const float *ring_scale, cudaStream_t st);
cudaError_t launch_c2r_rows(const float2 *G, float *y, int64_t R, int nlon, int M, const float2 *twiddle,
                            const RadixPlan &rp, cudaStream_t st);

// Longitude synthesis from folded Gw[m][p][k'][ldc]:
//   u_kj = ring_scale[k] * sum_m c_m Re(G_k(m) e^{2 pi i j m / nlon})
// with G_k = G_even + G_odd (north row k'), G_kbar = G_even - G_odd.
cudaError_t launch_c2r(const float *Gw, float *y, int nlat, int nlon, int M,
                       int B, FoldLayout fl, const float2 *twiddle,
                       const RadixPlan &rp, const float *ring_scale,
                       int inverse_weights, cudaStream_t st);

// Forward Legendre contraction, FP32 CUDA cores:
//   xhat[b][l][m] = sum_k' T[m][p][i][k'] Fw[m][p][k'][2b + {re, im}]
cudaError_t launch_leg_fwd_f32(const TableF32 &T, const LegTile *tiles,
                               int ntiles, const float *Fw, float2 *xhat,
                               int L, int M, int Kh, int ldc, int B,
                               cudaStream_t st);

// Inverse Legendre contraction, FP32 CUDA cores:
//   Gw[m][p][k'][2b + {re, im}] = sum_i T[m][p][i][k'] yhat[b][m + p + 2 i][m]
cudaError_t launch_leg_inv_f32(const TableF32 &T, const LegTile *tiles,
                               int ntiles, const float2 *yhat, float *Gw,
                               int L, int M, int Kh, int ldc, int B,
                               cudaStream_t st);

// One problem of a grouped FP32 Legendre launch (the arguments of
// launch_leg_fwd_f32: T, tiles, Fw -> xhat; or of launch_leg_inv_f32:
// T, tiles, yhat -> Gw).
constexpr int kMaxLegGroup = 8;
struct F32LegItem {
  TableF32 T;
  const LegTile *tiles;
  int ntiles;
  const float *Fw;
  float2 *xhat;
  const float2 *yhat;
  float *Gw;
  int L, M, Kh, ldc, B;
};
cudaError_t launch_leg_f32_group(int inverse, const F32LegItem *items, int n, cudaStream_t st);
// Zero fill of the l < m parts of up to kMaxLegGroup problems in one launch.
cudaError_t launch_zero_upper_group(float2 *const *xhat, const int *L, const int *M, const int64_t *B, int n,
                                    cudaStream_t st);

// Zero the l < m part of B dense [L][M] coefficient blocks.
cudaError_t launch_zero_upper(float2 *xhat, int L, int M, int64_t B,
                              cudaStream_t st);

// Spectral filter (adjoint = 0) or its input adjoint (adjoint = 1):
//   adjoint 0: y[b][o][l][m] = sum_i W[l][o][i] x[b][i][l][m]
//   adjoint 1: y[b][i][l][m] = sum_o conj(W[l][o][i]) x[b][o][l][m]
// Output is zero for m > l.
cudaError_t launch_filter(const float2 *x, const float2 *W, float2 *y, int L,
                          int M, int64_t Bm, int Cin, int Cout, int adjoint,
                          cudaStream_t st);

// Wt[l][i][o] = conj(W[l][o][i]) for W [L][Cout][Cin].
cudaError_t launch_transpose_conj(const float2 *W, float2 *Wt, int L, int Cout, int Cin, cudaStream_t st);
// Weight adjoint gW[l][o][i] (+)= sum_{b, m <= l} gy[b][o][l][m] conj(x[b][i][l][m])
// (accumulate = 0 overwrites).
cudaError_t launch_filter_dw(const float2 *gy, const float2 *x, float2 *gW,
                             int L, int M, int64_t Bm, int Cin, int Cout,
                             cudaStream_t st, int accumulate = 0);

// FP64 generation of the folded FP32 table on the device.
cudaError_t launch_table_gen_f32(float *table, const int64_t *off, int Khp,
                                 const double *xk, const double *sk,
                                 const double *a, const double *b,
                                 const double *seed, int L, int M, int Kh,
                                 cudaStream_t st);

}  // namespace shtgb

// Event record of the per-kernel profiler.
struct ProfileState {
  bool on = false;
  int capacity = 0;
  int used = 0;
  int64_t dropped = 0;
  std::vector<cudaEvent_t> start, stop;
  std::vector<int> kernel;
};

// The opaque plan.
struct sht_plan_s {
  ProfileState prof;
  int device = 0;
  int nlat = 0, nlon = 0, grid = 0, L = 0, M = 0, precision = 0;
  int64_t max_batch = 0;
  int Kh = 0;    // ceil(nlat / 2)
  int Khp = 0;   // Kh padded to a multiple of 16
  int ldc = 0;   // row stride (floats) of the folded Fourier workspace
  shtgb::FoldLayout lay_f{};  // layout of the workspace the analysis writes (FP32 ldc or bf16 ldcb rows)
  shtgb::FoldLayout lay_g{};  // layout of the FP32 workspace the synthesis reads
  shtgb::RadixPlan radix{};
  std::vector<double> x, s, w;  // nodes, sin(theta), latitude weights
  std::vector<int64_t> tab_off;  // host copy of the table offsets
  int64_t table_bytes = 0;
  int64_t workspace_bytes = 0;

  // device memory (all owned)
  unsigned *d_err = nullptr;   // error word of bounded device waits
  shtgb::TcPlanView tc{};      // tensor-core view (bf16 precisions)
  __nv_bfloat16 *d_tf_hi = nullptr, *d_tf_lo = nullptr;  // bf16 table (one layout for both directions)
  int table_source = 0;        // 0: streamed bf16 table, 1: on-chip recurrence, 2: forward streamed, inverse on chip
  void *d_seeds = nullptr;     // recurrence seeds of the on-chip table
  float4 *d_coef = nullptr;    // two-step recurrence coefficients [(2m + p) ldC + i]
  float *d_x2h = nullptr, *d_x2l = nullptr;  // squared latitudes as FP32 hi + lo
  int ldcb = 0;                // bf16 row stride of the workspaces (elements)
  int64_t srows = 0;           // rows of the internal coefficient layout
  int ldx = 0;                 // columns of the l-major forward rows
  int ldr = 0;                 // columns of the FP32 forward rows (in spec_b)
  int max_channels = 0;        // capacity of the real filter weights
  __nv_bfloat16 *d_x_hi = nullptr, *d_x_lo = nullptr;  // l-major forward rows [L M][ldx]
  // second l-major rows buffer (the weight gradient's ISHT^T(gy) rows) and
  // the tensor-core view whose forward-row maps describe it; allocated by
  // the first weight-gradient call
  __nv_bfloat16 *d_g_hi = nullptr, *d_g_lo = nullptr;
  shtgb::TcPlanView tc_g{};
  // conj-transposed weights of the adjoint block (large W), grown on demand
  float2 *d_wt = nullptr;
  size_t wt_bytes = 0;
  void *d_ftiles = nullptr;    // filter tiles (l, m0)
  int n_ftiles = 0;
  __nv_bfloat16 *d_s_hi = nullptr, *d_s_lo = nullptr;  // bf16 internal rows [srows][ldcb]
  int *d_roff = nullptr;
  float *d_table = nullptr;
  int64_t *d_tab_off = nullptr;
  float2 *d_twiddle = nullptr;
  float *d_ring_w = nullptr;  // w_k * 2 pi / nlon
  float *d_zonal_c = nullptr; // 2 pi sin(theta_k) (2 pi / nlon)^2 (zonal power spectrum)
  shtgb::LegTile *d_fwd_tiles = nullptr;
  int n_fwd_tiles = 0;
  shtgb::LegTile *d_inv_tiles = nullptr;
  int n_inv_tiles = 0;
  int2 *d_fwd_krange = nullptr;  // K-chunk ranges of the tiles (streamed bf16 table only)
  int2 *d_inv_krange = nullptr;
  std::vector<int> fwd_tile_m, inv_tile_m;  // first tile of each order m (M + 1 entries)
  float *d_work = nullptr;    // folded Fourier workspace [M][2][Kh][ldc]
  float2 *d_spec_a = nullptr;  // [max_batch][L][M] spectral buffer
  float2 *d_spec_b = nullptr;  // [max_batch][L][M] spectral buffer
};
