/*
 * shtgb: spherical harmonic transforms and per-degree spectral filtering on
 * one NVIDIA GB300 GPU (sm_103a).  C ABI.
 *
 * The operation is the global convolution inside FourCastNet 3's spherical
 * neural-operator blocks (arXiv 2507.12144):
 *
 *   forward SHT   xhat_lm = int u conj(Y_lm) dmu                       Eq. (sht)
 *                 = sum_k w_k (2 pi / nlon) Phat_l^m(x_k) sum_j u_kj e^{-i m phi_j}
 *                 (longitude FFT, then a Legendre contraction whose
 *                 quadrature weights are folded in: Sec. B.3, Sec. G.2.2
 *                 Algorithm 1)
 *   filter        yhat[b][o][l][m] = sum_i W[l][o][i] xhat[b][i][l][m]
 *                 (the convolution theorem Eq. (s2_spectral_conv), with the
 *                 per-degree scalar generalised to complex channel mixing)
 *   inverse SHT   u_kj = sum_{m} c_m Re(G_k(m) e^{i m phi_j}),
 *                 G_k(m) = sum_l Phat_l^m(x_k) yhat_lm                  Eq. (isht)
 *                 c_0 = 1, c_{nlon/2} = 1 (Nyquist), c_m = 2 otherwise.
 *
 * Y_l^m(theta, phi) = Phat_l^m(cos theta) e^{i m phi} with the orthonormal
 * normalisation and one factor (-1)^m (Eq. spherical_harmonics).
 *
 * Around the transforms (sections further down): ensemble scores of the
 * coefficients and the grid (power spectra, spectral and spatial CRPS with
 * the loss gradient; Sec. D.4, E.1, F.7), the DISCO convolution's sparse
 * contraction and its transpose (Sec. B.5), and one step of the spherical
 * diffusion process that makes the noise channels (Sec. B.7).
 *
 * Conventions
 *   - lmax and mmax are COUNTS: 0 <= l < lmax, 0 <= m < mmax, and
 *     1 <= mmax <= lmax, mmax <= nlon/2 + 1.  Gaussian grids need
 *     lmax <= nlat.
 *   - Latitude row k = 0 is the northernmost.  Equiangular grids include
 *     both poles, theta_k = pi k / (nlat - 1).
 *   - Spatial arrays: float32 [B][nlat][nlon], row-major, contiguous.
 *   - Spectral arrays: complex64 (interleaved re, im float32) in the dense
 *     l-major rectangle [B][lmax][mmax] (the B x C x lmax x mmax layout of
 *     Algorithm 1).  Outputs have exact zeros at l < m; inputs are read only
 *     at l >= m.  The forward transform writes Im(m = 0) = 0 exactly, and
 *     the inverse ignores Im of m = 0 and of the Nyquist column.
 *   - Filter weights: complex64 W[lmax][Cout][Cin].
 *   - Adjoints are taken under the real inner product <a, b> = Re sum
 *     conj(a) b, which is PyTorch's convention for complex gradients.
 *
 * Memory and streams
 *   - Every data pointer is a DEVICE pointer on the plan's device, owned by
 *     the caller, 16-byte aligned and contiguous.  The plan owns its tables
 *     and workspaces, all allocated in sht_plan().
 *   - Execute calls allocate nothing and do not synchronise; they enqueue
 *     work on `stream` (a cudaStream_t passed as void*, NULL = legacy
 *     default stream).  A plan's workspace is shared by its execute calls,
 *     so one plan must not be used from two streams at once.
 *   - Batches larger than the plan's max_batch are processed in chunks of
 *     max_batch fields inside one call.
 *
 * Errors
 *   - Argument errors are returned before anything is enqueued.
 *   - A CUDA launch error is returned as SHT_ERR_CUDA; asynchronous faults
 *     surface on a later call.  Nothing aborts or prints.
 *   - sht_last_error_message() gives a one-line description of the most
 *     recent failure on the calling thread.
 */
#ifndef SHTGB_SHT_H_
#define SHTGB_SHT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sht_plan_s *sht_plan_t;

typedef enum {
  SHT_GRID_GAUSS = 0,             /* Gauss-Legendre latitudes (Sec. B.1)   */
  SHT_GRID_EQUIANGULAR_CC = 1,    /* pole-inclusive equiangular,
                                     Clenshaw-Curtis weights (footnote to
                                     Eq. latlon_quad_weights)              */
  SHT_GRID_EQUIANGULAR_TRAPZ = 2  /* pole-inclusive equiangular, weights
                                     sin(theta) dtheta (Eq.
                                     latlon_quad_weights)                  */
} sht_grid_t;

typedef enum {
  SHT_OK = 0,
  SHT_ERR_INVALID_ARG = 1,
  SHT_ERR_UNSUPPORTED = 2,
  SHT_ERR_OOM = 3,
  SHT_ERR_CUDA = 4,
  SHT_ERR_TIMEOUT = 5,
  SHT_ERR_INTERNAL = 6
} sht_status_t;

/* Arithmetic of the Legendre contractions (the dominant cost, Sec. B.3).
 * With a = a_hi + a_lo, a_hi = bf16(a), a_lo = bf16(a - a_hi):
 * FP32: FP32 table and data, FP32 accumulation (CUDA cores).
 * BF16: data rounded to bf16, table split; T_hi D + T_lo D on the tensor
 *   cores (tcgen05, operands by TMA), FP32 accumulation.  The table keeps
 *   its lo part because a bf16-rounded table carries errors shared by every
 *   field, up to the bf16 unit roundoff 2^-8.
 * SPLIT_BF16: table and data split; T_hi D_hi + T_hi D_lo + T_lo D_hi,
 *   FP32 accumulation.
 * Training in the paper uses bf16 mixed precision (Sec. E.3). */
typedef enum {
  SHT_PREC_FP32 = 0,
  SHT_PREC_BF16 = 1,
  SHT_PREC_SPLIT_BF16 = 2
} sht_precision_t;

/* Source of the Legendre table Phat_l^m(x_k) (Eq. sht_legendre_recursion)
 * for the tensor-core precisions; FP32 plans always stream an FP32 table.
 * STREAMED: bf16 hi/lo tables built once in FP64 at plan time and read by
 *   TMA on every call (table bytes re-read per call, no recurrence work).
 *   A streamed contraction skips, per tile, the leading latitudes (forward)
 *   or degrees (inverse) whose table entries are all below 2^-40 in
 *   magnitude: near the poles the high orders' Phat are zero to working
 *   precision, and what is left out changes a coefficient by at most 2^-40
 *   times the sum of |data| over it.
 * RECURRENCE: only seeds every 32 degrees are stored (FP64-computed, kept
 *   as FP32 pairs); extra warps of the Legendre kernels run the three-term
 *   recurrence in FP32 on chip (about 1/16 of the table bytes, more
 *   instructions per call).  The inverse keeps its generated table in
 *   tensor memory and, for split BF16, in three bf16 parts.
 * MIXED: the forward contraction streams the table (forward layout only),
 *   the inverse generates it on chip as RECURRENCE does.
 * RECURRENCE and MIXED need lmax <= 1400, else sht_plan returns
 * UNSUPPORTED. */
typedef enum {
  SHT_TABLE_STREAMED = 0,
  SHT_TABLE_RECURRENCE = 1,
  SHT_TABLE_MIXED = 2
} sht_table_source_t;

typedef struct {
  int precision;      /* sht_precision_t, default SHT_PREC_FP32            */
  int device;         /* CUDA device ordinal, default: the current device  */
  int64_t max_batch;  /* fields per internal chunk, default 256            */
  int max_channels;   /* tensor-core plans: largest Cin / Cout accepted
                         by the fused block; 0 = min(max_batch, 128)        */
  int table_source;   /* sht_table_source_t, default SHT_TABLE_STREAMED    */
  int reserved[6];    /* must be zero                                      */
} sht_plan_opts;

/* Fill opts with the defaults (precision FP32, current device,
 * max_batch 256, max_channels 0, table_source STREAMED). */
void sht_plan_opts_default(sht_plan_opts *opts);

/* Create a plan for an (nlat x nlon) grid and lmax x mmax coefficients.
 * Computes the latitude nodes and weights (FP64, host), generates the
 * normalised Legendre table Phat_l^m(x_k) in FP64 on the GPU and stores it
 * in the precision's layout, and allocates the workspace for max_batch
 * fields.  Blocks until the tables are built.  On success *out owns all
 * device memory; release it with sht_plan_destroy.
 * Errors: INVALID_ARG (sizes outside the conventions above, nlat < 2 for an
 * equiangular grid, NULL out); UNSUPPORTED (nlon with a prime factor other
 * than 2, 3, 5, or nlon > 8192); OOM; CUDA. */
sht_status_t sht_plan(sht_plan_t *out, int nlat, int nlon, int grid,
                      int lmax, int mmax, const sht_plan_opts *opts);

sht_status_t sht_plan_destroy(sht_plan_t plan);

/* Sizes and state of a plan.  Any output pointer may be NULL. */
sht_status_t sht_plan_info(sht_plan_t plan, int *nlat, int *nlon, int *grid,
                           int *lmax, int *mmax, int *precision,
                           int64_t *max_batch, int64_t *table_bytes,
                           int64_t *workspace_bytes);

/* Wait for all work on the plan's device (cudaDeviceSynchronize) and report
 * device-side failures of the plan's kernels: SHT_ERR_TIMEOUT when a bounded
 * wait of a tensor-core kernel gave up (the error word is then cleared),
 * SHT_ERR_CUDA for a pending CUDA error, else SHT_OK. */
sht_status_t sht_plan_check(sht_plan_t plan);

/* Copy the plan's latitude nodes x_k = cos(theta_k) and weights w_k (FP64,
 * host arrays of nlat entries; the 2-D weight is w_k * 2 pi / nlon).
 * Either pointer may be NULL. */
sht_status_t sht_plan_grid(sht_plan_t plan, double *x, double *w);

/* Forward SHT, Eq. (sht).  x: float32 [B][nlat][nlon] -> xhat: complex64
 * [B][lmax][mmax].  B >= 0 (B = 0 is a no-op). */
sht_status_t sht_forward(sht_plan_t plan, const float *x, void *xhat,
                         int64_t B, void *stream);

/* Inverse SHT, Eq. (isht).  xhat: complex64 [B][lmax][mmax] -> x: float32
 * [B][nlat][nlon]. */
sht_status_t sht_inverse(sht_plan_t plan, const void *xhat, float *x,
                         int64_t B, void *stream);

/* Adjoint of sht_forward: gxhat [B][lmax][mmax] -> gx [B][nlat][nlon],
 *   gx_kj = w_k (2 pi / nlon) Re sum_m e^{i m phi_j} sum_l Phat_l^m(x_k) gy_lm
 * (every m with weight 1; this is not the inverse transform). */
sht_status_t sht_forward_adjoint(sht_plan_t plan, const void *gxhat,
                                 float *gx, int64_t B, void *stream);

/* Adjoint of sht_inverse: gx [B][nlat][nlon] -> gxhat [B][lmax][mmax],
 *   gy_lm = sum_k Phat_l^m(x_k) c_m sum_j gx_kj e^{-i m phi_j}. */
sht_status_t sht_inverse_adjoint(sht_plan_t plan, const float *gx,
                                 void *gxhat, int64_t B, void *stream);

/* Spectral filter (Eq. s2_spectral_conv with channel mixing).
 * xhat: complex64 [Bm][Cin][lmax][mmax], W: complex64 [lmax][Cout][Cin],
 * yhat: complex64 [Bm][Cout][lmax][mmax] (zero at l < m).  FP32 arithmetic. */
sht_status_t spectral_filter(sht_plan_t plan, const void *xhat, const void *W,
                             void *yhat, int64_t Bm, int Cin, int Cout,
                             void *stream);

/* Adjoint of the filter in both arguments:
 *   gx[b][i][l][m] = sum_o conj(W[l][o][i]) gy[b][o][l][m]
 *   gW[l][o][i]    = sum_{b, m <= l} gy[b][o][l][m] conj(xhat[b][i][l][m])
 * gx and gW may each be NULL (not computed); gW is overwritten. */
sht_status_t spectral_filter_adjoint(sht_plan_t plan, const void *gy,
                                     const void *W, const void *xhat,
                                     void *gx, void *gW, int64_t Bm, int Cin,
                                     int Cout, void *stream);

/* One spectral block: y = ISHT(filter(SHT(x), W)) with the intermediates
 * kept in the plan's workspace.  x: float32 [Bm][Cin][nlat][nlon],
 * W: complex64 [lmax][Cout][Cin], y: float32 [Bm][Cout][nlat][nlon]. */
sht_status_t sht_spectral_block(sht_plan_t plan, const float *x,
                                const void *W, float *y, int64_t Bm, int Cin,
                                int Cout, void *stream);

/* Adjoint of the spectral block in x (Sec. B.8, the differentiable SHT):
 * gx = SHT^T(W^H ISHT^T(gy)), the gradient of <gy, y> with y =
 * sht_spectral_block(x).  gy: float32 [Bm][Cout][nlat][nlon], W: complex64
 * [lmax][Cout][Cin] (the forward's weights), gx: float32
 * [Bm][Cin][nlat][nlon].  Tensor-core plans run it on the block's kernels
 * (the analysis with the inverse's mode weights, the filter with
 * conj(W[l][o][i]) built on chip, the synthesis with the latitude weights);
 * FP32 plans on the CUDA-core kernels.  Limits and errors as
 * sht_spectral_block. */
sht_status_t sht_spectral_block_adjoint(sht_plan_t plan, const float *gy,
                                        const void *W, float *gx, int64_t Bm,
                                        int Cin, int Cout, void *stream);

/* Weight gradient of the spectral block (Sec. B.8): the gradient of
 * <gy, y> with respect to W for y = sht_spectral_block(x, W),
 *   gW[l][o][i] = sum_{b, m <= l} ISHT^T(gy)[b][o][l][m] conj(SHT(x)[b][i][l][m]).
 * x: float32 [Bm][Cin][nlat][nlon], gy: float32 [Bm][Cout][nlat][nlon],
 * gW: complex64 [lmax][Cout][Cin] (overwritten; device memory).  Tensor-
 * core plans compute both transforms into split (or single) bf16 l-major
 * rows and contract them per degree on the tensor cores (the first call
 * allocates a second rows buffer of the size of the plan's forward rows);
 * FP32 plans run the API transforms and an FP32 CUDA-core contraction.
 * Limits and errors as sht_spectral_block. */
sht_status_t sht_spectral_block_weight_grad(sht_plan_t plan, const float *x,
                                            const float *gy, void *gW,
                                            int64_t Bm, int Cin, int Cout,
                                            void *stream);

/* The block's backward in one call: gx as sht_spectral_block_adjoint and gW
 * as sht_spectral_block_weight_grad (either may be NULL: not computed; x is
 * read only for gW, W only for gx).  Tensor-core plans compute ISHT^T(gy)
 * once into the gradient rows and read it for both (the two separate calls
 * compute it twice); FP32 plans run the two calls.  Limits and errors as
 * sht_spectral_block. */
sht_status_t sht_spectral_block_backward(sht_plan_t plan, const float *x,
                                         const float *gy, const void *W,
                                         float *gx, void *gW, int64_t Bm,
                                         int Cin, int Cout, void *stream);

/* Fused filter + inverse SHT: y = ISHT(filter(xhat, W)).  xhat: complex64
 * [Bm][Cin][lmax][mmax], y: float32 [Bm][Cout][nlat][nlon]. */
sht_status_t spectral_filter_inverse(sht_plan_t plan, const void *xhat,
                                     const void *W, float *y, int64_t Bm,
                                     int Cin, int Cout, void *stream);

/* Forward SHT that allocates nothing: the same result as sht_forward, with
 * its scratch (the folded longitude coefficients of a chunk of fields) in a
 * 16 MiB static device array compiled into the library instead of the
 * plan's workspace.  The paper has no counterpart.  It is meant for callers
 * that may not request device memory while they run: hosts that own all
 * device memory through their own pool and forbid cudaMalloc in plug-ins,
 * or services held to a fixed memory budget.  The plan itself must have
 * been made beforehand (sht_plan allocates its tables).
 *   - Limit: the smallest chunk must fit.  A chunk row holds 4 floats
 *     (the re and im parts of two fields; the kernel loads them 16 bytes at
 *     a time) for every (order, parity, latitude), so the grid needs
 *     32 * mmax * ceil(nlat/2) bytes <= 16 MiB, also for a single field;
 *     larger grids get SHT_ERR_INVALID_ARG.  Larger batches are processed
 *     in chunks that fit.
 *   - FP32 plans only (SHT_ERR_UNSUPPORTED otherwise).
 *   - The array exists once per GPU that loads the library and stays until
 *     the process exits.  Every call on a device shares it: calls whose
 *     work overlaps on the GPU (two streams, or two host threads) race.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream
 *     capture.  The address is kept for the life of the process: after a
 *     cudaDeviceReset of that device, do not call this entry point again.
 *   - SHT_ERR_CUDA if the plan's device cannot be made current. */
sht_status_t sht_forward_static_scratch(sht_plan_t plan, const float *x,
                                        void *xhat, int64_t B, void *stream);

/* ---------------------------------------------------------------------------
 * Partial transforms: the local steps of the distributed (pencil) transform
 * of Algorithm 1 (appendix, "Distributed spherical Harmonic transforms").
 * A rank of a pencil decomposition holds a block of latitude rows for the
 * longitude steps and a block of orders over all latitudes for the Legendre
 * steps; the exchanges between the steps (all-to-alls over the polar and
 * azimuth groups) are the caller's.  The forward SHT is
 * legendre_orders(forward) of analysis_rows of every row, the inverse SHT
 * is synthesis_rows of legendre_orders(inverse).  All data on the plan's
 * device, 16-byte aligned, caller-owned; stream-ordered, no allocation.
 * Longitude steps use the generic mixed-radix FFT in FP32 on any plan;
 * the Legendre steps use the FP32 plan's table (SHT_ERR_UNSUPPORTED on
 * tensor-core plans).
 *
 * sht_analysis_rows: F[b][r][m] = w_k (2 pi / nlon) sum_j x[b][r][j]
 *   e^{-2 pi i j m / nlon} for m < mmax, k = k0 + r (Algorithm 1's
 *   2 pi FFT_1D_R2C and truncation; w_k the latitude weight of Sec. B.1).
 *   x: float32 [B][nrows][nlon], F: complex64 [B][nrows][mmax];
 *   0 <= k0, k0 + nrows <= nlat, else SHT_ERR_INVALID_ARG. */
sht_status_t sht_analysis_rows(sht_plan_t plan, const float *x, void *F,
                               int64_t B, int k0, int nrows, void *stream);

/* sht_synthesis_rows: y[b][r][j] = sum_{m < mmax} c_m Re(G[b][r][m]
 *   e^{2 pi i j m / nlon}), c_0 = 1, c_m = 2, c_{nlon/2} = 1 (Eq. isht for a
 *   real field; the imaginary parts of m = 0 and of the Nyquist mode are
 *   ignored).  G: complex64 [B][nrows][mmax], y: float32 [B][nrows][nlon];
 *   k0 and nrows as for sht_analysis_rows (the rows carry no weight). */
sht_status_t sht_synthesis_rows(sht_plan_t plan, const void *G, float *y,
                                int64_t B, int k0, int nrows, void *stream);

/* sht_legendre_orders: the Legendre step for orders m0 .. m0 + mcount - 1
 *   over all latitudes (Algorithm 1's "Legendre-Gauss quadrature via tensor
 *   contraction" on an order block; Eq. isht's sum over l for the inverse).
 *   inverse = 0: in = F complex64 [B][nlat][mcount] (weights applied, as
 *     sht_analysis_rows gives them), out = xhat complex64 [B][lmax][mcount],
 *     xhat[b][l][j] = sum_k Phat_l^m(x_k) F[b][k][j], m = m0 + j, zero for
 *     l < m.
 *   inverse = 1: in = yhat complex64 [B][lmax][mcount] (entries l < m are
 *     ignored), out = G complex64 [B][nlat][mcount], G[b][k][j] =
 *     sum_l Phat_l^m(x_k) yhat[b][l][j].
 *   0 <= m0, m0 + mcount <= mmax, else SHT_ERR_INVALID_ARG; FP32 plans only
 *   (SHT_ERR_UNSUPPORTED).  Uses the plan's workspaces: one stream at a
 *   time per plan, like the other execute calls. */
sht_status_t sht_legendre_orders(sht_plan_t plan, int inverse, const void *in,
                                 void *out, int64_t B, int m0, int mcount,
                                 void *stream);

/* ---------------------------------------------------------------------------
 * Host-resident fields through the spectral block.  A pipe owns `depth`
 * device staging slots (one input and one output array of the block's
 * shape each) and two copy streams.  sht_pipe_block(x_host -> y_host) is
 * asynchronous: it queues the host-to-device copy of x_host on the pipe's
 * input stream, sht_spectral_block on `stream` once that copy landed, and
 * the device-to-host copy into y_host on the pipe's output stream, with
 * events so that successive calls overlap (the next input copy and the
 * previous output copy run while a block computes) and a slot is reused
 * only after its previous input was consumed and its output drained.
 *   - x_host: float32 [Bm][Cin][nlat][nlon], y_host: float32
 *     [Bm][Cout][nlat][nlon], host memory, 16-byte aligned; page-locked
 *     (cudaHostAlloc / pinned) memory is needed for the copies to overlap.
 *     The caller keeps x_host unchanged, and reads y_host only, after
 *     sht_pipe_wait.  W: device complex64 [lmax][Cout][Cin], read when
 *     the block runs.
 *   - Errors: argument errors before anything is queued; CUDA errors as
 *     SHT_ERR_CUDA; the block's own conditions as sht_spectral_block.
 *   - The paper has no counterpart (it trains from data already on the
 *     GPU); this is the serving path for fields held by the host. */
typedef struct sht_pipe_s *sht_pipe_t;

/* depth: 1 .. 4 slots (2 overlaps input copy, block and output copy of
 * neighbouring calls).  Allocates depth * (in + out) bytes of device
 * memory on the plan's device.  The plan must outlive the pipe. */
sht_status_t sht_pipe_create(sht_pipe_t *out, sht_plan_t plan, int64_t Bm,
                             int Cin, int Cout, int depth);
sht_status_t sht_pipe_block(sht_pipe_t pipe, const float *x_host,
                            const void *W, float *y_host, void *stream);
/* Block the calling thread until every queued output copy has finished. */
sht_status_t sht_pipe_wait(sht_pipe_t pipe);
/* Wait for the pipe's copies, then free its slots, streams and events. */
sht_status_t sht_pipe_destroy(sht_pipe_t pipe);

/* ---------------------------------------------------------------------------
 * Batched transforms over several grids.  Ensemble members are independent
 * of one another (the ensemble-parallel computations of the section on
 * simultaneous model-, data- and ensemble-parallelism are embarrassingly
 * parallel), so many fields on grids of different
 * sizes can be transformed together.  A batch binds up to 8 items, each a
 * plan (its grid, table and workspace) with a fixed count of fields and
 * fixed input and output buffers, and records the whole transform of all
 * items as one CUDA graph: one grouped longitude launch, one persistent
 * Legendre launch over the tiles of every item, one grouped epilogue launch
 * (for the forward: the transpose of the tensor-core rows into the API
 * layout, or the zero fill of the FP32 path; before the inverse on the
 * tensor-core precisions: the transpose into the internal rows).
 * sht_batch_run replays it.
 *
 * Items:
 *   plan   a plan, at most once per batch; all plans of a batch share the
 *          device, the precision and the table source.
 *   count  fields, 1 <= count <= the plan's max_batch.
 *   in     forward: float [count][nlat][nlon]; inverse: complex64
 *          [count][lmax][mmax] (same contract as sht_forward / sht_inverse).
 *   out    forward: complex64 [count][lmax][mmax]; inverse: float
 *          [count][nlat][nlon].
 * The buffers stay owned by the caller and must outlive the batch; their
 * contents are read and written by every run.  The plans' workspaces are
 * used by the runs: a plan must not execute other calls concurrently.
 *
 * Tuning (opts.tune = 1): creation times the Legendre launch for candidate
 * launch shapes (column tile widths 256, 128 and 64 for the tensor-core
 * precisions; item orders) on the bound buffers — so it writes the outputs
 * — and keeps the fastest.  With opts.tune_cache set, the choice is looked
 * up in that text file by the batch's key first, and appended to it after
 * tuning.  opts.profile = 1 adds CUDA event nodes between the kernels of
 * the graph for sht_batch_profile_*.
 *
 * Errors: INVALID_ARG (n outside 1..8, NULL or repeated plans, mixed
 * device, precision or table source, counts outside the range, NULL
 * buffers); CUDA / OOM from tuning, capture or instantiation.
 * No paper counterpart as an interface: it serves the batched form.
 * ------------------------------------------------------------------------- */
typedef struct sht_batch_s *sht_batch_t;

typedef enum {
  SHT_BATCH_FORWARD = 0,   /* sht_forward of every item */
  SHT_BATCH_INVERSE = 1    /* sht_inverse of every item */
} sht_batch_direction_t;

typedef struct {
  sht_plan_t plan;
  int64_t count;
  const void *in;
  void *out;
} sht_batch_item;

typedef struct {
  int direction;           /* sht_batch_direction_t, default FORWARD     */
  int tune;                /* 1 (default): time candidate launch shapes  */
  const char *tune_cache;  /* NULL (default) or a text file of choices   */
  int profile;             /* 0 (default) or 1: event nodes in the graph */
  int reserved[8];         /* must be zero                               */
} sht_batch_opts;

void sht_batch_opts_default(sht_batch_opts *opts);

/* Validate, tune, record and instantiate.  `stream` (may be NULL) orders
 * the tuning runs after the caller's earlier work on it; creation returns
 * after they finished. */
sht_status_t sht_batch_create(sht_batch_t *out, const sht_batch_item *items,
                              int n, const sht_batch_opts *opts,
                              void *stream);

/* Launch the recorded graph on `stream` (NULL: the legacy default stream).
 * Asynchronous; errors of earlier device work surface as SHT_ERR_CUDA. */
sht_status_t sht_batch_run(sht_batch_t batch, void *stream);

/* NUL-terminated description of the launch shape in use and how it was
 * chosen, e.g. "legendre: tile<=128, order=cost; tuned 412.3 us". */
sht_status_t sht_batch_describe(sht_batch_t batch, char *buf, int len);

/* Kernels of the graph, in launch order ("r2c", "leg_fwd", "zero", ...). */
int sht_batch_stage_count(sht_batch_t batch);
const char *sht_batch_stage_name(sht_batch_t batch, int stage);

/* Per-stage device time of profiled runs (batches created with
 * opts.profile = 1).  begin: record the next `capacity` runs; collect: wait
 * for them and return the number of recorded runs and the summed
 * milliseconds per stage (array of sht_batch_stage_count entries), then
 * reset the record. */
sht_status_t sht_batch_profile_begin(sht_batch_t batch, int capacity);
sht_status_t sht_batch_profile_collect(sht_batch_t batch, int64_t *runs,
                                       double *ms);

/* Release the graph and the batch (not the plans or the buffers). */
sht_status_t sht_batch_destroy(sht_batch_t batch);

/* ------------------------------------------------------------------------
 * Ensemble scores (Sec. D.4, Sec. E.1, Sec. F.7)
 *
 * Scores of E-member ensembles against one observation, computed on the
 * coefficients a forward transform produces (or on the grid).  They need no
 * plan except the spatial CRPS, which takes the grid's quadrature weights
 * from one.  Every result is summed in a fixed order (deterministic).
 * FP32 arithmetic.  Pointers as everywhere else: device, 16-byte aligned,
 * contiguous, on the current device (the plan's for sht_spatial_crps).
 * ------------------------------------------------------------------------ */

/* Angular power spectrum, Eq. (psd), of B coefficient arrays:
 *   psd[b][l] = |xhat[b][l][0]|^2 + 2 sum_{m = 1}^{min(l, mmax - 1)} |xhat[b][l][m]|^2
 * (the sum over |m| <= l of a real field, whose m < 0 coefficients have the
 * moduli of m > 0).  xhat: complex64 [B][lmax][mmax], read at l >= m only;
 * psd: float32 [B][lmax].  Needs 1 <= mmax <= lmax; B = 0 is a no-op. */
sht_status_t sht_angular_psd(const void *xhat, float *psd, int64_t B, int lmax,
                             int mmax, void *stream);

/* Zonal power spectrum, Eq. (zonal_psd), of B fields on the plan's grid:
 *   zpsd[b][k][m] = 2 pi sin(theta_k) |(2 pi / nlon) sum_j x[b][k][j] e^{-i m phi_j}|^2
 * for m < mmax (each m >= 0 once; the longitude integral by the grid's
 * uniform longitude quadrature).  x: float32 [B][nlat][nlon], zpsd: float32
 * [B][nlat][mmax].  Runs the plan's longitude FFT in FP32 whatever the
 * plan's precision, with an FP32 buffer of the plan as scratch (the
 * analysis workspace of FP32 plans, the spectral buffer of tensor-core
 * plans); SHT_ERR_UNSUPPORTED when a tensor-core plan's buffer cannot hold
 * one field (lmax < nlat / 2).  B = 0 is a no-op. */
sht_status_t sht_zonal_psd(sht_plan_t plan, const float *x, float *zpsd,
                           int64_t B, void *stream);

/* Spectral CRPS, Eq. (spectral_loss): for every channel c and degree l
 *   crps_l[c][l] = sum_{|m| <= l} CRPS(u_l^m) = c_l0 + 2 sum_{m >= 1} c_lm,
 *   c_lm = CRPS(Re ens[.][c][l][m], Re obs[c][l][m])
 *        + CRPS(Im ens[.][c][l][m], Im obs[c][l][m]),
 * with the ensemble CRPS of Eq. (spread_skill_crps) (fair = 0) or the fair
 * CRPS of Eq. (fair_spread_skill_crps) (fair = 1), computed on the sorted
 * members.
 *   ens:     complex64 [E][C][lmax][mmax], members first (the layout of
 *            sht_forward applied to E x C fields), read at l >= m only;
 *   obs:     complex64 [C][lmax][mmax];
 *   crps_l:  float32 [C][lmax], required;
 *   crps_lm: float32 [C][lmax][mmax] or NULL: c_lm, 0 at l < m;
 *   loss:    float32 [C] or NULL: sum_{l_lo <= l < l_hi} crps_l[c][l].
 * 1 <= E <= 64 (E >= 2 for the fair form), 0 <= l_lo <= l_hi <= lmax,
 * C >= 0 (C = 0 is a no-op). */
sht_status_t sht_spectral_crps(const void *ens, const void *obs, float *crps_l,
                               float *crps_lm, float *loss, int E, int64_t C,
                               int lmax, int mmax, int fair, int l_lo,
                               int l_hi, void *stream);

/* Gradient of the loss output of sht_spectral_crps, for training with it:
 *   gens[e][c][l][m] = gloss[c] d loss[c] / d ens[e][c][l][m],
 *   gobs[c][l][m]    = gloss[c] d loss[c] / d obs[c][l][m]   (gobs NULL: skipped),
 * complex64, each entry d/dRe + i d/dIm (PyTorch's convention for a real
 * function of complex values).  Per real value with members u_e and
 * observation u*,
 *   d CRPS / d u_e = sign(u_e - u*) / E - (1/D) sum_i sign(u_e - u_i),
 *   d CRPS / d u*  = -(1/E) sum_e sign(u_e - u*),       sign(0) = 0
 * (at ties the subgradient that averages the tied ranks), D = E^2
 * (fair = 0) or E (E - 1) (fair = 1); m > 0 counts twice.  Both
 * outputs are written everywhere: zero outside l_lo <= l < l_hi and at
 * l < m.  gloss: float32 [C]; other arguments as for sht_spectral_crps. */
sht_status_t sht_spectral_crps_backward(const void *ens, const void *obs,
                                        const float *gloss, void *gens, void *gobs,
                                        int E, int64_t C, int lmax, int mmax,
                                        int fair, int l_lo, int l_hi,
                                        void *stream);

/* Spatial CRPS, Eq. (spatial_loss): the point-wise CRPS averaged over the
 * sphere with the plan's grid and quadrature,
 *   crps_k[c][k] = (1 / (4 pi)) w_k (2 pi / nlon) sum_j CRPS(ens[.][c][k][j], obs[c][k][j]),
 *   loss[c]      = sum_k crps_k[c][k].
 * ens: float32 [E][C][nlat][nlon], obs: float32 [C][nlat][nlon], crps_k:
 * float32 [C][nlat] (required), loss: float32 [C] or NULL.  E and fair as
 * for sht_spectral_crps. */
sht_status_t sht_spatial_crps(sht_plan_t plan, const float *ens, const float *obs,
                              float *crps_k, float *loss, int E, int64_t C,
                              int fair, void *stream);

/* ------------------------------------------------------------------------
 * Spherical diffusion process (Sec. B.7)
 * ------------------------------------------------------------------------ */

/* One step of Eq. (spherical_diffusion) for B noise fields, in place on
 * their coefficients:
 *   zhat[b][l][m] = phi zhat[b][l][m] + sigma_l xi[b][l][m],
 *   phi = exp(-lambda), sigma_l = F0 exp(-(kT / 2) l (l + 1)),
 *   F0 = sigma sqrt(2 pi (1 - phi^2) / sum_{l=1}^{lmax-1} (2l+1) exp(-kT l (l+1))),
 * for 1 <= l < lmax and m <= l; the l = 0 entry is set to 0 (no l = 0
 * term) and entries with m > l are neither read nor written (the inverse
 * transform ignores them).  xi = eta for m > 0 (real and imaginary part standard normal) and
 * sqrt(2) Re(eta) at m = 0, so that the real field (sht_inverse of zhat)
 * has the stationary variance sigma^2 at every point.
 *   zhat: complex64 [B][lmax][mmax] device, updated in place;
 *   eta:  complex64 [B][lmax][mmax] device standard normals, or NULL: drawn
 *         on the GPU from Philox4x32-10 with key = seed: for the flat
 *         coefficient index idx = b lmax mmax + l mmax + m, the generator
 *         at counter (idx >> 1, step) gives words w0 .. w3, of which idx
 *         takes (wa, wb) = (w0, w1) if idx is even and (w2, w3) if odd,
 *         then the Box-Muller transform u1 = ((wa >> 8) + 1) 2^-24,
 *         u2 = (wb >> 8) 2^-24, eta = sqrt(-2 ln u1) e^{2 pi i u2};
 *   kT:   HOST array of nk (1 .. 16) length scales; field b uses kT[b % nk].
 * lambda > 0, sigma >= 0, lmax >= 2, 1 <= mmax <= lmax; B = 0 is a no-op. */
sht_status_t sht_diffusion_step(void *zhat, const void *eta, int64_t B, int lmax,
                                int mmax, const double *kT, int nk,
                                double lambda, double sigma, uint64_t seed,
                                uint64_t step, void *stream);

/* ------------------------------------------------------------------------
 * DISCO convolution (Sec. B.5, Eq. disco_convolution_formula)
 *
 * The contraction of a field with the sparse convolution tensor psi of a
 * locally supported filter basis, for every shift in longitude:
 *   y[c][k][h][w] = sum_{h', w'} psi[k][h][h'][w'] x[c][h'][(w' + s w) mod nlon_in],
 *   psi[k][h][h'][w'] = kb_k(R_h^{-1} x_{h', w'}) w_{h'} 2 pi / nlon_in,
 * nlon_in = s nlon_out, R_h the rotation taking the north pole to the
 * output point (theta_h, longitude 0), and the basis kb_k of Sec. B.5.1 on
 * the cap of radius theta_cutoff: with vartheta' = vartheta / theta_cutoff
 * <= 1 and the azimuth varphi of the rotated input point,
 * cos^2(pi vartheta' / 2) times cos or sin of pi (l vartheta' sin varphi +
 * m vartheta' cos varphi), 0 <= l, m < basis_n: the cosines for all (l, m),
 * then the sines without l = m = 0, K = 2 basis_n^2 - 1 functions.  The
 * mixing of channels and basis functions with learnable weights, a dense
 * GEMM over (c, k), is left to the caller.
 * ------------------------------------------------------------------------ */
typedef struct sht_disco_s *sht_disco_t;

/* Build psi (FP64 on the host, FP32 on the device) for an input grid
 * (nlat_in, nlon_in, grid_in) and an output grid (nlat_out, nlon_out,
 * grid_out); nlon_in a multiple of nlon_out, basis_n 1 .. 4,
 * 0 < theta_cutoff <= pi (radians), on CUDA device `device`. */
sht_status_t sht_disco_create(sht_disco_t *out, int nlat_in, int nlon_in,
                              int grid_in, int nlat_out, int nlon_out,
                              int grid_out, int basis_n, double theta_cutoff,
                              int device);

/* K and the number of (output latitude, input point) entries of psi. */
sht_status_t sht_disco_info(sht_disco_t disco, int *nbasis, int64_t *nnz);

/* x: float32 [C][nlat_in][nlon_in] -> y: float32 [C][K][nlat_out][nlon_out]. */
sht_status_t sht_disco_forward(sht_disco_t disco, const float *x, float *y,
                               int64_t C, void *stream);

/* The transpose of sht_disco_forward (its backward): gy: float32
 * [C][K][nlat_out][nlon_out] -> gx: float32 [C][nlat_in][nlon_in]
 * (overwritten).  On equal longitude grids whose nlon is a multiple of 4
 * and of 3, 5 or 9 it runs by runs of consecutive longitude offsets, with
 * the K gradient rows of each run staged in shared memory by bulk copies
 * and waits bounded in time; a wait that runs out leaves gx unwritten and
 * is reported by sht_disco_check.  Both pointers 16-byte aligned. */
sht_status_t sht_disco_backward(sht_disco_t disco, const float *gy, float *gx,
                                int64_t C, void *stream);

/* Synchronise the handle's device and report (then clear) a timed-out wait
 * of an earlier backward: SHT_ERR_TIMEOUT, else SHT_OK. */
sht_status_t sht_disco_check(sht_disco_t disco);

sht_status_t sht_disco_destroy(sht_disco_t disco);

/* ---------------------------------------------------------------------------
 * Per-kernel timing.  While profiling is on, every kernel a plan's execute
 * calls launch is bracketed by two CUDA events recorded on the launch
 * stream (up to `capacity` launches; later launches run unrecorded and are
 * counted as dropped).  sht_profile_collect waits for the recorded events,
 * adds each launch's duration to its kernel's total and resets the record.
 * No paper counterpart: this is the library's tracing facility.
 * ------------------------------------------------------------------------- */
typedef enum {
  SHT_KERNEL_R2C = 0,        /* longitude analysis (FFT), parity fold     */
  SHT_KERNEL_LEG_FWD = 1,    /* forward Legendre contraction              */
  SHT_KERNEL_ZERO = 2,       /* zero fill of l < m                        */
  SHT_KERNEL_FILTER = 3,     /* spectral filter or its input adjoint      */
  SHT_KERNEL_FILTER_DW = 4,  /* weight adjoint of the filter              */
  SHT_KERNEL_LEG_INV = 5,    /* inverse Legendre contraction              */
  SHT_KERNEL_C2R = 6,        /* longitude synthesis (inverse FFT)         */
  SHT_KERNEL_PACK = 7,       /* API coefficients -> internal bf16 rows    */
  SHT_KERNEL_FILTER_PREP = 8, /* weight preparation: the conj-transposed
                                 W of an adjoint block with large W       */
  SHT_KERNEL_FINALIZE = 9,   /* FP32 l-major rows -> API xhat (+ zeros)   */
  SHT_KERNEL_COUNT = 10
} sht_kernel_t;

/* Start recording (capacity >= 1 launches); creates the events on the
 * plan's device.  Calling it again while on resets the record. */
sht_status_t sht_profile_begin(sht_plan_t plan, int capacity);

/* Wait for the recorded launches and report, per sht_kernel_t id, the
 * launch count and the summed device milliseconds (arrays of
 * SHT_KERNEL_COUNT entries, either may be NULL); *dropped (may be NULL)
 * receives the launches beyond capacity.  Recording continues. */
sht_status_t sht_profile_collect(sht_plan_t plan, int64_t *launches,
                                 double *ms, int64_t *dropped);

/* Stop recording and release the events. */
sht_status_t sht_profile_end(sht_plan_t plan);

/* Name of a kernel id ("r2c", "leg_fwd", ...), or "?" when out of range. */
const char *sht_kernel_name(int kernel);

const char *sht_status_string(sht_status_t status);
const char *sht_last_error_message(void);

/* Library version, e.g. "0.1.0". */
const char *sht_version(void);

/* Test hook for failure handling: the n-th device allocation made by later
 * sht_plan calls fails as if the device were out of memory (n = 0: the next
 * one; n < 0: off).  The plan call then returns SHT_ERR_OOM and frees what
 * it had allocated.  Not thread-safe; for tests only. */
void sht_debug_fail_alloc_after(int n);

/* Test hook for device-side failure detection: queue on `stream` one kernel
 * that waits on a shared-memory barrier nothing ever completes, through the
 * same bounded wait the tensor-core kernels use, with a limit of
 * timeout_ns (1 .. 2e9).  The wait gives up, records the timeout in the
 * plan's error word and the kernel returns normally; sht_plan_check then
 * reports SHT_ERR_TIMEOUT (and clears the word), and the plan stays usable.
 * For tests only. */
sht_status_t sht_debug_stall(sht_plan_t plan, int64_t timeout_ns, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SHTGB_SHT_H_ */
