// C ABI of shtgb: plan construction (grids, weights, FP64 Legendre table on
// the GPU, workspaces) and the execute calls.  See include/sht.h for the
// contract of every entry point.
#include <algorithm>
#include <cmath>
#include <new>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "sht_internal.cuh"

namespace shtgb {

static thread_local std::string g_last_error = "";
static int g_fail_alloc_after = -1;  // test hook: fail the n-th allocation

sht_status_t fail(sht_status_t st, const std::string &msg) {
  g_last_error = msg;
  return st;
}

sht_status_t cuda_fail(cudaError_t err, const char *what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(err);
  return err == cudaErrorMemoryAllocation ? SHT_ERR_OOM : SHT_ERR_CUDA;
}

namespace {

#define SHT_TRY(expr)                    \
  do {                                   \
    sht_status_t _s = (expr);            \
    if (_s != SHT_OK) return _s;         \
  } while (0)

constexpr double kPi = 3.14159265358979323846264338327950288;

struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
      changed = cudaSetDevice(dev) == cudaSuccess;
    }
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

cudaError_t dev_alloc(void **p, size_t bytes) {
  if (g_fail_alloc_after == 0) {
    g_fail_alloc_after = -1;
    return cudaErrorMemoryAllocation;
  }
  if (g_fail_alloc_after > 0) g_fail_alloc_after--;
  if (bytes == 0) bytes = 16;
  return cudaMalloc(p, bytes);
}

// Legendre polynomial P_n and P_{n-1} at z by Bonnet's recurrence.
void bonnet(int n, double z, double &pn, double &pn1) {
  double a = 1.0, b = z;
  if (n == 0) {
    pn = 1.0;
    pn1 = 0.0;
    return;
  }
  for (int j = 1; j < n; j++) {
    double c = ((2 * j + 1) * z * b - j * a) / (j + 1);
    a = b;
    b = c;
  }
  pn = b;
  pn1 = a;
}

// Latitude nodes (x = cos theta, s = sin theta) and weights w for the
// northern half including the equator; the southern half mirrors it.
void make_grid(int grid, int nlat, std::vector<double> &x, std::vector<double> &s, std::vector<double> &w) {
  x.assign(nlat, 0.0);
  s.assign(nlat, 0.0);
  w.assign(nlat, 0.0);
  const int half = (nlat + 1) / 2;
  for (int k = 0; k < half; k++) {
    double xk, sk, wk;
    if (grid == SHT_GRID_GAUSS) {
      // k-th root of P_nlat from the north, Newton from the asymptotic guess
      double z = std::cos(kPi * (4.0 * k + 3.0) / (4.0 * nlat + 2.0));
      if (2 * k + 1 == nlat) z = 0.0;
      double pn, pn1;
      for (int it = 0; it < 64 && 2 * k + 1 != nlat; it++) {
        bonnet(nlat, z, pn, pn1);
        double dp = nlat * (pn1 - z * pn) / ((1.0 - z) * (1.0 + z));
        double dz = pn / dp;
        z -= dz;
        if (std::fabs(dz) < 1e-17) break;
      }
      bonnet(nlat, z, pn, pn1);
      double omz = (1.0 - z) * (1.0 + z);
      double dp = nlat * (pn1 - z * pn) / omz;
      xk = z;
      sk = std::sqrt(omz);
      wk = 2.0 / (omz * dp * dp);
    } else {
      const int N = nlat - 1;
      double t = kPi * (double)k / (double)N;
      xk = std::cos(t);
      sk = std::sin(t);
      if (2 * k == N) xk = 0.0, sk = 1.0;
      if (grid == SHT_GRID_EQUIANGULAR_CC) {
        double acc = 1.0;
        for (int j = 1; 2 * j <= N; j++) {
          double bj = (2 * j == N) ? 1.0 : 2.0;
          acc -= bj * std::cos(2.0 * j * t) / (4.0 * (double)j * j - 1.0);
        }
        wk = ((k == 0) ? 1.0 : 2.0) * acc / (double)N;
      } else {
        wk = kPi / (double)N * sk;
      }
    }
    x[k] = xk;
    s[k] = sk;
    w[k] = wk;
    x[nlat - 1 - k] = -xk;
    s[nlat - 1 - k] = sk;
    w[nlat - 1 - k] = wk;
  }
}

bool factor_radix(int n, RadixPlan &rp) {
  rp.n = n;
  rp.nstages = 0;
  int r = n;
  auto push = [&](int v) {
    if (rp.nstages >= kMaxRadices) return false;
    rp.r[rp.nstages++] = v;
    return true;
  };
  while (r % 4 == 0) {
    if (!push(4)) return false;
    r /= 4;
  }
  while (r % 2 == 0) {
    if (!push(2)) return false;
    r /= 2;
  }
  while (r % 3 == 0) {
    if (!push(3)) return false;
    r /= 3;
  }
  while (r % 5 == 0) {
    if (!push(5)) return false;
    r /= 5;
  }
  return r == 1;
}

template <class T>
cudaError_t upload(T **dst, const std::vector<T> &src) {
  cudaError_t e = dev_alloc((void **)dst, sizeof(T) * src.size());
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
}

void profile_release(ProfileState &pr);

void free_plan(sht_plan_s *p) {
  if (!p) return;
  DeviceGuard g(p->device);
  profile_release(p->prof);
  cudaFree(p->d_err);
  cudaFree(p->d_tf_hi);
  cudaFree(p->d_tf_lo);
  cudaFree(p->d_seeds);
  cudaFree(p->d_coef);
  cudaFree(p->d_x2h);
  cudaFree(p->d_x2l);
  cudaFree(p->d_roff);
  cudaFree(p->d_x_hi);
  cudaFree(p->d_x_lo);
  cudaFree(p->d_g_hi);
  cudaFree(p->d_g_lo);
  cudaFree(p->d_wt);
  cudaFree(p->d_ftiles);
  cudaFree(p->d_s_hi);
  cudaFree(p->d_s_lo);
  cudaFree(p->d_table);
  cudaFree(p->d_tab_off);
  cudaFree(p->d_twiddle);
  cudaFree(p->d_ring_w);
  cudaFree(p->d_zonal_c);
  cudaFree(p->d_fwd_tiles);
  cudaFree(p->d_inv_tiles);
  cudaFree(p->d_fwd_krange);
  cudaFree(p->d_inv_krange);
  cudaFree(p->d_work);
  cudaFree(p->d_spec_a);
  cudaFree(p->d_spec_b);
  delete p;
}

TableF32 table_view(const sht_plan_s *p) { return TableF32{p->d_table, p->d_tab_off, p->Khp}; }

// Launch through the profiler: brackets the launch with the next pair of
// events when profiling is on.
template <class F>
cudaError_t traced(sht_plan_s *p, int kernel, cudaStream_t st, F &&launch) {
  ProfileState &pr = p->prof;
  const bool rec = pr.on && pr.used < pr.capacity;
  if (pr.on && !rec) pr.dropped++;
  if (rec) {
    cudaError_t e = cudaEventRecord(pr.start[pr.used], st);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = launch();
  if (e != cudaSuccess) return e;
  if (rec) {
    e = cudaEventRecord(pr.stop[pr.used], st);
    if (e != cudaSuccess) return e;
    pr.kernel[pr.used] = kernel;
    pr.used++;
  }
  return cudaSuccess;
}

void profile_release(ProfileState &pr) {
  for (auto ev : pr.start) cudaEventDestroy(ev);
  for (auto ev : pr.stop) cudaEventDestroy(ev);
  pr.start.clear();
  pr.stop.clear();
  pr.kernel.clear();
  pr.on = false;
  pr.capacity = pr.used = 0;
  pr.dropped = 0;
}

// ---- chunked execute bodies -------------------------------------------------

bool is_tc(const sht_plan_s *p) { return p->precision != SHT_PREC_FP32; }

__nv_bfloat16 *f_hi(sht_plan_s *p) { return reinterpret_cast<__nv_bfloat16 *>(p->d_work); }
__nv_bfloat16 *f_lo(sht_plan_s *p) { return f_hi(p) + (size_t)p->M * 2 * p->Kh * p->ldcb; }
// FP32 l-major rows of the forward into the API layout (in the spec_b
// workspace, row stride ldr floats).
float *rows_f32(sht_plan_s *p) { return reinterpret_cast<float *>(p->d_spec_b); }
// The lo half of the data exists only for split precision.
__nv_bfloat16 *data_lo(sht_plan_s *p, __nv_bfloat16 *lo) { return p->precision == SHT_PREC_SPLIT_BF16 ? lo : nullptr; }

// Destination of the forward contraction in the tensor-core block path: the
// Column block of one member in the l-major rows of the fused block.
int block_kx(int Cin) { return (2 * Cin + 7) / 8 * 8; }

// l-major bf16 rows with members of cin channels in blocks of kx columns;
// T: the tensor-core view whose forward-row maps describe these rows (NULL:
// the plan's own view and rows).
struct RowsOut {
  __nv_bfloat16 *hi, *lo;
  int ldo, cin, kx;
  const TcPlanView *T = nullptr;
};

// Forward transform (or the inverse adjoint) of B fields; the coefficients
// go to the API layout xhat, or, when rows_out is set (tensor-core plans
// only, one chunk), to the l-major rows.
sht_status_t analysis(sht_plan_s *p, const float *x, float2 *xhat, int64_t B, cudaStream_t st, bool adjoint,
                      bool zero_upper, const RowsOut *rows_out = nullptr) {
  const int64_t LM = (int64_t)p->L * p->M;
  for (int64_t b0 = 0; b0 < B; b0 += p->max_batch) {
    const int nb = (int)std::min<int64_t>(p->max_batch, B - b0);
    const float *xb = x + b0 * p->nlat * (int64_t)p->nlon;
    const float *ring = adjoint ? nullptr : p->d_ring_w;
    const int wts = adjoint ? 1 : 0;
    cudaError_t e;
    if (!is_tc(p)) {
      e = traced(p, SHT_KERNEL_R2C, st, [&] {
        if (fft45_supported(p->nlon))
          return launch_r2c45(xb, p->d_work, nullptr, nullptr, p->nlat, p->nlon, p->M, nb, p->lay_f, p->d_twiddle,
                              ring, wts, st, p->d_err);
        return launch_r2c(xb, p->d_work, p->nlat, p->nlon, p->M, nb, p->lay_f, p->d_twiddle, p->radix, ring, wts, st);
      });
      if (e != cudaSuccess) return cuda_fail(e, "longitude analysis launch");
      e = traced(p, SHT_KERNEL_LEG_FWD, st, [&] {
        return launch_leg_fwd_f32(table_view(p), p->d_fwd_tiles, p->n_fwd_tiles, p->d_work, xhat + b0 * LM, p->L,
                                  p->M, p->Kh, p->ldc, nb, st);
      });
    } else {
      e = traced(p, SHT_KERNEL_R2C, st, [&] {
        if (fft45_supported(p->nlon))
          return launch_r2c45(xb, nullptr, f_hi(p), data_lo(p, f_lo(p)), p->nlat, p->nlon, p->M, nb, p->lay_f,
                              p->d_twiddle, ring, wts, st, p->d_err);
        return launch_r2c_bf16(xb, f_hi(p), data_lo(p, f_lo(p)), p->nlat, p->nlon, p->M, nb, p->lay_f, p->d_twiddle,
                               p->radix, ring, wts, st);
      });
      if (e != cudaSuccess) return cuda_fail(e, "longitude analysis launch");
      e = traced(p, SHT_KERNEL_LEG_FWD, st, [&] {
        TcLegItem it{};
        it.T = rows_out && rows_out->T ? rows_out->T : &p->tc;
        it.tiles = p->d_fwd_tiles;
        it.krange = p->d_fwd_krange;
        it.ntiles = p->n_fwd_tiles;
        it.B = nb;
        if (rows_out) {
          it.rows_hi = rows_out->hi;
          it.rows_lo = rows_out->lo;
          it.ldo = rows_out->ldo;
          it.cin = rows_out->cin;
          it.kx = rows_out->kx;
        } else {
          // FP32 l-major rows, turned into the API layout below
          it.rowsf = rows_f32(p);
          it.ldr = p->ldr;
        }
        return launch_leg_tc_group(0, &it, 1, TcLaunch{}, st);
      });
      if (e == cudaSuccess && !rows_out) {
        e = traced(p, SHT_KERNEL_FINALIZE, st, [&] {
          RowsItem r{rows_f32(p), xhat + b0 * LM, nullptr, nullptr, p->L, p->M, nb, p->ldr};
          return launch_rows_transpose(false, &r, 1, st);
        });
        if (e != cudaSuccess) return cuda_fail(e, "coefficient transpose launch");
        continue;
      }
    }
    if (e != cudaSuccess) return cuda_fail(e, "forward Legendre launch");
    if (zero_upper && !rows_out) {
      e = traced(p, SHT_KERNEL_ZERO, st, [&] { return launch_zero_upper(xhat + b0 * LM, p->L, p->M, nb, st); });
      if (e != cudaSuccess) return cuda_fail(e, "zero fill launch");
    }
    if (rows_out && B > p->max_batch) return fail(SHT_ERR_INTERNAL, "internal rows hold one chunk only");
  }
  return SHT_OK;
}

// Longitude synthesis from the FP32 folded workspace.
cudaError_t c2r_any(sht_plan_s *p, float *y, int nb, bool adjoint, cudaStream_t st) {
  const float *ring = adjoint ? p->d_ring_w : nullptr;
  const int wts = adjoint ? 0 : 1;
  if (fft45_supported(p->nlon))
    return launch_c2r45(p->d_work, y, p->nlat, p->nlon, p->M, nb, p->lay_g, p->d_twiddle, ring, wts, st, p->d_err);
  return launch_c2r(p->d_work, y, p->nlat, p->nlon, p->M, nb, p->lay_g, p->d_twiddle, p->radix, ring, wts, st);
}

// Inverse Legendre + longitude synthesis of B fields whose coefficients are
// already in the tensor-core internal rows (bf16 hi/lo).
sht_status_t synthesis_rows(sht_plan_s *p, float *y, int nb, cudaStream_t st, bool adjoint) {
  cudaError_t e = traced(p, SHT_KERNEL_LEG_INV, st, [&] {
    return launch_leg_inv_tc(p->tc, p->d_inv_tiles, p->d_inv_krange, p->n_inv_tiles, p->d_work, p->ldc, nb, st);
  });
  if (e != cudaSuccess) return cuda_fail(e, "inverse Legendre launch");
  e = traced(p, SHT_KERNEL_C2R, st, [&] { return c2r_any(p, y, nb, adjoint, st); });
  if (e != cudaSuccess) return cuda_fail(e, "longitude synthesis launch");
  return SHT_OK;
}

sht_status_t synthesis(sht_plan_s *p, const float2 *yhat, float *y, int64_t B, cudaStream_t st, bool adjoint) {
  const int64_t LM = (int64_t)p->L * p->M;
  for (int64_t b0 = 0; b0 < B; b0 += p->max_batch) {
    const int nb = (int)std::min<int64_t>(p->max_batch, B - b0);
    float *yb = y + b0 * p->nlat * (int64_t)p->nlon;
    if (is_tc(p)) {
      cudaError_t e = traced(p, SHT_KERNEL_PACK, st, [&] {
        RowsItem r{nullptr, const_cast<float2 *>(yhat + b0 * LM), p->d_s_hi, data_lo(p, p->d_s_lo), p->L, p->M, nb, p->ldcb};
        return launch_rows_transpose(true, &r, 1, st);
      });
      if (e != cudaSuccess) return cuda_fail(e, "coefficient repack launch");
      SHT_TRY(synthesis_rows(p, yb, nb, st, adjoint));
      continue;
    }
    cudaError_t e = traced(p, SHT_KERNEL_LEG_INV, st, [&] {
      return launch_leg_inv_f32(table_view(p), p->d_inv_tiles, p->n_inv_tiles, yhat + b0 * LM, p->d_work, p->L,
                                p->M, p->Kh, p->ldc, nb, st);
    });
    if (e != cudaSuccess) return cuda_fail(e, "inverse Legendre launch");
    e = traced(p, SHT_KERNEL_C2R, st, [&] { return c2r_any(p, yb, nb, adjoint, st); });
    if (e != cudaSuccess) return cuda_fail(e, "longitude synthesis launch");
  }
  return SHT_OK;
}

sht_status_t filter_body(sht_plan_s *p, const float2 *x, const float2 *W, float2 *y, int64_t Bm, int Cin, int Cout,
                         int adjoint, cudaStream_t st) {
  const int64_t LM = (int64_t)p->L * p->M;
  const int64_t chunk = 65535;
  const int cin = adjoint ? Cout : Cin, cout = adjoint ? Cin : Cout;
  for (int64_t b0 = 0; b0 < Bm; b0 += chunk) {
    const int64_t nb = std::min<int64_t>(chunk, Bm - b0);
    cudaError_t e = traced(p, SHT_KERNEL_FILTER, st, [&] {
      return launch_filter(x + b0 * cin * LM, W, y + b0 * cout * LM, p->L, p->M, nb, Cin, Cout, adjoint, st);
    });
    if (e != cudaSuccess) return cuda_fail(e, "filter launch");
  }
  return SHT_OK;
}

// One chunk of nb members through the tensor-core block path: forward into
// the l-major rows, real filter weights, tensor-core filter into the split
// rows of the inverse, inverse + synthesis.  adjoint: the block's adjoint in
// x, ISHT^T -> W^H -> SHT^T on the same kernels (the analysis with the
// inverse's mode weights and no latitude weights, the filter with
// conj(W[l][i][o]), the synthesis with the latitude weights); x then has
// Cin = the forward's Cout channels, W is the forward's [L][Cin][Cout].
// Weights above this size (bytes) go through a conj-transposed copy in the
// adjoint block (the strided reads of the on-chip adjoint builder then miss L2).
constexpr size_t kAdjointTransposeBytes = size_t(64) << 20;

// The tensor-core filter of nb members from l-major rows (rows_hi / rows_lo,
// Cin channels per member at kx = block_kx(Cin) columns) into the inverse's
// split rows S; adjoint: output i from input o by conj(W[l][i][o]).
sht_status_t filter_rows_tc(sht_plan_s *p, const __nv_bfloat16 *rows_hi, const __nv_bfloat16 *rows_lo,
                            const void *W, int64_t nb, int Cin, int Cout, bool adjoint, cudaStream_t st) {
  // members' columns packed at kx = 2 Cin rounded to 8: the 64-column K
  // chunks of one member run into the next member's columns, which meet
  // zero weight columns, or past the last member outside the map (read as
  // zero without memory traffic)
  const int kx = block_kx(Cin);
  const int nwr = (2 * Cout + 15) / 16 * 16;
  CUtensorMap ta_hi, ta_lo;
  const int64_t width = std::max<int64_t>(64, nb * (int64_t)kx);
  if (!tc_encode_2d(&ta_hi, rows_hi, width, (int64_t)p->L * p->M, 64, 128, p->ldx) ||
      !tc_encode_2d(&ta_lo, rows_lo ? rows_lo : rows_hi, width, (int64_t)p->L * p->M, 64, 128, p->ldx))
    return fail(SHT_ERR_CUDA, "cuTensorMapEncodeTiled failed for the forward rows");
  cudaError_t e;
  // the adjoint reads conj(W[l][i][o]) along i for each o: strided, which
  // costs little while W sits in L2; a larger W is conj-transposed once per
  // call so that the filter reads it as forward weights, row by row
  const float2 *Wf = (const float2 *)W;
  int wadj = adjoint ? 1 : 0;
  const size_t wbytes = sizeof(float2) * (size_t)p->L * Cin * Cout;
  if (adjoint && wbytes > kAdjointTransposeBytes) {
    if (p->wt_bytes < wbytes) {
      cudaFree(p->d_wt);
      p->d_wt = nullptr;
      p->wt_bytes = 0;
      if ((e = dev_alloc((void **)&p->d_wt, wbytes)) != cudaSuccess) return cuda_fail(e, "adjoint weight allocation");
      p->wt_bytes = wbytes;
    }
    // W is [L][Cin][Cout] in this call's channel names (the forward's [L][Cout][Cin])
    e = traced(p, SHT_KERNEL_FILTER_PREP, st,
               [&] { return launch_transpose_conj((const float2 *)W, p->d_wt, p->L, Cin, Cout, st); });
    if (e != cudaSuccess) return cuda_fail(e, "weight transpose launch");
    Wf = p->d_wt;
    wadj = 0;
  }
  e = traced(p, SHT_KERNEL_FILTER, st, [&] {
    return launch_filter_tc(p->tc, p->d_ftiles, p->n_ftiles, ta_hi, ta_lo, Wf, p->d_s_hi, data_lo(p, p->d_s_lo),
                            p->ldcb, kx, nwr, (int)nb, Cin, Cout, wadj, st);
  });
  if (e != cudaSuccess) return cuda_fail(e, "filter launch");
  return SHT_OK;
}

sht_status_t block_tc(sht_plan_s *p, const float *x, const void *W, float *y, int64_t nb, int Cin, int Cout,
                      cudaStream_t st, bool adjoint = false) {
  const bool split = p->precision == SHT_PREC_SPLIT_BF16;
  RowsOut ro{p->d_x_hi, split ? p->d_x_lo : nullptr, p->ldx, Cin, block_kx(Cin)};
  SHT_TRY(analysis(p, x, nullptr, nb * Cin, st, adjoint, false, &ro));
  SHT_TRY(filter_rows_tc(p, p->d_x_hi, split ? p->d_x_lo : nullptr, W, nb, Cin, Cout, adjoint, st));
  return synthesis_rows(p, y, (int)(nb * Cout), st, adjoint);
}

sht_status_t check_plan(sht_plan_t plan) {
  if (!plan) return fail(SHT_ERR_INVALID_ARG, "plan is NULL");
  return SHT_OK;
}

sht_status_t check_batch(int64_t B) {
  if (B < 0) return fail(SHT_ERR_INVALID_ARG, "batch must be >= 0");
  return SHT_OK;
}

sht_status_t check_ptr(const void *ptr, const char *name) {
  if (!ptr) return fail(SHT_ERR_INVALID_ARG, std::string(name) + " is NULL");
  if (((uintptr_t)ptr) & 15) return fail(SHT_ERR_INVALID_ARG, std::string(name) + " is not 16-byte aligned");
  return SHT_OK;
}

sht_status_t check_channels(sht_plan_s *p, int Cin, int Cout, bool block) {
  if (Cin < 1 || Cout < 1) return fail(SHT_ERR_INVALID_ARG, "channel counts must be >= 1");
  if (block && (int64_t)std::max(Cin, Cout) > p->max_batch)
    return fail(SHT_ERR_INVALID_ARG, "max(Cin, Cout) exceeds the plan's max_batch");
  return SHT_OK;
}


}  // namespace

void grid_nodes(int grid, int nlat, std::vector<double> &x, std::vector<double> &s, std::vector<double> &w) {
  make_grid(grid, nlat, x, s, w);
}

}  // namespace shtgb

using namespace shtgb;

extern "C" {

void sht_plan_opts_default(sht_plan_opts *opts) {
  if (!opts) return;
  std::memset(opts, 0, sizeof(*opts));
  opts->precision = SHT_PREC_FP32;
  opts->device = -1;
  opts->max_batch = 256;
}

sht_status_t sht_plan(sht_plan_t *out, int nlat, int nlon, int grid, int lmax, int mmax, const sht_plan_opts *opts) {
  NvtxRange nvtx_range("sht_plan");
  if (!out) return fail(SHT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  sht_plan_opts o;
  sht_plan_opts_default(&o);
  if (opts) o = *opts;
  if (grid != SHT_GRID_GAUSS && grid != SHT_GRID_EQUIANGULAR_CC && grid != SHT_GRID_EQUIANGULAR_TRAPZ)
    return fail(SHT_ERR_INVALID_ARG, "unknown grid type");
  if (nlat < 1 || nlon < 1 || lmax < 1 || mmax < 1)
    return fail(SHT_ERR_INVALID_ARG, "nlat, nlon, lmax, mmax must be >= 1");
  if (grid != SHT_GRID_GAUSS && nlat < 2) return fail(SHT_ERR_INVALID_ARG, "equiangular grids need nlat >= 2");
  if (mmax > lmax) return fail(SHT_ERR_INVALID_ARG, "mmax must be <= lmax");
  if (mmax > nlon / 2 + 1) return fail(SHT_ERR_INVALID_ARG, "mmax must be <= nlon/2 + 1");
  if (grid == SHT_GRID_GAUSS && lmax > nlat) return fail(SHT_ERR_INVALID_ARG, "Gaussian grids need lmax <= nlat");
  if (o.precision != SHT_PREC_FP32 && o.precision != SHT_PREC_BF16 && o.precision != SHT_PREC_SPLIT_BF16)
    return fail(SHT_ERR_INVALID_ARG, "unknown precision");
  if (o.max_batch < 1) return fail(SHT_ERR_INVALID_ARG, "max_batch must be >= 1");
  for (int r : o.reserved)
    if (r != 0) return fail(SHT_ERR_INVALID_ARG, "reserved option fields must be zero");
  if (o.max_channels < 0) return fail(SHT_ERR_INVALID_ARG, "max_channels must be >= 0");
  if (o.table_source != SHT_TABLE_STREAMED && o.table_source != SHT_TABLE_RECURRENCE &&
      o.table_source != SHT_TABLE_MIXED)
    return fail(SHT_ERR_INVALID_ARG, "unknown table_source");
  if (o.table_source != SHT_TABLE_STREAMED && o.precision != SHT_PREC_FP32 && leg_rows(lmax, 0, 0) > 700)
    return fail(SHT_ERR_UNSUPPORTED, "the on-chip recurrence supports lmax <= 1400");
  if (nlon > kMaxNlon) return fail(SHT_ERR_UNSUPPORTED, "nlon above 8192 is not supported");
  RadixPlan rp;
  if (!factor_radix(nlon, rp)) return fail(SHT_ERR_UNSUPPORTED, "nlon must factor into 2, 3 and 5");

  int dev = o.device;
  if (dev < 0) {
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (dev >= ndev) return fail(SHT_ERR_INVALID_ARG, "device ordinal out of range");
  DeviceGuard guard(dev);

  sht_plan_s *p = new (std::nothrow) sht_plan_s();
  if (!p) return fail(SHT_ERR_OOM, "host allocation failed");
  p->device = dev;
  p->nlat = nlat;
  p->nlon = nlon;
  p->grid = grid;
  p->L = lmax;
  p->M = mmax;
  p->precision = o.precision;
  p->table_source = o.precision == SHT_PREC_FP32 ? SHT_TABLE_STREAMED : o.table_source;
  p->max_batch = o.max_batch;
  p->Kh = (nlat + 1) / 2;
  p->Khp = (p->Kh + 15) / 16 * 16;
  // FP32 workspace row: 2 max_batch columns, rounded to 4 (FP32 plans) or to
  // the 16-column groups of the parity-paired layout (tensor-core plans)
  p->ldc = o.precision == SHT_PREC_FP32 ? (int)((2 * o.max_batch + 3) / 4 * 4)
                                        : (int)((2 * o.max_batch + 15) / 16 * 16);
  p->radix = rp;
  make_grid(grid, nlat, p->x, p->s, p->w);

  auto bail = [&](cudaError_t err, const char *what) {
    sht_status_t st = cuda_fail(err, what);
    free_plan(p);
    return st;
  };

  // table offsets (floats) of the folded blocks (m, p)
  std::vector<int64_t> off(2 * (size_t)mmax + 1);
  int64_t acc = 0;
  for (int m = 0; m < mmax; m++)
    for (int q = 0; q < 2; q++) {
      off[2 * m + q] = acc;
      acc += (int64_t)leg_rows(lmax, m, q) * p->Khp;
    }
  off[2 * mmax] = acc;
  p->tab_off = off;
  p->table_bytes = acc * (int64_t)sizeof(float);

  // tile lists: row tiles of 64 (CUDA cores) or 128 (tensor cores)
  const bool tc = o.precision != SHT_PREC_FP32;
  const int trow = tc ? 128 : 64;
  // block-major order: the row tiles of one (m, p) block run back to back
  // and share its Fourier rows in L2
  std::vector<LegTile> ft, it;
  int64_t frows_acc = 0;
  std::vector<int> roff_h(2 * (size_t)mmax);
  for (int m = 0; m < mmax; m++)
    for (int q = 0; q < 2; q++) {
      roff_h[2 * m + q] = (int)frows_acc;
      frows_acc += leg_rows(lmax, m, q);
    }
  for (int m = 0; m < mmax; m++)
    for (int q = 0; q < 2; q++)
      for (int r0 = 0; r0 < leg_rows(lmax, m, q); r0 += trow)
        ft.push_back(LegTile{m, q, r0, roff_h[2 * m + q] + r0});
  // every (m, p) block gets inverse tiles, also the empty one (m = lmax-1,
  // odd parity): its tiles write the zeros that the synthesis reads
  for (int m = 0; m < mmax; m++)
    for (int q = 0; q < 2; q++)
      for (int k0 = 0; k0 < p->Kh; k0 += trow) it.push_back(LegTile{m, q, k0, m + q});
  p->n_fwd_tiles = (int)ft.size();
  p->n_inv_tiles = (int)it.size();
  // the tiles of one order are consecutive: first tile of each m
  p->fwd_tile_m.assign(mmax + 1, (int)ft.size());
  p->inv_tile_m.assign(mmax + 1, (int)it.size());
  for (int t = (int)ft.size() - 1; t >= 0; t--) p->fwd_tile_m[ft[t].m] = t;
  for (int t = (int)it.size() - 1; t >= 0; t--) p->inv_tile_m[it[t].m] = t;
  for (int m = mmax - 1; m >= 0; m--) {
    p->fwd_tile_m[m] = std::min(p->fwd_tile_m[m], p->fwd_tile_m[m + 1]);
    p->inv_tile_m[m] = std::min(p->inv_tile_m[m], p->inv_tile_m[m + 1]);
  }

  // device tables
  if ((e = dev_alloc((void **)&p->d_err, sizeof(unsigned))) != cudaSuccess) return bail(e, "error word allocation");
  if ((e = cudaMemset(p->d_err, 0, sizeof(unsigned))) != cudaSuccess) return bail(e, "error word memset");
  if (!tc) {
    if ((e = dev_alloc((void **)&p->d_table, (size_t)p->table_bytes)) != cudaSuccess)
      return bail(e, "table allocation");
    if ((e = cudaMemset(p->d_table, 0, (size_t)p->table_bytes)) != cudaSuccess) return bail(e, "table memset");
  } else {
    p->table_bytes = 0;
  }
  if ((e = upload(&p->d_tab_off, off)) != cudaSuccess) return bail(e, "offset upload");
  if ((e = upload(&p->d_fwd_tiles, ft)) != cudaSuccess) return bail(e, "tile upload");
  if ((e = upload(&p->d_inv_tiles, it)) != cudaSuccess) return bail(e, "tile upload");
  std::vector<float2> tw(nlon);
  for (int q = 0; q < nlon; q++) {
    double ph = 2.0 * kPi * (double)q / (double)nlon;
    tw[q] = make_float2((float)std::cos(ph), (float)-std::sin(ph));
  }
  if ((e = upload(&p->d_twiddle, tw)) != cudaSuccess) return bail(e, "twiddle upload");
  std::vector<float> ringw(nlat);
  for (int k = 0; k < nlat; k++) ringw[k] = (float)(p->w[k] * 2.0 * kPi / (double)nlon);
  if ((e = upload(&p->d_ring_w, ringw)) != cudaSuccess) return bail(e, "weight upload");
  std::vector<float> zonal(nlat);
  for (int k = 0; k < nlat; k++) {
    const double d = 2.0 * kPi / (double)nlon;
    zonal[k] = (float)(2.0 * kPi * p->s[k] * d * d);
  }
  if ((e = upload(&p->d_zonal_c, zonal)) != cudaSuccess) return bail(e, "weight upload");

  // FP64 generation of the table on the device
  {
    std::vector<double> a((size_t)lmax * mmax, 0.0), b((size_t)lmax * mmax, 0.0), seed(mmax + 1, 0.0);
    for (int m = 0; m < mmax; m++)
      for (int l = m + 2; l < lmax; l++) {
        double dl = l, dm = m;
        a[(size_t)l * mmax + m] = std::sqrt((4.0 * dl * dl - 1.0) / (dl * dl - dm * dm));
        b[(size_t)l * mmax + m] = std::sqrt(((dl - 1.0) * (dl - 1.0) - dm * dm) / (4.0 * (dl - 1.0) * (dl - 1.0) - 1.0));
      }
    for (int i = 1; i <= mmax; i++) seed[i] = -std::sqrt((2.0 * i + 1.0) / (2.0 * i));
    std::vector<double> xh(p->x.begin(), p->x.begin() + p->Kh), sh(p->s.begin(), p->s.begin() + p->Kh);
    double *d_x = nullptr, *d_s = nullptr, *d_a = nullptr, *d_b = nullptr, *d_seed = nullptr;
    e = upload(&d_x, xh);
    if (e == cudaSuccess) e = upload(&d_s, sh);
    if (e == cudaSuccess) e = upload(&d_a, a);
    if (e == cudaSuccess) e = upload(&d_b, b);
    if (e == cudaSuccess) e = upload(&d_seed, seed);
    if (e == cudaSuccess && !tc)
      e = launch_table_gen_f32(p->d_table, p->d_tab_off, p->Khp, d_x, d_s, d_a, d_b, d_seed, lmax, mmax, p->Kh, 0);
    if (e == cudaSuccess && tc) {
      // tensor-core plans: the Legendre table either as bf16 hi/lo tables
      // streamed by TMA (one layout [rows][Kp64] for both directions), or
      // generated on chip from seeds every 32
      // rows of every (m, p) (FP64, stored as FP32), FP32 recurrence coefficients (zero past
      // lmax) and the latitudes as hi + lo
      const bool split = o.precision == SHT_PREC_SPLIT_BF16;
      // the forward streams the table unless it is generated everywhere;
      // the inverse generates it unless it is streamed everywhere
      const bool gen_fwd = o.table_source == SHT_TABLE_RECURRENCE;
      const bool gen_inv = o.table_source != SHT_TABLE_STREAMED;
      std::vector<int> roff(2 * (size_t)mmax);
      int64_t frows = 0;
      for (int m = 0; m < mmax; m++)
        for (int q = 0; q < 2; q++) {
          roff[2 * m + q] = (int)frows;
          frows += leg_rows(lmax, m, q);
        }
      e = upload(&p->d_roff, roff);
      TcPlanView &T = p->tc;
      T.gen_fwd = gen_fwd;
      T.gen_inv = gen_inv;
      p->table_bytes = 0;
      if (!gen_fwd) {
        // streamed table: the forward layout [rows i of the (m, p) blocks]
        // [Kp64 latitudes k']; the forward contraction reads it K-major
        // (boxes of 64 k' x 128 rows), the inverse MN-major (boxes of 64 k'
        // x 64 rows: A = T^T with k' contiguous), so one table serves both
        const int Kp64 = (p->Kh + 63) / 64 * 64;
        const size_t fbytes = sizeof(__nv_bfloat16) * (size_t)frows * Kp64;
        if (e == cudaSuccess) e = dev_alloc((void **)&p->d_tf_hi, fbytes);
        if (e == cudaSuccess) e = dev_alloc((void **)&p->d_tf_lo, fbytes);
        if (e == cudaSuccess) e = cudaMemset(p->d_tf_hi, 0, fbytes);
        if (e == cudaSuccess) e = cudaMemset(p->d_tf_lo, 0, fbytes);
        if (e == cudaSuccess)
          e = launch_table_gen_bf16(p->d_tf_hi, p->d_tf_lo, p->d_roff, Kp64, d_x, d_s, d_a,
                                    d_b, d_seed, lmax, mmax, p->Kh, 0);
        p->table_bytes += (int64_t)fbytes * 2;
        // the K chunks of each tile that hold non-negligible table entries
        // (polar latitudes of high orders hold none)
        if (e == cudaSuccess) e = dev_alloc((void **)&p->d_fwd_krange, sizeof(int2) * (size_t)p->n_fwd_tiles);
        if (e == cudaSuccess)
          e = launch_tile_krange(p->d_tf_hi, Kp64, p->d_roff, p->d_fwd_tiles, p->n_fwd_tiles, 0, lmax, p->Kh,
                                 p->d_fwd_krange, 0);
        if (e == cudaSuccess && !gen_inv)
          e = dev_alloc((void **)&p->d_inv_krange, sizeof(int2) * (size_t)p->n_inv_tiles);
        if (e == cudaSuccess && !gen_inv)
          e = launch_tile_krange(p->d_tf_hi, Kp64, p->d_roff, p->d_inv_tiles, p->n_inv_tiles, 1, lmax, p->Kh,
                                 p->d_inv_krange, 0);
        if (e == cudaSuccess &&
            // maps Kh columns wide (row pitch Kp64): the boxes' columns past
            // Kh read zeros without memory traffic
            !(tc_encode_2d(&T.tab_fwd_hi, p->d_tf_hi, p->Kh, frows, 64, 128, Kp64) &&
              tc_encode_2d(&T.tab_fwd_lo, p->d_tf_lo, p->Kh, frows, 64, 128, Kp64) &&
              tc_encode_2d(&T.tab_inv_hi, p->d_tf_hi, p->Kh, frows, 64, 64, Kp64) &&
              tc_encode_2d(&T.tab_inv_lo, p->d_tf_lo, p->Kh, frows, 64, 64, Kp64)))
          e = cudaErrorInvalidValue;
      }
      if (gen_inv) {
        const int NB = (leg_rows(lmax, 0, 0) + 31) / 32 + 1;
        const size_t seed_bytes = sizeof(float2) * (size_t)mmax * 2 * NB * p->Kh;
        // two-step coefficients of row i (l = m + p + 2 i): the step to the
        // row after next, zero where that row is past lmax
        const int ldC = (leg_rows(lmax, 0, 0) + 63) / 64 * 64 + 64;
        auto A = [](double n, double m) { return std::sqrt((4.0 * n * n - 1.0) / (n * n - m * m)); };
        auto Bc = [](double n, double m) {
          return std::sqrt(((n - 1.0) * (n - 1.0) - m * m) / (4.0 * (n - 1.0) * (n - 1.0) - 1.0));
        };
        std::vector<float4> coef((size_t)mmax * 2 * ldC, make_float4(0.f, 0.f, 0.f, 0.f));
        for (int m = 0; m < mmax; m++)
          for (int q = 0; q < 2; q++)
            for (int i = 0; i < leg_rows(lmax, m, q); i++) {
              const int l = m + q + 2 * i;
              if (l + 2 >= lmax) continue;
              const double a2 = A(l + 2, m), a1 = A(l + 1, m), b2 = Bc(l + 2, m), b1 = Bc(l + 1, m);
              double al = a2 * a1, be, ga;
              if (l == m) {
                be = -a2 * b2;
                ga = 0.0;
              } else {
                const double a0 = A(l, m), b0 = Bc(l, m);
                be = -a2 * (b2 + a1 * b1 / a0);
                ga = -a2 * a1 * b1 * b0;
              }
              coef[((size_t)m * 2 + q) * ldC + i] = make_float4((float)al, (float)be, (float)ga, 0.f);
            }
        std::vector<float> x2hv(p->Kh), x2lv(p->Kh);
        for (int k = 0; k < p->Kh; k++) {
          const double x2 = p->x[k] * p->x[k];
          x2hv[k] = (float)x2;
          x2lv[k] = (float)(x2 - (double)x2hv[k]);
        }
        if (e == cudaSuccess) e = upload(&p->d_coef, coef);
        if (e == cudaSuccess) e = upload(&p->d_x2h, x2hv);
        if (e == cudaSuccess) e = upload(&p->d_x2l, x2lv);
        if (e == cudaSuccess) e = dev_alloc(&p->d_seeds, seed_bytes);
        if (e == cudaSuccess) e = cudaMemset(p->d_seeds, 0, seed_bytes);
        if (e == cudaSuccess)
          e = launch_seed_gen(p->d_seeds, NB, d_x, d_s, d_a, d_b, d_seed, lmax, mmax, p->Kh, 0);
        p->table_bytes += (int64_t)(seed_bytes + sizeof(float4) * coef.size());
        T.seeds = p->d_seeds;
        T.coef = p->d_coef;
        T.x2h = p->d_x2h;
        T.x2l = p->d_x2l;
        T.NB = NB;
        T.ldC = ldC;
      }
      T.roff = p->d_roff;
      T.L = lmax;
      T.M = mmax;
      T.Kh = p->Kh;
      T.split = split;
      T.err = p->d_err;
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d_x);
    cudaFree(d_s);
    cudaFree(d_a);
    cudaFree(d_b);
    cudaFree(d_seed);
    if (e != cudaSuccess) return bail(e, "table generation");
  }

  // workspaces
  p->ldcb = (int)std::max<int64_t>(64, (2 * o.max_batch + 7) / 8 * 8);
  // folded Fourier workspaces.  The analysis output is (m, p)-major: the
  // forward contraction reads whole (m, p) blocks of contiguous rows.  The
  // synthesis input of the tensor-core plans is parity-paired, so that the
  // longitude synthesis reads E and O of 8 fields as one 128-byte line
  // (the inverse contraction stores whole 16-column groups through TMA);
  // the FP32 contraction writes (m, p)-major rows.  (A ring-major layout
  // measured no faster for the longitude kernels at 721 x 1440 and slower
  // for the tensor-core gathers.)
  p->lay_f = classic_layout(p->Kh, tc ? p->ldcb : p->ldc);
  p->lay_g = tc ? pair_layout(p->Kh, p->ldc) : classic_layout(p->Kh, p->ldc);
  const size_t frow = (size_t)mmax * 2 * p->Kh;
  const size_t work = std::max(sizeof(float) * frow * p->ldc, tc ? 2 * sizeof(__nv_bfloat16) * frow * p->ldcb : 0);
  // spec_b also holds the FP32 l-major rows of the tensor-core forward into
  // the API layout: [lmax mmax][ldr] floats, ldr = 2 max_batch rounded to 4
  p->ldr = (int)((2 * o.max_batch + 3) / 4 * 4);
  const size_t spec = std::max(sizeof(float2) * (size_t)o.max_batch * lmax * mmax,
                               tc ? sizeof(float) * (size_t)lmax * mmax * p->ldr : 0);
  size_t extra = 0;
  if ((e = dev_alloc((void **)&p->d_work, work)) != cudaSuccess) return bail(e, "workspace allocation");
  if (!tc && (e = dev_alloc((void **)&p->d_spec_a, spec)) != cudaSuccess) return bail(e, "workspace allocation");
  if ((e = dev_alloc((void **)&p->d_spec_b, spec)) != cudaSuccess) return bail(e, "workspace allocation");
  if ((e = cudaMemset(p->d_work, 0, work)) != cudaSuccess) return bail(e, "workspace memset");
  if (tc) {
    // internal coefficient rows S, l-major [lmax][mmax][ldcb] (rows m > l unused)
    p->srows = (int64_t)lmax * mmax;
    const size_t sbytes = sizeof(__nv_bfloat16) * (size_t)p->srows * p->ldcb;
    if ((e = dev_alloc((void **)&p->d_s_hi, sbytes)) != cudaSuccess) return bail(e, "workspace allocation");
    if ((e = dev_alloc((void **)&p->d_s_lo, sbytes)) != cudaSuccess) return bail(e, "workspace allocation");
    if ((e = cudaMemset(p->d_s_hi, 0, sbytes)) != cudaSuccess) return bail(e, "workspace memset");
    if ((e = cudaMemset(p->d_s_lo, 0, sbytes)) != cudaSuccess) return bail(e, "workspace memset");
    // l-major forward rows for the tensor-core filter, real filter weights,
    // filter tiles (l, m0)
    p->max_channels = o.max_channels > 0 ? o.max_channels : (int)std::min<int64_t>(o.max_batch, 128);
    p->ldx = (int)std::max<int64_t>(64, (2 * o.max_batch + 63) / 64 * 64);
    const size_t xbytes = sizeof(__nv_bfloat16) * (size_t)lmax * mmax * p->ldx;
    std::vector<int2> ftl;
    for (int l = 0; l < lmax; l++)
      for (int m0 = 0; m0 < std::min(l + 1, mmax); m0 += 128) ftl.push_back(make_int2(l, m0));
    p->n_ftiles = (int)ftl.size();
    if ((e = dev_alloc((void **)&p->d_x_hi, xbytes)) != cudaSuccess) return bail(e, "workspace allocation");
    if ((e = dev_alloc((void **)&p->d_x_lo, xbytes)) != cudaSuccess) return bail(e, "workspace allocation");
    if ((e = upload((int2 **)&p->d_ftiles, ftl)) != cudaSuccess) return bail(e, "tile upload");
    // the padding columns stay zero: the filter's K chunks read them
    if ((e = cudaMemset(p->d_x_hi, 0, xbytes)) != cudaSuccess) return bail(e, "workspace memset");
    if ((e = cudaMemset(p->d_x_lo, 0, xbytes)) != cudaSuccess) return bail(e, "workspace memset");
    extra = 2 * sbytes + 2 * xbytes;
    TcPlanView &T = p->tc;
    if (!(tc_encode_2d(&T.x_hi, p->d_x_hi, p->ldx, (int64_t)lmax * mmax, 64, 128) &&
          tc_encode_2d(&T.x_lo, p->d_x_lo, p->ldx, (int64_t)lmax * mmax, 64, 128))) {
      free_plan(p);
      return fail(SHT_ERR_CUDA, "cuTensorMapEncodeTiled failed for the forward rows");
    }
    T.gw = p->d_work;
    T.gw_ldc = p->ldc;
    T.gpair = p->lay_g.cg;
    T.xrows_hi = p->d_x_hi;
    T.ldx = p->ldx;
    T.srows_hi = p->d_s_hi;
    T.lds = p->ldcb;
    T.frows = reinterpret_cast<const float *>(p->d_spec_b);
    T.ldr = p->ldr;
    if (!(tc_encode_lrows_bf16(&T.xo32_hi, p->d_x_hi, p->ldx, mmax, lmax, 32) &&
          tc_encode_lrows_bf16(&T.xo32_lo, p->d_x_lo, p->ldx, mmax, lmax, 32) &&
          tc_encode_lrows_bf16(&T.xo16_hi, p->d_x_hi, p->ldx, mmax, lmax, 16) &&
          tc_encode_lrows_bf16(&T.xo16_lo, p->d_x_lo, p->ldx, mmax, lmax, 16) &&
          tc_encode_lrows_f32(&T.ro32, T.frows, p->ldr, mmax, lmax, 32) &&
          tc_encode_lrows_f32(&T.ro16, T.frows, p->ldr, mmax, lmax, 16))) {
      free_plan(p);
      return fail(SHT_ERR_CUDA, "cuTensorMapEncodeTiled failed for the forward rows");
    }
    if (!(tc_encode_fold_f32(&T.g32, p->d_work, p->lay_g, p->ldc, 2 * mmax, p->Kh, 32) &&
          tc_encode_fold_f32(&T.g16, p->d_work, p->lay_g, p->ldc, 2 * mmax, p->Kh, 16))) {
      free_plan(p);
      return fail(SHT_ERR_CUDA, "cuTensorMapEncodeTiled failed for the inverse output");
    }
    if (!(tc_encode_fold_bf16(&T.f_hi, f_hi(p), p->lay_f, p->ldcb, 2 * mmax, p->Kh, 64) &&
          tc_encode_fold_bf16(&T.f_lo, f_lo(p), p->lay_f, p->ldcb, 2 * mmax, p->Kh, 64) &&
          tc_encode_fold_bf16(&T.fh_hi, f_hi(p), p->lay_f, p->ldcb, 2 * mmax, p->Kh, 32) &&
          tc_encode_fold_bf16(&T.fh_lo, f_lo(p), p->lay_f, p->ldcb, 2 * mmax, p->Kh, 32) &&
          tc_encode_srows_bf16(&T.s_hi, p->d_s_hi, p->ldcb, mmax, lmax, true, 64) &&
          tc_encode_srows_bf16(&T.s_lo, p->d_s_lo, p->ldcb, mmax, lmax, true, 64) &&
          tc_encode_srows_bf16(&T.sh_hi, p->d_s_hi, p->ldcb, mmax, lmax, true, 64, 32) &&
          tc_encode_srows_bf16(&T.sh_lo, p->d_s_lo, p->ldcb, mmax, lmax, true, 64, 32) &&
          tc_encode_srows_bf16(&T.so32_hi, p->d_s_hi, p->ldcb, mmax, lmax, false, 32) &&
          tc_encode_srows_bf16(&T.so32_lo, p->d_s_lo, p->ldcb, mmax, lmax, false, 32) &&
          tc_encode_srows_bf16(&T.so16_hi, p->d_s_hi, p->ldcb, mmax, lmax, false, 16) &&
          tc_encode_srows_bf16(&T.so16_lo, p->d_s_lo, p->ldcb, mmax, lmax, false, 16))) {
      free_plan(p);
      return fail(SHT_ERR_CUDA, "cuTensorMapEncodeTiled failed for the workspaces");
    }
  }
  p->workspace_bytes = (int64_t)(work + (tc ? 1 : 2) * spec + extra);

  *out = p;
  return SHT_OK;
}

sht_status_t sht_plan_destroy(sht_plan_t plan) {
  if (!plan) return fail(SHT_ERR_INVALID_ARG, "plan is NULL");
  cudaError_t pending;
  {
    DeviceGuard g(plan->device);
    pending = cudaGetLastError();
  }
  free_plan(plan);
  if (pending != cudaSuccess) return cuda_fail(pending, "pending CUDA error");
  return SHT_OK;
}

sht_status_t sht_plan_info(sht_plan_t p, int *nlat, int *nlon, int *grid, int *lmax, int *mmax, int *precision,
                           int64_t *max_batch, int64_t *table_bytes, int64_t *workspace_bytes) {
  SHT_TRY(check_plan(p));
  if (nlat) *nlat = p->nlat;
  if (nlon) *nlon = p->nlon;
  if (grid) *grid = p->grid;
  if (lmax) *lmax = p->L;
  if (mmax) *mmax = p->M;
  if (precision) *precision = p->precision;
  if (max_batch) *max_batch = p->max_batch;
  if (table_bytes) *table_bytes = p->table_bytes;
  if (workspace_bytes) *workspace_bytes = p->workspace_bytes;
  return SHT_OK;
}

sht_status_t sht_plan_grid(sht_plan_t p, double *x, double *w) {
  SHT_TRY(check_plan(p));
  if (x) std::memcpy(x, p->x.data(), sizeof(double) * p->nlat);
  if (w) std::memcpy(w, p->w.data(), sizeof(double) * p->nlat);
  return SHT_OK;
}

sht_status_t sht_forward(sht_plan_t p, const float *x, void *xhat, int64_t B, void *stream) {
  NvtxRange nvtx_range("sht_forward");
  SHT_TRY(check_plan(p));
  SHT_TRY(check_batch(B));
  if (B == 0) return SHT_OK;
  SHT_TRY(check_ptr(x, "x"));
  SHT_TRY(check_ptr(xhat, "xhat"));
  DeviceGuard g(p->device);
  return analysis(p, x, (float2 *)xhat, B, (cudaStream_t)stream, false, true);
}

sht_status_t sht_inverse_adjoint(sht_plan_t p, const float *gx, void *gxhat, int64_t B, void *stream) {
  NvtxRange nvtx_range("sht_inverse_adjoint");
  SHT_TRY(check_plan(p));
  SHT_TRY(check_batch(B));
  if (B == 0) return SHT_OK;
  SHT_TRY(check_ptr(gx, "gx"));
  SHT_TRY(check_ptr(gxhat, "gxhat"));
  DeviceGuard g(p->device);
  return analysis(p, gx, (float2 *)gxhat, B, (cudaStream_t)stream, true, true);
}

sht_status_t sht_inverse(sht_plan_t p, const void *xhat, float *x, int64_t B, void *stream) {
  NvtxRange nvtx_range("sht_inverse");
  SHT_TRY(check_plan(p));
  SHT_TRY(check_batch(B));
  if (B == 0) return SHT_OK;
  SHT_TRY(check_ptr(xhat, "xhat"));
  SHT_TRY(check_ptr(x, "x"));
  DeviceGuard g(p->device);
  return synthesis(p, (const float2 *)xhat, x, B, (cudaStream_t)stream, false);
}

sht_status_t sht_forward_adjoint(sht_plan_t p, const void *gxhat, float *gx, int64_t B, void *stream) {
  NvtxRange nvtx_range("sht_forward_adjoint");
  SHT_TRY(check_plan(p));
  SHT_TRY(check_batch(B));
  if (B == 0) return SHT_OK;
  SHT_TRY(check_ptr(gxhat, "gxhat"));
  SHT_TRY(check_ptr(gx, "gx"));
  DeviceGuard g(p->device);
  return synthesis(p, (const float2 *)gxhat, gx, B, (cudaStream_t)stream, true);
}

sht_status_t spectral_filter(sht_plan_t p, const void *xhat, const void *W, void *yhat, int64_t Bm, int Cin, int Cout,
                             void *stream) {
  NvtxRange nvtx_range("spectral_filter");
  SHT_TRY(check_plan(p));
  SHT_TRY(check_batch(Bm));
  SHT_TRY(check_channels(p, Cin, Cout, false));
  if (Bm == 0) return SHT_OK;
  SHT_TRY(check_ptr(xhat, "xhat"));
  SHT_TRY(check_ptr(W, "W"));
  SHT_TRY(check_ptr(yhat, "yhat"));
  DeviceGuard g(p->device);
  return filter_body(p, (const float2 *)xhat, (const float2 *)W, (float2 *)yhat, Bm, Cin, Cout, 0,
                     (cudaStream_t)stream);
}

sht_status_t spectral_filter_adjoint(sht_plan_t p, const void *gy, const void *W, const void *xhat, void *gx, void *gW,
                                     int64_t Bm, int Cin, int Cout, void *stream) {
  NvtxRange nvtx_range("spectral_filter_adjoint");
  SHT_TRY(check_plan(p));
  SHT_TRY(check_batch(Bm));
  SHT_TRY(check_channels(p, Cin, Cout, false));
  SHT_TRY(check_ptr(gy, "gy"));
  SHT_TRY(check_ptr(W, "W"));
  if (gW) SHT_TRY(check_ptr(xhat, "xhat"));
  if (gx) SHT_TRY(check_ptr(gx, "gx"));
  if (gW) SHT_TRY(check_ptr(gW, "gW"));
  DeviceGuard g(p->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (gx && Bm > 0) SHT_TRY(filter_body(p, (const float2 *)gy, (const float2 *)W, (float2 *)gx, Bm, Cin, Cout, 1, st));
  if (gW) {
    cudaError_t e = traced(p, SHT_KERNEL_FILTER_DW, st, [&] {
      return launch_filter_dw((const float2 *)gy, (const float2 *)xhat, (float2 *)gW, p->L, p->M, Bm, Cin, Cout, st);
    });
    if (e != cudaSuccess) return cuda_fail(e, "weight adjoint launch");
  }
  return SHT_OK;
}

sht_status_t sht_spectral_block(sht_plan_t p, const float *x, const void *W, float *y, int64_t Bm, int Cin, int Cout,
                                void *stream) {
  NvtxRange nvtx_range("sht_spectral_block");
  SHT_TRY(check_plan(p));
  SHT_TRY(check_batch(Bm));
  SHT_TRY(check_channels(p, Cin, Cout, true));
  if (Bm == 0) return SHT_OK;
  SHT_TRY(check_ptr(x, "x"));
  SHT_TRY(check_ptr(W, "W"));
  SHT_TRY(check_ptr(y, "y"));
  DeviceGuard g(p->device);
  cudaStream_t st = (cudaStream_t)stream;
  int64_t per = p->max_batch / std::max(Cin, Cout);
  if (is_tc(p)) {
    if (std::max(Cin, Cout) > p->max_channels)
      return fail(SHT_ERR_INVALID_ARG, "max(Cin, Cout) exceeds the plan's max_channels");
    per = std::min<int64_t>(per, p->ldx / block_kx(Cin));
  }
  const int64_t npix = (int64_t)p->nlat * p->nlon;
  for (int64_t b0 = 0; b0 < Bm; b0 += per) {
    const int64_t nb = std::min(per, Bm - b0);
    if (is_tc(p)) {
      SHT_TRY(block_tc(p, x + b0 * Cin * npix, W, y + b0 * Cout * npix, nb, Cin, Cout, st));
      continue;
    }
    SHT_TRY(analysis(p, x + b0 * Cin * npix, p->d_spec_a, nb * Cin, st, false, false));
    SHT_TRY(filter_body(p, p->d_spec_a, (const float2 *)W, p->d_spec_b, nb, Cin, Cout, 0, st));
    SHT_TRY(synthesis(p, p->d_spec_b, y + b0 * Cout * npix, nb * Cout, st, false));
  }
  return SHT_OK;
}

sht_status_t sht_spectral_block_adjoint(sht_plan_t p, const float *gy, const void *W, float *gx, int64_t Bm, int Cin,
                                        int Cout, void *stream) {
  NvtxRange nvtx_range("sht_spectral_block_adjoint");
  SHT_TRY(check_plan(p));
  SHT_TRY(check_batch(Bm));
  SHT_TRY(check_channels(p, Cin, Cout, true));
  if (Bm == 0) return SHT_OK;
  SHT_TRY(check_ptr(gy, "gy"));
  SHT_TRY(check_ptr(W, "W"));
  SHT_TRY(check_ptr(gx, "gx"));
  DeviceGuard g(p->device);
  cudaStream_t st = (cudaStream_t)stream;
  int64_t per = p->max_batch / std::max(Cin, Cout);
  if (is_tc(p)) {
    if (std::max(Cin, Cout) > p->max_channels)
      return fail(SHT_ERR_INVALID_ARG, "max(Cin, Cout) exceeds the plan's max_channels");
    per = std::min<int64_t>(per, p->ldx / block_kx(Cout));
  }
  const int64_t npix = (int64_t)p->nlat * p->nlon;
  for (int64_t b0 = 0; b0 < Bm; b0 += per) {
    const int64_t nb = std::min(per, Bm - b0);
    const float *gyb = gy + b0 * Cout * npix;
    float *gxb = gx + b0 * Cin * npix;
    if (is_tc(p)) {
      SHT_TRY(block_tc(p, gyb, W, gxb, nb, Cout, Cin, st, true));
      continue;
    }
    SHT_TRY(analysis(p, gyb, p->d_spec_a, nb * Cout, st, true, true));
    SHT_TRY(filter_body(p, p->d_spec_a, (const float2 *)W, p->d_spec_b, nb, Cin, Cout, 1, st));
    SHT_TRY(synthesis(p, p->d_spec_b, gxb, nb * Cin, st, true));
  }
  return SHT_OK;
}

namespace {
// The weight gradient's second rows buffer (ISHT^T(gy) rows) and its view:
// a copy of the plan's tensor-core view with the forward-row maps re-encoded
// for it.  Rows m > l stay zero (the forward writes l >= m only), as the
// contraction requires.
sht_status_t ensure_grad_rows(sht_plan_s *p, cudaStream_t st) {
  if (p->d_g_hi) return SHT_OK;
  const size_t xbytes = sizeof(__nv_bfloat16) * (size_t)p->L * p->M * p->ldx;
  cudaError_t e;
  if ((e = dev_alloc((void **)&p->d_g_hi, xbytes)) != cudaSuccess) return cuda_fail(e, "gradient rows allocation");
  if ((e = dev_alloc((void **)&p->d_g_lo, xbytes)) != cudaSuccess) {
    cudaFree(p->d_g_hi);
    p->d_g_hi = nullptr;
    return cuda_fail(e, "gradient rows allocation");
  }
  if ((e = cudaMemsetAsync(p->d_g_hi, 0, xbytes, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(p->d_g_lo, 0, xbytes, st)) != cudaSuccess)
    return cuda_fail(e, "gradient rows memset");
  TcPlanView &T = p->tc_g;
  T = p->tc;
  T.xrows_hi = p->d_g_hi;
  if (!(tc_encode_2d(&T.x_hi, p->d_g_hi, p->ldx, (int64_t)p->L * p->M, 64, 128) &&
        tc_encode_2d(&T.x_lo, p->d_g_lo, p->ldx, (int64_t)p->L * p->M, 64, 128) &&
        tc_encode_lrows_bf16(&T.xo32_hi, p->d_g_hi, p->ldx, p->M, p->L, 32) &&
        tc_encode_lrows_bf16(&T.xo32_lo, p->d_g_lo, p->ldx, p->M, p->L, 32) &&
        tc_encode_lrows_bf16(&T.xo16_hi, p->d_g_hi, p->ldx, p->M, p->L, 16) &&
        tc_encode_lrows_bf16(&T.xo16_lo, p->d_g_lo, p->ldx, p->M, p->L, 16)))
    return fail(SHT_ERR_CUDA, "cuTensorMapEncodeTiled failed for the gradient rows");
  p->workspace_bytes += (int64_t)(2 * xbytes);
  return SHT_OK;
}
}  // namespace

sht_status_t sht_spectral_block_weight_grad(sht_plan_t p, const float *x, const float *gy, void *gW, int64_t Bm,
                                            int Cin, int Cout, void *stream) {
  NvtxRange nvtx_range("sht_spectral_block_weight_grad");
  SHT_TRY(check_plan(p));
  SHT_TRY(check_batch(Bm));
  SHT_TRY(check_channels(p, Cin, Cout, true));
  SHT_TRY(check_ptr(gW, "gW"));
  DeviceGuard g(p->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t LM = (int64_t)p->L * p->M;
  if (Bm == 0) {
    const cudaError_t e = cudaMemsetAsync(gW, 0, sizeof(float2) * (size_t)p->L * Cout * Cin, st);
    return e == cudaSuccess ? SHT_OK : cuda_fail(e, "gradient memset");
  }
  SHT_TRY(check_ptr(x, "x"));
  SHT_TRY(check_ptr(gy, "gy"));
  const int64_t npix = (int64_t)p->nlat * p->nlon;
  int64_t per = p->max_batch / std::max(Cin, Cout);
  if (is_tc(p)) {
    if (std::max(Cin, Cout) > p->max_channels)
      return fail(SHT_ERR_INVALID_ARG, "max(Cin, Cout) exceeds the plan's max_channels");
    SHT_TRY(ensure_grad_rows(p, st));
    const int kxa = block_kx(Cout), kxb = block_kx(Cin);
    per = std::min<int64_t>(per, p->ldx / std::max(kxa, kxb));
    const bool split = p->precision == SHT_PREC_SPLIT_BF16;
    for (int64_t b0 = 0; b0 < Bm; b0 += per) {
      const int64_t nb = std::min(per, Bm - b0);
      RowsOut rx{p->d_x_hi, split ? p->d_x_lo : nullptr, p->ldx, Cin, kxb, &p->tc};
      SHT_TRY(analysis(p, x + b0 * Cin * npix, nullptr, nb * Cin, st, false, false, &rx));
      RowsOut rg{p->d_g_hi, split ? p->d_g_lo : nullptr, p->ldx, Cout, kxa, &p->tc_g};
      SHT_TRY(analysis(p, gy + b0 * Cout * npix, nullptr, nb * Cout, st, true, false, &rg));
      const cudaError_t e = traced(p, SHT_KERNEL_FILTER_DW, st, [&] {
        return launch_dw_tc(p->d_g_hi, split ? p->d_g_lo : nullptr, p->d_x_hi, split ? p->d_x_lo : nullptr, p->ldx,
                            (float2 *)gW, p->L, p->M, (int)nb, Cin, Cout, kxa, kxb, b0 > 0 ? 1 : 0, p->d_err, st);
      });
      if (e != cudaSuccess) return cuda_fail(e, "weight gradient launch");
    }
    return SHT_OK;
  }
  // FP32 plans: the API transforms into the spectral buffers and the FP32
  // contraction, accumulated over member chunks
  for (int64_t b0 = 0; b0 < Bm; b0 += per) {
    const int64_t nb = std::min(per, Bm - b0);
    SHT_TRY(analysis(p, x + b0 * Cin * npix, p->d_spec_a, nb * Cin, st, false, true));
    SHT_TRY(analysis(p, gy + b0 * Cout * npix, p->d_spec_b, nb * Cout, st, true, true));
    const cudaError_t e = traced(p, SHT_KERNEL_FILTER_DW, st, [&] {
      return launch_filter_dw(p->d_spec_b, p->d_spec_a, (float2 *)gW, p->L, p->M, nb, Cin, Cout, st, b0 > 0 ? 1 : 0);
    });
    if (e != cudaSuccess) return cuda_fail(e, "weight gradient launch");
  }
  (void)LM;
  return SHT_OK;
}

sht_status_t sht_spectral_block_backward(sht_plan_t p, const float *x, const float *gy, const void *W, float *gx,
                                         void *gW, int64_t Bm, int Cin, int Cout, void *stream) {
  NvtxRange nvtx_range("sht_spectral_block_backward");
  SHT_TRY(check_plan(p));
  SHT_TRY(check_batch(Bm));
  SHT_TRY(check_channels(p, Cin, Cout, true));
  if (!gx && !gW) return SHT_OK;
  if (gx) SHT_TRY(check_ptr(W, "W"));
  if (!is_tc(p)) {
    // FP32 plans: the two calls (no shared intermediate on this path)
    if (gx) SHT_TRY(sht_spectral_block_adjoint(p, gy, W, gx, Bm, Cin, Cout, stream));
    if (gW) SHT_TRY(sht_spectral_block_weight_grad(p, x, gy, gW, Bm, Cin, Cout, stream));
    return SHT_OK;
  }
  DeviceGuard g(p->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (std::max(Cin, Cout) > p->max_channels)
    return fail(SHT_ERR_INVALID_ARG, "max(Cin, Cout) exceeds the plan's max_channels");
  if (Bm == 0) {
    if (gW) {
      const cudaError_t e = cudaMemsetAsync(gW, 0, sizeof(float2) * (size_t)p->L * Cout * Cin, st);
      if (e != cudaSuccess) return cuda_fail(e, "gradient memset");
    }
    return SHT_OK;
  }
  SHT_TRY(check_ptr(gy, "gy"));
  if (gW) SHT_TRY(check_ptr(x, "x"));
  SHT_TRY(ensure_grad_rows(p, st));
  const int kxa = block_kx(Cout), kxb = block_kx(Cin);
  int64_t per = p->max_batch / std::max(Cin, Cout);
  per = std::min<int64_t>(per, p->ldx / std::max(kxa, kxb));
  const bool split = p->precision == SHT_PREC_SPLIT_BF16;
  const int64_t npix = (int64_t)p->nlat * p->nlon;
  for (int64_t b0 = 0; b0 < Bm; b0 += per) {
    const int64_t nb = std::min(per, Bm - b0);
    // ISHT^T(gy) once, into the gradient rows: the input gradient's filter
    // and the weight gradient both read it
    RowsOut rg{p->d_g_hi, split ? p->d_g_lo : nullptr, p->ldx, Cout, kxa, &p->tc_g};
    SHT_TRY(analysis(p, gy + b0 * Cout * npix, nullptr, nb * Cout, st, true, false, &rg));
    if (gx) {
      SHT_TRY(filter_rows_tc(p, p->d_g_hi, split ? p->d_g_lo : nullptr, W, nb, Cout, Cin, true, st));
      SHT_TRY(synthesis_rows(p, gx + b0 * Cin * npix, (int)(nb * Cin), st, true));
    }
    if (gW) {
      RowsOut rx{p->d_x_hi, split ? p->d_x_lo : nullptr, p->ldx, Cin, kxb, &p->tc};
      SHT_TRY(analysis(p, x + b0 * Cin * npix, nullptr, nb * Cin, st, false, false, &rx));
      const cudaError_t e = traced(p, SHT_KERNEL_FILTER_DW, st, [&] {
        return launch_dw_tc(p->d_g_hi, split ? p->d_g_lo : nullptr, p->d_x_hi, split ? p->d_x_lo : nullptr, p->ldx,
                            (float2 *)gW, p->L, p->M, (int)nb, Cin, Cout, kxa, kxb, b0 > 0 ? 1 : 0, p->d_err, st);
      });
      if (e != cudaSuccess) return cuda_fail(e, "weight gradient launch");
    }
  }
  return SHT_OK;
}

sht_status_t spectral_filter_inverse(sht_plan_t p, const void *xhat, const void *W, float *y, int64_t Bm, int Cin,
                                     int Cout, void *stream) {
  NvtxRange nvtx_range("spectral_filter_inverse");
  SHT_TRY(check_plan(p));
  SHT_TRY(check_batch(Bm));
  SHT_TRY(check_channels(p, Cin, Cout, true));
  if (Bm == 0) return SHT_OK;
  SHT_TRY(check_ptr(xhat, "xhat"));
  SHT_TRY(check_ptr(W, "W"));
  SHT_TRY(check_ptr(y, "y"));
  DeviceGuard g(p->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t per = p->max_batch / std::max(Cin, Cout);
  const int64_t LM = (int64_t)p->L * p->M;
  const int64_t npix = (int64_t)p->nlat * p->nlon;
  for (int64_t b0 = 0; b0 < Bm; b0 += per) {
    const int64_t nb = std::min(per, Bm - b0);
    SHT_TRY(filter_body(p, (const float2 *)xhat + b0 * Cin * LM, (const float2 *)W, p->d_spec_b, nb, Cin, Cout, 0, st));
    SHT_TRY(synthesis(p, p->d_spec_b, y + b0 * Cout * npix, nb * Cout, st, false));
  }
  return SHT_OK;
}

sht_status_t sht_plan_check(sht_plan_t p) {
  SHT_TRY(check_plan(p));
  DeviceGuard g(p->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "device synchronize");
  unsigned word = 0;
  e = cudaMemcpy(&word, p->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "error word read");
  if (word != 0) {
    cudaMemset(p->d_err, 0, sizeof(unsigned));
    return fail(SHT_ERR_TIMEOUT, "a bounded wait in a tensor-core kernel timed out");
  }
  return SHT_OK;
}

sht_status_t sht_profile_begin(sht_plan_t p, int capacity) {
  SHT_TRY(check_plan(p));
  if (capacity < 1) return fail(SHT_ERR_INVALID_ARG, "capacity must be >= 1");
  DeviceGuard g(p->device);
  profile_release(p->prof);
  ProfileState &pr = p->prof;
  pr.start.resize(capacity);
  pr.stop.resize(capacity);
  pr.kernel.assign(capacity, -1);
  for (int i = 0; i < capacity; i++) {
    cudaError_t e1 = cudaEventCreate(&pr.start[i]);
    cudaError_t e2 = cudaEventCreate(&pr.stop[i]);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
      pr.start.resize(e1 == cudaSuccess ? i + 1 : i);
      pr.stop.resize(e2 == cudaSuccess ? i + 1 : i);
      profile_release(pr);
      return cuda_fail(e1 != cudaSuccess ? e1 : e2, "cudaEventCreate");
    }
  }
  pr.capacity = capacity;
  pr.used = 0;
  pr.dropped = 0;
  pr.on = true;
  return SHT_OK;
}

sht_status_t sht_profile_collect(sht_plan_t p, int64_t *launches, double *ms, int64_t *dropped) {
  SHT_TRY(check_plan(p));
  ProfileState &pr = p->prof;
  if (launches)
    for (int k = 0; k < SHT_KERNEL_COUNT; k++) launches[k] = 0;
  if (ms)
    for (int k = 0; k < SHT_KERNEL_COUNT; k++) ms[k] = 0.0;
  if (dropped) *dropped = pr.dropped;
  if (!pr.on) return SHT_OK;
  DeviceGuard g(p->device);
  for (int i = 0; i < pr.used; i++) {
    cudaError_t e = cudaEventSynchronize(pr.stop[i]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    float t = 0.f;
    e = cudaEventElapsedTime(&t, pr.start[i], pr.stop[i]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
    const int k = pr.kernel[i];
    if (k >= 0 && k < SHT_KERNEL_COUNT) {
      if (launches) launches[k]++;
      if (ms) ms[k] += t;
    }
  }
  pr.used = 0;
  pr.dropped = 0;
  return SHT_OK;
}

sht_status_t sht_profile_end(sht_plan_t p) {
  SHT_TRY(check_plan(p));
  DeviceGuard g(p->device);
  profile_release(p->prof);
  return SHT_OK;
}

const char *sht_kernel_name(int k) {
  static const char *names[SHT_KERNEL_COUNT] = {"r2c", "leg_fwd", "zero_upper", "filter", "filter_dw", "leg_inv",
                                                "c2r", "pack", "filter_prep", "finalize"};
  return (k >= 0 && k < SHT_KERNEL_COUNT) ? names[k] : "?";
}

const char *sht_status_string(sht_status_t s) {
  switch (s) {
    case SHT_OK: return "SHT_OK";
    case SHT_ERR_INVALID_ARG: return "SHT_ERR_INVALID_ARG";
    case SHT_ERR_UNSUPPORTED: return "SHT_ERR_UNSUPPORTED";
    case SHT_ERR_OOM: return "SHT_ERR_OOM";
    case SHT_ERR_CUDA: return "SHT_ERR_CUDA";
    case SHT_ERR_TIMEOUT: return "SHT_ERR_TIMEOUT";
    case SHT_ERR_INTERNAL: return "SHT_ERR_INTERNAL";
  }
  return "SHT_ERR_UNKNOWN";
}

const char *sht_last_error_message(void) { return g_last_error.c_str(); }

const char *sht_version(void) { return "0.1.0"; }

/* Test hook: make the n-th device allocation of later sht_plan calls fail
 * (n = 0 fails the next one; n < 0 disables). */
void sht_debug_fail_alloc_after(int n) { g_fail_alloc_after = n; }

sht_status_t sht_debug_stall(sht_plan_t p, int64_t timeout_ns, void *stream) {
  SHT_TRY(check_plan(p));
  if (timeout_ns < 1 || timeout_ns > 2000000000ll) return fail(SHT_ERR_INVALID_ARG, "timeout_ns must be 1 .. 2e9");
  DeviceGuard g(p->device);
  const cudaError_t e = launch_debug_stall(p->d_err, timeout_ns, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "stall launch");
  return SHT_OK;
}

}  // extern "C"
