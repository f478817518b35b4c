// Batched transforms over several grids: the items' kernels are recorded
// once into a CUDA graph — the longitude step (one grouped launch, or one
// persistent launch per item), one persistent Legendre launch over the
// tiles of every item (tensor cores) or one grouped tile grid (FP32), one
// grouped epilogue launch — and replayed per run.  The launch shape
// (Legendre column tile width, item order and pipeline stages; grouped or
// per-item longitude launches) is chosen by timing candidates at creation,
// optionally through a text cache.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "sht_internal.cuh"

namespace shtgb {
namespace {

constexpr int kMaxItems = 8;

struct Shape {
  int nt_cap = 256;  // widest column tile of the tensor-core Legendre launch
  int order = 0;     // 0: items as given, 1: most expensive tiles first
  int stages = 0;    // Legendre pipeline stages (0: as many as fit)
  int fft = 0;       // longitude step: 0 one grouped launch, 1 one launch per item
};

struct BatchProfile {
  int capacity = 0, used = 0;
  std::vector<cudaEvent_t> ev;  // capacity x (stages + 1)
};

}  // namespace
}  // namespace shtgb

struct sht_batch_s {
  int device = 0;
  int direction = SHT_BATCH_FORWARD;
  bool tc = false;
  std::vector<sht_batch_item> items;
  std::vector<sht_plan_s *> plans;
  std::vector<const char *> stages;
  shtgb::Shape shape;
  std::string how;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // profiling: event record nodes around the stages
  bool profile = false;
  std::vector<cudaEvent_t> cap_ev;
  std::vector<cudaGraphNode_t> ev_nodes;
  shtgb::BatchProfile prof;
};

namespace shtgb {
namespace {

struct DevGuard {
  int prev = -1;
  bool changed = false;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DevGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

__nv_bfloat16 *work_hi(sht_plan_s *p) { return reinterpret_cast<__nv_bfloat16 *>(p->d_work); }
__nv_bfloat16 *work_lo(sht_plan_s *p) {
  if (p->precision != SHT_PREC_SPLIT_BF16) return nullptr;
  return work_hi(p) + (size_t)p->M * 2 * p->Kh * p->ldcb;
}
__nv_bfloat16 *srow_lo(sht_plan_s *p) { return p->precision == SHT_PREC_SPLIT_BF16 ? p->d_s_lo : nullptr; }

// Relative cost of one tile of item i (K chunks): order key of the
// persistent launch.
int tile_cost(const sht_batch_s *b, int i) {
  const sht_plan_s *p = b->plans[i];
  if (b->direction == SHT_BATCH_FORWARD) return (p->Kh + 63) / 64;
  return (leg_rows(p->L, 0, 0) + 63) / 64;
}

std::vector<int> item_order(const sht_batch_s *b, int order) {
  std::vector<int> perm(b->items.size());
  std::iota(perm.begin(), perm.end(), 0);
  if (order == 1)
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int c) { return tile_cost(b, a) > tile_cost(b, c); });
  return perm;
}

// Column tile of B fields under a cap: balanced tiles, multiples of 16.
int column_tile(int64_t B, int cap) {
  const int64_t C2 = 2 * B;
  const int64_t n = (C2 + cap - 1) / cap;
  return (int)(((C2 + n - 1) / n + 15) / 16 * 16);
}

bool all_fft45(const sht_batch_s *b) {
  for (auto *p : b->plans)
    if (!fft45_supported(p->nlon)) return false;
  return true;
}

// ---- the stages -----------------------------------------------------------

cudaError_t stage_r2c(sht_batch_s *b, const Shape &sh, cudaStream_t st) {
  const int n = (int)b->items.size();
  if (all_fft45(b) && sh.fft == 0) {
    Fft45Item it[kMaxItems];
    for (int i = 0; i < n; i++) {
      sht_plan_s *p = b->plans[i];
      it[i] = Fft45Item{static_cast<const float *>(b->items[i].in),
                        b->tc ? nullptr : p->d_work,
                        b->tc ? work_hi(p) : nullptr,
                        b->tc ? work_lo(p) : nullptr,
                        p->d_twiddle,
                        p->d_ring_w,
                        p->lay_f,
                        p->nlat,
                        p->nlon,
                        p->M,
                        (int)b->items[i].count,
                        0};
    }
    return launch_r2c45_grouped(it, n, b->tc, st);
  }
  for (int i = 0; i < n; i++) {
    sht_plan_s *p = b->plans[i];
    const float *x = static_cast<const float *>(b->items[i].in);
    const int nb = (int)b->items[i].count;
    cudaError_t e;
    if (fft45_supported(p->nlon))
      e = b->tc ? launch_r2c45(x, nullptr, work_hi(p), work_lo(p), p->nlat, p->nlon, p->M, nb, p->lay_f,
                               p->d_twiddle, p->d_ring_w, 0, st, p->d_err)
                : launch_r2c45(x, p->d_work, nullptr, nullptr, p->nlat, p->nlon, p->M, nb, p->lay_f, p->d_twiddle,
                               p->d_ring_w, 0, st, p->d_err);
    else
      e = b->tc ? launch_r2c_bf16(x, work_hi(p), work_lo(p), p->nlat, p->nlon, p->M, nb, p->lay_f, p->d_twiddle,
                                  p->radix, p->d_ring_w, 0, st)
                : launch_r2c(x, p->d_work, p->nlat, p->nlon, p->M, nb, p->lay_f, p->d_twiddle, p->radix, p->d_ring_w,
                             0, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t stage_c2r(sht_batch_s *b, const Shape &sh, cudaStream_t st) {
  const int n = (int)b->items.size();
  if (all_fft45(b) && sh.fft == 0) {
    Fft45Item it[kMaxItems];
    for (int i = 0; i < n; i++) {
      sht_plan_s *p = b->plans[i];
      it[i] = Fft45Item{p->d_work, static_cast<float *>(b->items[i].out), nullptr, nullptr, p->d_twiddle, nullptr,
                        p->lay_g, p->nlat, p->nlon, p->M, (int)b->items[i].count, 1};
    }
    return launch_c2r45_grouped(it, n, st);
  }
  for (int i = 0; i < n; i++) {
    sht_plan_s *p = b->plans[i];
    float *y = static_cast<float *>(b->items[i].out);
    const int nb = (int)b->items[i].count;
    cudaError_t e =
        fft45_supported(p->nlon)
            ? launch_c2r45(p->d_work, y, p->nlat, p->nlon, p->M, nb, p->lay_g, p->d_twiddle, nullptr, 1, st, p->d_err)
            : launch_c2r(p->d_work, y, p->nlat, p->nlon, p->M, nb, p->lay_g, p->d_twiddle, p->radix, nullptr, 1, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t stage_legendre(sht_batch_s *b, const Shape &sh, cudaStream_t st) {
  const bool inverse = b->direction == SHT_BATCH_INVERSE;
  const std::vector<int> perm = item_order(b, sh.order);
  const int n = (int)perm.size();
  if (b->tc) {
    TcLegItem it[kMaxItems];
    for (int j = 0; j < n; j++) {
      const int i = perm[j];
      sht_plan_s *p = b->plans[i];
      TcLegItem &q = it[j];
      q = TcLegItem{};
      q.T = &p->tc;
      q.tiles = inverse ? p->d_inv_tiles : p->d_fwd_tiles;
      q.krange = inverse ? p->d_inv_krange : p->d_fwd_krange;
      q.ntiles = inverse ? p->n_inv_tiles : p->n_fwd_tiles;
      q.B = (int)b->items[i].count;
      q.Nt = column_tile(q.B, sh.nt_cap);
      if (!inverse) {
        q.rowsf = reinterpret_cast<float *>(p->d_spec_b);
        q.ldr = p->ldr;
        q.cin = 1;
      } else {
        q.Gw = p->d_work;
        q.ldc = p->ldc;
      }
    }
    return launch_leg_tc_group(inverse ? 1 : 0, it, n, TcLaunch{0, sh.stages}, st);
  }
  F32LegItem it[kMaxItems];
  for (int j = 0; j < n; j++) {
    const int i = perm[j];
    sht_plan_s *p = b->plans[i];
    F32LegItem &q = it[j];
    q = F32LegItem{};
    q.T = TableF32{p->d_table, p->d_tab_off, p->Khp};
    q.tiles = inverse ? p->d_inv_tiles : p->d_fwd_tiles;
    q.ntiles = inverse ? p->n_inv_tiles : p->n_fwd_tiles;
    q.L = p->L;
    q.M = p->M;
    q.Kh = p->Kh;
    q.ldc = p->ldc;
    q.B = (int)b->items[i].count;
    if (!inverse) {
      q.Fw = p->d_work;
      q.xhat = static_cast<float2 *>(b->items[i].out);
    } else {
      q.yhat = static_cast<const float2 *>(b->items[i].in);
      q.Gw = p->d_work;
    }
  }
  return launch_leg_f32_group(inverse ? 1 : 0, it, n, st);
}

cudaError_t stage_zero(sht_batch_s *b, cudaStream_t st) {
  const int n = (int)b->items.size();
  float2 *xh[kMaxItems];
  int L[kMaxItems], M[kMaxItems];
  int64_t B[kMaxItems];
  for (int i = 0; i < n; i++) {
    xh[i] = static_cast<float2 *>(b->items[i].out);
    L[i] = b->plans[i]->L;
    M[i] = b->plans[i]->M;
    B[i] = b->items[i].count;
  }
  return launch_zero_upper_group(xh, L, M, B, n, st);
}

cudaError_t stage_pack(sht_batch_s *b, cudaStream_t st) {
  const int n = (int)b->items.size();
  RowsItem it[kMaxItems];
  for (int i = 0; i < n; i++) {
    sht_plan_s *p = b->plans[i];
    it[i] = RowsItem{nullptr, static_cast<float2 *>(const_cast<void *>(b->items[i].in)), p->d_s_hi, srow_lo(p), p->L, p->M, (int)b->items[i].count, p->ldcb};
  }
  return launch_rows_transpose(true, it, n, st);
}

// FP32 rows of the tensor-core forward -> API layout, zeros included.
cudaError_t stage_finalize(sht_batch_s *b, cudaStream_t st) {
  const int n = (int)b->items.size();
  RowsItem it[kMaxItems];
  for (int i = 0; i < n; i++) {
    sht_plan_s *p = b->plans[i];
    it[i] = RowsItem{reinterpret_cast<const float *>(p->d_spec_b), static_cast<float2 *>(b->items[i].out), nullptr,
                     nullptr, p->L, p->M, (int)b->items[i].count, p->ldr};
  }
  return launch_rows_transpose(false, it, n, st);
}

void stage_names(sht_batch_s *b) {
  b->stages.clear();
  if (b->direction == SHT_BATCH_FORWARD) {
    b->stages = {"r2c", "leg_fwd", b->tc ? "finalize" : "zero"};
  } else if (b->tc) {
    b->stages = {"pack", "leg_inv", "c2r"};
  } else {
    b->stages = {"leg_inv", "c2r"};
  }
}

cudaError_t run_stage(sht_batch_s *b, int k, const Shape &sh, cudaStream_t st) {
  const char *name = b->stages[k];
  if (!strcmp(name, "r2c")) return stage_r2c(b, sh, st);
  if (!strcmp(name, "leg_fwd") || !strcmp(name, "leg_inv")) return stage_legendre(b, sh, st);
  if (!strcmp(name, "zero")) return stage_zero(b, st);
  if (!strcmp(name, "finalize")) return stage_finalize(b, st);
  if (!strcmp(name, "pack")) return stage_pack(b, st);
  return stage_c2r(b, sh, st);
}

int legendre_stage(const sht_batch_s *b) {
  for (size_t k = 0; k < b->stages.size(); k++)
    if (!strncmp(b->stages[k], "leg_", 4)) return (int)k;
  return 0;
}

int longitude_stage(const sht_batch_s *b) {
  for (size_t k = 0; k < b->stages.size(); k++)
    if (!strcmp(b->stages[k], "r2c") || !strcmp(b->stages[k], "c2r")) return (int)k;
  return 0;
}

// ---- tuning -----------------------------------------------------------------

std::string batch_key(const sht_batch_s *b) {
  char buf[160];
  std::string key;
  const sht_plan_s *p0 = b->plans[0];
  snprintf(buf, sizeof(buf), "dir=%d prec=%d table=%d", b->direction, p0->precision, p0->table_source);
  key = buf;
  for (size_t i = 0; i < b->items.size(); i++) {
    const sht_plan_s *p = b->plans[i];
    snprintf(buf, sizeof(buf), " %dx%d/g%d/L%d/M%d/B%lld", p->nlat, p->nlon, p->grid, p->L, p->M,
             (long long)b->items[i].count);
    key += buf;
  }
  return key;
}

std::mutex g_cache_mutex;

bool cache_lookup(const char *path, const std::string &key, Shape &sh) {
  std::lock_guard<std::mutex> lock(g_cache_mutex);
  FILE *f = fopen(path, "r");
  if (!f) return false;
  char line[2048];
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    char *tab = strchr(line, '\t');
    if (!tab) continue;
    *tab = 0;
    if (key != line) continue;
    int cap = 0, order = 0, stages = 0, fft = 0;
    const int got = sscanf(tab + 1, "%d %d %d %d", &cap, &order, &stages, &fft);
    if (got >= 2 && (cap == 64 || cap == 128 || cap == 256) && (order == 0 || order == 1) && stages >= 0 &&
        stages <= 16 && (fft == 0 || fft == 1)) {
      sh.nt_cap = cap;
      sh.order = order;
      sh.stages = got >= 3 ? stages : 0;
      sh.fft = got >= 4 ? fft : 0;
      found = true;  // the last entry of a key wins
    }
  }
  fclose(f);
  return found;
}

void cache_store(const char *path, const std::string &key, const Shape &sh, double us) {
  std::lock_guard<std::mutex> lock(g_cache_mutex);
  FILE *f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s\t%d %d %d %d %.1f\n", key.c_str(), sh.nt_cap, sh.order, sh.stages, sh.fft, us);
  fclose(f);
}

// Median device time of stage k under one shape (us).
cudaError_t time_stage(sht_batch_s *b, int k, const Shape &sh, cudaStream_t st, double &us) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  std::vector<double> t;
  for (int rep = 0; rep < 4 && e == cudaSuccess; rep++) {
    // the stage's inputs come from the stages before it
    for (int j = 0; j < k && e == cudaSuccess; j++) e = run_stage(b, j, sh, st);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = run_stage(b, k, sh, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0) t.push_back(ms * 1000.0);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  std::sort(t.begin(), t.end());
  us = t[t.size() / 2];
  return cudaSuccess;
}

void release(sht_batch_s *b) {
  if (!b) return;
  DevGuard g(b->device);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto ev : b->cap_ev) cudaEventDestroy(ev);
  for (auto ev : b->prof.ev) cudaEventDestroy(ev);
  delete b;
}

}  // namespace
}  // namespace shtgb

using namespace shtgb;

extern "C" {

void sht_batch_opts_default(sht_batch_opts *opts) {
  if (!opts) return;
  memset(opts, 0, sizeof(*opts));
  opts->direction = SHT_BATCH_FORWARD;
  opts->tune = 1;
}

sht_status_t sht_batch_create(sht_batch_t *out, const sht_batch_item *items, int n, const sht_batch_opts *opts,
                              void *stream) {
  NvtxRange nvtx_range("sht_batch_create");
  if (!out) return fail(SHT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  sht_batch_opts o;
  sht_batch_opts_default(&o);
  if (opts) o = *opts;
  for (int r : o.reserved)
    if (r != 0) return fail(SHT_ERR_INVALID_ARG, "reserved option fields must be zero");
  if (o.direction != SHT_BATCH_FORWARD && o.direction != SHT_BATCH_INVERSE)
    return fail(SHT_ERR_INVALID_ARG, "unknown direction");
  if (n < 1 || n > kMaxItems) return fail(SHT_ERR_INVALID_ARG, "a batch holds 1 to 8 items");
  if (!items) return fail(SHT_ERR_INVALID_ARG, "items is NULL");
  for (int i = 0; i < n; i++) {
    const sht_batch_item &it = items[i];
    if (!it.plan) return fail(SHT_ERR_INVALID_ARG, "item plan is NULL");
    if (!it.in || !it.out) return fail(SHT_ERR_INVALID_ARG, "item buffer is NULL");
    for (int j = 0; j < i; j++)
      if (items[j].plan == it.plan) return fail(SHT_ERR_INVALID_ARG, "a plan appears twice in the batch");
    const sht_plan_s *p = it.plan;
    const sht_plan_s *p0 = items[0].plan;
    if (p->device != p0->device || p->precision != p0->precision || p->table_source != p0->table_source)
      return fail(SHT_ERR_INVALID_ARG, "batch plans differ in device, precision or table source");
    if (it.count < 1 || it.count > p->max_batch)
      return fail(SHT_ERR_INVALID_ARG, "item count outside 1..max_batch of its plan");
  }
  sht_batch_s *b = new (std::nothrow) sht_batch_s();
  if (!b) return fail(SHT_ERR_OOM, "host allocation failed");
  b->device = items[0].plan->device;
  b->direction = o.direction;
  b->tc = items[0].plan->precision != SHT_PREC_FP32;
  b->items.assign(items, items + n);
  for (int i = 0; i < n; i++) b->plans.push_back(items[i].plan);
  b->profile = o.profile != 0;
  stage_names(b);
  DevGuard guard(b->device);
  auto bail = [&](cudaError_t e, const char *what) {
    sht_status_t s = cuda_fail(e, what);
    release(b);
    return s;
  };

  cudaStream_t ts;
  cudaError_t e = cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking);
  if (e != cudaSuccess) return bail(e, "stream creation");
  // order the tuning and the capture after the caller's work
  if (stream) {
    cudaEvent_t dep;
    e = cudaEventCreateWithFlags(&dep, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(dep, static_cast<cudaStream_t>(stream));
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ts, dep, 0);
    cudaEventDestroy(dep);
    if (e != cudaSuccess) {
      cudaStreamDestroy(ts);
      return bail(e, "stream ordering");
    }
  }

  // launch shape: cache, tuning, or the default
  const std::string key = batch_key(b);
  Shape best;
  char how[200];
  if (o.tune_cache && cache_lookup(o.tune_cache, key, best)) {
    snprintf(how, sizeof(how), "cached");
  } else if (o.tune) {
    // the Legendre stage over (column tile, item order, pipeline stages),
    // then the longitude stage over (grouped, per item) with the best
    // Legendre shape; the two stages do not interact
    std::vector<Shape> cand;
    const int caps_tc[3] = {256, 128, 64};
    for (int order = 0; order < 2; order++) {
      if (b->tc) {
        for (int cap : caps_tc)
          for (int stages : {0, 4}) cand.push_back(Shape{cap, order, stages, 0});
      } else {
        cand.push_back(Shape{256, order, 0, 0});
      }
    }
    double best_us = 1e300, best_fft_us = 0.0;
    int tried = 0;
    auto fail_tuning = [&](cudaError_t err) {
      cudaStreamDestroy(ts);
      return bail(err, "tuning run");
    };
    for (const Shape &sh : cand) {
      double us = 0.0;
      if ((e = time_stage(b, legendre_stage(b), sh, ts, us)) != cudaSuccess) return fail_tuning(e);
      tried++;
      if (us < best_us) {
        best_us = us;
        best = sh;
      }
    }
    if (all_fft45(b)) {
      double us_mode[2] = {0.0, 0.0};
      for (int mode = 0; mode < 2; mode++) {
        Shape sh = best;
        sh.fft = mode;
        if ((e = time_stage(b, longitude_stage(b), sh, ts, us_mode[mode])) != cudaSuccess) return fail_tuning(e);
        tried++;
      }
      best.fft = us_mode[1] < us_mode[0] ? 1 : 0;
      best_fft_us = us_mode[best.fft];
    }
    snprintf(how, sizeof(how), "tuned over %d shapes, legendre %.1f us, longitude %.1f us", tried, best_us,
             best_fft_us);
    if (o.tune_cache) cache_store(o.tune_cache, key, best, best_us + best_fft_us);
  } else {
    snprintf(how, sizeof(how), "default");
  }
  b->shape = best;
  char desc[400];
  snprintf(desc, sizeof(desc), "legendre: tile<=%d, order=%s, stages=%s; longitude: %s; %s", best.nt_cap,
           best.order ? "cost" : "given", best.stages ? std::to_string(best.stages).c_str() : "max",
           best.fft ? "per item" : "grouped", how);
  b->how = desc;

  // record the graph
  const int S = (int)b->stages.size();
  if (b->profile) {
    b->cap_ev.resize(S + 1, nullptr);
    for (int k = 0; k <= S && e == cudaSuccess; k++) e = cudaEventCreate(&b->cap_ev[k]);
    if (e != cudaSuccess) {
      cudaStreamDestroy(ts);
      return bail(e, "event creation");
    }
  }
  e = cudaStreamBeginCapture(ts, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(ts);
    return bail(e, "stream capture");
  }
  cudaError_t le = cudaSuccess;
  for (int k = 0; k < S && le == cudaSuccess; k++) {
    if (b->profile) le = cudaEventRecordWithFlags(b->cap_ev[k], ts, cudaEventRecordExternal);
    if (le == cudaSuccess) le = run_stage(b, k, b->shape, ts);
  }
  if (b->profile && le == cudaSuccess) le = cudaEventRecordWithFlags(b->cap_ev[S], ts, cudaEventRecordExternal);
  e = cudaStreamEndCapture(ts, &b->graph);
  cudaStreamDestroy(ts);
  if (le != cudaSuccess) return bail(le, "recording the batch");
  if (e != cudaSuccess) return bail(e, "stream capture");
  e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) return bail(e, "graph instantiation");
  if (b->profile) {
    // the event record nodes, in stage order
    size_t nn = 0;
    e = cudaGraphGetNodes(b->graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (e == cudaSuccess && nn) e = cudaGraphGetNodes(b->graph, nodes.data(), &nn);
    b->ev_nodes.assign(S + 1, nullptr);
    for (size_t i = 0; i < nn && e == cudaSuccess; i++) {
      cudaGraphNodeType t;
      e = cudaGraphNodeGetType(nodes[i], &t);
      if (e != cudaSuccess || t != cudaGraphNodeTypeEventRecord) continue;
      cudaEvent_t ev;
      e = cudaGraphEventRecordNodeGetEvent(nodes[i], &ev);
      for (int k = 0; k <= S && e == cudaSuccess; k++)
        if (b->cap_ev[k] == ev) b->ev_nodes[k] = nodes[i];
    }
    if (e != cudaSuccess) return bail(e, "graph inspection");
    for (auto nd : b->ev_nodes)
      if (!nd) {
        release(b);
        return fail(SHT_ERR_INTERNAL, "event node missing from the recorded graph");
      }
  }
  *out = b;
  return SHT_OK;
}

sht_status_t sht_batch_run(sht_batch_t b, void *stream) {
  NvtxRange nvtx_range("sht_batch_run");
  if (!b || !b->exec) return fail(SHT_ERR_INVALID_ARG, "batch is NULL");
  DevGuard guard(b->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  BatchProfile &pr = b->prof;
  const int S = (int)b->stages.size();
  if (b->profile && pr.used < pr.capacity) {
    for (int k = 0; k <= S; k++) {
      cudaError_t e = cudaGraphExecEventRecordNodeSetEvent(b->exec, b->ev_nodes[k], pr.ev[pr.used * (S + 1) + k]);
      if (e != cudaSuccess) return cuda_fail(e, "profile event update");
    }
    pr.used++;
  }
  cudaError_t e = cudaGraphLaunch(b->exec, st);
  if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  return SHT_OK;
}

sht_status_t sht_batch_describe(sht_batch_t b, char *buf, int len) {
  if (!b || !buf || len < 1) return fail(SHT_ERR_INVALID_ARG, "batch or buffer is NULL");
  snprintf(buf, (size_t)len, "%s", b->how.c_str());
  return SHT_OK;
}

int sht_batch_stage_count(sht_batch_t b) { return b ? (int)b->stages.size() : 0; }

const char *sht_batch_stage_name(sht_batch_t b, int stage) {
  if (!b || stage < 0 || stage >= (int)b->stages.size()) return "?";
  return b->stages[stage];
}

sht_status_t sht_batch_profile_begin(sht_batch_t b, int capacity) {
  if (!b) return fail(SHT_ERR_INVALID_ARG, "batch is NULL");
  if (!b->profile) return fail(SHT_ERR_INVALID_ARG, "batch was created without profile = 1");
  if (capacity < 1) return fail(SHT_ERR_INVALID_ARG, "capacity must be >= 1");
  DevGuard guard(b->device);
  for (auto ev : b->prof.ev) cudaEventDestroy(ev);
  b->prof = BatchProfile{};
  const int S = (int)b->stages.size();
  b->prof.ev.resize((size_t)capacity * (S + 1), nullptr);
  for (auto &ev : b->prof.ev) {
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return cuda_fail(e, "event creation");
  }
  b->prof.capacity = capacity;
  return SHT_OK;
}

sht_status_t sht_batch_profile_collect(sht_batch_t b, int64_t *runs, double *ms) {
  if (!b) return fail(SHT_ERR_INVALID_ARG, "batch is NULL");
  DevGuard guard(b->device);
  BatchProfile &pr = b->prof;
  const int S = (int)b->stages.size();
  std::vector<double> tot(S, 0.0);
  for (int r = 0; r < pr.used; r++)
    for (int k = 0; k < S; k++) {
      cudaError_t e = cudaEventSynchronize(pr.ev[r * (S + 1) + k + 1]);
      float t = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, pr.ev[r * (S + 1) + k], pr.ev[r * (S + 1) + k + 1]);
      if (e != cudaSuccess) return cuda_fail(e, "profile events");
      tot[k] += t;
    }
  if (runs) *runs = pr.used;
  if (ms)
    for (int k = 0; k < S; k++) ms[k] = tot[k];
  pr.used = 0;
  return SHT_OK;
}

sht_status_t sht_batch_destroy(sht_batch_t b) {
  if (!b) return fail(SHT_ERR_INVALID_ARG, "batch is NULL");
  release(b);
  return SHT_OK;
}

}  // extern "C"
