// Host-to-host execution of the spectral block (SHT -> filter -> ISHT, Eq.
// sht_forward, the per-degree filter of Sec. 3 and Eq. sht_inverse) for
// fields that live in host memory: a pipe owns device staging slots and two
// copy streams, and every run is
//   copy-in stream:  wait until the slot's input is free, x_host -> x_slot
//   caller's stream: wait for the input and for the slot's output to be
//                    drained, sht_spectral_block(x_slot -> y_slot)
//   copy-out stream: wait for the block, y_slot -> y_host
// so that run i+1's host-to-device copy and run i-1's device-to-host copy
// proceed while run i computes.  The data path is the device block; the
// pipe only orders copies and kernels with events.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sht_internal.cuh"

struct sht_pipe_s {
  sht_plan_t plan = nullptr;
  int device = 0;
  int64_t Bm = 0;
  int Cin = 0, Cout = 0, depth = 0;
  size_t in_bytes = 0, out_bytes = 0;
  cudaStream_t s_in = nullptr, s_out = nullptr;
  std::vector<float *> x_dev, y_dev;
  // per slot: input copied, input consumed, output written, output drained
  std::vector<cudaEvent_t> ev_in, ev_x_free, ev_y_ready, ev_y_free;
  std::vector<char> used;  // slot used by an earlier run (its events are recorded)
  int64_t runs = 0;
};

namespace shtgb {
namespace {

struct PipeDevice {
  int prev = -1;
  bool changed = false;
  explicit PipeDevice(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = cudaSetDevice(dev) == cudaSuccess;
  }
  ~PipeDevice() {
    if (changed) cudaSetDevice(prev);
  }
};

void free_pipe(sht_pipe_s *q) {
  if (!q) return;
  PipeDevice g(q->device);
  if (q->s_in) cudaStreamSynchronize(q->s_in);
  if (q->s_out) cudaStreamSynchronize(q->s_out);
  for (float *p : q->x_dev) cudaFree(p);
  for (float *p : q->y_dev) cudaFree(p);
  for (auto *v : {&q->ev_in, &q->ev_x_free, &q->ev_y_ready, &q->ev_y_free})
    for (cudaEvent_t e : *v)
      if (e) cudaEventDestroy(e);
  if (q->s_in) cudaStreamDestroy(q->s_in);
  if (q->s_out) cudaStreamDestroy(q->s_out);
  delete q;
}

}  // namespace
}  // namespace shtgb

using namespace shtgb;

extern "C" {

sht_status_t sht_pipe_create(sht_pipe_t *out, sht_plan_t plan, int64_t Bm, int Cin, int Cout, int depth) {
  if (!out) return fail(SHT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!plan) return fail(SHT_ERR_INVALID_ARG, "plan is NULL");
  if (Bm < 1 || Cin < 1 || Cout < 1) return fail(SHT_ERR_INVALID_ARG, "Bm, Cin and Cout must be >= 1");
  if (depth < 1 || depth > 4) return fail(SHT_ERR_INVALID_ARG, "depth must be 1 .. 4");
  if ((int64_t)std::max(Cin, Cout) > plan->max_batch)
    return fail(SHT_ERR_INVALID_ARG, "max(Cin, Cout) exceeds the plan's max_batch");
  const int device = plan->device;
  sht_pipe_s *q = new (std::nothrow) sht_pipe_s();
  if (!q) return fail(SHT_ERR_OOM, "host allocation failed");
  q->plan = plan;
  q->device = device;
  q->Bm = Bm;
  q->Cin = Cin;
  q->Cout = Cout;
  q->depth = depth;
  const size_t npix = (size_t)plan->nlat * plan->nlon;
  q->in_bytes = sizeof(float) * (size_t)Bm * Cin * npix;
  q->out_bytes = sizeof(float) * (size_t)Bm * Cout * npix;
  PipeDevice g(device);
  auto bail = [&](cudaError_t e, const char *what) {
    const sht_status_t s = cuda_fail(e, what);
    free_pipe(q);
    return s;
  };
  cudaError_t e = cudaStreamCreateWithFlags(&q->s_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&q->s_out, cudaStreamNonBlocking);
  if (e != cudaSuccess) return bail(e, "pipe stream creation");
  q->x_dev.assign(depth, nullptr);
  q->y_dev.assign(depth, nullptr);
  for (auto *v : {&q->ev_in, &q->ev_x_free, &q->ev_y_ready, &q->ev_y_free}) v->assign(depth, nullptr);
  q->used.assign(depth, 0);
  for (int s = 0; s < depth; s++) {
    if ((e = cudaMalloc((void **)&q->x_dev[s], q->in_bytes)) != cudaSuccess) return bail(e, "pipe staging allocation");
    if ((e = cudaMalloc((void **)&q->y_dev[s], q->out_bytes)) != cudaSuccess) return bail(e, "pipe staging allocation");
    for (auto *v : {&q->ev_in, &q->ev_x_free, &q->ev_y_ready, &q->ev_y_free})
      if ((e = cudaEventCreateWithFlags(&(*v)[s], cudaEventDisableTiming)) != cudaSuccess)
        return bail(e, "pipe event creation");
  }
  *out = q;
  return SHT_OK;
}

sht_status_t sht_pipe_block(sht_pipe_t q, const float *x_host, const void *W, float *y_host, void *stream) {
  NvtxRange nvtx_range("sht_pipe_block");
  if (!q) return fail(SHT_ERR_INVALID_ARG, "pipe is NULL");
  if (!x_host || !W || !y_host) return fail(SHT_ERR_INVALID_ARG, "x_host, W and y_host must not be NULL");
  if ((((uintptr_t)x_host) | ((uintptr_t)y_host)) & 15)
    return fail(SHT_ERR_INVALID_ARG, "x_host and y_host must be 16-byte aligned");
  PipeDevice g(q->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int s = (int)(q->runs % q->depth);
  cudaError_t e = cudaSuccess;
  // input: the slot's previous block must have consumed it
  if (q->used[s]) e = cudaStreamWaitEvent(q->s_in, q->ev_x_free[s], 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(q->x_dev[s], x_host, q->in_bytes, cudaMemcpyHostToDevice, q->s_in);
  if (e == cudaSuccess) e = cudaEventRecord(q->ev_in[s], q->s_in);
  // block: after the input arrived and the slot's previous output drained
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, q->ev_in[s], 0);
  if (e == cudaSuccess && q->used[s]) e = cudaStreamWaitEvent(st, q->ev_y_free[s], 0);
  if (e != cudaSuccess) return cuda_fail(e, "pipe input ordering");
  sht_status_t r = sht_spectral_block(q->plan, q->x_dev[s], W, q->y_dev[s], q->Bm, q->Cin, q->Cout, stream);
  if (r != SHT_OK) return r;
  e = cudaEventRecord(q->ev_x_free[s], st);
  if (e == cudaSuccess) e = cudaEventRecord(q->ev_y_ready[s], st);
  // output
  if (e == cudaSuccess) e = cudaStreamWaitEvent(q->s_out, q->ev_y_ready[s], 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(y_host, q->y_dev[s], q->out_bytes, cudaMemcpyDeviceToHost, q->s_out);
  if (e == cudaSuccess) e = cudaEventRecord(q->ev_y_free[s], q->s_out);
  if (e != cudaSuccess) return cuda_fail(e, "pipe output ordering");
  q->used[s] = 1;
  q->runs++;
  return SHT_OK;
}

sht_status_t sht_pipe_wait(sht_pipe_t q) {
  if (!q) return fail(SHT_ERR_INVALID_ARG, "pipe is NULL");
  PipeDevice g(q->device);
  for (int s = 0; s < q->depth; s++) {
    if (!q->used[s]) continue;
    const cudaError_t e = cudaEventSynchronize(q->ev_y_free[s]);
    if (e != cudaSuccess) return cuda_fail(e, "pipe wait");
  }
  return SHT_OK;
}

sht_status_t sht_pipe_destroy(sht_pipe_t q) {
  if (!q) return SHT_OK;
  free_pipe(q);
  return SHT_OK;
}

}  // extern "C"
