// Forward SHT whose scratch memory is a fixed static device array.
//
// sht_forward keeps the folded longitude coefficients of a chunk of fields
// in the plan's workspace.  This variant keeps them in `g_fourier_scratch`
// below instead, so the call itself never asks the CUDA runtime for memory:
// it suits callers that must not allocate device memory while they run --
// host frameworks that hand out all device memory from their own pool and
// forbid cudaMalloc in plug-ins, or code paths with a fixed memory budget.
// The paper has no counterpart; it is a property of this library's API.
//
// The array is 16 MiB and lives on every GPU that loads the library until
// the process exits.  Calls share it, so calls whose work overlaps on the
// GPU (different streams, or different host threads on one device) race.
//
// Size limit: the Legendre kernel reads the coefficients of two fields per
// 16-byte load, so a chunk row holds at least 4 floats (two fields' re and
// im) for every (order, parity, latitude): 32 * mmax * ceil(nlat/2) bytes
// must fit in the 16 MiB, even when a single field is transformed.
//
// The array's device address is looked up once per device and kept for the
// life of the process.  A cudaDeviceReset of that device ends the validity
// of this address together with every plan made on the device before the
// reset; plans made afterwards must not be used with this entry point.
#include <algorithm>
#include <mutex>
#include <string>

#include "sht_internal.cuh"

namespace shtgb {
namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB

static __device__ __align__(256) unsigned char g_fourier_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the array on the current device (looked up once per
// device; the host-side symbol itself is not a device address).
sht_status_t scratch_address(int device, void **out) {
  if (device < 0 || device >= kMaxDevices) return fail(SHT_ERR_UNSUPPORTED, "device ordinal above 63");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[device]) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_fourier_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the static scratch");
    g_scratch_ptr[device] = ptr;
  }
  *out = g_scratch_ptr[device];
  return SHT_OK;
}

// Makes `dev` the current device for the life of the object and restores
// the previous one afterwards; `ok` is false when the switch failed, so
// that nothing is looked up or launched on another device.
struct DeviceSwitch {
  int prev = -1;
  bool changed = false, ok = false;
  explicit DeviceSwitch(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) return;
    if (prev != dev) {
      if (cudaSetDevice(dev) != cudaSuccess) return;
      changed = true;
    }
    int now = -1;
    ok = cudaGetDevice(&now) == cudaSuccess && now == dev;
  }
  ~DeviceSwitch() {
    if (changed) cudaSetDevice(prev);
  }
};

}  // namespace
}  // namespace shtgb

using namespace shtgb;

extern "C" sht_status_t sht_forward_static_scratch(sht_plan_t p, const float *x, void *xhat, int64_t B,
                                                   void *stream) {
  shtgb::NvtxRange nvtx_range("sht_forward_static_scratch");
  if (!p) return fail(SHT_ERR_INVALID_ARG, "plan is NULL");
  if (p->precision != SHT_PREC_FP32) return fail(SHT_ERR_UNSUPPORTED, "static-scratch forward is FP32 only");
  if (B < 0) return fail(SHT_ERR_INVALID_ARG, "batch must be >= 0");
  if (B == 0) return SHT_OK;
  if (!x || !xhat) return fail(SHT_ERR_INVALID_ARG, "x or xhat is NULL");
  if ((((uintptr_t)x) | ((uintptr_t)xhat)) & 15) return fail(SHT_ERR_INVALID_ARG, "x or xhat not 16-byte aligned");
  // The scratch holds the folded longitude coefficients [M][2][Kh][ldc] of
  // a chunk of nb fields, ldc = 2 nb rounded up to a multiple of 4 floats.
  // Nothing in it needs clearing: the analysis kernel writes every entry the
  // Legendre kernel reads for live fields; padding columns may keep an
  // earlier call's values and only feed outputs that are discarded.
  // A chunk row is at least 4 floats wide (the kernel's 16-byte loads take
  // two fields), so the smallest chunk needs 4 columns whatever B is.
  const size_t column_bytes = (size_t)p->M * 2 * p->Kh * sizeof(float);
  const size_t ldc_max = (kStaticScratchBytes / column_bytes) / 4 * 4;
  if (ldc_max < 4)
    return fail(SHT_ERR_INVALID_ARG,
                "grid too large for the 16 MiB static scratch: the smallest chunk (4 columns, two fields) needs "
                "32 * mmax * ceil(nlat/2) = " + std::to_string(column_bytes * 4) + " bytes");
  const int64_t chunk = (int64_t)(ldc_max / 2);  // fields per chunk
  DeviceSwitch g(p->device);
  if (!g.ok) return fail(SHT_ERR_CUDA, "could not make the plan's device current");
  void *scratch = nullptr;
  sht_status_t st = scratch_address(p->device, &scratch);
  if (st != SHT_OK) return st;
  float *Fw = (float *)scratch;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t LM = (int64_t)p->L * p->M;
  TableF32 T{p->d_table, p->d_tab_off, p->Khp};
  for (int64_t b0 = 0; b0 < B; b0 += chunk) {
    const int nb = (int)std::min<int64_t>(chunk, B - b0);
    const int ldc = (2 * nb + 3) / 4 * 4;
    cudaError_t e = launch_r2c(x + b0 * p->nlat * (int64_t)p->nlon, Fw, p->nlat, p->nlon, p->M, nb,
                               classic_layout(p->Kh, ldc),
                               p->d_twiddle, p->radix, p->d_ring_w, 0, s);
    if (e != cudaSuccess) return cuda_fail(e, "longitude analysis launch");
    e = launch_leg_fwd_f32(T, p->d_fwd_tiles, p->n_fwd_tiles, Fw, (float2 *)xhat + b0 * LM, p->L, p->M, p->Kh, ldc,
                           nb, s);
    if (e != cudaSuccess) return cuda_fail(e, "forward Legendre launch");
    e = launch_zero_upper((float2 *)xhat + b0 * LM, p->L, p->M, nb, s);
    if (e != cudaSuccess) return cuda_fail(e, "zero fill launch");
  }
  return SHT_OK;
}
