// DeepClean FP32 forward that allocates no device memory.
//
// Some callers cannot allocate: a real-time acquisition or control loop that
// reserves all of its device memory up front and must never block in
// cudaMalloc (which can synchronise the device and take milliseconds), or a
// host framework that owns the GPU's memory plan and forbids allocations from
// plug-in libraries after start-up.  gw_deepclean_forward grows a workspace
// on demand; this variant instead runs the same FP32 layer kernels on a
// fixed scratch array that is part of the library image itself.
//
// The scratch is a file-scope __device__ array: every GPU that loads the
// library holds it (GW_NOALLOC_MAX_SAMPLES * 16 floats = 2 MiB) until the
// process exits.  Host code must not use the array's name as a device address
// (on the host it is only a stand-in symbol), so the device address is looked
// up with cudaGetSymbolAddress once per device, on that device's first call.
#include <mutex>

#include "gw_internal.h"

namespace {

// B * L of one call may not exceed this many samples (e.g. one 8 s window at
// 4096 Hz, or eight 1 s windows).
constexpr int64_t kMaxSamples = 32768;
constexpr int kMaxDevices = 64;

// Two ping-pong activation buffers of B * 8 * L floats each.  Every layer
// writes all of its outputs before the next layer reads them, so nothing in
// the array needs to start at zero and a call never depends on what the
// previous call left behind.
static __device__ __align__(256) float g_scratch[2 * 8 * kMaxSamples];

std::mutex g_mu;
float* g_addr[kMaxDevices] = {};

float* scratch_address(int device) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess)
      throw gw::Error(GW_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_addr[device] = static_cast<float*>(p);
  }
  return g_addr[device];
}

}  // namespace

extern "C" int gw_deepclean_forward_noalloc(gw_model_t m, const float* x, int64_t ld, int64_t window_stride,
                                            int B, int L, float* y, void* cuda_stream) {
  try {
    GW_CHECK_ARG(m && x && y, "NULL argument");
    GW_CHECK_ARG(m->kind == GW_MODEL_DEEPCLEAN, "model is not a DeepClean model");
    if (m->precision != GW_FP32) throw gw::Error(GW_ENOTIMPL, "the no-allocation forward runs FP32 models only");
    GW_CHECK_ARG(B >= 1 && L >= 8 && L % 8 == 0, "need B >= 1 and L a positive multiple of 8");
    GW_CHECK_ARG(ld >= L && window_stride >= 0, "bad ld / window_stride");
    if ((int64_t)B * L > kMaxSamples)
      throw gw::Error(GW_EINVAL, "B * L exceeds the no-allocation scratch limit of 32768 samples");
    int device = 0;
    GW_CUDA(cudaGetDevice(&device));
    GW_CHECK_ARG(device >= 0 && device < kMaxDevices, "device index out of range");
    // the weights, the input statistics and the caller's buffers live on the
    // model's device; the scratch address and the launches must be that device's
    GW_CHECK_ARG(device == m->ctx->device, "the current CUDA device is not the model's device");
    float* buf = scratch_address(device);
    const int64_t per = (int64_t)B * 8 * L;
    gw::deepclean_f32(m, x, window_stride, ld, true, B, L, y, L, buf, buf + per, (cudaStream_t)cuda_stream);
    return GW_OK;
  } catch (const gw::Error& e) {
    gw::set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    gw::set_last_error(e.what());
    return GW_EINVAL;
  }
}
