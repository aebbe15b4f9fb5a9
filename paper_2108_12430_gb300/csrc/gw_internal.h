// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/gwstream.h"

namespace gw {

// ---- errors ---------------------------------------------------------------
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};
void set_last_error(const std::string& msg);

#define GW_CHECK_ARG(cond, msg) \
  do { if (!(cond)) throw ::gw::Error(GW_EINVAL, msg); } while (0)
#define GW_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      throw ::gw::Error(GW_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define GW_LAUNCH_CHECK() GW_CUDA(cudaGetLastError())

// Body of every extern "C" entry point: no exception crosses the ABI.
#define GW_API_BEGIN try {
#define GW_API_END                                \
  }                                               \
  catch (const gw::Error& e) {                    \
    gw::set_last_error(e.what());                 \
    return e.code;                                \
  }                                               \
  catch (const std::bad_alloc&) {                 \
    gw::set_last_error("host allocation failed"); \
    return GW_ENOMEM;                             \
  }                                               \
  catch (const std::exception& e) {               \
    gw::set_last_error(e.what());                 \
    return GW_EINVAL;                             \
  }                                               \
  return GW_OK;

// ---- layer description ----------------------------------------------------
enum Act { ACT_NONE = 0, ACT_TANH = 1, ACT_RELU = 2 };

struct LayerSpec {
  bool transposed = false;
  int cin = 0, cout = 0, k = 1, stride = 1, pad_l = 0, pad_r = 0, out_pad = 0;
  bool bn = false;
  int act = ACT_NONE;
  int lout(int lin) const {
    return transposed ? (lin - 1) * stride - pad_l - pad_r + k + out_pad
                      : (lin + pad_l + pad_r - k) / stride + 1;
  }
};

std::vector<LayerSpec> deepclean_specs(int n_in);
std::vector<LayerSpec> bbhnet_specs(int n_in);

// Weights of one layer on the device after the BatchNorm fold.
struct LayerDev {
  LayerSpec s;
  float* w = nullptr;      // FP32 [C_out][C_in][K] (transposed convs re-indexed to this order)
  float* b = nullptr;      // FP32 [C_out]
  // tensor-core path (BF16 / FP8): packed operand image and per-K-step table
  void* wq = nullptr;      // packed B operand image (bf16 or e4m3)
  uint32_t* table = nullptr;
  std::vector<uint32_t> table_h;  // the same slice codes on the host (launch planning)
  float* wscale = nullptr; // FP8: per-output-channel dequant scale (weight scale * act scale)
  int n_steps = 0;         // K-steps (MMA instructions per M sub-tile)
  int npad = 0;            // N (output channels) padded for the MMA
  int gin = 0;             // input channel groups of 8 (or 16 for FP8)
  int pin = 1;             // input phase planes the layer reads
  int n_chains = 1;        // output positions folded into one MMA row (Q)
  int coutp = 8;           // output channels per position in the MMA columns
  int dspan = 0;           // extra input rows per plane (tap shift range)
  int dmin = 0;            // smallest tap row shift
  int J = 0;               // output positions folded per row (0 = chosen by the lowering)
  float act_scale = 1.f;   // FP8: scale of this layer's input activations
  float out_scale = 1.f;   // FP8: scale applied to the outputs for the next layer
};

struct FusedPlan;

}  // namespace gw

// ---- public object structs --------------------------------------------------
struct gw_ctx {
  int device = 0;
  size_t budget = 0;
  size_t in_use = 0;
  bool alive = true;
};

struct gw_model {
  gw_ctx* ctx = nullptr;
  int kind = 0, precision = 0, n_in = 0;
  std::vector<gw::LayerDev> layers;
  float* head_w = nullptr;   // BBHnet linear head [256]
  float* head_b = nullptr;   // [1]
  float* in_mean = nullptr;  // [n_in]
  float* in_istd = nullptr;  // [n_in] 1/std
  std::vector<void*> allocs;
  size_t bytes = 0;
  // workspace for offline forwards (grown on demand)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int* err = nullptr;        // device error flag of the tensor-core kernels (bounded waits)
  // FP8: host copies of each layer's per-output-channel weight scales, the
  // scale of the last block's output (read by the pooling head), and whether
  // activation scales have been set (at create or by calibration)
  std::vector<std::vector<float>> fp8_wscale;
  float fp8_final_scale = 1.f;
  bool fp8_scaled = false;
  // FP8 BBHnet: the stem (2 input channels) on BF16 operands, writing the
  // first block's e4m3 input; an e4m3 K step would pad its 2 channels to 32
  gw::LayerDev stem16;
  bool has_stem16 = false;
  // BF16 DeepClean: the whole-network tensor-core kernel's plan (or null)
  gw::FusedPlan* fused = nullptr;
  // tensor-core BBHnet: a second stream on which each residual block's
  // shortcut conv runs beside the block's first conv (both read the block
  // input), forked from and joined back to the caller's stream by events
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
};

struct gw_fir {
  gw_ctx* ctx = nullptr;
  int ntaps = 0, precision = 0;
  std::vector<double> taps;
  float* d_taps = nullptr;
  // BF16: the FIR as an 8 -> 8 channel conv over the space-to-depth view of
  // the signal (Toeplitz weights W[r][e][c] = h[8 c + e - r])
  gw::LayerDev tc;
  std::vector<void*> allocs;
  int* err = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  size_t bytes = 0;
};

namespace gw {

// Makes `device` current for a scope (device < 0: leaves it as it is) and
// gives the caller's device back at its end (object teardown synchronises
// and frees on the object's device).
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int device) {
    if (device < 0 || cudaGetDevice(&prev) != cudaSuccess) {
      prev = -1;
      return;
    }
    if (prev != device) cudaSetDevice(device);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// ---- instrumentation -------------------------------------------------------
// Every launch site opens a Prof scope: it counts the launch and, when
// profiling is on, records CUDA events around it on the launching stream.
struct Prof {
  Prof(const char* name, cudaStream_t st);
  ~Prof();
  int slot;
  int64_t gen;  // the record list's generation when the slot was taken
  cudaStream_t st;
};
void prof_set_capturing(bool on);  // this thread is capturing a CUDA graph
void add_launches(int64_t n);      // kernels launched by a graph replay

// ---- per-device launch state ----------------------------------------------
// A kernel's dynamic shared-memory limit is a per-device attribute: it is set
// once per (device, kernel), on the calling thread's current device, the first
// time that device launches the kernel.  Thread-safe.
void set_smem_limit_once(const void* func, int bytes);
template <typename... A>
void set_smem_limit_once(void (*func)(A...), int bytes) {
  set_smem_limit_once(reinterpret_cast<const void*>(func), bytes);
}
// Multiprocessor count of the calling thread's current device (cached per device).
int current_sm_count();

// ---- device memory accounting --------------------------------------------
void* dev_alloc(gw_ctx* ctx, size_t bytes, size_t* counter);
void dev_free(gw_ctx* ctx, void* p, size_t bytes, size_t* counter);

// ---- FP32 SIMT kernels (k_f32.cu) --------------------------------------------
struct ConvF32Args {
  const float* x; int64_t xb, xc;     // input element (b, c, t) at x + b*xb + c*xc + t
  float* y; int64_t yb, yc;           // output element (b, c, t)
  const float* res; int64_t rb, rc;   // optional residual added before the activation
  const float* w; const float* bias;  // folded weights [C_out][C_in][K], bias [C_out]
  const float* in_mean; const float* in_istd;  // optional input standardisation
  const float* const* item_ptr;       // optional device table: address of item b's (0, 0) (replaces x + b*xb)
  const float* gy; int64_t gyb, gyc;  // optional: multiply the output by act'(gy) (gy = that activation's output)
  int gact;
  int B, lin, lout;
  LayerSpec s;
};
void launch_conv_f32(const ConvF32Args& a, cudaStream_t st);
// y[r][n] = scale * sum_k h'[k] x[r][n + k + x_off] for n < lout, x zero outside
// [0, x_len) (x_len < 0: lout + ntaps - 1, valid mode), h' = h or h reversed.
void launch_fir_f32(const float* x, int64_t x_row, float* y, int64_t y_row, int rows,
                    const float* taps, int ntaps, int lout, cudaStream_t st, int x_off = 0, int x_len = -1,
                    int rev = 0, float scale = 1.f);
void launch_gap_linear_f32(const float* h, int64_t hb, int64_t hc, int B, int C, int L,
                           const float* w, const float* b, float* out, cudaStream_t st);

// DeepClean forward in FP32 over B windows (api.cu): input element (b, c, t)
// at x + b*xb + c*xc + t, output [B][y_ld]; buf0 / buf1 each hold B*8*L floats.
void deepclean_f32(gw_model* m, const float* x, int64_t xb, int64_t xc, bool standardise, int B, int L,
                   float* y, int64_t y_ld, float* buf0, float* buf1, cudaStream_t st,
                   const float* const* item_ptr = nullptr);

// ---- model runners (api.cu) ------------------------------------------------------
struct TcIn;
struct TcOut;
// amax (optional, device [n_layers + 1], zeroed by the caller): max |.| of
// every conv layer's input and, in the output slot of each residual block,
// of the shortcut output and the block output (FP8 calibration).
void bbhnet_f32(gw_model* m, const float* x, int B, int L, float* logits, float* ws, cudaStream_t st,
                float* amax = nullptr);
size_t bbhnet_tc_ws_bytes(int B, int L);
size_t bbhnet_f32_ws_bytes(int B, int L);

// ---- stream kernels (k_stream.cu) -------------------------------------------
// skip (optional device flag): when set at run time the kernel writes nothing
// (a push whose input was rejected leaves the state unchanged).
void launch_ring_push_f32(const float* src, int64_t src_ld, int C, int n, float* ring,
                          int64_t R, int64_t head, const float* mean, const float* istd,
                          int* status, cudaStream_t st, const int* skip = nullptr);
// Blocked BF16 ring [G][P][2R / P][8]: ring position q (0 <= q < 2R) of
// channel group g sits in plane q % P, row q / P.
void launch_ring_push_bf16(const float* src, int64_t src_ld, int C, int G, int n,
                           __nv_bfloat16* ring, int64_t R, int64_t head, int P, const float* mean,
                           const float* istd, int* status, cudaStream_t st, const int* skip = nullptr);
// Sets every position of a witness ring (2R = R2 positions per channel) to
// the standardised zero sample (-mean_c / std_c), or to 0 when mean is null.
void launch_ring_fill(void* ring, int bf16, int C, int G, int64_t R2, const float* mean, const float* istd,
                      cudaStream_t st);
void launch_strain_push(const float* src, int n, float* ring, int64_t R, int64_t head,
                        int* status, cudaStream_t st, const int* skip = nullptr);
// launch_ring_push_bf16 and launch_strain_push in one launch (programmatic
// dependent of the previous kernel in the stream).
void launch_stream_push_bf16(const float* src, int64_t src_ld, int C, int G, int n, __nv_bfloat16* ring, int64_t R,
                             int64_t head, int P, const float* mean, const float* istd, const float* strain_src,
                             float* strain_ring, int* status, cudaStream_t st, const int* skip = nullptr);
// pring (optional): instead of subtracting, store the aggregated prediction of
// every emitted time t >= 0 at pring[t mod Rp] (post-processing follows).
// skip_copy (optional): receives *skip (0 without skip) before anything else.
void launch_sub_ola(const float* pred, int64_t pred_ld, int n, int S, int W, int64_t R,
                    int64_t head, int mode, int delta, float* acc, const float* strain_ring,
                    float* out, cudaStream_t st, const int* skip = nullptr, float* pring = nullptr,
                    int64_t Rp = 0, int* skip_copy = nullptr);
// out[i] = strain[t] - sum_k h[k] p[t + k - c] for t = t0 + i, i < count,
// c = (K - 1) / 2, p read from the ring pring (0 before time 0), strain from
// its ring (0 before time 0).
void launch_post_sub(const float* pring, int64_t Rp, const float* h, int K, const float* strain_ring, int64_t R,
                     int64_t t0, int count, float* out, cudaStream_t st, const int* skip = nullptr);
// Sets *flag to 1 when any of the n floats at x is not finite (the caller zeroes it).
void launch_check_finite(const float* x, int64_t n, int* flag, cudaStream_t st);

// ---- tensor-core conv path (k_tc.cu) ---------------------------------------------
// Activation layout of the tensor-core path ("blocked"): channels in groups of
// 8 (bf16) or 16 (e4m3) so that one position of one group is a 16-byte row;
// rows of a group are split into P phase planes (P = the stride of the layer
// that consumes them), so a stride-2 conv reads each tap as a plain row
// offset.  Element (b, c, t) sits at
//   base + off0 + b*bstride + (c / cg)*gstride + (t % P)*pstride + (t / P + b*boff)*cg + c % cg
// with cg = 8 (bf16) or 16 (e4m3).  boff lets B overlapping ring windows be
// views of one buffer.
struct TcIn {
  const void* p;
  int64_t off0, bstride, boff, gstride, pstride;
  int P, L;
  // optional device table: address of element (b, 0, 0) of item b (replaces
  // base + off0 + b*bstride + b*boff*cg), so that one launch reads windows of
  // many streams' rings
  const void* const* item_ptr = nullptr;
};
struct TcOut {
  void* p;               // blocked activations, or FP32 [B][bstride] when fp32_single
  int64_t bstride, gstride, pstride;
  int P;
  int fp32_single;       // write channel 0 as FP32 (the DeepClean prediction)
  const void* res;       // optional residual in blocked layout, added before the activation
  int64_t rbstride, rgstride, rpstride;
  int rP;
  int fp8_out;           // write e4m3 (scaled by out_scale) instead of bf16
  int fp32_d2s;          // 8-channel layer: write FP32 [B][bstride], channel o of position u at 8 u + o
  // FP32 [B][C][L] output (training): channel o of position u at p + b bstride + o gstride + u (floats),
  // optionally times the derivative of an activation whose output is gy (same layout, strides gy_b,
  // gy_c): 1 - gy^2 (tanh) or gy > 0 (ReLU)
  int fp32_full;
  const float* gy;
  int64_t gy_b, gy_c;
  int gact;
  // with fp32_full, optionally the same values also in a blocked BF16 layout
  // (the next conv's input: blk_P phase planes, strides in elements)
  void* blk;
  int64_t blk_b, blk_g, blk_p;
  int blk_P;
};
// Blocked output of `cout` channels x `lout` positions in P planes, and its view
// as the next layer's input (api.cu).
TcOut blocked_out(void* buf, int cout, int lout, int P, bool fp8 = false);
TcIn as_input(const TcOut& o, int lout);
int64_t deepclean_tc_act_elems(int L);
// DeepClean on B windows through the tensor-core kernels: `in` is the first
// layer's blocked input, y gets FP32 [B][y_ld]; buf0/buf1 hold
// B * deepclean_tc_act_elems(L) elements each; fresh_x0, fresh_dx as for
// launch_deepclean_fused.
void deepclean_tc(gw_model* m, TcIn in, int B, int L, float* y, int64_t y_ld, void* buf0, void* buf1, int* err,
                  cudaStream_t st, int fresh_x0 = 0, int fresh_dx = 0);
// BBHnet on B items of FP32 [2][L]; ws holds bbhnet_tc_ws_bytes(B, L).
void bbhnet_tc(gw_model* m, const float* x, int B, int L, float* logits, char* ws, cudaStream_t st);
// The same on e4m3 operands with the model's static activation scales.
void bbhnet_fp8(gw_model* m, const float* x, int B, int L, float* logits, char* ws, cudaStream_t st);
int tc_supported();
// Packs a layer's folded weights for the tensor-core kernel; FP8 also returns
// the per-output-channel weight scales (max |w| -> 448) in wscale_out.
void tc_pack_layer(LayerDev& L, const std::vector<double>& wfold, int precision, gw_ctx* ctx,
                   size_t* counter, std::vector<void*>& allocs, std::vector<float>* wscale_out = nullptr);
// BF16 lowering of one folded layer (L.J > 0 fixes the positions folded per
// MMA row): packed B-operand image [steps][2 K-halves][npad rows][16 bytes]
// and the per-step slice codes; fills the lowering fields of L.
void tc_lower_layer(LayerDev& L, const std::vector<double>& wf, std::vector<uint8_t>& img,
                    std::vector<uint32_t>& table);
// Byte offset of slice `code` in a buffer of P planes per channel group and
// `rows` 16-byte rows per plane.
uint32_t tc_slice_offset(uint32_t code, int P, int rows);
// Tensor-core layer whose weights change on the device (training): the
// lowering's operand image is allocated on the device and refilled by
// launch_tc_pack from FP32 weights; src_of maps a weight in the layer's own
// [C_out][C_in][K] order to its index in the array given to launch_tc_pack.
// Returns the device map (image element -> weight index, or -1) and its length.
void tc_prepare_trainable(LayerDev& L, gw_ctx* ctx, size_t* counter, std::vector<void*>& allocs,
                          const std::vector<int32_t>& src_of, const int32_t** d_map, int64_t* n_map);
void launch_tc_pack(const float* w, const int32_t* map, int64_t n, void* img, cudaStream_t st);
// Several packs in one launch (at most kTcPackMax).
struct TcPackSeg {
  const float* w;
  const int32_t* map;
  int64_t n;
  void* img;
};
constexpr int kTcPackMax = 24;
void launch_tc_pack_many(const TcPackSeg* segs, int n_segs, cudaStream_t st);

// ---- fused DeepClean (k_fused.cu) ------------------------------------------------
struct FusedPlan;
// Lowers the folded layers (wfold[l] = FP64 folded weights, b32[l] = FP32
// bias) for the fused kernel and uploads its weight images; nullptr when the
// layer table does not fit the kernel.
FusedPlan* fused_plan_create(gw_model* m, const std::vector<std::vector<double>>& wfold,
                             const std::vector<std::vector<float>>& bias);
void fused_plan_destroy(FusedPlan* f);
// True when windows of L samples can run through the fused kernel.
bool fused_supported(gw_model* m, int L);
// DeepClean on B windows of L samples: `in` is the first layer's blocked
// input (ring windows, a converted batch, or per-window addresses in
// in.item_ptr), y gets FP32 [B][y_ld].
// fresh_x0 > 0: the previous kernel on the stream writes only positions
// x >= fresh_x0 - b fresh_dx of window b (a stream's ring update); tiles that
// read none of them start before it ends (else every tile waits for it).
void launch_deepclean_fused(gw_model* m, const TcIn& in, int B, int L, float* y, int64_t y_ld, int* err,
                            cudaStream_t st, int fresh_x0 = 0, int fresh_dx = 0);

// max |x| over n floats, combined into *amax (atomic max of non-negative floats).
void launch_absmax(const float* x, int64_t n, float* amax, cudaStream_t st);
// The calling thread's next tensor-core launch (launch_conv_tc or
// launch_deepclean_fused) leaves one input stage of CTA 0 unarmed, so that a
// bounded wait runs out (testing of the failure path).
void conv_tc_arm_stall_test();
bool tc_take_stall_test();
void launch_conv_tc(const LayerDev& L, const TcIn& in, int lout, const TcOut& out, int B, int* err_flag,
                    cudaStream_t st);
// FP32 element (b, c, t) at x + b*xb + c*xc + t*ts -> blocked bf16 / e4m3,
// optionally standardised (ts = 8, xc = 1: space-to-depth of one signal).
// y (optional): the (standardised) FP32 values also written to y[b yb + c yc + t].
void launch_to_blocked(const float* x, int64_t xb, int64_t xc, int B, int C, int L, const float* mean,
                       const float* istd, float scale, const TcOut& out, int fp8, cudaStream_t st,
                       int64_t ts = 1, float* y = nullptr, int64_t yb = 0, int64_t yc = 0);
// Global average pool over a blocked activation + linear head -> FP32 logits.
void launch_gap_linear_blocked(const TcIn& in, int C, int fp8, float in_scale, const float* w,
                               const float* b, float* out, int B, cudaStream_t st);
}  // namespace gw
