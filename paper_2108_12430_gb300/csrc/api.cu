// Host runtime behind the C ABI: contexts, models (FP64 BatchNorm fold and
// packing), whitening FIR design (FP64), offline forwards and streams.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <map>
#include <map>
#include <mutex>
#include <set>

#include "gw_internal.h"

namespace gw {

static thread_local std::string g_last_error;
void set_last_error(const std::string& msg) { g_last_error = msg; }

// ---- instrumentation ---------------------------------------------------------
static std::mutex g_prof_mu;
static std::atomic<bool> g_prof_on{false};  // set by the caller, read by every launching thread
static std::atomic<int64_t> g_launches{0};
struct ProfRec {
  std::string name;
  cudaEvent_t a, b;
};
static std::vector<ProfRec> g_prof;
// bumped whenever g_prof is cleared, so that a scope opened before a clear
// (on another thread) does not touch a slot of the new list
static int64_t g_prof_gen = 0;

// While a CUDA graph is being captured on this thread, launches are neither
// counted nor timed here: the graph's kernels are counted at each replay.
static thread_local bool g_capturing = false;
void prof_set_capturing(bool on) { g_capturing = on; }
void add_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

Prof::Prof(const char* name, cudaStream_t s) : slot(-1), gen(0), st(s) {
  if (g_capturing) return;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_prof_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ProfRec r;
  r.name = name;
  if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return;
  cudaEventRecord(r.a, st);
  g_prof.push_back(r);
  slot = (int)g_prof.size() - 1;
  gen = g_prof_gen;
}

Prof::~Prof() {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (gen == g_prof_gen) cudaEventRecord(g_prof[slot].b, st);
}

static void prof_clear() {
  for (auto& r : g_prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_prof.clear();
  ++g_prof_gen;
}

// ---- per-device launch state ----------------------------------------------
static std::mutex g_dev_mu;
static std::set<std::pair<int, const void*>> g_smem_limit_set;
static std::map<int, int> g_sm_count;

void set_smem_limit_once(const void* func, int bytes) {
  int dev = 0;
  GW_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_dev_mu);
  const auto key = std::make_pair(dev, func);
  if (g_smem_limit_set.count(key)) return;
  GW_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  g_smem_limit_set.insert(key);
}

int current_sm_count() {
  int dev = 0;
  GW_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_dev_mu);
  auto it = g_sm_count.find(dev);
  if (it != g_sm_count.end()) return it->second;
  int n = 0;
  GW_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  g_sm_count[dev] = n > 0 ? n : 152;
  return g_sm_count[dev];
}

// ---- device memory with a per-context budget ------------------------------
static std::mutex g_alloc_mu;
static std::atomic<int64_t> g_dev_allocs{0};

void* dev_alloc(gw_ctx* ctx, size_t bytes, size_t* counter) {
  if (bytes == 0) return nullptr;
  g_dev_allocs.fetch_add(1, std::memory_order_relaxed);
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (ctx->budget && ctx->in_use + bytes > ctx->budget)
      throw Error(GW_EBUDGET, "HBM budget exceeded: " + std::to_string(ctx->in_use + bytes) + " > " +
                                  std::to_string(ctx->budget) + " bytes");
    ctx->in_use += bytes;
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    ctx->in_use -= bytes;
    throw Error(GW_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  if (counter) *counter += bytes;
  return p;
}

void dev_free(gw_ctx* ctx, void* p, size_t bytes, size_t* counter) {
  if (!p) return;
  cudaFree(p);
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  ctx->in_use -= bytes;
  if (counter) *counter -= bytes;
}

// ---- layer tables ----------------------------------------------------------
std::vector<LayerSpec> deepclean_specs(int n_in) {
  std::vector<LayerSpec> v;
  v.push_back({false, n_in, 8, 7, 1, 3, 3, 0, true, ACT_TANH});
  v.push_back({false, 8, 16, 7, 2, 3, 3, 0, true, ACT_TANH});
  v.push_back({false, 16, 32, 7, 2, 3, 3, 0, true, ACT_TANH});
  v.push_back({false, 32, 64, 7, 2, 3, 3, 0, true, ACT_TANH});
  v.push_back({true, 64, 32, 7, 2, 3, 3, 1, true, ACT_TANH});
  v.push_back({true, 32, 16, 7, 2, 3, 3, 1, true, ACT_TANH});
  v.push_back({true, 16, 8, 7, 2, 3, 3, 1, true, ACT_TANH});
  v.push_back({false, 8, 1, 7, 1, 3, 3, 0, false, ACT_NONE});
  return v;
}

std::vector<LayerSpec> bbhnet_specs(int n_in) {
  std::vector<LayerSpec> v;
  v.push_back({false, n_in, 32, 16, 1, 7, 8, 0, true, ACT_RELU});
  int cin = 32;
  for (int cout : {32, 64, 128, 256}) {
    v.push_back({false, cin, cout, 7, 2, 3, 3, 0, true, ACT_RELU});
    v.push_back({false, cout, cout, 7, 1, 3, 3, 0, true, ACT_NONE});
    v.push_back({false, cin, cout, 1, 2, 0, 0, 0, true, ACT_NONE});
    cin = cout;
  }
  return v;
}

static size_t layer_param_count(const LayerSpec& s) {
  return (size_t)s.cin * s.cout * s.k + s.cout + (s.bn ? 4 * (size_t)s.cout : 0);
}

static std::vector<LayerSpec> specs_for(int kind, int n_in) {
  if (kind == GW_MODEL_DEEPCLEAN) return deepclean_specs(n_in);
  if (kind == GW_MODEL_BBHNET) return bbhnet_specs(n_in);
  throw Error(GW_EINVAL, "unknown model kind");
}

// FP64 BatchNorm fold (eval statistics, eps = 1e-5):
//   a = gamma / sqrt(var + eps); w' = w a (per output channel); b' = (b - mean) a + beta.
// The folded weights come back in [C_out][C_in][K] order for both conv kinds.
static void fold_layer(const LayerSpec& s, const float* p, std::vector<double>& w, std::vector<double>& b) {
  const size_t nw = (size_t)s.cin * s.cout * s.k;
  const float* pw = p;
  const float* pb = p + nw;
  w.assign(nw, 0.0);
  b.assign(s.cout, 0.0);
  std::vector<double> a(s.cout, 1.0), shift(s.cout, 0.0);
  if (s.bn) {
    const float* g = pb + s.cout;
    const float* be = g + s.cout;
    const float* mu = be + s.cout;
    const float* var = mu + s.cout;
    for (int o = 0; o < s.cout; ++o) {
      a[o] = (double)g[o] / std::sqrt((double)var[o] + 1e-5);
      b[o] = ((double)pb[o] - (double)mu[o]) * a[o] + (double)be[o];
    }
  } else {
    for (int o = 0; o < s.cout; ++o) b[o] = pb[o];
  }
  for (int o = 0; o < s.cout; ++o)
    for (int i = 0; i < s.cin; ++i)
      for (int k = 0; k < s.k; ++k) {
        const double raw = s.transposed ? pw[((size_t)i * s.cout + o) * s.k + k] : pw[((size_t)o * s.cin + i) * s.k + k];
        w[((size_t)o * s.cin + i) * s.k + k] = raw * a[o];
      }
}

template <typename T>
static T* upload(gw_model* m, const std::vector<T>& host) {
  T* d = (T*)dev_alloc(m->ctx, host.size() * sizeof(T), &m->bytes);
  m->allocs.push_back(d);
  GW_CUDA(cudaMemcpy(d, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice));
  return d;
}

static void model_free(gw_model* m) {
  if (!m) return;
  DeviceGuard dg(m->ctx ? m->ctx->device : -1);
  cudaDeviceSynchronize();
  for (void* p : m->allocs) cudaFree(p);
  if (m->ws) cudaFree(m->ws);
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    m->ctx->in_use -= m->bytes + m->ws_bytes;
  }
  fused_plan_destroy(m->fused);
  if (m->fork_ev) cudaEventDestroy(m->fork_ev);
  if (m->join_ev) cudaEventDestroy(m->join_ev);
  if (m->side) cudaStreamDestroy(m->side);
  delete m;
}

static void* model_workspace(gw_model* m, size_t bytes) {
  if (bytes <= m->ws_bytes) return m->ws;
  GW_CUDA(cudaDeviceSynchronize());
  if (m->ws) dev_free(m->ctx, m->ws, m->ws_bytes, nullptr);
  m->ws = nullptr;
  m->ws_bytes = 0;
  m->ws = dev_alloc(m->ctx, bytes, nullptr);
  m->ws_bytes = bytes;
  return m->ws;
}

// ---- FIR design (FP64) -----------------------------------------------------
// Zero-phase inverse real DFT of the amplitude A_j = sqrt(2 / (fs S_j)),
// centred on tap (ntaps-1)/2, truncated and Hann-windowed:
//   h0[n] = (A_0 + A_{N/2} cos(pi n) + 2 sum_{j=1}^{N/2-1} A_j cos(2 pi j n / N)) / N.
// Zero-phase FIR from real amplitudes A_j on the DFT grid j = 0 .. N/2
// (N = 2 (n_amp - 1)): the centred inverse real DFT
//   h0[n] = (A_0 + A_{N/2} (-1)^n + 2 sum_{j=1}^{N/2-1} A_j cos(2 pi j n / N)) / N,
// n = -(ntaps-1)/2 .. (ntaps-1)/2, times a Hann window over the taps (FP64).
static std::vector<double> design_zero_phase(const std::vector<double>& A, int ntaps) {
  const int n_amp = (int)A.size();
  const int N = 2 * (n_amp - 1);
  std::vector<double> ctab(N);
  for (int m = 0; m < N; ++m) ctab[m] = std::cos(2.0 * M_PI * (double)m / (double)N);
  const int c = (ntaps - 1) / 2;
  std::vector<double> h(ntaps);
  for (int n = 0; n <= c; ++n) {
    double s = A[0] + A[N / 2] * ((n & 1) ? -1.0 : 1.0);
    double acc = 0.0;
    long long jn = 0;
    for (int j = 1; j < N / 2; ++j) {
      jn += n;
      if (jn >= N) jn -= N;
      acc += A[j] * ctab[jn];
    }
    const double h0 = (s + 2.0 * acc) / (double)N;
    const int k1 = c + n, k2 = c - n;
    h[k1] = h0 * 0.5 * (1.0 - std::cos(2.0 * M_PI * k1 / (ntaps - 1)));
    h[k2] = h0 * 0.5 * (1.0 - std::cos(2.0 * M_PI * k2 / (ntaps - 1)));
  }
  return h;
}

// Whitening: A(f) = sqrt(2 / (fs S(f))), unit variance for a one-sided PSD.
static std::vector<double> design_whitening(const double* psd, int n_psd, double fs, int ntaps) {
  std::vector<double> A(n_psd);
  for (int j = 0; j < n_psd; ++j) A[j] = std::sqrt(2.0 / (fs * psd[j]));
  return design_zero_phase(A, ntaps);
}

// Band-limited inverse-PSD loss weight: |G(f)|^2 = T(f) S(f_ref) / S(f), with
// T a Tukey band (1 on [f1 + ramp, f2 - ramp], raised-cosine ramps to 0 at f1
// and f2) and S(f_ref) interpolated linearly on the grid.
// 1 on [f1 + ramp, f2 - ramp], raised-cosine ramps to 0 at f1 and f2.
static double tukey_band(double f, double f1, double f2, double ramp) {
  if (f >= f1 + ramp && f <= f2 - ramp) return 1.0;
  if (f > f1 && f < f1 + ramp) return 0.5 * (1.0 - std::cos(M_PI * (f - f1) / ramp));
  if (f > f2 - ramp && f < f2) return 0.5 * (1.0 - std::cos(M_PI * (f2 - f) / ramp));
  return 0.0;
}

static std::vector<double> design_band_loss(const double* psd, int n_psd, double fs, int ntaps, double f1, double f2,
                                            double ramp, double f_ref) {
  const int N = 2 * (n_psd - 1);
  const double df = fs / N;
  double pos = f_ref / df;
  pos = std::min(std::max(pos, 0.0), (double)(n_psd - 1));
  const int j0 = std::min((int)pos, n_psd - 2);
  const double s_ref = psd[j0] + (pos - j0) * (psd[j0 + 1] - psd[j0]);
  std::vector<double> A(n_psd);
  for (int j = 0; j < n_psd; ++j) A[j] = std::sqrt(tukey_band(j * df, f1, f2, ramp) * s_ref / psd[j]);
  return design_zero_phase(A, ntaps);
}

// ---- forward runners ---------------------------------------------------------
static const char* kDcNames[8] = {"conv_f32.enc1", "conv_f32.enc2", "conv_f32.enc3", "conv_f32.enc4",
                                  "conv_f32.dec1", "conv_f32.dec2", "conv_f32.dec3", "conv_f32.out"};
// DeepClean on B windows in FP32.  Input element (b, c, t) at
// x + b*xb + c*xc + t; the first layer standardises when mean != null.
void deepclean_f32(gw_model* m, const float* x, int64_t xb, int64_t xc, bool standardise, int B, int L,
                   float* y, int64_t y_ld, float* buf0, float* buf1, cudaStream_t st, const float* const* item_ptr) {
  const auto& Ls = m->layers;
  const float* in = x;
  int64_t ib = xb, ic = xc;
  int lin = L;
  float* bufs[2] = {buf0, buf1};
  for (size_t li = 0; li < Ls.size(); ++li) {
    const LayerSpec& s = Ls[li].s;
    const int lout = s.lout(lin);
    ConvF32Args a{};
    a.x = in; a.xb = ib; a.xc = ic;
    const bool last = (li + 1 == Ls.size());
    if (last) {
      a.y = y; a.yb = y_ld; a.yc = 0;
    } else {
      a.y = bufs[li & 1]; a.yb = (int64_t)s.cout * lout; a.yc = lout;
    }
    a.res = nullptr;
    a.w = Ls[li].w; a.bias = Ls[li].b;
    a.in_mean = (li == 0 && standardise) ? m->in_mean : nullptr;
    a.in_istd = (li == 0 && standardise) ? m->in_istd : nullptr;
    a.item_ptr = li == 0 ? item_ptr : nullptr;
    a.B = B; a.lin = lin; a.lout = lout; a.s = s;
    {
      Prof p(kDcNames[li], st);
      launch_conv_f32(a, st);
    }
    in = a.y; ib = a.yb; ic = a.yc;
    lin = lout;
  }
}

void bbhnet_f32(gw_model* m, const float* x, int B, int L, float* logits, float* ws, cudaStream_t st,
                float* amax) {
  const auto& Ls = m->layers;
  const size_t per = (size_t)B * 32 * L;
  float* buf[3] = {ws, ws + per, ws + 2 * per};
  auto track = [&](const float* t, int64_t n, int slot) {
    if (!amax) return;
    Prof p("absmax", st);
    launch_absmax(t, n, amax + slot, st);
  };
  track(x, (int64_t)B * m->n_in * L, 0);
  auto conv = [&](const LayerDev& Ld, const float* in, int64_t ib, int64_t ic, int lin, float* out,
                  const float* res, int act) {
    LayerSpec s = Ld.s;
    s.act = act;
    const int lout = s.lout(lin);
    ConvF32Args a{};
    a.x = in; a.xb = ib; a.xc = ic;
    a.y = out; a.yb = (int64_t)s.cout * lout; a.yc = lout;
    a.res = res; a.rb = a.yb; a.rc = a.yc;
    a.w = Ld.w; a.bias = Ld.b;
    a.B = B; a.lin = lin; a.lout = lout; a.s = s;
    Prof p("conv_f32.bbhnet", st);
    launch_conv_f32(a, st);
    return lout;
  };
  int l = conv(Ls[0], x, 2LL * L, L, L, buf[0], nullptr, ACT_RELU);
  track(buf[0], (int64_t)B * 32 * l, 1);
  int cin = 32, h = 0;
  for (int blk = 0; blk < 4; ++blk) {
    const LayerDev& c1 = Ls[1 + 3 * blk];
    const LayerDev& c2 = Ls[2 + 3 * blk];
    const LayerDev& sc = Ls[3 + 3 * blk];
    const int cout = c1.s.cout;
    const int a_i = (h + 1) % 3, o_i = (h + 2) % 3;
    const int64_t hb = (int64_t)cin * l, hc = l;
    const int l2 = conv(c1, buf[h], hb, hc, l, buf[a_i], nullptr, ACT_RELU);
    track(buf[a_i], (int64_t)B * cout * l2, 2 + 3 * blk);
    // the shortcut output and the block output share the block's output slot
    const int out_slot = blk < 3 ? 1 + 3 * (blk + 1) : (int)Ls.size();
    conv(sc, buf[h], hb, hc, l, buf[o_i], nullptr, ACT_NONE);
    track(buf[o_i], (int64_t)B * cout * l2, out_slot);
    conv(c2, buf[a_i], (int64_t)cout * l2, l2, l2, buf[o_i], buf[o_i], ACT_RELU);
    track(buf[o_i], (int64_t)B * cout * l2, out_slot);
    h = o_i;
    l = l2;
    cin = cout;
  }
  Prof p("gap_linear_f32", st);
  launch_gap_linear_f32(buf[h], (int64_t)cin * l, l, B, cin, l, m->head_w, m->head_b, logits, st);
}

// ---- tensor-core runners -------------------------------------------------------
// Blocked activation of `cout` channels x `lout` positions in P phase planes
// (element strides; rows of 8 bf16 channels).
TcOut blocked_out(void* buf, int cout, int lout, int P, bool fp8) {
  TcOut o{};
  const int cg = fp8 ? 16 : 8;  // channels per 16-byte row
  const int G = (cout + cg - 1) / cg;
  const int64_t Lp = (lout + P - 1) / P;
  o.p = buf;
  o.pstride = Lp * cg;
  o.gstride = (int64_t)P * Lp * cg;
  o.bstride = (int64_t)G * o.gstride;
  o.P = P;
  o.fp8_out = fp8 ? 1 : 0;
  return o;
}

TcIn as_input(const TcOut& o, int lout) {
  TcIn i{};
  i.p = o.p;
  i.bstride = o.bstride;
  i.gstride = o.gstride;
  i.pstride = o.pstride;
  i.P = o.P;
  i.L = lout;
  return i;
}

static const char* kDcTcNames[8] = {"conv_tc.enc1", "conv_tc.enc2", "conv_tc.enc3", "conv_tc.enc4",
                                    "conv_tc.dec1", "conv_tc.dec2", "conv_tc.dec3", "conv_tc.out"};

// Per-item elements of the largest inter-layer activation of a DeepClean window.
int64_t deepclean_tc_act_elems(int L) { return 8LL * L + 2048; }

// DeepClean on B windows through the tensor-core kernels.  `in` is the
// blocked BF16 input (ring windows or a converted batch); y gets FP32 [B][y_ld].
void deepclean_tc(gw_model* m, TcIn in, int B, int L, float* y, int64_t y_ld, void* buf0, void* buf1,
                         int* err, cudaStream_t st, int fresh_x0, int fresh_dx) {
  if (fused_supported(m, L)) {
    // the whole network in one launch, activations in shared memory
    Prof p("deepclean_fused", st);
    launch_deepclean_fused(m, in, B, L, y, y_ld, err, st, fresh_x0, fresh_dx);
    return;
  }
  const auto& Ls = m->layers;
  void* bufs[2] = {buf0, buf1};
  int lin = L;
  for (size_t li = 0; li < Ls.size(); ++li) {
    const LayerSpec& s = Ls[li].s;
    const int lout = s.lout(lin);
    TcOut o{};
    if (li + 1 == Ls.size()) {
      o.p = y;
      o.bstride = y_ld;
      o.P = 1;
      o.fp32_single = 1;
    } else {
      o = blocked_out(bufs[li & 1], s.cout, lout, Ls[li + 1].pin);
      GW_CHECK_ARG(o.bstride <= deepclean_tc_act_elems(L), "activation buffer too small");
    }
    {
      Prof p(kDcTcNames[li], st);
      launch_conv_tc(Ls[li], in, lout, o, B, err, st);
    }
    in = as_input(o, lout);
    lin = lout;
  }
}

// Profile scope names of BBHnet's 13 conv launches in launch order: the stem,
// then per block its first conv, its shortcut and its second conv.
static const char* kBbhNames[2][13] = {
    {"conv_tc.bbhnet.stem", "conv_tc.bbhnet.b1c1", "conv_tc.bbhnet.b1sc", "conv_tc.bbhnet.b1c2",
     "conv_tc.bbhnet.b2c1", "conv_tc.bbhnet.b2sc", "conv_tc.bbhnet.b2c2", "conv_tc.bbhnet.b3c1",
     "conv_tc.bbhnet.b3sc", "conv_tc.bbhnet.b3c2", "conv_tc.bbhnet.b4c1", "conv_tc.bbhnet.b4sc",
     "conv_tc.bbhnet.b4c2"},
    {"conv_tc.bbhnet_fp8.stem", "conv_tc.bbhnet_fp8.b1c1", "conv_tc.bbhnet_fp8.b1sc", "conv_tc.bbhnet_fp8.b1c2",
     "conv_tc.bbhnet_fp8.b2c1", "conv_tc.bbhnet_fp8.b2sc", "conv_tc.bbhnet_fp8.b2c2", "conv_tc.bbhnet_fp8.b3c1",
     "conv_tc.bbhnet_fp8.b3sc", "conv_tc.bbhnet_fp8.b3c2", "conv_tc.bbhnet_fp8.b4c1", "conv_tc.bbhnet_fp8.b4sc",
     "conv_tc.bbhnet_fp8.b4c2"}};

// BBHnet on B items of [2][L] FP32 through the tensor-core kernels.
void bbhnet_tc(gw_model* m, const float* x, int B, int L, float* logits, char* ws, cudaStream_t st) {
  const auto& Ls = m->layers;
  const int64_t per = (int64_t)B * 32 * L;  // elements of the largest activation
  void* in0 = ws;
  void* buf[3] = {ws + (size_t)B * 8 * L * 2, ws + (size_t)B * 8 * L * 2 + per * 2,
                  ws + (size_t)B * 8 * L * 2 + 2 * per * 2};
  TcOut xin = blocked_out(in0, m->n_in, L, Ls[0].pin);
  {
    Prof p("to_blocked", st);
    launch_to_blocked(x, (int64_t)m->n_in * L, L, B, m->n_in, L, nullptr, nullptr, 1.f, xin, 0, st);
  }
  int l = Ls[0].s.lout(L);
  TcOut h = blocked_out(buf[0], Ls[0].s.cout, l, Ls[1].pin);
  {
    Prof p(kBbhNames[0][0], st);
    launch_conv_tc(Ls[0], as_input(xin, L), l, h, B, m->err, st);
  }
  int hi = 0;
  for (int blk = 0; blk < 4; ++blk) {
    const LayerDev& c1 = Ls[1 + 3 * blk];
    LayerDev c2 = Ls[2 + 3 * blk];
    const LayerDev& sc = Ls[3 + 3 * blk];
    c2.s.act = ACT_RELU;  // relu(conv2 + shortcut)
    GW_CHECK_ARG(c1.pin == sc.pin, "block convs must read the same input layout");
    const int a_i = (hi + 1) % 3, o_i = (hi + 2) % 3;
    const int l2 = c1.s.lout(l);
    const int next_P = blk < 3 ? Ls[1 + 3 * (blk + 1)].pin : 1;
    TcOut a = blocked_out(buf[a_i], c1.s.cout, l2, c2.pin);
    TcOut o = blocked_out(buf[o_i], c2.s.cout, l2, next_P);
    // the shortcut on the side stream, beside the first conv; the second
    // conv (which adds the shortcut) waits for both
    GW_CUDA(cudaEventRecord(m->fork_ev, st));
    GW_CUDA(cudaStreamWaitEvent(m->side, m->fork_ev, 0));
    {
      Prof p(kBbhNames[0][2 + 3 * blk], m->side);
      launch_conv_tc(sc, as_input(h, l), l2, o, B, m->err, m->side);
    }
    GW_CUDA(cudaEventRecord(m->join_ev, m->side));
    {
      Prof p(kBbhNames[0][1 + 3 * blk], st);
      launch_conv_tc(c1, as_input(h, l), l2, a, B, m->err, st);
    }
    GW_CUDA(cudaStreamWaitEvent(st, m->join_ev, 0));
    TcOut o2 = o;
    o2.res = o.p;
    o2.rbstride = o.bstride;
    o2.rgstride = o.gstride;
    o2.rpstride = o.pstride;
    o2.rP = o.P;
    {
      Prof p(kBbhNames[0][3 + 3 * blk], st);
      launch_conv_tc(c2, as_input(a, l2), l2, o2, B, m->err, st);
    }
    h = o;
    hi = o_i;
    l = l2;
  }
  Prof p("gap_linear_tc", st);
  launch_gap_linear_blocked(as_input(h, l), Ls.back().s.cout, 0, 1.f, m->head_w, m->head_b, logits, B, st);
}

size_t bbhnet_tc_ws_bytes(int B, int L) { return (size_t)B * 8 * L * 2 + 3 * (size_t)B * 32 * L * 2; }
size_t bbhnet_f32_ws_bytes(int B, int L) { return 3 * (size_t)B * 32 * L * 4; }

// BBHnet on e4m3 operands (FP32 accumulation).  Every activation tensor is
// stored as e4m3 rows of 16 channels, quantised by its consumer's static
// scale s (q = e4m3(x s)); a layer dequantises its accumulator by
// wscale[o] / s_in per output channel in the epilogue.  A block's shortcut
// output is stored with the block output's scale, which its second conv's
// epilogue divides out before adding it.
void bbhnet_fp8(gw_model* m, const float* x, int B, int L, float* logits, char* ws, cudaStream_t st) {
  const auto& Ls = m->layers;
  if (!m->fp8_scaled)
    throw Error(GW_ESTATE, "FP8 BBHnet has no activation scales: pass act_scales or call gw_model_calibrate");
  const int64_t per = (int64_t)B * 32 * L;  // bytes of the largest activation (and then some)
  void* in0 = ws;
  void* buf[3] = {ws + (size_t)B * 16 * L, ws + (size_t)B * 16 * L + per, ws + (size_t)B * 16 * L + 2 * per};
  // the stem on BF16 operands (when built), its output in e4m3 at the first block's scale
  const LayerDev& stem = m->has_stem16 ? m->stem16 : Ls[0];
  const int in_fp8 = m->has_stem16 ? 0 : 1;
  TcOut xin = blocked_out(in0, m->n_in, L, stem.pin, in_fp8 != 0);
  {
    Prof p("to_blocked", st);
    launch_to_blocked(x, (int64_t)m->n_in * L, L, B, m->n_in, L, nullptr, nullptr, in_fp8 ? Ls[0].act_scale : 1.f,
                      xin, in_fp8, st);
  }
  int l = Ls[0].s.lout(L);
  TcOut h = blocked_out(buf[0], Ls[0].s.cout, l, Ls[1].pin, true);
  {
    Prof p(kBbhNames[1][0], st);
    launch_conv_tc(stem, as_input(xin, L), l, h, B, m->err, st);
  }
  int hi = 0;
  for (int blk = 0; blk < 4; ++blk) {
    const LayerDev& c1 = Ls[1 + 3 * blk];
    LayerDev c2 = Ls[2 + 3 * blk];
    const LayerDev& sc = Ls[3 + 3 * blk];
    c2.s.act = ACT_RELU;  // relu(conv2 + shortcut)
    GW_CHECK_ARG(c1.pin == sc.pin, "block convs must read the same input layout");
    const int a_i = (hi + 1) % 3, o_i = (hi + 2) % 3;
    const int l2 = c1.s.lout(l);
    const int next_P = blk < 3 ? Ls[1 + 3 * (blk + 1)].pin : 1;
    TcOut a = blocked_out(buf[a_i], c1.s.cout, l2, c2.pin, true);
    TcOut o = blocked_out(buf[o_i], c2.s.cout, l2, next_P, true);
    // the shortcut on the side stream, beside the first conv; the second
    // conv (which adds the shortcut) waits for both
    GW_CUDA(cudaEventRecord(m->fork_ev, st));
    GW_CUDA(cudaStreamWaitEvent(m->side, m->fork_ev, 0));
    {
      Prof p(kBbhNames[1][2 + 3 * blk], m->side);
      launch_conv_tc(sc, as_input(h, l), l2, o, B, m->err, m->side);
    }
    GW_CUDA(cudaEventRecord(m->join_ev, m->side));
    {
      Prof p(kBbhNames[1][1 + 3 * blk], st);
      launch_conv_tc(c1, as_input(h, l), l2, a, B, m->err, st);
    }
    GW_CUDA(cudaStreamWaitEvent(st, m->join_ev, 0));
    TcOut o2 = o;
    o2.res = o.p;
    o2.rbstride = o.bstride;
    o2.rgstride = o.gstride;
    o2.rpstride = o.pstride;
    o2.rP = o.P;
    {
      Prof p(kBbhNames[1][3 + 3 * blk], st);
      launch_conv_tc(c2, as_input(a, l2), l2, o2, B, m->err, st);
    }
    h = o;
    hi = o_i;
    l = l2;
  }
  Prof p("gap_linear_tc", st);
  launch_gap_linear_blocked(as_input(h, l), Ls.back().s.cout, 1, 1.f / m->fp8_final_scale, m->head_w, m->head_b,
                            logits, B, st);
}

// FP8 activation scales from per-layer input scales s[l] (l < n_layers; a
// shortcut's own entry is not used, its input is its block's first conv's)
// and the last block's output scale s[n_layers]: sets every layer's input and
// output scale and uploads its dequantisation factors wscale / s_in.
static void set_fp8_scales(gw_model* m, const std::vector<float>& s) {
  auto& Ls = m->layers;
  const int n = (int)Ls.size();
  for (int li = 0; li < n; ++li)
    GW_CHECK_ARG(s[li] > 0 && std::isfinite(s[li]), "activation scales must be positive and finite");
  GW_CHECK_ARG(s[n] > 0 && std::isfinite(s[n]), "activation scales must be positive and finite");
  for (int li = 0; li < n; ++li) {
    LayerDev& L = Ls[li];
    const bool shortcut = li >= 3 && (li - 3) % 3 == 0;
    L.act_scale = shortcut ? s[li - 2] : s[li];
    if (li == 0) {
      L.out_scale = s[1];
    } else {
      const int blk = (li - 1) / 3, role = (li - 1) % 3;  // 0: conv1, 1: conv2, 2: shortcut
      const float block_out = blk < 3 ? s[1 + 3 * (blk + 1)] : s[n];
      L.out_scale = role == 0 ? s[2 + 3 * blk] : block_out;
    }
    std::vector<float> deq(L.s.cout);
    for (int o = 0; o < L.s.cout; ++o) deq[o] = m->fp8_wscale[li][o] / L.act_scale;
    GW_CUDA(cudaMemcpy(L.wscale, deq.data(), deq.size() * 4, cudaMemcpyHostToDevice));
  }
  if (m->has_stem16) m->stem16.out_scale = Ls[0].out_scale;
  m->fp8_final_scale = s[n];
  m->fp8_scaled = true;
}

}  // namespace gw

// ---- stream object ------------------------------------------------------------
struct gw_stream {
  gw_ctx* ctx = nullptr;
  gw_stream_desc d{};
  gw_model* dc[2] = {nullptr, nullptr};
  int64_t R = 0;
  int64_t head = 0;
  float* ring_f32[2] = {nullptr, nullptr};
  __nv_bfloat16* ring_bf16[2] = {nullptr, nullptr};
  float* strain[2] = {nullptr, nullptr};
  float* acc[2] = {nullptr, nullptr};
  float* pred = nullptr;
  void* act0 = nullptr;
  void* act1 = nullptr;
  float* stage_in = nullptr;
  float* stage_out = nullptr;
  int* status = nullptr;
  int* err = nullptr;
  int* reject = nullptr;    // device: this host-mode push's input had a non-finite sample
  int* reject_h = nullptr;  // pinned host copies: [0] for a synchronous push, [1 + k] for queued push k
  // pushes queued by gw_stream_push_async and not yet synchronised: the head
  // before each, and the CUDA stream they were queued on
  int pending = 0;
  std::vector<int64_t> head_q;
  cudaStream_t async_st = nullptr;
  // Queued pushes alternate between two staging sets; their input copies run
  // on cs_in and their output copies on cs_out, so that the copies of pushes
  // k + 1 and k - 1 overlap the compute of push k.  Events: ev_in[b] inputs
  // of set b staged, ev_done[b] compute on set b finished, ev_out[b] outputs of
  // set b copied out.  reject_q[k]: the reject flag as push k's compute left it.
  float* stage_in_q[2] = {nullptr, nullptr};
  float* stage_out_q[2] = {nullptr, nullptr};
  int* reject_q = nullptr;
  cudaStream_t cs_in = nullptr, cs_out = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
  // post-processing FIR of the aggregated prediction (optional)
  float* post_taps = nullptr;
  int post_K = 0;
  float* pring[2] = {nullptr, nullptr};  // aggregated prediction per detector, ring of Rp
  int64_t Rp = 0;
  size_t bytes = 0;
  std::vector<void*> allocs;
};

namespace gw {

static void stream_free(gw_stream* s) {
  if (!s) return;
  DeviceGuard dg(s->ctx ? s->ctx->device : -1);
  cudaDeviceSynchronize();
  for (void* p : s->allocs) cudaFree(p);
  if (s->reject_h) cudaFreeHost(s->reject_h);
  for (int b = 0; b < 2; ++b) {
    if (s->ev_in[b]) cudaEventDestroy(s->ev_in[b]);
    if (s->ev_done[b]) cudaEventDestroy(s->ev_done[b]);
    if (s->ev_out[b]) cudaEventDestroy(s->ev_out[b]);
  }
  if (s->cs_in) cudaStreamDestroy(s->cs_in);
  if (s->cs_out) cudaStreamDestroy(s->cs_out);
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    s->ctx->in_use -= s->bytes;
  }
  delete s;
}

template <typename T>
static T* salloc(gw_stream* s, size_t count) {
  T* p = (T*)dev_alloc(s->ctx, count * sizeof(T), &s->bytes);
  s->allocs.push_back(p);
  GW_CUDA(cudaMemset(p, 0, count * sizeof(T)));
  return p;
}

}  // namespace gw

using namespace gw;

extern "C" {

const char* gw_last_error(void) { return gw::g_last_error.c_str(); }
const char* gw_version(void) { return "gwstream 0.1 (sm_103a)"; }

int gw_profile_enable(int on) {
  GW_API_BEGIN
  std::lock_guard<std::mutex> lk(g_prof_mu);
  prof_clear();
  g_prof_on.store(on != 0, std::memory_order_relaxed);
  GW_API_END
}

int gw_profile_read(char* names, size_t names_len, double* total_ms, int64_t* launches, int max_entries) {
  try {
    GW_CHECK_ARG(names && total_ms && launches && max_entries > 0, "NULL argument");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::map<std::string, std::pair<double, int64_t>> agg;
    for (auto& r : g_prof) {
      GW_CUDA(cudaEventSynchronize(r.b));
      float ms = 0.f;
      GW_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
      auto& e = agg[r.name];
      e.first += ms;
      e.second += 1;
    }
    std::string buf;
    int n = 0;
    for (auto& kv : agg) {
      if (n >= max_entries) break;
      total_ms[n] = kv.second.first;
      launches[n] = kv.second.second;
      buf += kv.first + "\n";
      ++n;
    }
    GW_CHECK_ARG(buf.size() < names_len, "names buffer too small");
    memcpy(names, buf.c_str(), buf.size() + 1);
    return n;
  } catch (const gw::Error& e) {
    gw::set_last_error(e.what());
    return e.code;
  }
}

int64_t gw_launch_count(void) { return g_launches.load(); }
int64_t gw_alloc_count(void) { return g_dev_allocs.load(); }

int gw_ctx_create(int device, size_t hbm_budget_bytes, gw_ctx_t* out) {
  GW_API_BEGIN
  GW_CHECK_ARG(out, "out is NULL");
  *out = nullptr;
  int n = 0;
  GW_CUDA(cudaGetDeviceCount(&n));
  GW_CHECK_ARG(device >= 0 && device < n, "device index out of range");
  GW_CUDA(cudaSetDevice(device));
  auto* c = new gw_ctx();
  c->device = device;
  c->budget = hbm_budget_bytes;
  *out = c;
  GW_API_END
}

int gw_ctx_destroy(gw_ctx_t ctx) {
  GW_API_BEGIN
  GW_CHECK_ARG(ctx, "ctx is NULL");
  delete ctx;
  GW_API_END
}

size_t gw_ctx_bytes_in_use(gw_ctx_t ctx) { return ctx ? ctx->in_use : 0; }

size_t gw_model_param_count(int kind, int n_in) {
  if (n_in <= 0) return 0;
  if (kind != GW_MODEL_DEEPCLEAN && kind != GW_MODEL_BBHNET) return 0;
  size_t n = 0;
  for (const auto& s : specs_for(kind, n_in)) n += layer_param_count(s);
  if (kind == GW_MODEL_BBHNET) n += 257;
  return n;
}

int gw_model_create(gw_ctx_t ctx, const gw_model_desc* d, gw_model_t* out) {
  gw_model* m = nullptr;
  GW_API_BEGIN
  GW_CHECK_ARG(ctx && d && out, "NULL argument");
  *out = nullptr;
  GW_CHECK_ARG(d->kind == GW_MODEL_DEEPCLEAN || d->kind == GW_MODEL_BBHNET, "unknown model kind");
  GW_CHECK_ARG(d->precision >= GW_FP32 && d->precision <= GW_FP8, "unknown precision");
  GW_CHECK_ARG(d->n_in >= 1 && d->n_in <= 256, "n_in out of range");
  GW_CHECK_ARG(d->params, "params is NULL");
  GW_CHECK_ARG(d->n_params == gw_model_param_count(d->kind, d->n_in), "n_params does not match the layer table");
  if (d->precision == GW_FP8 && d->kind != GW_MODEL_BBHNET)
    throw Error(GW_ENOTIMPL, "FP8 is implemented for the BBHnet model only");
  if (d->precision != GW_FP32 && !tc_supported())
    throw Error(GW_ENOTIMPL, "tensor-core path needs an sm_103 device");
  GW_CUDA(cudaSetDevice(ctx->device));
  m = new gw_model();
  try {
  m->ctx = ctx;
  m->kind = d->kind;
  m->precision = d->precision;
  m->n_in = d->n_in;
  const auto specs = specs_for(d->kind, d->n_in);
  const float* p = d->params;
  std::vector<std::vector<double>> wfold;
  std::vector<std::vector<float>> bfold;
  for (size_t li = 0; li < specs.size(); ++li) {
    const LayerSpec& s = specs[li];
    std::vector<double> wf, bf;
    fold_layer(s, p, wf, bf);
    p += layer_param_count(s);
    LayerDev L;
    L.s = s;
    std::vector<float> w32(wf.begin(), wf.end()), b32(bf.begin(), bf.end());
    wfold.push_back(wf);
    bfold.push_back(b32);
    L.w = upload(m, w32);
    L.b = upload(m, b32);
    if (d->precision != GW_FP32) {
      // a BBHnet shortcut reads the same input as its block's first conv, so it
      // takes that conv's output folding (and with it the same input phases)
      if (d->kind == GW_MODEL_BBHNET && li >= 3 && (li - 3) % 3 == 0) L.J = m->layers[li - 2].J;
      std::vector<float> wscale;
      tc_pack_layer(L, wf, d->precision, ctx, &m->bytes, m->allocs, &wscale);
      if (d->precision == GW_FP8) m->fp8_wscale.push_back(wscale);
      if (d->kind == GW_MODEL_BBHNET && d->precision == GW_FP8 && li == 0) {
        LayerDev S;
        S.s = s;
        S.w = L.w;
        S.b = L.b;
        tc_pack_layer(S, wf, GW_BF16, ctx, &m->bytes, m->allocs);
        m->stem16 = S;
        m->has_stem16 = true;
      }
    }
    m->layers.push_back(L);
  }
  if (d->kind == GW_MODEL_DEEPCLEAN && d->precision == GW_BF16) m->fused = fused_plan_create(m, wfold, bfold);
  if (d->kind == GW_MODEL_BBHNET && d->precision != GW_FP32) {
    GW_CUDA(cudaStreamCreateWithFlags(&m->side, cudaStreamNonBlocking));
    GW_CUDA(cudaEventCreateWithFlags(&m->fork_ev, cudaEventDisableTiming));
    GW_CUDA(cudaEventCreateWithFlags(&m->join_ev, cudaEventDisableTiming));
  }
  if (d->precision == GW_FP8 && d->act_scales) {
    GW_CHECK_ARG(d->n_act_scales == (int)specs.size() + 1,
                 "act_scales must have one entry per conv layer plus the final output scale");
    set_fp8_scales(m, std::vector<float>(d->act_scales, d->act_scales + d->n_act_scales));
  }
  if (d->kind == GW_MODEL_BBHNET) {
    std::vector<float> hw(p, p + 256), hb(p + 256, p + 257);
    m->head_w = upload(m, hw);
    m->head_b = upload(m, hb);
  }
  std::vector<float> mean(d->n_in, 0.f), istd(d->n_in, 1.f);
  for (int c = 0; c < d->n_in; ++c) {
    if (d->in_mean) mean[c] = d->in_mean[c];
    if (d->in_std) {
      GW_CHECK_ARG(d->in_std[c] > 0.f, "in_std must be positive");
      istd[c] = 1.0f / d->in_std[c];
    }
  }
  m->in_mean = upload(m, mean);
  m->in_istd = upload(m, istd);
  m->err = upload(m, std::vector<int>(1, 0));
  } catch (...) {
    model_free(m);
    m = nullptr;
    throw;
  }
  *out = m;
  m = nullptr;
  GW_API_END
}

int gw_model_destroy(gw_model_t m) {
  GW_API_BEGIN
  GW_CHECK_ARG(m, "model is NULL");
  model_free(m);
  GW_API_END
}

int gw_deepclean_forward(gw_model_t m, const float* x, int64_t ld, int64_t window_stride, int B, int L, float* y,
                         void* cuda_stream) {
  GW_API_BEGIN
  GW_CHECK_ARG(m && x && y, "NULL argument");
  GW_CHECK_ARG(m->kind == GW_MODEL_DEEPCLEAN, "model is not a DeepClean model");
  GW_CHECK_ARG(B >= 1 && L >= 8 && L % 8 == 0, "need B >= 1 and L a positive multiple of 8");
  GW_CHECK_ARG(ld >= L && window_stride >= 0, "bad ld / window_stride");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (m->precision == GW_FP32) {
    const size_t per = (size_t)B * 8 * L;
    float* ws = (float*)model_workspace(m, 2 * per * sizeof(float));
    deepclean_f32(m, x, window_stride, ld, true, B, L, y, L, ws, ws + per, st);
  } else {
    // standardise + cast the windows into the blocked BF16 layout, then run
    TcOut xin = blocked_out(nullptr, m->n_in, L, m->layers[0].pin);
    const size_t in_elems = (size_t)B * xin.bstride;
    const size_t act = (size_t)B * deepclean_tc_act_elems(L);
    char* ws = (char*)model_workspace(m, (in_elems + 2 * act) * 2);
    xin.p = ws;
    {
      Prof p("to_blocked", st);
      launch_to_blocked(x, window_stride, ld, B, m->n_in, L, m->in_mean, m->in_istd, 1.f, xin, 0, st);
    }
    deepclean_tc(m, as_input(xin, L), B, L, y, L, ws + in_elems * 2, ws + (in_elems + act) * 2, m->err, st);
  }
  GW_API_END
}

int gw_model_status(gw_model_t m, void* cuda_stream) {
  GW_API_BEGIN
  GW_CHECK_ARG(m, "model is NULL");
  int h = 0;
  GW_CUDA(cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)cuda_stream));
  GW_CUDA(cudaStreamSynchronize((cudaStream_t)cuda_stream));
  if (h) throw Error(GW_ETIMEOUT, "a tensor-core kernel gave up a bounded wait (flag " + std::to_string(h) + ")");
  GW_API_END
}

int gw_model_test_wait_timeout(gw_model_t m, int* observed, void* cuda_stream) {
  GW_API_BEGIN
  GW_CHECK_ARG(m && observed, "NULL argument");
  GW_CHECK_ARG(m->kind == GW_MODEL_DEEPCLEAN && m->precision != GW_FP32, "needs a tensor-core DeepClean model");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int B = 1, L = 4096;
  float* x = nullptr;
  float* y = nullptr;
  GW_CUDA(cudaMalloc(&x, (size_t)m->n_in * L * sizeof(float)));
  GW_CUDA(cudaMalloc(&y, (size_t)L * sizeof(float)));
  int rc = GW_OK;
  try {
    GW_CUDA(cudaMemsetAsync(x, 0, (size_t)m->n_in * L * sizeof(float), st));
    int h = -1;
    auto run = [&](bool stall) {
      if (stall) conv_tc_arm_stall_test();
      const int r = gw_deepclean_forward(m, x, L, 0, B, L, y, st);
      if (r != GW_OK) throw Error(r, "forward failed");
      GW_CUDA(cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, st));
      GW_CUDA(cudaStreamSynchronize(st));
    };
    run(true);
    *observed = h ? GW_ETIMEOUT : GW_OK;
    GW_CUDA(cudaMemsetAsync(m->err, 0, sizeof(int), st));
    run(false);  // the context and the model still work
    if (h) rc = GW_ETIMEOUT;
  } catch (...) {
    cudaFree(x);
    cudaFree(y);
    throw;
  }
  GW_CUDA(cudaFree(x));
  GW_CUDA(cudaFree(y));
  return rc;
  GW_API_END
}

int gw_bbhnet_score(gw_model_t m, const float* x, int B, int L, float* logits, void* cuda_stream) {
  GW_API_BEGIN
  GW_CHECK_ARG(m && x && logits, "NULL argument");
  GW_CHECK_ARG(m->kind == GW_MODEL_BBHNET, "model is not a BBHnet model");
  GW_CHECK_ARG(B >= 1 && L >= 16 && L % 16 == 0, "need B >= 1 and L a positive multiple of 16");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (m->precision == GW_FP32) {
    float* ws = (float*)model_workspace(m, 3 * (size_t)B * 32 * L * sizeof(float));
    bbhnet_f32(m, x, B, L, logits, ws, st);
  } else if (m->precision == GW_BF16) {
    char* ws = (char*)model_workspace(m, bbhnet_tc_ws_bytes(B, L));
    bbhnet_tc(m, x, B, L, logits, ws, st);
  } else {
    char* ws = (char*)model_workspace(m, bbhnet_tc_ws_bytes(B, L));
    bbhnet_fp8(m, x, B, L, logits, ws, st);
  }
  GW_API_END
}

int gw_model_calibrate(gw_model_t m, const float* x, int B, int L, float headroom, float* scales_out,
                       void* cuda_stream) {
  GW_API_BEGIN
  GW_CHECK_ARG(m && x, "NULL argument");
  GW_CHECK_ARG(m->kind == GW_MODEL_BBHNET && m->precision == GW_FP8, "calibration is for FP8 BBHnet models");
  GW_CHECK_ARG(B >= 1 && L >= 16 && L % 16 == 0, "need B >= 1 and L a positive multiple of 16");
  GW_CHECK_ARG(headroom >= 1.f && std::isfinite(headroom), "headroom must be >= 1");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int n = (int)m->layers.size();
  const size_t f32_ws = bbhnet_f32_ws_bytes(B, L);
  char* ws = (char*)model_workspace(m, f32_ws + 64 * sizeof(float) + (size_t)B * sizeof(float));
  float* amax = (float*)(ws + f32_ws);
  float* logits = amax + 64;
  GW_CUDA(cudaMemsetAsync(amax, 0, 64 * sizeof(float), st));
  // the FP8 model keeps its folded FP32 weights: run them and record ranges
  bbhnet_f32(m, x, B, L, logits, (float*)ws, st, amax);
  std::vector<float> h(n + 1);
  GW_CUDA(cudaMemcpyAsync(h.data(), amax, (n + 1) * sizeof(float), cudaMemcpyDeviceToHost, st));
  GW_CUDA(cudaStreamSynchronize(st));
  // scale = 448 / (headroom * max |x|): the largest calibration value lands
  // at 448 / headroom (e4m3's largest finite is 448)
  std::vector<float> s(n + 1, 1.f);
  for (int i = 0; i <= n; ++i) s[i] = h[i] > 0 && std::isfinite(h[i]) ? 448.f / (headroom * h[i]) : 1.f;
  set_fp8_scales(m, s);
  if (scales_out)
    for (int i = 0; i <= n; ++i) scales_out[i] = s[i];
  GW_API_END
}

// Uploads FP64-designed taps (and, for BF16, their Toeplitz conv lowering).
static gw_fir* fir_from_taps(gw_ctx_t ctx, std::vector<double> taps, int precision) {
  const int ntaps = (int)taps.size();
  gw_fir* f = nullptr;
  GW_CUDA(cudaSetDevice(ctx->device));
  f = new gw_fir();
  f->ctx = ctx;
  f->ntaps = ntaps;
  f->precision = precision;
  f->taps = std::move(taps);
  std::vector<float> t32(f->taps.begin(), f->taps.end());
  try {
    f->d_taps = (float*)dev_alloc(ctx, t32.size() * 4, &f->bytes);
    GW_CUDA(cudaMemcpy(f->d_taps, t32.data(), t32.size() * 4, cudaMemcpyHostToDevice));
    if (precision == GW_BF16) {
      // y[8 t + r] = sum_{e, c} h[8 c + e - r] x[8 (t + c) + e]: an 8 -> 8
      // channel conv with K = (ntaps - 1) / 8 + 1 taps over the signal viewed
      // as 8 "channels" of consecutive samples
      GW_CHECK_ARG(!tc_supported() ? false : true, "tensor-core path needs an sm_103 device");
      if ((ntaps - 1) % 8 != 0) throw Error(GW_ENOTIMPL, "BF16 whitening needs ntaps = 8 q + 1");
      const int K = (ntaps - 1) / 8 + 1;
      std::vector<double> wf((size_t)64 * K, 0.0);
      for (int r = 0; r < 8; ++r)
        for (int e = 0; e < 8; ++e)
          for (int c = 0; c < K; ++c) {
            const int k = 8 * c + e - r;
            if (k >= 0 && k < ntaps) wf[((size_t)r * 8 + e) * K + c] = f->taps[k];
          }
      f->tc.s = LayerSpec{false, 8, 8, K, 1, 0, 0, 0, false, ACT_NONE};
      std::vector<float> zero8(8, 0.f);
      f->tc.b = (float*)dev_alloc(ctx, 32, &f->bytes);
      f->allocs.push_back(f->tc.b);
      GW_CUDA(cudaMemcpy(f->tc.b, zero8.data(), 32, cudaMemcpyHostToDevice));
      tc_pack_layer(f->tc, wf, GW_BF16, ctx, &f->bytes, f->allocs);
      f->err = (int*)dev_alloc(ctx, sizeof(int), &f->bytes);
      f->allocs.push_back(f->err);
      GW_CUDA(cudaMemset(f->err, 0, sizeof(int)));
    }
  } catch (...) {
    gw_fir_destroy(f);
    throw;
  }
  return f;
}

// Hann-windowed sinc low-pass normalised to unit gain at DC, in FP64.
static std::vector<double> design_lowpass(double fc, double fs, int ntaps) {
  std::vector<double> h(ntaps);
  const double c = 0.5 * (ntaps - 1), nu = 2.0 * fc / fs;
  double sum = 0.0;
  for (int j = 0; j < ntaps; ++j) {
    const double x = nu * (j - c);
    const double sinc = x == 0.0 ? 1.0 : std::sin(M_PI * x) / (M_PI * x);
    const double win = ntaps > 1 ? 0.5 - 0.5 * std::cos(2.0 * M_PI * j / (ntaps - 1)) : 1.0;
    h[j] = nu * sinc * win;
    sum += h[j];
  }
  for (double& v : h) v /= sum;
  return h;
}

int gw_fir_create_whitening(gw_ctx_t ctx, const double* psd, int n_psd, double fs, int ntaps, int precision,
                            gw_fir_t* out) {
  GW_API_BEGIN
  GW_CHECK_ARG(ctx && psd && out, "NULL argument");
  *out = nullptr;
  GW_CHECK_ARG(n_psd >= 3 && fs > 0, "bad PSD grid");
  const int N = 2 * (n_psd - 1);
  GW_CHECK_ARG(ntaps >= 1 && (ntaps & 1) && ntaps <= N, "ntaps must be odd and <= nfft");
  GW_CHECK_ARG(precision == GW_FP32 || precision == GW_BF16, "FIR precision must be FP32 or BF16");
  for (int j = 0; j < n_psd; ++j) GW_CHECK_ARG(psd[j] > 0 && std::isfinite(psd[j]), "PSD must be positive and finite");
  *out = fir_from_taps(ctx, design_whitening(psd, n_psd, fs, ntaps), precision);
  GW_API_END
}

int gw_fir_create_bandpass(gw_ctx_t ctx, double fs, int nfft, int ntaps, double f1, double f2, double ramp,
                           int precision, gw_fir_t* out) {
  GW_API_BEGIN
  GW_CHECK_ARG(ctx && out, "NULL argument");
  *out = nullptr;
  GW_CHECK_ARG(fs > 0 && nfft >= 4 && nfft % 2 == 0, "need fs > 0 and an even nfft");
  GW_CHECK_ARG(ntaps >= 1 && (ntaps & 1) && ntaps <= nfft, "ntaps must be odd and <= nfft");
  GW_CHECK_ARG(f1 >= 0 && ramp > 0 && f1 + 2 * ramp <= f2 && f2 <= 0.5 * fs, "need 0 <= f1, f1 + 2 ramp <= f2 <= fs/2");
  GW_CHECK_ARG(precision == GW_FP32, "the post-processing band-pass is FP32");
  const int n = nfft / 2 + 1;
  const double df = fs / nfft;
  std::vector<double> A(n);
  for (int j = 0; j < n; ++j) A[j] = tukey_band(j * df, f1, f2, ramp);
  *out = fir_from_taps(ctx, design_zero_phase(A, ntaps), precision);
  GW_API_END
}

int gw_fir_create_band_loss(gw_ctx_t ctx, const double* psd, int n_psd, double fs, int ntaps, double f1, double f2,
                            double ramp, double f_ref, int precision, gw_fir_t* out) {
  GW_API_BEGIN
  GW_CHECK_ARG(ctx && psd && out, "NULL argument");
  *out = nullptr;
  GW_CHECK_ARG(n_psd >= 3 && fs > 0, "bad PSD grid");
  const int N = 2 * (n_psd - 1);
  GW_CHECK_ARG(ntaps >= 1 && (ntaps & 1) && ntaps <= N, "ntaps must be odd and <= nfft");
  GW_CHECK_ARG(f1 >= 0 && ramp > 0 && f1 + 2 * ramp <= f2 && f2 <= 0.5 * fs, "need 0 <= f1, f1 + 2 ramp <= f2 <= fs/2");
  GW_CHECK_ARG(f_ref >= 0 && f_ref <= 0.5 * fs, "f_ref outside [0, fs/2]");
  GW_CHECK_ARG(precision == GW_FP32 || precision == GW_BF16, "FIR precision must be FP32 or BF16");
  for (int j = 0; j < n_psd; ++j) GW_CHECK_ARG(psd[j] > 0 && std::isfinite(psd[j]), "PSD must be positive and finite");
  *out = fir_from_taps(ctx, design_band_loss(psd, n_psd, fs, ntaps, f1, f2, ramp, f_ref), precision);
  GW_API_END
}

int gw_fir_create_lowpass(gw_ctx_t ctx, double fc, double fs, int ntaps, int precision, gw_fir_t* out) {
  GW_API_BEGIN
  GW_CHECK_ARG(ctx && out, "NULL argument");
  *out = nullptr;
  GW_CHECK_ARG(fs > 0 && fc > 0 && fc < 0.5 * fs, "cutoff must lie in (0, fs / 2)");
  GW_CHECK_ARG(ntaps >= 1 && (ntaps & 1) && ntaps <= 65537, "ntaps must be odd and <= 65537");
  GW_CHECK_ARG(precision == GW_FP32 || precision == GW_BF16, "FIR precision must be FP32 or BF16");
  *out = fir_from_taps(ctx, design_lowpass(fc, fs, ntaps), precision);
  GW_API_END
}

int gw_fir_destroy(gw_fir_t f) {
  GW_API_BEGIN
  GW_CHECK_ARG(f, "fir is NULL");
  DeviceGuard dg(f->ctx ? f->ctx->device : -1);
  cudaDeviceSynchronize();
  if (f->d_taps) cudaFree(f->d_taps);
  for (void* p : f->allocs) cudaFree(p);
  if (f->ws) cudaFree(f->ws);
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    f->ctx->in_use -= f->bytes + f->ws_bytes;
  }
  delete f;
  GW_API_END
}

int gw_fir_ntaps(gw_fir_t f) { return f ? f->ntaps : GW_EINVAL; }

int gw_fir_taps(gw_fir_t f, double* taps_out) {
  GW_API_BEGIN
  GW_CHECK_ARG(f && taps_out, "NULL argument");
  memcpy(taps_out, f->taps.data(), f->taps.size() * sizeof(double));
  GW_API_END
}

int gw_whiten(gw_fir_t f, const float* x, int B, int C, int L_in, float* y, void* cuda_stream) {
  GW_API_BEGIN
  GW_CHECK_ARG(f && x && y, "NULL argument");
  GW_CHECK_ARG(B >= 1 && C >= 1 && L_in >= f->ntaps, "need B, C >= 1 and L_in >= ntaps");
  const int lout = L_in - f->ntaps + 1;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (f->precision == GW_FP32) {
    Prof p("fir_f32", st);
    launch_fir_f32(x, L_in, y, lout, B * C, f->d_taps, f->ntaps, lout, st);
  } else {
    GW_CHECK_ARG(L_in % 8 == 0, "BF16 whitening needs L_in a multiple of 8");
    const int lin8 = L_in / 8, lout8 = lout / 8;
    TcOut xin = blocked_out(nullptr, 8, lin8, f->tc.pin);
    const size_t need = (size_t)B * C * xin.bstride * 2;
    if (need > f->ws_bytes) {
      GW_CUDA(cudaDeviceSynchronize());
      if (f->ws) dev_free(f->ctx, f->ws, f->ws_bytes, nullptr);
      f->ws = nullptr;
      f->ws_bytes = 0;
      f->ws = dev_alloc(f->ctx, need, nullptr);
      f->ws_bytes = need;
    }
    xin.p = f->ws;
    {
      Prof p("to_blocked", st);
      launch_to_blocked(x, L_in, 1, B * C, 8, lin8, nullptr, nullptr, 1.f, xin, 0, st, 8);
    }
    TcOut o{};
    o.p = y;
    o.bstride = lout;
    o.P = 1;
    o.fp32_d2s = 1;
    Prof p("conv_tc.whiten", st);
    launch_conv_tc(f->tc, as_input(xin, lin8), lout8, o, B * C, f->err, st);
  }
  GW_API_END
}

int gw_stream_create(gw_ctx_t ctx, const gw_stream_desc* d, const gw_model_t* deepclean, gw_stream_t* out) {
  gw_stream* s = nullptr;
  GW_API_BEGIN
  GW_CHECK_ARG(ctx && d && deepclean && out, "NULL argument");
  *out = nullptr;
  GW_CHECK_ARG(d->n_det == 1 || d->n_det == 2, "n_det must be 1 or 2");
  GW_CHECK_ARG(d->stride >= 8 && d->stride % 8 == 0, "stride must be a positive multiple of 8");
  GW_CHECK_ARG(d->window >= d->stride && d->window % d->stride == 0 && d->window % 8 == 0,
               "window must be a multiple of stride and of 8");
  GW_CHECK_ARG(d->max_batch >= 1 && d->max_batch <= 4096, "max_batch out of range");
  GW_CHECK_ARG(d->agg_mode == GW_AGG_LATEST || d->agg_mode == GW_AGG_AVERAGE, "unknown aggregation mode");
  GW_CHECK_ARG(d->agg_delay >= 0 && d->agg_delay <= d->window - d->stride, "agg_delay out of range");
  GW_CHECK_ARG(!d->post || (d->post->precision == GW_FP32 && (d->post->ntaps & 1) && d->post->ntaps <= 16385),
               "post-processing FIR must be FP32 with an odd number of taps (<= 16385)");
  for (int i = 0; i < d->n_det; ++i) {
    GW_CHECK_ARG(deepclean[i] && deepclean[i]->kind == GW_MODEL_DEEPCLEAN, "need one DeepClean model per detector");
    GW_CHECK_ARG(deepclean[i]->n_in == d->n_witness, "model n_in != n_witness");
    GW_CHECK_ARG(deepclean[i]->precision == deepclean[0]->precision, "detectors must share a precision");
  }
  GW_CUDA(cudaSetDevice(ctx->device));
  s = new gw_stream();
  s->ctx = ctx;
  s->d = *d;
  const int prec = deepclean[0]->precision;
  for (int i = 0; i < d->n_det; ++i) s->dc[i] = deepclean[i];
  const int64_t W = d->window, S = d->stride, nb = d->max_batch, C = d->n_witness;
  const int64_t post_c = d->post ? (d->post->ntaps - 1) / 2 : 0;
  // the strain ring also serves the post-processed outputs, c samples older
  s->R = W + (nb - 1) * S + post_c;
  s->R = (s->R + 15) / 16 * 16;  // whole rows in every phase plane of the ring
  const int G = (int)((C + 7) / 8);
  try {
    for (int i = 0; i < d->n_det; ++i) {
      if (prec == GW_FP32)
        s->ring_f32[i] = salloc<float>(s, (size_t)C * 2 * s->R);
      else
        s->ring_bf16[i] = salloc<__nv_bfloat16>(s, (size_t)G * 2 * s->R * 8);
      launch_ring_fill(prec == GW_FP32 ? (void*)s->ring_f32[i] : (void*)s->ring_bf16[i], prec != GW_FP32, (int)C, G,
                       2 * s->R, deepclean[i]->in_mean, deepclean[i]->in_istd, nullptr);
      s->strain[i] = salloc<float>(s, (size_t)s->R);
      s->acc[i] = salloc<float>(s, (size_t)s->R);
    }
    s->pred = salloc<float>(s, (size_t)nb * W);
    const size_t act_elems = (size_t)nb * deepclean_tc_act_elems((int)W);
    const size_t esz = prec == GW_FP32 ? 4 : 2;
    s->act0 = salloc<char>(s, act_elems * esz);
    s->act1 = salloc<char>(s, act_elems * esz);
    s->stage_in = salloc<float>(s, (size_t)d->n_det * (C + 1) * nb * S);
    s->stage_out = salloc<float>(s, (size_t)d->n_det * nb * S);
    if (d->post) {
      s->post_K = d->post->ntaps;
      s->post_taps = salloc<float>(s, (size_t)s->post_K);
      GW_CUDA(cudaMemcpy(s->post_taps, d->post->d_taps, (size_t)s->post_K * sizeof(float), cudaMemcpyDeviceToDevice));
      // the FIR of a push reads predictions from c before its first output to
      // c after its last one
      s->Rp = (nb * S + 2 * post_c + 64 + 63) / 64 * 64;
      for (int i = 0; i < d->n_det; ++i) s->pring[i] = salloc<float>(s, (size_t)s->Rp);
    }
    s->status = salloc<int>(s, 3);
    s->err = s->status + 1;
    s->reject = s->status + 2;
    GW_CUDA(cudaHostAlloc((void**)&s->reject_h, (1 + GW_STREAM_MAX_PENDING) * sizeof(int), cudaHostAllocDefault));
    s->head_q.resize(GW_STREAM_MAX_PENDING);
    s->stage_in_q[0] = s->stage_in;
    s->stage_out_q[0] = s->stage_out;
    s->stage_in_q[1] = salloc<float>(s, (size_t)d->n_det * (C + 1) * nb * S);
    s->stage_out_q[1] = salloc<float>(s, (size_t)d->n_det * nb * S);
    s->reject_q = salloc<int>(s, GW_STREAM_MAX_PENDING);
    GW_CUDA(cudaStreamCreateWithFlags(&s->cs_in, cudaStreamNonBlocking));
    GW_CUDA(cudaStreamCreateWithFlags(&s->cs_out, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
      GW_CUDA(cudaEventCreateWithFlags(&s->ev_in[b], cudaEventDisableTiming));
      GW_CUDA(cudaEventCreateWithFlags(&s->ev_done[b], cudaEventDisableTiming));
      GW_CUDA(cudaEventCreateWithFlags(&s->ev_out[b], cudaEventDisableTiming));
    }
    GW_CUDA(cudaDeviceSynchronize());
  } catch (...) {
    stream_free(s);
    s = nullptr;
    throw;
  }
  *out = s;
  s = nullptr;
  GW_API_END
}

int gw_stream_destroy(gw_stream_t s) {
  GW_API_BEGIN
  GW_CHECK_ARG(s, "stream is NULL");
  stream_free(s);
  GW_API_END
}

int64_t gw_stream_head(gw_stream_t s) { return s ? s->head : GW_EINVAL; }

int gw_stream_status(gw_stream_t s, void* cuda_stream) {
  GW_API_BEGIN
  GW_CHECK_ARG(s, "stream is NULL");
  int h[2] = {0, 0};
  GW_CUDA(cudaMemcpyAsync(h, s->status, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)cuda_stream));
  GW_CUDA(cudaStreamSynchronize((cudaStream_t)cuda_stream));
  if (h[0]) return h[0];
  if (h[1]) return GW_ETIMEOUT;
  GW_API_END
}

// Queues the device work of one push of n_snap snapshots on st: wit / str /
// out are device buffers in the layouts of gw_stream_push; skip (device, may
// be null) is the reject flag that the state-changing kernels obey, and
// skip_copy (device, may be null) receives its value as this push left it.
static void stream_compute(gw_stream* s, int n_snap, const float* wit, const float* str, float* out,
                           const int* skip, int* skip_copy, cudaStream_t st) {
  GW_CHECK_ARG(n_snap >= 1 && n_snap <= s->d.max_batch, "n_snap out of range [1, max_batch]");
  const int C = s->d.n_witness, S = s->d.stride, W = s->d.window, nd = s->d.n_det;
  const int64_t n = (int64_t)n_snap * S;
  const int64_t R = s->R, head = s->head;
  const int G = (C + 7) / 8;
  for (int d = 0; d < nd; ++d) {
    gw_model* m = s->dc[d];
    const float* wd = wit + (size_t)d * C * n;
    if (m->precision == GW_FP32) {
      {
        Prof p("ring_push", st);
        launch_ring_push_f32(wd, n, C, (int)n, s->ring_f32[d], R, head, m->in_mean, m->in_istd, s->status, st, skip);
      }
      Prof p("strain_push", st);
      launch_strain_push(str + (size_t)d * n, (int)n, s->strain[d], R, head, s->status, st, skip);
    } else {
      Prof p("stream_push", st);
      launch_stream_push_bf16(wd, n, C, G, (int)n, s->ring_bf16[d], R, head, m->layers[0].pin, m->in_mean,
                              m->in_istd, str + (size_t)d * n, s->strain[d], s->status, st, skip);
    }
    // window j of this batch ends at head + (j+1) S; in the double-mapped ring
    // the batch's windows are views at uniform stride S from p0.
    int64_t p0 = (head + S - W) % R;
    if (p0 < 0) p0 += R;
    if (m->precision == GW_FP32) {
      deepclean_f32(m, s->ring_f32[d] + p0, S, 2 * R, false, n_snap, W, s->pred, W, (float*)s->act0,
                    (float*)s->act1, st);
    } else {
      // the first layer reads the windows in place from the blocked BF16 ring,
      // stored in the P phase planes the layer consumes (window starts are
      // multiples of P because S and W are)
      const int P = m->layers[0].pin;
      GW_CHECK_ARG(S % P == 0 && W % P == 0 && p0 % P == 0 && R % P == 0,
                   "stride and window must be multiples of the first layer's phase count");
      TcIn in{};
      in.p = s->ring_bf16[d];
      in.off0 = (p0 / P) * 8;
      in.bstride = 0;
      in.boff = S / P;
      in.gstride = 2 * R * 8;
      in.pstride = (2 * R / P) * 8;
      in.P = P;
      in.L = W;
      // the ring update before this launch writes the batch's newest n samples:
      // positions x >= W - (j+1) S of window j
      deepclean_tc(m, in, n_snap, W, s->pred, W, s->act0, s->act1, s->err, st, W - S, S);
    }
    {
      Prof p("sub_ola", st);
      launch_sub_ola(s->pred, W, n_snap, S, W, R, head, s->d.agg_mode, s->d.agg_delay, s->acc[d], s->strain[d],
                     out + (size_t)d * n, st, skip, s->pring[d], s->Rp, d == 0 ? skip_copy : nullptr);
    }
    if (s->post_K) {
      Prof p("post", st);
      launch_post_sub(s->pring[d], s->Rp, s->post_taps, s->post_K, s->strain[d], R,
                      head - s->d.agg_delay - (s->post_K - 1) / 2, (int)n, out + (size_t)d * n, st, skip);
    }
  }
}


int gw_stream_push(gw_stream_t s, int n_snap, const float* witness, const float* strain, float* clean_out, int mem,
                   void* cuda_stream) {
  GW_API_BEGIN
  GW_CHECK_ARG(s && witness && strain && clean_out, "NULL argument");
  GW_CHECK_ARG(mem == GW_MEM_HOST || mem == GW_MEM_DEVICE, "mem must be GW_MEM_HOST or GW_MEM_DEVICE");
  if (s->pending) throw Error(GW_ESTATE, "asynchronous pushes are pending: call gw_stream_sync first");
  GW_CHECK_ARG(n_snap >= 1 && n_snap <= s->d.max_batch, "n_snap out of range [1, max_batch]");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (mem == GW_MEM_DEVICE) {
    stream_compute(s, n_snap, witness, strain, clean_out, nullptr, nullptr, st);
  } else {
    // Host mode rejects a push with a non-finite sample before the state
    // changes: the staged input is checked on the device, the state-changing
    // kernels (ring, strain and aggregation updates) skip their writes when
    // the check failed, and the verdict is read back with the results.
    const size_t n = (size_t)n_snap * s->d.stride, nd = s->d.n_det;
    const size_t nw = nd * s->d.n_witness * n, ns = nd * n;
    GW_CUDA(cudaMemsetAsync(s->reject, 0, sizeof(int), st));
    GW_CUDA(cudaMemcpyAsync(s->stage_in, witness, nw * 4, cudaMemcpyHostToDevice, st));
    GW_CUDA(cudaMemcpyAsync(s->stage_in + nw, strain, ns * 4, cudaMemcpyHostToDevice, st));
    launch_check_finite(s->stage_in, (int64_t)(nw + ns), s->reject, st);
    stream_compute(s, n_snap, s->stage_in, s->stage_in + nw, s->stage_out, s->reject, nullptr, st);
    GW_CUDA(cudaMemcpyAsync(clean_out, s->stage_out, ns * 4, cudaMemcpyDeviceToHost, st));
    GW_CUDA(cudaMemcpyAsync(s->reject_h, s->reject, sizeof(int), cudaMemcpyDeviceToHost, st));
    GW_CUDA(cudaStreamSynchronize(st));
    if (*s->reject_h) throw Error(GW_ENONFINITE, "non-finite input sample");
  }
  s->head += (int64_t)n_snap * s->d.stride;
  GW_API_END
}

int gw_stream_push_async(gw_stream_t s, int n_snap, const float* witness, const float* strain, float* clean_out,
                         void* cuda_stream) {
  GW_API_BEGIN
  GW_CHECK_ARG(s && witness && strain && clean_out, "NULL argument");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (s->pending) {
    GW_CHECK_ARG(st == s->async_st, "pending asynchronous pushes were queued on another CUDA stream");
    if (s->pending >= GW_STREAM_MAX_PENDING)
      throw Error(GW_ESTATE, "GW_STREAM_MAX_PENDING pushes pending: call gw_stream_sync first");
  }
  GW_CHECK_ARG(n_snap >= 1 && n_snap <= s->d.max_batch, "n_snap out of range [1, max_batch]");
  const int k = s->pending, b = k & 1;
  const size_t n = (size_t)n_snap * s->d.stride, nd = s->d.n_det;
  const size_t nw = nd * s->d.n_witness * n, ns = nd * n;
  float* in = s->stage_in_q[b];
  float* out = s->stage_out_q[b];
  // inputs: once the compute of the push before last (same set) is done
  GW_CUDA(cudaStreamWaitEvent(s->cs_in, s->ev_done[b], 0));
  GW_CUDA(cudaMemcpyAsync(in, witness, nw * 4, cudaMemcpyHostToDevice, s->cs_in));
  GW_CUDA(cudaMemcpyAsync(in + nw, strain, ns * 4, cudaMemcpyHostToDevice, s->cs_in));
  GW_CUDA(cudaEventRecord(s->ev_in[b], s->cs_in));
  // compute: once the inputs are staged and the outputs of the push before
  // last (same set) are copied out.  The device flag is cleared once per
  // sequence of queued pushes: a rejected push leaves it set, so every later
  // push of the sequence skips its state updates as well and the state stays
  // that before the rejected push.
  GW_CUDA(cudaStreamWaitEvent(st, s->ev_in[b], 0));
  GW_CUDA(cudaStreamWaitEvent(st, s->ev_out[b], 0));
  if (k == 0) GW_CUDA(cudaMemsetAsync(s->reject, 0, sizeof(int), st));
  launch_check_finite(in, (int64_t)(nw + ns), s->reject, st);
  stream_compute(s, n_snap, in, in + nw, out, s->reject, s->reject_q + k, st);
  GW_CUDA(cudaEventRecord(s->ev_done[b], st));
  // outputs and this push's verdict
  GW_CUDA(cudaStreamWaitEvent(s->cs_out, s->ev_done[b], 0));
  GW_CUDA(cudaMemcpyAsync(clean_out, out, ns * 4, cudaMemcpyDeviceToHost, s->cs_out));
  GW_CUDA(cudaMemcpyAsync(s->reject_h + 1 + k, s->reject_q + k, sizeof(int), cudaMemcpyDeviceToHost, s->cs_out));
  GW_CUDA(cudaEventRecord(s->ev_out[b], s->cs_out));
  s->async_st = st;
  s->head_q[s->pending++] = s->head;
  s->head += (int64_t)n_snap * s->d.stride;
  GW_API_END
}

int gw_stream_sync(gw_stream_t s, int* first_rejected) {
  GW_API_BEGIN
  GW_CHECK_ARG(s, "stream is NULL");
  if (first_rejected) *first_rejected = -1;
  if (!s->pending) return GW_OK;
  const int n = s->pending;
  s->pending = 0;
  GW_CUDA(cudaStreamSynchronize(s->cs_out));
  GW_CUDA(cudaStreamSynchronize(s->async_st));
  for (int k = 0; k < n; ++k) {
    if (s->reject_h[1 + k]) {
      // push k and every later one skipped their state updates: rewind
      s->head = s->head_q[k];
      if (first_rejected) *first_rejected = k;
      GW_CUDA(cudaMemsetAsync(s->reject, 0, sizeof(int), s->async_st));
      GW_CUDA(cudaStreamSynchronize(s->async_st));
      throw Error(GW_ENONFINITE, "non-finite input sample in queued push " + std::to_string(k) +
                                     "; it and the later queued pushes were not applied");
    }
  }
  GW_API_END
}

}  // extern "C"
