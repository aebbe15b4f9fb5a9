// DeepClean training step: forward with a tape, band-limited PSD-weighted
// loss, hand-written backward to the raw (unfolded) parameters, Adam.
//
// The paper retrains DeepClean regularly on recent data (main text, model
// validity and retraining) without giving the loss; the loss here is the
// reading of the band-limited inverse-PSD-weighted mean square error
//   L = (1 / N) sum_{b,n} r[b][n]^2,  r = g (*) (s - y_hat)  (valid mode),
// with |G(f)|^2 = T(f) S(f_ref) / S(f) on the 55-65 Hz band.  BatchNorm runs
// with its running statistics (eval mode), so it folds into the weights; the
// trained parameters are the raw w, b, gamma, beta of every layer, kept by the
// caller in FP32 ("master weights") and folded on the device at every forward.
//
// Backward per layer (from the output down), with v = folded conv output and
// y = act(v):
//   dv = dy * act'(y)                         (fused into the data gradient)
//   dW' = wgrad(input, dv), db' = sum dv      (fixed-order reductions)
//   raw: dw = dW' sc, db = db' sc, dbeta = db', dgamma = a (sum w dW' + db' (b - mean))
//   d input = conv-transpose of dv with W'^T (conv) / conv of dv with W'^T (transposed conv)
// Weight gradients: FP32 (SIMT FMA, fixed-order reductions) or, with
// precision GW_BF16, on the tensor cores (BF16 operands, FP32 accumulation in
// TMEM, per-CTA partials summed in a fixed order; k_wgrad_tc.cu).
// Activation checkpointing: with `checkpoint`, only the inputs of the four
// blocks (enc1-enc2, enc3-enc4, dec1-dec2, dec3-out) are kept and the first
// layer's output of each block is recomputed during the backward.
#include "gw_train.h"

namespace gw {
namespace {

struct TrainLayer {
  LayerSpec s;
  int lin = 0, lout = 0;
  FoldArgs f{};
  // tensor-core forward / data gradient (tc_data): the layer and the layer
  // that maps its output gradient to its input gradient, with operand images
  // refilled from the folded weights at every forward (maps: image element ->
  // index into wf / wT)
  LayerDev tf, td;
  const int32_t* map_f = nullptr;
  const int32_t* map_d = nullptr;
  int64_t n_f = 0, n_d = 0;
};

// The weight-gradient contraction of a layer (operand pointers left to the
// caller): conv, A = the output gradient and Bm = the input; transposed conv,
// A = the input and Bm = the output gradient.  The tensor-core kernel also
// gives the bias gradient (bias 1: conv, 2: transposed conv).
WgradArgs wgrad_plan(const TrainLayer& T) {
  const LayerSpec& s = T.s;
  WgradArgs w = s.transposed ? plan_wgrad(s.cin, s.cout, s.k, s.stride, T.lin)
                             : plan_wgrad(s.cout, s.cin, s.k, s.stride, T.lout);
  w.LB = s.transposed ? T.lout : T.lin;
  w.p = s.pad_l;
  w.bias = s.transposed ? 2 : 1;
  if (!wgrad_tc_supported(w)) w.bias = 0;
  return w;
}

}  // namespace
}  // namespace gw

struct gw_trainer {
  gw_ctx* ctx = nullptr;
  int n_in = 0, max_batch = 0, L = 0, checkpoint = 0, wgrad_tc = 0, tc_data = 0;
  // tc_data: blocked BF16 inputs of the tensor-core convs; [0] and [1] alternate
  // along the forward and along the backward (each conv writes its successor's
  // input beside its FP32 output), [2] serves the recomputed layers
  char* blk[3] = {nullptr, nullptr, nullptr};
  std::vector<void*> tc_allocs;  // operand images, slice tables and weight maps of the tensor-core layers
  size_t tc_bytes = 0;
  int* err = nullptr;  // device: a tensor-core kernel gave up a bounded wait
  size_t n_params = 0;
  std::vector<gw::TrainLayer> layers;
  float* in_mean = nullptr;
  float* in_istd = nullptr;
  float* x_std = nullptr;
  std::vector<float*> act;  // output of layer l (l < n_layers - 1), or null when recomputed
  float* scratch = nullptr; // recomputed activation
  float* dv[2] = {nullptr, nullptr};
  float* partial = nullptr;
  // per layer: the folded parameters' gradients, unfolded after the backward
  std::vector<float*> dWf, dbf;
  float* bpart = nullptr;
  float* zero_bias = nullptr;
  const float* params = nullptr;  // raw parameters of the last forward
  int B = 0;
  std::vector<std::pair<void*, size_t>> allocs;
  size_t bytes = 0;
};

namespace gw {
namespace {

template <typename T>
T* talloc(gw_trainer* t, size_t count) {
  const size_t b = std::max<size_t>(count * sizeof(T), 256);
  T* p = (T*)dev_alloc(t->ctx, b, &t->bytes);
  t->allocs.push_back({p, b});
  GW_CUDA(cudaMemset(p, 0, b));
  return p;
}

void trainer_free(gw_trainer* t) {
  if (!t) return;
  DeviceGuard dg(t->ctx ? t->ctx->device : -1);
  cudaDeviceSynchronize();
  for (auto& a : t->allocs) dev_free(t->ctx, a.first, a.second, nullptr);
  bool first = true;  // the tensor-core layers' bytes are returned to the budget with the first of their buffers
  for (void* p : t->tc_allocs) {
    dev_free(t->ctx, p, first ? t->tc_bytes : 0, nullptr);
    first = false;
  }
  delete t;
}

const char* kWgradNames[8] = {"train.wgrad.enc1", "train.wgrad.enc2", "train.wgrad.enc3", "train.wgrad.enc4",
                              "train.wgrad.dec1", "train.wgrad.dec2", "train.wgrad.dec3", "train.wgrad.out"};
const char* kWgradTcNames[8] = {"train.wgrad_tc.enc1", "train.wgrad_tc.enc2", "train.wgrad_tc.enc3",
                                "train.wgrad_tc.enc4", "train.wgrad_tc.dec1", "train.wgrad_tc.dec2",
                                "train.wgrad_tc.dec3", "train.wgrad_tc.out"};

bool recomputed(const gw_trainer* t, int l) { return t->checkpoint && (l % 2 == 0) && l + 1 < (int)t->layers.size(); }

// Forward of layer l from `in` into `out` (out strides: item cout*lout, channel lout).
// Tensor-core forward of layer l (tc_data): its input in the blocked BF16
// layout is at in_blk (converted from `in` into t->blk[2] when null); writes
// FP32 [B][C][L] (the output layer: FP32 [B][L]) and, when out_blk is given,
// the same values blocked for the next layer.
void layer_forward_tc(gw_trainer* t, int l, const float* in, const TcOut* in_blk, float* out, int64_t yb, int64_t yc,
                      const TcOut* out_blk, int B, cudaStream_t st) {
  const TrainLayer& T = t->layers[l];
  TcOut blk;
  if (in_blk) {
    blk = *in_blk;
  } else {
    blk = blocked_out(t->blk[2], T.s.cin, T.lin, T.tf.pin);
    Prof p("train.to_blocked", st);
    launch_to_blocked(in, (int64_t)T.s.cin * T.lin, T.lin, B, T.s.cin, T.lin, nullptr, nullptr, 1.f, blk, 0, st);
  }
  TcOut o{};
  o.p = out;
  o.bstride = yb;
  o.gstride = yc;
  o.P = 1;
  if (T.s.cout == 1) {
    o.fp32_single = 1;
  } else {
    o.fp32_full = 1;
    if (out_blk) {
      o.blk = out_blk->p;
      o.blk_b = out_blk->bstride;
      o.blk_g = out_blk->gstride;
      o.blk_p = out_blk->pstride;
      o.blk_P = out_blk->P;
    }
  }
  Prof p("train.conv_fwd_tc", st);
  launch_conv_tc(T.tf, as_input(blk, T.lin), T.lout, o, B, t->err, st);
}

void layer_forward(gw_trainer* t, int l, const float* in, float* out, int64_t yb, int64_t yc, int B, cudaStream_t st) {
  const TrainLayer& T = t->layers[l];
  if (t->tc_data) {
    layer_forward_tc(t, l, in, nullptr, out, yb, yc, nullptr, B, st);
    return;
  }
  ConvF32Args a{};
  a.x = in;
  a.xb = (int64_t)T.s.cin * T.lin;
  a.xc = T.lin;
  a.y = out;
  a.yb = yb;
  a.yc = yc;
  a.w = T.f.wf;
  a.bias = T.f.bf;
  a.B = B;
  a.lin = T.lin;
  a.lout = T.lout;
  a.s = T.s;
  Prof p("train.conv_fwd", st);
  launch_conv_f32(a, st);
}

const float* layer_input(gw_trainer* t, int l) { return l == 0 ? t->x_std : (t->act[l - 1] ? t->act[l - 1] : t->scratch); }

}  // namespace
}  // namespace gw

using namespace gw;

extern "C" {

int gw_trainer_create(gw_ctx_t ctx, const gw_trainer_desc* d, const float* in_mean, const float* in_std,
                      gw_trainer_t* out) {
  gw_trainer* t = nullptr;
  GW_API_BEGIN
  GW_CHECK_ARG(ctx && d && out, "NULL argument");
  *out = nullptr;
  GW_CHECK_ARG(d->n_in >= 1 && d->n_in <= 256, "n_in out of range");
  GW_CHECK_ARG(d->max_batch >= 1 && d->max_batch <= 4096, "max_batch out of range");
  GW_CHECK_ARG(d->length >= 16 && d->length % 8 == 0, "length must be a multiple of 8, >= 16");
  GW_CHECK_ARG(d->checkpoint == 0 || d->checkpoint == 1, "checkpoint must be 0 or 1");
  GW_CHECK_ARG(d->precision == GW_FP32 || d->precision == GW_BF16, "trainer precision must be FP32 or BF16");
  GW_CHECK_ARG(d->precision == GW_FP32 || tc_supported(), "BF16 weight gradients need the sm_103a tensor cores");
  GW_CHECK_ARG(d->tc_data == 0 || (d->tc_data == 1 && d->precision == GW_BF16),
               "tc_data (forward and data gradients on the tensor cores) needs precision GW_BF16");
  GW_CUDA(cudaSetDevice(ctx->device));
  t = new gw_trainer();
  try {
    t->ctx = ctx;
    t->n_in = d->n_in;
    t->max_batch = d->max_batch;
    t->L = d->length;
    t->checkpoint = d->checkpoint;
    t->wgrad_tc = d->precision == GW_BF16;
    t->tc_data = d->tc_data;
    const auto specs = deepclean_specs(d->n_in);
    int64_t off = 0;
    int lin = d->length;
    size_t max_act = 0, max_partial = 0;
    int max_c = 0;
    for (const auto& s : specs) {
      TrainLayer T;
      T.s = s;
      T.lin = lin;
      T.lout = s.lout(lin);
      FoldArgs& f = T.f;
      f.cin = s.cin;
      f.cout = s.cout;
      f.K = s.k;
      f.transposed = s.transposed;
      f.bn = s.bn;
      f.off_w = off;
      off += (int64_t)s.cin * s.cout * s.k;
      f.off_b = off;
      off += s.cout;
      if (s.bn) {
        f.off_g = off;
        f.off_be = off + s.cout;
        f.off_mu = off + 2 * s.cout;
        f.off_var = off + 3 * s.cout;
        off += 4 * s.cout;
      }
      max_act = std::max(max_act, (size_t)std::max(s.cin * T.lin, s.cout * T.lout));
      const size_t nw = (size_t)s.cin * s.cout * s.k;
      max_c = std::max(max_c, std::max(s.cin, s.cout));
      const WgradArgs w = wgrad_plan(T);
      max_partial = std::max(max_partial, (size_t)d->max_batch * w.chunks_per_b * nw);
      if (d->precision == GW_BF16 && wgrad_tc_supported(w))
        max_partial = std::max(max_partial, wgrad_tc_partial_floats(w, d->max_batch));
      t->layers.push_back(T);
      lin = T.lout;
    }
    GW_CHECK_ARG(lin == d->length, "length does not round-trip through the network");
    t->n_params = (size_t)off;
    const int Bm = d->max_batch;
    for (auto& T : t->layers) {
      const size_t nw = (size_t)T.s.cin * T.s.cout * T.s.k;
      T.f.wf = talloc<float>(t, nw);
      T.f.wT = talloc<float>(t, nw);
      T.f.bf = talloc<float>(t, T.s.cout);
    }
    std::vector<float> mean(d->n_in, 0.f), istd(d->n_in, 1.f);
    for (int c = 0; c < d->n_in; ++c) {
      if (in_mean) mean[c] = in_mean[c];
      if (in_std) {
        GW_CHECK_ARG(in_std[c] > 0 && std::isfinite(in_std[c]), "in_std must be positive");
        istd[c] = 1.f / in_std[c];
      }
    }
    t->in_mean = talloc<float>(t, d->n_in);
    t->in_istd = talloc<float>(t, d->n_in);
    GW_CUDA(cudaMemcpy(t->in_mean, mean.data(), d->n_in * 4, cudaMemcpyHostToDevice));
    GW_CUDA(cudaMemcpy(t->in_istd, istd.data(), d->n_in * 4, cudaMemcpyHostToDevice));
    t->x_std = talloc<float>(t, (size_t)Bm * d->n_in * d->length);
    const int nl = (int)t->layers.size();
    t->act.assign(nl - 1, nullptr);
    for (int l = 0; l + 1 < nl; ++l)
      if (!recomputed(t, l))
        t->act[l] = talloc<float>(t, (size_t)Bm * t->layers[l].s.cout * t->layers[l].lout);
    if (t->checkpoint) t->scratch = talloc<float>(t, (size_t)Bm * max_act);
    t->dv[0] = talloc<float>(t, (size_t)Bm * max_act);
    t->dv[1] = talloc<float>(t, (size_t)Bm * max_act);
    t->partial = talloc<float>(t, max_partial);
    for (const TrainLayer& T : t->layers) {
      t->dWf.push_back(talloc<float>(t, (size_t)T.s.cin * T.s.cout * T.s.k));
      t->dbf.push_back(talloc<float>(t, T.s.cout));
    }
    t->bpart = talloc<float>(t, (size_t)Bm * max_c);
    t->zero_bias = talloc<float>(t, max_c);
    t->err = talloc<int>(t, 1);
    if (t->tc_data) {
      // per layer: the forward conv (weights: wf, as stored) and the conv that
      // maps its output gradient to its input gradient (weights: wT; a
      // stride-2 conv's is a transposed conv and vice versa, a stride-1 conv's
      // is a stride-1 conv with the taps reversed and padding K - 1 - p)
      size_t max_blk = 0;
      for (int l = 0; l < nl; ++l) {
        TrainLayer& T = t->layers[l];
        const LayerSpec& s = T.s;
        const size_t nw = (size_t)s.cin * s.cout * s.k;
        std::vector<int32_t> src(nw);
        for (size_t i = 0; i < nw; ++i) src[i] = (int32_t)i;
        T.tf.s = s;
        T.tf.b = T.f.bf;
        tc_prepare_trainable(T.tf, ctx, &t->tc_bytes, t->tc_allocs, src, &T.map_f, &T.n_f);
        max_blk = std::max(max_blk, (size_t)blocked_out(nullptr, s.cin, T.lin, T.tf.pin).bstride);
        if (l == 0) continue;  // the network input needs no gradient
        LayerSpec ds{};
        ds.cin = s.cout;
        ds.cout = s.cin;
        ds.k = s.k;
        ds.out_pad = 0;
        ds.bn = false;
        ds.act = ACT_NONE;
        if (s.stride == 2) {
          ds.transposed = !s.transposed;
          ds.stride = 2;
          ds.pad_l = s.pad_l;
          ds.pad_r = s.pad_r;
        } else {
          GW_CHECK_ARG(!s.transposed && s.stride == 1, "unsupported layer for the tensor-core data gradient");
          ds.transposed = false;
          ds.stride = 1;
          ds.pad_l = ds.pad_r = s.k - 1 - s.pad_l;
          for (int c = 0; c < s.cin; ++c)
            for (int o = 0; o < s.cout; ++o)
              for (int k = 0; k < s.k; ++k)
                src[((size_t)c * s.cout + o) * s.k + k] = (int32_t)(((size_t)c * s.cout + o) * s.k + (s.k - 1 - k));
        }
        T.td.s = ds;
        T.td.b = t->zero_bias;
        tc_prepare_trainable(T.td, ctx, &t->tc_bytes, t->tc_allocs, src, &T.map_d, &T.n_d);
        max_blk = std::max(max_blk, (size_t)blocked_out(nullptr, s.cout, T.lout, T.td.pin).bstride);
      }
      for (int i = 0; i < 3; ++i) t->blk[i] = talloc<char>(t, (size_t)Bm * max_blk * 2);
    }
  } catch (...) {
    trainer_free(t);
    throw;
  }
  *out = t;
  GW_API_END
}

int gw_trainer_status(gw_trainer_t t, void* cuda_stream) {
  GW_API_BEGIN
  GW_CHECK_ARG(t, "trainer is NULL");
  int h = 0;
  GW_CUDA(cudaMemcpyAsync(&h, t->err, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)cuda_stream));
  GW_CUDA(cudaStreamSynchronize((cudaStream_t)cuda_stream));
  if (h) throw Error(GW_ETIMEOUT, "a tensor-core kernel gave up a bounded wait (flag " + std::to_string(h) + ")");
  GW_API_END
}

int gw_trainer_destroy(gw_trainer_t t) {
  GW_API_BEGIN
  GW_CHECK_ARG(t, "trainer is NULL");
  trainer_free(t);
  GW_API_END
}

int64_t gw_trainer_param_count(gw_trainer_t t) { return t ? (int64_t)t->n_params : GW_EINVAL; }

int64_t gw_trainer_bytes(gw_trainer_t t) { return t ? (int64_t)t->bytes : GW_EINVAL; }

int gw_trainer_forward(gw_trainer_t t, const float* params, const float* x, int B, float* y_hat, void* cuda_stream) {
  GW_API_BEGIN
  GW_CHECK_ARG(t && params && x && y_hat, "NULL argument");
  GW_CHECK_ARG(B >= 1 && B <= t->max_batch, "B out of range [1, max_batch]");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  t->params = params;
  t->B = B;
  std::vector<TcPackSeg> packs;
  std::vector<FoldArgs> folds;
  for (auto& T : t->layers) {
    T.f.p = params;
    folds.push_back(T.f);
  }
  {
    Prof p("train.fold", st);
    launch_fold_many(folds.data(), (int)folds.size(), st);
  }
  for (auto& T : t->layers) {
    if (t->tc_data) {
      packs.push_back({T.f.wf, T.map_f, T.n_f, T.tf.wq});
      if (T.map_d) packs.push_back({T.f.wT, T.map_d, T.n_d, T.td.wq});
    }
  }
  if (!packs.empty()) {
    // this step's folded weights into the tensor-core operand images
    Prof p("train.pack", st);
    launch_tc_pack_many(packs.data(), (int)packs.size(), st);
  }
  const int nl = (int)t->layers.size();
  const float* in = t->x_std;
  TcOut cur{};
  if (t->tc_data) {
    // one pass: the standardised input in FP32 (the tape) and blocked BF16 (the first conv's operand)
    const TrainLayer& T0 = t->layers[0];
    cur = blocked_out(t->blk[0], T0.s.cin, T0.lin, T0.tf.pin);
    Prof p("train.standardise", st);
    const int64_t xb = (int64_t)T0.s.cin * T0.lin;
    launch_to_blocked(x, xb, T0.lin, B, T0.s.cin, T0.lin, t->in_mean, t->in_istd, 1.f, cur, 0, st, 1, t->x_std, xb,
                      T0.lin);
  } else {
    Prof p("train.standardise", st);
    launch_standardise(x, B, t->n_in, t->L, t->in_mean, t->in_istd, t->x_std, st);
  }
  for (int l = 0; l < nl; ++l) {
    const TrainLayer& T = t->layers[l];
    float* out;
    int64_t yb = (int64_t)T.s.cout * T.lout, yc = T.lout;
    if (l + 1 == nl) {
      out = y_hat;
      yb = t->L;
      yc = t->L;
    } else {
      out = t->act[l] ? t->act[l] : t->scratch;
    }
    if (t->tc_data) {
      TcOut next{};
      if (l + 1 < nl) next = blocked_out(t->blk[(l + 1) & 1], T.s.cout, T.lout, t->layers[l + 1].tf.pin);
      layer_forward_tc(t, l, in, &cur, out, yb, yc, l + 1 < nl ? &next : nullptr, B, st);
      cur = next;
    } else {
      layer_forward(t, l, in, out, yb, yc, B, st);
    }
    in = out;
  }
  GW_API_END
}

int gw_trainer_backward(gw_trainer_t t, const float* dy_hat, float* dparams, void* cuda_stream) {
  GW_API_BEGIN
  GW_CHECK_ARG(t && dy_hat && dparams, "NULL argument");
  GW_CHECK_ARG(t->params && t->B >= 1, "backward before forward");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int B = t->B, nl = (int)t->layers.size();
  const float* g = dy_hat;  // gradient w.r.t. the current layer's (pre-activation) output
  int64_t gb = t->L, gn = t->L;
  int cur = 0;
  TcOut gnext{};  // tc_data: the next data gradient's input, blocked by the previous one
  for (int l = nl - 1; l >= 0; --l) {
    const TrainLayer& T = t->layers[l];
    const LayerSpec& s = T.s;
    if (l > 0 && recomputed(t, l - 1)) {
      // the checkpointed block input is the output of layer l - 2 (or x)
      const TrainLayer& P = t->layers[l - 1];
      layer_forward(t, l - 1, layer_input(t, l - 1), t->scratch, (int64_t)P.s.cout * P.lout, P.lout, B, st);
    }
    const float* xin = layer_input(t, l);
    const int64_t xb = (int64_t)s.cin * T.lin, xc = T.lin;
    WgradArgs w = wgrad_plan(T);
    if (!s.transposed) {
      w.A = g; w.ab = gb; w.aa = gn;
      w.Bm = xin; w.bb = xb; w.bc = xc;
    } else {
      w.A = xin; w.ab = xb; w.aa = xc;
      w.Bm = g; w.bb = gb; w.bc = gn;
    }
    w.partial = t->partial;
    bool db_done = false;
    if (t->wgrad_tc && wgrad_tc_supported(w)) {
      // the bias gradient comes with the weight gradient (a row of ones in the GEMM)
      Prof p(l < 8 ? kWgradTcNames[l] : "train.wgrad_tc", st);
      launch_wgrad_tc(w, B, t->partial, t->dWf[l], w.bias ? t->dbf[l] : nullptr, t->err, st);
      db_done = w.bias != 0;
    } else {
      w.bias = 0;
      {
        Prof p(l < 8 ? kWgradNames[l] : "train.wgrad", st);
        launch_wgrad_partial(w, B, st);
      }
      {
        Prof p("train.wgrad_reduce", st);
        launch_wgrad_reduce(w, B, t->dWf[l], st);
      }
    }
    if (!db_done) {
      Prof p("train.bgrad", st);
      launch_bias_grad(g, gb, gn, B, s.cout, T.lout, t->bpart, t->dbf[l], st);
    }
    if (l == 0) break;
    // data gradient, times the derivative of layer l-1's activation (whose
    // output is this layer's input)
    if (t->tc_data) {
      float* dst = t->dv[cur];
      TcOut gblk;
      if (l == nl - 1) {
        // the loss gradient, blocked once; later layers' come with their FP32 copies
        gblk = blocked_out(t->blk[0], s.cout, T.lout, T.td.pin);
        Prof p("train.to_blocked", st);
        launch_to_blocked(g, gb, gn, B, s.cout, T.lout, nullptr, nullptr, 1.f, gblk, 0, st);
      } else {
        gblk = gnext;
      }
      if (l - 1 >= 1) gnext = blocked_out(t->blk[(gblk.p == t->blk[0]) ? 1 : 0], s.cin, T.lin, t->layers[l - 1].td.pin);
      TcOut o{};
      o.p = dst;
      o.bstride = xb;
      o.gstride = xc;
      o.P = 1;
      o.fp32_full = 1;
      o.gy = xin;
      o.gy_b = xb;
      o.gy_c = xc;
      o.gact = t->layers[l - 1].s.act;
      if (l - 1 >= 1) {
        o.blk = gnext.p;
        o.blk_b = gnext.bstride;
        o.blk_g = gnext.gstride;
        o.blk_p = gnext.pstride;
        o.blk_P = gnext.P;
      }
      {
        Prof p("train.dgrad_tc", st);
        launch_conv_tc(T.td, as_input(gblk, T.lout), T.lin, o, B, t->err, st);
      }
      g = dst;
      gb = xb;
      gn = xc;
      cur ^= 1;
      continue;
    }
    ConvF32Args a{};
    a.x = g;
    a.xb = gb;
    a.xc = gn;
    float* dst = t->dv[cur];
    a.y = dst;
    a.yb = xb;
    a.yc = xc;
    a.w = T.f.wT;
    a.bias = t->zero_bias;
    a.B = B;
    a.lin = T.lout;
    a.lout = T.lin;
    LayerSpec ds{};
    ds.transposed = !s.transposed;
    ds.cin = s.cout;
    ds.cout = s.cin;
    ds.k = s.k;
    ds.stride = s.stride;
    ds.pad_l = s.pad_l;
    ds.pad_r = s.pad_r;
    ds.out_pad = 0;
    ds.bn = false;
    ds.act = ACT_NONE;
    a.s = ds;
    a.gy = xin;
    a.gyb = xb;
    a.gyc = xc;
    a.gact = t->layers[l - 1].s.act;
    {
      Prof p("train.dgrad", st);
      launch_conv_f32(a, st);
    }
    g = dst;
    gb = xb;
    gn = xc;
    cur ^= 1;
  }
  {
    // every layer's chain rule from the folded to the raw parameters, one launch
    std::vector<UnfoldItem> u;
    for (int l = 0; l < nl; ++l)
      u.push_back({t->layers[l].f, t->dWf[l], t->layers[l].s.transposed ? 1 : 0, t->dbf[l]});
    Prof p("train.unfold", st);
    for (int i = 0; i < nl; i += kFoldMax) launch_unfold_many(u.data() + i, std::min(kFoldMax, nl - i), dparams, st);
  }
  GW_API_END
}

int gw_band_loss(gw_fir_t f, const float* strain, const float* y_hat, int B, int L, float* loss, float* r,
                 void* cuda_stream) {
  GW_API_BEGIN
  GW_CHECK_ARG(f && strain && y_hat && loss && r, "NULL argument");
  GW_CHECK_ARG(B >= 1 && L >= f->ntaps, "need B >= 1 and L >= ntaps");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t need = ((size_t)B * L + (size_t)B) * sizeof(float);
  if (need > f->ws_bytes) {
    GW_CUDA(cudaStreamSynchronize(st));
    if (f->ws) dev_free(f->ctx, f->ws, f->ws_bytes, nullptr);
    f->ws = nullptr;
    f->ws_bytes = 0;
    f->ws = dev_alloc(f->ctx, need, nullptr);
    f->ws_bytes = need;
  }
  float* e = (float*)f->ws;
  Prof p("band_loss", st);
  launch_band_loss(strain, y_hat, B, L, f->d_taps, f->ntaps, e, r, e + (size_t)B * L, loss, st);
  GW_API_END
}

int gw_band_loss_backward(gw_fir_t f, const float* r, int B, int L, const float* dloss, float* dy_hat,
                          void* cuda_stream) {
  GW_API_BEGIN
  GW_CHECK_ARG(f && r && dy_hat, "NULL argument");
  GW_CHECK_ARG(B >= 1 && L >= f->ntaps, "need B >= 1 and L >= ntaps");
  Prof p("band_loss_bwd", (cudaStream_t)cuda_stream);
  launch_band_loss_backward(r, B, L, f->d_taps, f->ntaps, dloss, dy_hat, (cudaStream_t)cuda_stream);
  GW_API_END
}

int gw_fir_backward(gw_fir_t f, const float* dy, int B, int C, int L_in, float* dx, void* cuda_stream) {
  GW_API_BEGIN
  GW_CHECK_ARG(f && dy && dx, "NULL argument");
  GW_CHECK_ARG(B >= 1 && C >= 1 && L_in >= f->ntaps, "need B, C >= 1 and L_in >= ntaps");
  const int K = f->ntaps, lout = L_in - K + 1;
  Prof p("fir_bwd", (cudaStream_t)cuda_stream);
  launch_fir_f32(dy, lout, dx, L_in, B * C, f->d_taps, K, L_in, (cudaStream_t)cuda_stream, -(K - 1), lout, 1, 1.f);
  GW_API_END
}

int gw_adam_step(float* params, const float* grads, float* m, float* v, int64_t n, int step, float lr, float beta1,
                 float beta2, float eps, void* cuda_stream) {
  GW_API_BEGIN
  GW_CHECK_ARG(params && grads && m && v, "NULL argument");
  GW_CHECK_ARG(n >= 1 && step >= 1, "need n >= 1 and step >= 1");
  GW_CHECK_ARG(beta1 >= 0 && beta1 < 1 && beta2 >= 0 && beta2 < 1 && eps > 0 && lr >= 0, "bad Adam hyper-parameters");
  Prof p("adam", (cudaStream_t)cuda_stream);
  launch_adam(params, grads, m, v, n, step, lr, beta1, beta2, eps, (cudaStream_t)cuda_stream);
  GW_API_END
}

int gw_adam_step_dev(float* params, const float* grads, float* m, float* v, int64_t n, int* step, float lr,
                     float beta1, float beta2, float eps, void* cuda_stream) {
  GW_API_BEGIN
  GW_CHECK_ARG(params && grads && m && v && step, "NULL argument");
  GW_CHECK_ARG(n >= 1, "need n >= 1");
  GW_CHECK_ARG(beta1 >= 0 && beta1 < 1 && beta2 >= 0 && beta2 < 1 && eps > 0 && lr >= 0, "bad Adam hyper-parameters");
  Prof p("adam", (cudaStream_t)cuda_stream);
  add_launches(1);  // the step counter's kernel
  launch_adam_dev(params, grads, m, v, n, step, lr, beta1, beta2, eps, (cudaStream_t)cuda_stream);
  GW_API_END
}

}  // extern "C"
