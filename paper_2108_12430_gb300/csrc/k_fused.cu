// Whole-network DeepClean forward on the tensor cores (BF16 operands, FP32
// accumulation): the eight layers of the DeepClean-shaped autoencoder (Sec. 1,
// "DeepClean") for one time tile of one window run inside one CTA, with every
// intermediate activation in shared memory.
//
// Work items.  A window of Lw samples is cut into tiles of T = 864 output
// samples; an item is (window b, tile t).  For the tile's outputs [t T,
// t T + T) the host-side rule of fused_tile_rows walks the layers backwards:
// the last layer needs its outputs there, every layer needs the inputs its
// needed outputs read (the receptive field grows by the taps of every layer),
// and each layer computes the one 128-row MMA tile that starts at the row
// holding its first needed output.  With T = 864 the needed rows of every
// layer fit one 128-row tile (checked on the host for every tile).
//
// Layers.  Each layer is the implicit GEMM of the per-layer kernel (k_tc.cu):
// an MMA row holds Q consecutive output positions, the K-steps are pairs of
// 16-byte "slices" (8 channels of one input phase plane at one row shift), so
// the A operand of a step is a descriptor into the layer's input buffer with
// no im2col.  A layer's input buffer holds G channel groups x P phase planes x
// `rows` 16-byte rows; the previous layer's epilogue writes its outputs
// straight into that layout (zero outside the layer's valid range: the next
// layer's padding), so no activation ever leaves the SM.  The first layer's
// input is copied by bulk copies from the blocked BF16 input (a stream's
// ring: every window is a view), the last layer writes the FP32 prediction.
//
// Scheduling.  One persistent CTA per SM keeps kSlots items in flight, one
// per slot, each with two TMEM accumulators (even and odd layers), an
// MMA-issuing thread and epilogue warps: while one slot's epilogue drains its
// accumulator of layer l, the other slots' MMAs keep the tensor pipe busy.
// An item's activations live in one buffer per slot, rewritten in place layer
// after layer (a layer's epilogue runs only once all of the layer's MMAs, the
// buffer's readers, have completed); the first layer's inputs, three times
// larger, have two buffers that the CTA's items use in turn.  A hidden
// layer's epilogue drains its 64 columns in two halves and signals after the
// first: the next layer's K-steps that read only that half's outputs come
// first in its step table and are issued then, the rest once the whole
// epilogue is stored; an item's first layer reads only the input buffer and
// does not wait for the previous item's last epilogue.  The CTA takes its
// items in rounds of kSlots, all with the same weights: a layer's B-operand
// image is streamed from global memory in chunks of whole K-steps through a
// kWStages-deep ring, each chunk released once every slot has read it.
//
// Warps: 0 stages the first-layer input of the next items (bulk copies, zero
// rows at the window edges), 1 streams the weight chunks, one warp per slot
// issues its MMAs from one thread, and kEpiW warps per slot (one per TMEM lane
// quarter) drain the accumulator (bias, tanh, BF16 rounding) into the slot's
// buffer.  Every wait is bounded (about 1 s); on timeout the kernel records an
// error bit and unwinds.
#include <cuda_fp16.h>

#include <algorithm>

#include "fused_tables.h"
#include "gw_internal.h"
#include "tc_ptx.h"

namespace gw {

namespace {

using namespace ptx;

constexpr int kLayers = 8;
constexpr int kTileT = 864;        // output samples per item
constexpr int kRowsM = 128;        // MMA rows per layer and item
constexpr int kWStages = 5;        // weight ring
constexpr int kWChunk = 12288;     // bytes per weight chunk (whole K-steps of one layer)
#ifndef GW_FUSED_SLOTS
#define GW_FUSED_SLOTS 4
#endif
constexpr int kSlots = GW_FUSED_SLOTS;  // items in flight per CTA
constexpr int kInBufs = 2;         // first-layer input buffers, used by the CTA's items in turn
constexpr int kEpiW = 4;           // epilogue warps per slot, one per TMEM lane quarter
// warps: 0 input producer, 1 weight producer, 2-3 MMA issue of slots 0-1,
// 4 .. 3 + kSlots kEpiW epilogue (kEpiW per slot, in slot order), then MMA
// issue of slots 2 .. kSlots - 1
constexpr int kWarpIn = 0, kWarpWeights = 1, kWarpEpi0 = 4, kWarpMmaHi = kWarpEpi0 + kSlots * kEpiW;
constexpr int kThreads = 32 * (kWarpMmaHi + kSlots - 2);
constexpr int kAccCols = 64;       // TMEM columns per accumulator
// two accumulators per slot, for even and odd layers: a layer's first MMAs
// may run while the previous layer's epilogue still reads its accumulator
constexpr int kTmemCols = 2 * kSlots * kAccCols <= 256 ? 256 : 512;
static_assert(kSlots >= 2 && 2 * kSlots * kAccCols <= 512, "slots");
__device__ __forceinline__ uint32_t acc_col(int s, int l) { return (uint32_t)((2 * s + (l & 1)) * kAccCols); }
static_assert(kWarpEpi0 % 4 == 0 && kEpiW == 4, "an epilogue warp's TMEM lane quarter is its warp index mod 4");
constexpr int kZeroRowsF = 256;
// Copies of the weight image in global memory: every CTA streams the same
// chunks at about the same time, and with one copy all of them would queue on
// the same L2 lines; CTA i reads copy i mod kWReps.
constexpr int kWReps = 16;
constexpr int kErrIn = 1, kErrW = 2, kErrAcc = 4, kErrAct = 8, kErrEmpty = 16, kErrDrain = 32;

// the layer tables (fused_tables.h) by index
template <int l> struct Lay;
template <> struct Lay<0> { using T = fz::L0; };
template <> struct Lay<1> { using T = fz::L1; };
template <> struct Lay<2> { using T = fz::L2; };
template <> struct Lay<3> { using T = fz::L3; };
template <> struct Lay<4> { using T = fz::L4; };
template <> struct Lay<5> { using T = fz::L5; };
template <> struct Lay<6> { using T = fz::L6; };
template <> struct Lay<7> { using T = fz::L7; };
// first bias of layer l in the bias table (each layer's biases padded to 8)
template <int l> struct BiasOff {
  static constexpr int v = BiasOff<l - 1>::v + (Lay<l - 1>::T::cout + 7) / 8 * 8;
};
template <> struct BiasOff<0> { static constexpr int v = 0; };
constexpr int kBiasCount = BiasOff<7>::v + 8;
// a layer's chunks all fit the ring at once (both items of a pair read them)
static_assert(fz::L0::n_chunks <= kWStages && fz::L1::n_chunks <= kWStages && fz::L2::n_chunks <= kWStages &&
                  fz::L3::n_chunks <= kWStages && fz::L4::n_chunks <= kWStages && fz::L5::n_chunks <= kWStages &&
                  fz::L6::n_chunks <= kWStages && fz::L7::n_chunks <= kWStages,
              "weight ring too small for a layer");
static_assert(fz::L0::n_steps + fz::L1::n_steps + fz::L2::n_steps + fz::L3::n_steps + fz::L4::n_steps +
                      fz::L5::n_steps + fz::L6::n_steps + fz::L7::n_steps <= 128,
              "step table");
static_assert(fz::L0::sps * fz::L0::step_bytes <= kWChunk && fz::L7::sps * fz::L7::step_bytes <= kWChunk,
              "weight chunk larger than a ring stage");
constexpr uint32_t idesc_for(int npad) {
  // D = F32, A = B = BF16, both K-major, N >> 3 at bit 17, M >> 4 at bit 24
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(npad >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __align__(128) uint4 g_zero_rows_f[kZeroRowsF];

struct FParams {
  uint32_t chunk_off[fz::kChunks];   // byte offset of each weight chunk in wimg
  uint32_t chunk_bytes[fz::kChunks];
  const char* wimg;                  // kWReps copies, wimg_stride bytes apart
  uint32_t wimg_stride;
  const float* bias;                 // kBiasCount floats
  int lout[kLayers];                 // output length of every layer for this window length
  // input: element (b, c, x) of window b at in + in_off0 + b in_b + (c / 8) in_g
  // + (x % P0) in_p + (x / P0 + b in_boff) 16 bytes
  const char* in;
  int64_t in_off0, in_b, in_boff, in_g, in_p;
  // optional per-window addresses of element (b, 0, 0), replacing in + in_off0
  // + b in_b + b in_boff 16 (the serving loop's windows in many streams' rings)
  const char* const* item_ptr;
  float* y;
  int64_t y_ld;
  // items run tile-major: item i is tile i / nb of window i % nb
  int Lw, T, tiles, nb, n_items;
  // early: the previous kernel (the stream's ring update) writes only the
  // newest samples, window positions x >= fresh_x0 - b fresh_dx of window b;
  // items whose input ends before them start without waiting for it
  int early, fresh_x0, fresh_dx;
  uint32_t in_bytes, act_bytes;
  int* err;
  // test of the bounded waits: CTA 0 never arms the input of its first item,
  // so its MMA thread's wait runs out and the launch unwinds with kErrIn
  int stall_test;
};

__host__ __device__ inline int floordiv_f(int a, int b) {
  const int q = a / b;
  return (q * b > a) ? q - 1 : q;
}

// The needed outputs [a, b) of layer l give its first computed row
// floor(a / Q) and the inputs they read, which are the needed outputs of
// layer l - 1 (see the file header).
template <int l>
__host__ __device__ inline void tile_rows_step(int& a, int& b, int* rm0, int* need_lo, int* need_hi) {
  using F = typename Lay<l>::T;
  rm0[l] = floordiv_f(a, F::Q);
  if (need_lo) {
    need_lo[l] = a;
    need_hi[l] = b;
  }
  int na, nb;
  if (!F::transposed) {
    // y[u] reads x[s u + k - p], k < K
    na = F::stride * a - F::pad;
    nb = F::stride * (b - 1) - F::pad + F::K;
  } else {
    // y[2 j + k - p] += x[j]: output v reads x[(v + p - k) / 2] for k < K
    na = floordiv_f(a + F::pad - (F::K - 1) + 1, 2);
    nb = floordiv_f(b - 1 + F::pad, 2) + 1;
  }
  a = na;
  b = nb;
}
__host__ __device__ inline void fused_tile_rows(int T, int Lw, int t, int* rm0, int* need_lo, int* need_hi) {
  int a = t * T, b = t * T + T < Lw ? t * T + T : Lw;
  tile_rows_step<7>(a, b, rm0, need_lo, need_hi);
  tile_rows_step<6>(a, b, rm0, need_lo, need_hi);
  tile_rows_step<5>(a, b, rm0, need_lo, need_hi);
  tile_rows_step<4>(a, b, rm0, need_lo, need_hi);
  tile_rows_step<3>(a, b, rm0, need_lo, need_hi);
  tile_rows_step<2>(a, b, rm0, need_lo, need_hi);
  tile_rows_step<1>(a, b, rm0, need_lo, need_hi);
  tile_rows_step<0>(a, b, rm0, need_lo, need_hi);
  if (need_lo) {
    need_lo[kLayers] = a;  // inputs of the first layer
    need_hi[kLayers] = b;
  }
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
// Shared-memory layout and barriers of the kernel.
struct Smem {
  uint32_t in0, act0, w;     // addresses: input buffers, activation buffers, weight ring
  uint32_t in_bytes, act_bytes;
  uint64_t* bars;
  volatile uint32_t* abort_flag;
  int* err;
  __device__ uint32_t bar(int i) const { return smem_u32(&bars[i]); }
  // the activation buffer of slot s (the input of layers 1-7, in their layouts)
  __device__ uint32_t act(int s) const { return act0 + (uint32_t)s * act_bytes; }
  // first-layer input buffer i
  __device__ uint32_t input(int i) const { return in0 + (uint32_t)i * in_bytes; }
};
// The input barriers: full per slot (a slot waits for its items' inputs in
// order, whichever buffer they are in; a barrier per buffer would let a slot
// wait for the buffer's next phase while its current one, another slot's
// item, is still pending, which a parity wait cannot tell apart), empty per
// buffer (only the producer waits on those, in order).
enum { kInFull = 0, kInEmpty = kInFull + kSlots, kWFull = kInEmpty + kInBufs, kWEmpty = kWFull + kWStages,
       kAccFull = kWEmpty + kWStages, kActReady = kAccFull + kSlots, kDrain = kActReady + kSlots,
       kActHalf = kDrain + kSlots, kNBars = kActHalf + kSlots };


// Descriptor words: low = start address >> 4 (14 bits) | LBO >> 4 << 16, high
// = SBO >> 4 (128 bytes) | the fixed 0b001 at bit 46.  Start addresses stay
// below 256 KB, so adding a buffer base to a step's low word never carries
// into the LBO field.
constexpr uint32_t kDescHi = (128u >> 4) | (1u << 14);

// MMAs of layer l for the item of round k in one slot, issued by the slot's
// own thread from the compile-time step table: the A operand of a step is a
// slice of the input buffer at a_addr, the B operand the step's rows of the
// weight chunk in the ring.  Every chunk is released by all slots' threads
// (its empty barrier counts kSlots arrivals), each committing after its last
// MMA on the chunk.  For l > 0 the first F::split steps read only what the
// first half of the previous layer's epilogue wrote (the caller waited for
// that half); before the rest, the whole epilogue (act_ready).
template <int l>
__device__ __forceinline__ bool issue_layer(const Smem& sm, uint32_t d, int k, uint32_t a_addr, int s, int& act_ph) {
  using F = typename Lay<l>::T;
  constexpr uint32_t b_lbo = (((uint32_t)F::npad * 16u) >> 4) << 16;
  constexpr uint32_t idesc = idesc_for(F::npad);
  constexpr uint32_t b_step = (uint32_t)F::step_bytes >> 4;
  const uint64_t hi = (uint64_t)kDescHi << 32;
  const uint32_t a_base = a_addr >> 4;
#pragma unroll
  for (int c = 0; c < F::n_chunks; ++c) {
    const int g = k * fz::kChunks + F::chunk0 + c, st = g % kWStages, use = g / kWStages;
    if (!mbar_spin(sm.bar(kWFull + st), (uint32_t)use & 1u, sm.abort_flag, sm.err, kErrW)) return false;
    tc_fence_after();
    const uint32_t b_base = ((sm.w + (uint32_t)st * kWChunk) >> 4) | b_lbo;
#pragma unroll
    for (int i = c * F::sps; i < (c + 1) * F::sps && i < F::n_steps; ++i) {
      if (l > 0 && i == F::split) {
        if (!mbar_spin(sm.bar(kActReady + s), (uint32_t)act_ph & 1u, sm.abort_flag, sm.err, kErrAct)) return false;
        ++act_ph;
        tc_fence_after();
      }
      mma_f16(d, hi | (a_base + F::apack(i)), hi | (b_base + (uint32_t)(i - c * F::sps) * b_step), idesc,
              i == 0 ? 0u : 1u);
    }
    mma_commit(sm.bar(kWEmpty + st));
  }
  if (l > 0 && F::split >= F::n_steps) {
    if (!mbar_spin(sm.bar(kActReady + s), (uint32_t)act_ph & 1u, sm.abort_flag, sm.err, kErrAct)) return false;
    ++act_ph;
  }
  return true;
}

// Layer l of the CTA's item j (round k) in slot s.
template <int l>
__device__ __forceinline__ bool mma_layer(const Smem& sm, uint32_t tmem, int k, int j, int s, int& act_ph,
                                          int& half_ph) {
  // the layer's input (or, for l > 0, the part its first F::split steps read)
  // is in place, and its accumulator (one of the slot's two, by the layer's
  // parity) was last read by the epilogue of layer l - 2, which ended before
  // the previous layer's epilogue began (for the first layer: the previous
  // item's layer 6, whose epilogue ended before that item's last layer took
  // its second part).  The first layer does not wait for the previous item's
  // last epilogue: its MMAs read only the input buffer, and its own epilogue,
  // which rewrites the slot's activation buffer, runs on the same warps after
  // that one and after all of this thread's earlier MMAs have completed.
  const int ib = j % kInBufs;
  if (l == 0 && !mbar_spin(sm.bar(kInFull + s), (uint32_t)k & 1u, sm.abort_flag, sm.err, kErrIn)) return false;
  if (l > 0) {
    if (!mbar_spin(sm.bar(kActHalf + s), (uint32_t)half_ph & 1u, sm.abort_flag, sm.err, kErrAct)) return false;
    ++half_ph;
  }
  tc_fence_after();
  if (!issue_layer<l>(sm, tmem + acc_col(s, l), k, l == 0 ? sm.input(ib) : sm.act(s), s, act_ph)) return false;
  mma_commit(sm.bar(kAccFull + s));
  if (l == 0) mma_commit(sm.bar(kInEmpty + ib));
  return true;
}

// Epilogue of one 32-column chunk of layer l (l < 7) for MMA row R (absolute):
// bias, tanh, bf16, written into the slot's buffer, in the next layer's
// layout, at its phase plane and row; positions outside the layer's output
// are the next layer's zero padding.
template <int l>
__device__ __forceinline__ void epi_hidden(const float (&v)[32], int half, int R, int rin0_next, uint32_t out_buf,
                                           int lout, const float* s_bias) {
  using F = typename Lay<l>::T;
  using N = typename Lay<l + 1>::T;
  // An MMA row of layer l holds Q consecutive outputs, and the next layer has
  // Q phase planes: the row's outputs land in one row of every plane.
  static_assert(F::Q == N::P, "output folding and next-layer phases differ");
  const int rn = R - rin0_next;  // that row of the next layer's buffer
  if ((unsigned)rn >= (unsigned)N::rows) return;
  const int u0 = R * F::Q;  // the row's first output position
  const bool all_in = u0 >= 0 && u0 + F::Q <= lout;
  const uint32_t row_addr = out_buf + ((uint32_t)rn << 4);
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const int n0 = half * 32 + h * 8;
    const int sg = n0 >> F::lgcoutp, o0 = n0 & (F::coutp - 1);
    const bool in_range = all_in || (u0 + sg >= 0 && u0 + sg < lout);
    const float4 b0 = *reinterpret_cast<const float4*>(s_bias + BiasOff<l>::v + o0);
    const float4 b1 = *reinterpret_cast<const float4*>(s_bias + BiasOff<l>::v + o0 + 4);
    uint32_t w0 = 0u, w1 = 0u, w2 = 0u, w3 = 0u;
    if (in_range) {
      w0 = pack_bf16x2(tanh_fast(v[h * 8 + 0] + b0.x), tanh_fast(v[h * 8 + 1] + b0.y));
      w1 = pack_bf16x2(tanh_fast(v[h * 8 + 2] + b0.z), tanh_fast(v[h * 8 + 3] + b0.w));
      w2 = pack_bf16x2(tanh_fast(v[h * 8 + 4] + b1.x), tanh_fast(v[h * 8 + 5] + b1.y));
      w3 = pack_bf16x2(tanh_fast(v[h * 8 + 6] + b1.z), tanh_fast(v[h * 8 + 7] + b1.w));
    }
    const uint32_t addr = row_addr + ((uint32_t)(((o0 >> 3) * N::P + sg) * N::rows) << 4);
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(w0), "r"(w1), "r"(w2), "r"(w3)
                 : "memory");
  }
}

struct EpiItem {
  int rm0[kLayers];
  int b, t;
};

// Named barrier 1 + s over the slot's epilogue warps with an AND-reduction:
// one warp polls the accumulator barrier, the others wait here, and all get
// the same verdict (so that they leave the loop together on an abort).
__device__ __forceinline__ bool epi_bar_and(int s, bool ok) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.and.pred q, %2, %3, p;\nselp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((uint32_t)ok), "r"(1 + s), "n"(32 * kEpiW)
      : "memory");
  return r != 0;
}

template <int l>
__device__ __forceinline__ bool epi_layer(const FParams& p, const Smem& sm, uint32_t tmem, int quarter, int lane,
                                          int s, bool poller, const EpiItem& e, int& acc_ph, const float* s_bias) {
  using F = typename Lay<l>::T;
  const int row = quarter * 32 + lane;  // MMA row = TMEM lane
  bool ok = true;
  if (poller) ok = mbar_spin(sm.bar(kAccFull + s), (uint32_t)acc_ph & 1u, sm.abort_flag, sm.err, kErrAcc);
  if (!epi_bar_and(s, ok)) return false;
  ++acc_ph;
  tc_fence_after();
  const int R = e.rm0[l] + row;
#pragma unroll
  for (int half = 0; half * 32 < F::npad; ++half) {
    float v[32];
    tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + acc_col(s, l) + (uint32_t)(half * 32), v);
    if constexpr (l + 1 < kLayers) {
      using N = typename Lay<l + 1>::T;
      const int rin0 = e.rm0[l + 1] + N::dmin;
      epi_hidden<l>(v, half, R, rin0, sm.act(s), p.lout[l], s_bias);
      if (half == 0) {
        // the next layer's first F::split steps read only what this half wrote
        static_assert(F::npad == 64, "a hidden layer's epilogue runs in two halves of 32 columns");
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(sm.bar(kActHalf + s));
      }
    } else {
      // output layer: one channel, Q positions per row -> FP32 prediction
      const int lo = e.t * p.T, hi2 = min(lo + p.T, p.Lw);
      float* y = p.y + (int64_t)e.b * p.y_ld;
      const float bias = s_bias[BiasOff<l>::v];
      const int u0 = R << F::lgQ;
#pragma unroll
      for (int sg = 0; sg < F::Q; ++sg) {
        const int u = u0 + sg;
        if (u >= lo && u < hi2) y[u] = v[sg] + bias;
      }
    }
  }
  tc_fence_before();
  if constexpr (l + 1 < kLayers) {
    fence_proxy_async_smem();  // the stores above feed the next layer's MMAs (async proxy)
    __syncwarp();
    if (lane == 0) mbar_arrive(sm.bar(kActReady + s));
  }
  return true;
}

__global__ void __launch_bounds__(kThreads, 1) deepclean_fused_kernel(const FParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t base = smem_u32(smem);
  // [IN 0][IN 1][ACT 0 .. ACT kSlots-1][W ring][barriers, flags, bias]
  Smem sm;
  sm.in0 = base;
  sm.in_bytes = p.in_bytes;
  sm.act_bytes = p.act_bytes;
  sm.act0 = base + kInBufs * p.in_bytes;
  sm.w = sm.act0 + kSlots * p.act_bytes;
  sm.bars = reinterpret_cast<uint64_t*>(smem + (sm.w - base) + kWStages * kWChunk);
  sm.abort_flag = reinterpret_cast<volatile uint32_t*>(sm.bars + kNBars);
  sm.err = p.err;
  uint32_t* tslot = (uint32_t*)(sm.abort_flag + 1);
  float* s_bias = reinterpret_cast<float*>(((uintptr_t)(tslot + 1) + 15) & ~(uintptr_t)15);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < kInBufs; ++i) mbar_init(sm.bar(kInEmpty + i), 1);
    for (int i = 0; i < kSlots; ++i) {
      mbar_init(sm.bar(kInFull + i), 1);
      mbar_init(sm.bar(kAccFull + i), 1);
      mbar_init(sm.bar(kActReady + i), kEpiW);
      mbar_init(sm.bar(kDrain + i), 1);
      mbar_init(sm.bar(kActHalf + i), kEpiW);
    }
    for (int i = 0; i < kWStages; ++i) {
      mbar_init(sm.bar(kWFull + i), 1);
      mbar_init(sm.bar(kWEmpty + i), kSlots);  // released by every slot
    }
    *sm.abort_flag = 0u;
    fence_barrier_init();
  }
  // Activation buffers start at zero: rows of a buffer that no layer writes
  // for an item are only read by MMA rows whose outputs are discarded, but a
  // non-finite value there would still poison them through the zero weights.
  {
    uint4* a = reinterpret_cast<uint4*>(smem + (sm.act0 - base));
    const int n16 = (int)(kSlots * p.act_bytes / 16);
    for (int i = tid; i < n16; i += kThreads) a[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  for (int i = tid; i < kBiasCount; i += kThreads) s_bias[i] = p.bias[i];

  fence_proxy_async_smem();
  if (warp == 2) tmem_alloc(smem_u32(tslot), kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  griddep_launch_dependents();

  const int G = gridDim.x;
  const int my_items = p.n_items > (int)blockIdx.x ? (p.n_items - (int)blockIdx.x + G - 1) / G : 0;
  const int n_rounds = (my_items + kSlots - 1) / kSlots;  // item j of the CTA: round j / kSlots, slot j % kSlots
  const int mma_slot = warp == 2 ? 0 : warp == 3 ? 1 : warp >= kWarpMmaHi ? 2 + (warp - kWarpMmaHi) : -1;

  if (warp == kWarpIn) {
    // ---------------- input producer: the first layer's buffer of each item ----------------
    using L0 = fz::L0;
    constexpr int planes = L0::G * L0::P;
    // the input is written by the previous kernel (ring update): wait for it
    // before the first item that reads what it writes
    bool waited = !p.early;
    if (waited) griddep_wait();
    // per slot: whether an input phase was armed, and the parity of the last one
    uint32_t armed_any = 0u, armed_par = 0u;
    for (int j = 0; j < my_items; ++j) {
      const int ib = j % kInBufs, use = j / kInBufs;
      if (use >= 1 && !mbar_wait(sm.bar(kInEmpty + ib), (uint32_t)(use - 1) & 1u, sm.abort_flag, p.err, kErrEmpty))
        break;
      if (p.stall_test && blockIdx.x == 0 && j == 0) continue;  // no arrival and no copy: nothing in flight
      const int item = (int)blockIdx.x + j * G;
      const int t = item / p.nb, b = item - t * p.nb;
      int rm0[kLayers];
      fused_tile_rows(p.T, p.Lw, t, rm0, nullptr, nullptr);
      const int rin0 = rm0[0] + L0::dmin;  // first input row of every plane
      if (!waited && min((rin0 + L0::rows) * L0::P, p.Lw) > p.fresh_x0 - b * p.fresh_dx) {
        griddep_wait();
        waited = true;
      }
      const char* src0 = p.item_ptr ? p.item_ptr[b] + (int64_t)rin0 * 16
                                    : p.in + p.in_off0 + (int64_t)b * p.in_b + ((int64_t)rin0 + (int64_t)b * p.in_boff) * 16;
      const int slot = j % kSlots;
      const uint32_t full = sm.bar(kInFull + slot), dst0 = sm.input(ib);
      if (lane == 0) mbar_expect_tx(full, (uint32_t)(planes * L0::rows) * 16u);
      armed_any |= 1u << slot;
      armed_par = (armed_par & ~(1u << slot)) | ((uint32_t)(j / kSlots) & 1u) << slot;
      __syncwarp();
      for (int plane = lane; plane < planes; plane += 32) {
        const int g = plane / L0::P, phi = plane - g * L0::P;
        const int plen = (p.Lw - phi + L0::P - 1) / L0::P;  // rows of this plane inside the window
        const int r0 = min(L0::rows, max(0, -rin0)), r1 = max(r0, min(L0::rows, plen - rin0));
        const uint32_t dst = dst0 + (uint32_t)(plane * L0::rows) * 16u;
        const char* src = src0 + (int64_t)g * p.in_g + (int64_t)phi * p.in_p;
        if (r0 > 0) bulk_g2s(dst, g_zero_rows_f, (uint32_t)r0 * 16u, full);
        if (r1 > r0) bulk_g2s(dst + (uint32_t)r0 * 16u, src + (int64_t)r0 * 16, (uint32_t)(r1 - r0) * 16u, full);
        if (L0::rows > r1) bulk_g2s(dst + (uint32_t)r1 * 16u, g_zero_rows_f, (uint32_t)(L0::rows - r1) * 16u, full);
      }
      __syncwarp();
      if (*sm.abort_flag) break;
    }
    // the copies of the last armed phase of each slot's barrier have landed
    if (lane == 0)
      for (int i = 0; i < kSlots; ++i)
        if (armed_any >> i & 1u) mbar_wait_landed(sm.bar(kInFull + i), armed_par >> i & 1u, p.err, kErrDrain);
    __syncwarp();
  } else if (warp == kWarpWeights) {
    // ---------------- weight producer: the layers' chunks, once per round ----------------
    if (lane == 0) {
      const char* wsrc = p.wimg + (size_t)(blockIdx.x % kWReps) * p.wimg_stride;
      int issued = 0;  // chunks whose copies were started
      for (int k = 0; k < n_rounds && !*sm.abort_flag; ++k) {
        for (int c = 0; c < fz::kChunks; ++c) {
          const int g = k * fz::kChunks + c, st = g % kWStages, use = g / kWStages;
          if (use >= 1 && !mbar_wait(sm.bar(kWEmpty + st), (uint32_t)(use - 1) & 1u, sm.abort_flag, p.err, kErrEmpty))
            break;
          mbar_expect_tx(sm.bar(kWFull + st), p.chunk_bytes[c]);
          bulk_g2s(sm.w + (uint32_t)st * kWChunk, wsrc + p.chunk_off[c], p.chunk_bytes[c], sm.bar(kWFull + st));
          issued = g + 1;
        }
      }
      // the last copy into every stage has landed
      for (int g = issued - kWStages; g < issued; ++g)
        if (g >= 0) mbar_wait_landed(sm.bar(kWFull + g % kWStages), (uint32_t)(g / kWStages) & 1u, p.err, kErrDrain);
    }
    __syncwarp();
  } else if (mma_slot >= 0) {
    // ---------------- MMA issue: one thread per slot ----------------
    const int s = mma_slot;
    if (lane == 0) {
      int act_ph = 0;   // act_ready phases consumed
      int half_ph = 0;  // act_half phases consumed
      for (int k = 0; k < n_rounds; ++k) {
        const int j = k * kSlots + s;
        if (j >= my_items) {
          // no item in this slot (the last round): release the round's weight
          // chunks in order, each once it has been loaded (so that the
          // arrival counts toward that chunk's phase)
          bool ok = true;
          for (int c = 0; c < fz::kChunks && ok; ++c) {
            const int g = k * fz::kChunks + c, st = g % kWStages, use = g / kWStages;
            ok = mbar_wait(sm.bar(kWFull + st), (uint32_t)use & 1u, sm.abort_flag, p.err, kErrW);
            if (ok) mbar_arrive(sm.bar(kWEmpty + st));
          }
          if (!ok) break;
          continue;
        }
        if (!mma_layer<0>(sm, tmem, k, j, s, act_ph, half_ph) || !mma_layer<1>(sm, tmem, k, j, s, act_ph, half_ph) ||
            !mma_layer<2>(sm, tmem, k, j, s, act_ph, half_ph) || !mma_layer<3>(sm, tmem, k, j, s, act_ph, half_ph) ||
            !mma_layer<4>(sm, tmem, k, j, s, act_ph, half_ph) || !mma_layer<5>(sm, tmem, k, j, s, act_ph, half_ph) ||
            !mma_layer<6>(sm, tmem, k, j, s, act_ph, half_ph) || !mma_layer<7>(sm, tmem, k, j, s, act_ph, half_ph))
          break;
      }
      // every MMA issued by this thread completes before TMEM is released
      mma_commit(sm.bar(kDrain + s));
      mbar_wait(sm.bar(kDrain + s), 0u, sm.abort_flag, p.err, kErrDrain);
    }
    __syncwarp();
  } else if (warp >= kWarpEpi0 && warp < kWarpMmaHi) {
    // ---------------- epilogue: kEpiW warps per slot ----------------
    const int s = (warp - kWarpEpi0) / kEpiW;      // slot this warp drains
    const int quarter = warp & 3;                  // TMEM lanes this warp may access
    const bool poller = quarter == 0;              // the slot's first epilogue warp polls the accumulator
    int acc_ph = 0;
    bool waited = false;
    for (int k = 0; k < n_rounds; ++k) {
      const int j = k * kSlots + s;
      if (j >= my_items) break;
      EpiItem e;
      const int item = (int)blockIdx.x + j * G;
      e.t = item / p.nb;
      e.b = item - e.t * p.nb;
      fused_tile_rows(p.T, p.Lw, e.t, e.rm0, nullptr, nullptr);
      if (!epi_layer<0>(p, sm, tmem, quarter, lane, s, poller, e, acc_ph, s_bias) ||
          !epi_layer<1>(p, sm, tmem, quarter, lane, s, poller, e, acc_ph, s_bias) ||
          !epi_layer<2>(p, sm, tmem, quarter, lane, s, poller, e, acc_ph, s_bias) ||
          !epi_layer<3>(p, sm, tmem, quarter, lane, s, poller, e, acc_ph, s_bias) ||
          !epi_layer<4>(p, sm, tmem, quarter, lane, s, poller, e, acc_ph, s_bias) ||
          !epi_layer<5>(p, sm, tmem, quarter, lane, s, poller, e, acc_ph, s_bias) ||
          !epi_layer<6>(p, sm, tmem, quarter, lane, s, poller, e, acc_ph, s_bias))
        break;
      if (!waited) {
        // the prediction buffer may still be read by the kernels before this one
        griddep_wait();
        waited = true;
      }
      if (!epi_layer<7>(p, sm, tmem, quarter, lane, s, poller, e, acc_ph, s_bias)) break;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

struct FusedPlan {
  FParams q{};
  size_t smem = 0;
  int lw_ok = -1;  // last window length checked
  bool lw_result = false;
};

namespace {

int lay_field(int l, int which) {
#define GW_FZ_CASE(i)                                                                                       \
  case i: {                                                                                                 \
    using F = Lay<i>::T;                                                                                    \
    const int v[] = {F::n_steps, F::npad, F::G, F::P, F::rows, F::dmin, F::Q, F::coutp, F::cout, F::cin,   \
                     F::transposed, F::stride, F::pad, F::K, F::step_bytes, F::sps, F::n_chunks, F::chunk0}; \
    return v[which];                                                                                        \
  }
  switch (l) {
    GW_FZ_CASE(0) GW_FZ_CASE(1) GW_FZ_CASE(2) GW_FZ_CASE(3) GW_FZ_CASE(4) GW_FZ_CASE(5) GW_FZ_CASE(6) GW_FZ_CASE(7)
  }
#undef GW_FZ_CASE
  return -1;
}
enum { fNSteps, fNpad, fG, fP, fRows, fDmin, fQ, fCoutp, fCout, fCin, fTr, fStride, fPad, fK, fStepBytes, fSps,
       fNChunks, fChunk0 };
uint32_t lay_apack(int l, int i) {
  switch (l) {
    case 0: return Lay<0>::T::apack(i);
    case 1: return Lay<1>::T::apack(i);
    case 2: return Lay<2>::T::apack(i);
    case 3: return Lay<3>::T::apack(i);
    case 4: return Lay<4>::T::apack(i);
    case 5: return Lay<5>::T::apack(i);
    case 6: return Lay<6>::T::apack(i);
    default: return Lay<7>::T::apack(i);
  }
}
int lay_order(int l, int i) {
  switch (l) {
    case 0: return Lay<0>::T::order(i);
    case 1: return Lay<1>::T::order(i);
    case 2: return Lay<2>::T::order(i);
    case 3: return Lay<3>::T::order(i);
    case 4: return Lay<4>::T::order(i);
    case 5: return Lay<5>::T::order(i);
    case 6: return Lay<6>::T::order(i);
    default: return Lay<7>::T::order(i);
  }
}

}  // namespace

// The compile-time tables describe DeepClean with 17-24 input channels; the
// plan is made only when the model's own lowering reproduces them exactly.
FusedPlan* fused_plan_create(gw_model* m, const std::vector<std::vector<double>>& wfold,
                             const std::vector<std::vector<float>>& bias) {
  if (m->kind != GW_MODEL_DEEPCLEAN || m->precision != GW_BF16 || m->layers.size() != (size_t)kLayers) return nullptr;
  if ((m->n_in + 7) / 8 != fz::L0::G) return nullptr;
  std::vector<uint8_t> all;
  std::vector<float> biases(kBiasCount, 0.f);
  FParams q{};
  uint32_t act_bytes = 0, in_bytes = 0;
  for (int l = 0; l < kLayers; ++l) {
    LayerDev Ld;
    Ld.s = m->layers[l].s;
    Ld.J = (l == 0 ? fz::L0::J : l == 1 ? fz::L1::J : l == 2 ? fz::L2::J : l == 3 ? fz::L3::J
            : l == 4 ? fz::L4::J : l == 5 ? fz::L5::J : l == 6 ? fz::L6::J : fz::L7::J);
    std::vector<uint8_t> img;
    std::vector<uint32_t> table;
    tc_lower_layer(Ld, wfold[l], img, table);
    const LayerSpec& s = Ld.s;
    const int rows = kRowsM + Ld.dspan;  // a plane's rows: the MMA rows and the layer's row shifts
    const bool same = lay_field(l, fNSteps) == Ld.n_steps && lay_field(l, fNpad) == Ld.npad &&
                      lay_field(l, fG) == Ld.gin && lay_field(l, fP) == Ld.pin && lay_field(l, fRows) == rows &&
                      lay_field(l, fDmin) == Ld.dmin && lay_field(l, fQ) == Ld.n_chains &&
                      lay_field(l, fCoutp) == Ld.coutp && lay_field(l, fCout) == s.cout &&
                      lay_field(l, fTr) == (s.transposed ? 1 : 0) && lay_field(l, fStride) == s.stride &&
                      lay_field(l, fPad) == s.pad_l && lay_field(l, fPad) == s.pad_r && lay_field(l, fK) == s.k &&
                      lay_field(l, fStepBytes) == 32 * Ld.npad &&
                      (l + 1 < kLayers ? s.act == ACT_TANH : s.act == ACT_NONE) &&
                      (!s.transposed || s.out_pad == 1);
    if (!same) return nullptr;
    // step i of the kernel is step order(i) of the host lowering (a permutation)
    std::vector<int> seen(Ld.n_steps, 0);
    for (int i = 0; i < Ld.n_steps; ++i) {
      const int h = lay_order(l, i);
      if (h < 0 || h >= Ld.n_steps || seen[h]++) return nullptr;
      const uint32_t o0 = tc_slice_offset(table[2 * h], Ld.pin, rows), o1 = tc_slice_offset(table[2 * h + 1], Ld.pin, rows);
      if (o1 < o0 || lay_apack(l, i) != ((o0 >> 4) | (((o1 - o0) >> 4) << 16))) return nullptr;
    }
    const uint32_t buf = (uint32_t)(Ld.gin * Ld.pin * rows * 16);
    if (l == 0)
      in_bytes = buf;
    else
      act_bytes = std::max(act_bytes, buf);
    const int sps = lay_field(l, fSps), step_bytes = lay_field(l, fStepBytes), c0 = lay_field(l, fChunk0);
    for (int c = 0; c < lay_field(l, fNChunks); ++c) {
      const int i0 = c * sps, i1 = std::min(Ld.n_steps, i0 + sps);
      q.chunk_off[c0 + c] = (uint32_t)all.size();
      q.chunk_bytes[c0 + c] = (uint32_t)((i1 - i0) * step_bytes);
      for (int i = i0; i < i1; ++i) {
        const size_t h = (size_t)lay_order(l, i);
        all.insert(all.end(), img.begin() + h * step_bytes, img.begin() + (h + 1) * step_bytes);
      }
    }
    const int b0 = (l == 0 ? BiasOff<0>::v : l == 1 ? BiasOff<1>::v : l == 2 ? BiasOff<2>::v : l == 3 ? BiasOff<3>::v
                    : l == 4 ? BiasOff<4>::v : l == 5 ? BiasOff<5>::v : l == 6 ? BiasOff<6>::v : BiasOff<7>::v);
    for (int o = 0; o < s.cout; ++o) biases[b0 + o] = bias[l][o];
  }
  FusedPlan* f = new FusedPlan();
  try {
    f->q = q;
    f->q.in_bytes = in_bytes;
    f->q.act_bytes = act_bytes;
    f->smem = 1024 + kInBufs * (size_t)in_bytes + kSlots * (size_t)act_bytes + (size_t)kWStages * kWChunk +
              8 * (size_t)kNBars + 32 + 4 * (size_t)kBiasCount;
    GW_CHECK_ARG(f->smem <= 227 * 1024, "fused plan: shared memory");
    const size_t stride = (all.size() + 127) / 128 * 128;
    all.resize(stride, 0);
    std::vector<uint8_t> reps(stride * kWReps);
    for (int r = 0; r < kWReps; ++r) std::copy(all.begin(), all.end(), reps.begin() + (size_t)r * stride);
    void* wimg = dev_alloc(m->ctx, reps.size(), &m->bytes);
    m->allocs.push_back(wimg);
    GW_CUDA(cudaMemcpy(wimg, reps.data(), reps.size(), cudaMemcpyHostToDevice));
    f->q.wimg_stride = (uint32_t)stride;
    float* bd = (float*)dev_alloc(m->ctx, biases.size() * sizeof(float), &m->bytes);
    m->allocs.push_back(bd);
    GW_CUDA(cudaMemcpy(bd, biases.data(), biases.size() * sizeof(float), cudaMemcpyHostToDevice));
    f->q.wimg = (const char*)wimg;
    f->q.bias = bd;
  } catch (...) {
    delete f;
    throw;
  }
  return f;
}

void fused_plan_destroy(FusedPlan* f) { delete f; }  // device buffers belong to the model's allocations

// Every tile's needed rows must fit one 128-row MMA tile per layer, the needed
// inputs of a layer must lie inside its input buffer, and the previous
// layer's computed rows must cover them.
static bool fused_check(int Lw, const int* lout) {
  if (lout[kLayers - 1] != Lw) return false;  // the network gives back the window length
  const int tiles = (Lw + kTileT - 1) / kTileT;
  for (int t = 0; t < tiles; ++t) {
    int rm0[kLayers], lo[kLayers + 1], hi[kLayers + 1];
    fused_tile_rows(kTileT, Lw, t, rm0, lo, hi);
    for (int l = 0; l < kLayers; ++l) {
      const int Q = lay_field(l, fQ), P = lay_field(l, fP), rows = lay_field(l, fRows), dmin = lay_field(l, fDmin);
      // needed outputs inside the computed rows
      if (floordiv_f(hi[l] - 1, Q) >= rm0[l] + kRowsM) return false;
      // needed inputs (the needed outputs of the layer before, or the
      // network input) inside the buffer rows
      const int ilo = l == 0 ? lo[kLayers] : lo[l - 1], ihi = l == 0 ? hi[kLayers] : hi[l - 1];
      const int rin0 = rm0[l] + dmin;
      if (floordiv_f(ilo, P) < rin0 || floordiv_f(ihi - 1, P) >= rin0 + rows) return false;
      // ... and computed by the previous layer
      if (l > 0) {
        const int Qp = lay_field(l - 1, fQ);
        if (ilo < Qp * rm0[l - 1] || ihi > Qp * (rm0[l - 1] + kRowsM)) return false;
      }
    }
  }
  return true;
}

static void layer_louts(gw_model* m, int L, int* lout) {
  int lin = L;
  for (int l = 0; l < kLayers; ++l) {
    lout[l] = m->layers[l].s.lout(lin);
    lin = lout[l];
  }
}

bool fused_supported(gw_model* m, int L) {
  FusedPlan* f = m->fused;
  if (!f || L < 8 || L % 8) return false;
  if (f->lw_ok != L) {
    int lout[kLayers];
    layer_louts(m, L, lout);
    f->lw_result = fused_check(L, lout);
    f->lw_ok = L;
  }
  return f->lw_result;
}

void launch_deepclean_fused(gw_model* m, const TcIn& in, int B, int L, float* y, int64_t y_ld, int* err,
                            cudaStream_t st, int fresh_x0, int fresh_dx) {
  FusedPlan* f = m->fused;
  GW_CHECK_ARG(f && fused_supported(m, L), "fused DeepClean does not support this window length");
  GW_CHECK_ARG(in.P == fz::L0::P, "fused DeepClean: unexpected input layout");
  FParams q = f->q;
  layer_louts(m, L, q.lout);
  q.in = (const char*)in.p;
  q.in_off0 = in.off0 * 2;
  q.in_b = in.bstride * 2;
  q.in_boff = in.boff;
  q.in_g = in.gstride * 2;
  q.in_p = in.pstride * 2;
  q.item_ptr = reinterpret_cast<const char* const*>(in.item_ptr);
  q.y = y;
  q.y_ld = y_ld;
  q.Lw = L;
  q.T = kTileT;
  q.tiles = (L + kTileT - 1) / kTileT;
  q.nb = B;
  q.n_items = q.tiles * B;
  q.early = fresh_x0 > 0 ? 1 : 0;
  q.fresh_x0 = fresh_x0;
  q.fresh_dx = fresh_dx;
  q.err = err;
  q.stall_test = tc_take_stall_test() ? 1 : 0;
  const int sms = current_sm_count();
  set_smem_limit_once(deepclean_fused_kernel, 227 * 1024);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(std::min(sms, q.n_items));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = f->smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  GW_CUDA(cudaLaunchKernelEx(&cfg, deepclean_fused_kernel, q));
}

}  // namespace gw
