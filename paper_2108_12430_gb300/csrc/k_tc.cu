// Tensor-core (tcgen05) implicit-GEMM convolution for sm_103a.
//
// Every Conv1d / ConvTranspose1d layer of the two networks runs here as
//   D[r][n] = sum_steps A_step[r][16 k] * B_step[n][16 k]
// with M = 128 "rows" r per MMA (one TMEM lane each), N output columns and
// K-steps of 16 BF16 (or 32 e4m3) inputs.
//
// Rows and columns.  A row r stands for Q consecutive output positions
// u = Q r + sigma (sigma < Q); column n = sigma * C' + o holds output channel o
// (C' = C_out rounded up to 8, or 1 for the single-channel prediction) of
// position sigma.  Q = J for a conv and Q = 2 J for a transposed conv: folding
// J output positions (and both phases of a stride-2 transposed conv) into N
// makes N >= 64 for the small channel counts of DeepClean instead of 8 or 16,
// which cuts the shared-memory operand traffic per useful MAC.
//
// K slices.  The layer's input is stored in P phase planes (P = stride x J for
// a conv, J for a transposed conv): input position x = P i + phi sits in plane
// phi, row i.  Output row r then reads, for every (tap, sigma), input row
// r + d of plane phi -- a fixed shift.  The distinct (phi, d) over all taps
// and sigma, times the channel groups of 8 (16 for e4m3), are the K "slices";
// two slices form a K-step.  Each slice is one 16-byte row per M row, so in
// the no-swizzle K-major core-matrix layout (16-byte rows, 8-row core
// matrices, SBO = 128 B) a slice is just a descriptor start address and the
// two slices of a step are LBO apart: the im2col matrix is never formed.
// B holds the folded weights arranged per (sigma, o) column and slice.
//
// Kernel.  Persistent and warp-specialised: warps 0 and 10 stage input tiles
// by bulk TMA into a ring of up to 6 stages (alternate tiles; zero rows for the
// padding at the edges), warp 1 issues the MMAs from one thread into a
// double-buffered TMEM accumulator, warps 2-9 drain TMEM with tcgen05.ld, add
// bias (and a residual), apply the activation and store the consumer's layout.
// Weights stay resident in shared memory when they fit, else stream per tile
// through a ring of stages (warp 0 then stages every input tile, and both
// producers fill the weight ring, each owning alternate stages).  The
// BatchNorm is folded into the weights on the host in FP64.  Every wait is
// bounded (1 s): on timeout the kernel records an error flag and unwinds.
#include <cuda_fp8.h>
#include <string.h>

#include <algorithm>
#include <set>

#include "gw_internal.h"
#include "tc_ptx.h"

namespace gw {

namespace {

using namespace ptx;

// warp 0 producer, warp 1 MMA, warps 2-9 epilogue: two epilogue warps per
// TMEM lane quarter (each takes every other 32-column chunk), so that every
// SM sub-partition has two warps to hide the epilogue's instruction latency.
// Warp 10 is a second producer: issuing a bulk copy blocks the issuing warp
// for about a memory round trip, so two warps taking alternate tiles keep
// twice the copies in flight.
constexpr int kEpiWarps = 8;
constexpr int kProdWarps = 2;
// CTAs per SM the planner may ask for (shared memory, TMEM columns and the
// register file permitting: 65536 / (kThreads * 96 registers))
constexpr int kMaxCtasPerSm = 2;
constexpr int kMaxA = 6;  // deepest input ring
constexpr int kMaxW = 8;  // deepest ring of streamed weight stages
constexpr int kTilesPerSm = 8;  // larger M tiles only while a layer keeps this many tiles per SM
constexpr int kWProd = 2;  // producer warps filling a streamed weight ring
// Bytes of a streamed weight stage: each stage costs its producer one issue
// round (wait, expect, copy) of about the same time whatever its size, so
// large layers get few large stages; the packed stages of split layers
// (small batches, few tiles) stay small.
constexpr int kWStage = 65536, kWStagePacked = 16384;
constexpr int kThreads = 32 * (kProdWarps + 1 + kEpiWarps);
constexpr int kErrWaitA = 1, kErrWaitW = 2, kErrWaitAcc = 4, kErrWaitEmpty = 8, kErrDrain = 16;
// Source of the zero padding rows of edge tiles (a stage plane holds at most
// kZeroRows rows; the planner checks it).
constexpr int kZeroRows = 2048;
__device__ __align__(128) uint4 g_zero_rows[kZeroRows];

struct TcParams {
  const char* in;
  int64_t in_off0, in_b, in_boff, in_g, in_p;  // bytes (boff in 16-byte rows)
  int in_P, in_L, G;
  int MT, rows, dmin, Q, coutp, mout, lout, tiles_per_item, n_tiles;
  const char* wimg;
  const uint32_t* table;
  int n_steps, npad, sps, nst, step_bytes, a_bytes, ncols, resident;
  int na;  // input stages in the A ring (2..kMaxA)
  // output-channel split: a tile is (M tile, column slice); each slice has
  // ncol = npad / nsplit columns (used when a layer has fewer tiles than SMs)
  int nsplit, ncol;
  // streamed weight stages: bytes per K-step in a stage (step_bytes, or with
  // wcompact = 1 only the slice's rows, packed [K-half][ncol rows] per step),
  // and the producer warps that fill them (1, or 2 with an even nst)
  int wstep, wcompact, wprod;
  uint32_t idesc;
  int fp8;
  const float* bias;
  const float* wscale;  // FP8: per output channel dequantisation scale
  int cout, act;
  char* out;
  int64_t out_b, out_g, out_p;  // bytes
  int out_P, fp32_single, fp8_out;
  float out_scale;
  const char* res;
  int64_t res_b, res_g, res_p;  // bytes
  int res_P, res_fp8;
  float res_scale;
  int* err;
  int coutp_log, out_P_log, res_P_log;  // power-of-two shifts for the epilogue addressing
  int min_plen;                          // rows of the shortest input plane
  int fp32_d2s;                          // write the 8 channels of position u as FP32 samples 8u..8u+7
  int fp32_full;                         // FP32 [B][C][L] output (out_g: bytes per channel)
  const float* gy;                       // with fp32_full: multiply by the derivative of an activation
  int64_t gy_b, gy_c;                    // whose output is gy (floats)
  int gact;
  char* blk;                             // with fp32_full: a blocked BF16 copy (bytes strides below)
  int64_t blk_b, blk_g, blk_p;
  int blk_P_log;
  const char* const* item_ptr;           // optional per-item input addresses (window start)
  int per_sm;                            // resident CTAs per SM the plan is sized for
  // Per K-step A operand, packed (start offset >> 4) | (LBO >> 4) << 16 relative
  // to the stage base, when n_steps <= kParamSteps (else 0 and the shared-memory
  // descriptor table is used).  Kernel parameters are uniform across the warp,
  // so the issue loop builds descriptors without per-MMA shared-memory reads.
  int param_desc;
  uint32_t apack[192];
  // test of the bounded waits: CTA 0 never arms the input stage of its first
  // tile, so its MMA thread's wait runs out and the launch unwinds with kErrWaitA
  int stall_test;
};
constexpr int kParamSteps = 192;

// Named barrier 1 over the epilogue warps with an AND-reduction of `ok`: every
// participating thread gets the same verdict, so the warps leave the tile loop
// together (a warp that left alone would strand the others in the barrier).
__device__ __forceinline__ bool epi_bar_and(bool ok) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.and.pred q, 1, %2, p;\nselp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((uint32_t)ok), "n"(32 * kEpiWarps)
      : "memory");
  return r != 0;
}
// Tile t -> (item b, first output row m0, column slice sl).  Within an item
// the M tiles are visited rotated by the item index, so that the item's edge
// tiles (first and last, which zero-fill padding rows on the slow path) fall
// on every CTA about equally often; with the plain order a persistent CTA
// whose stride is a multiple of half the tiles per item met an edge tile on
// every other step.
__device__ __forceinline__ void tile_coords(const TcParams& p, int t, int& b, int& m0, int& sl) {
  const int tm = t / p.nsplit;
  sl = t - tm * p.nsplit;
  b = tm / p.tiles_per_item;
  int j = tm - b * p.tiles_per_item + b % p.tiles_per_item;
  if (j >= p.tiles_per_item) j -= p.tiles_per_item;
  m0 = j * 128 * p.MT;
}
__device__ __forceinline__ float act_fn(float v, int act) {
  if (act == ACT_TANH) return tanh_fast(v);
  if (act == ACT_RELU) return fmaxf(v, 0.f);
  return v;
}

// Byte offset (M sub-tile 0) of the slice coded g | phi << 8 | dd << 14 in a
// tile of P planes per group, `rows` 16-byte rows per plane.
__host__ __device__ __forceinline__ uint32_t slice_off(uint32_t code, int P, int rows) {
  const uint32_t g = code & 255u, phi = (code >> 8) & 63u, dd = code >> 14;
  return ((g * (uint32_t)P + phi) * (uint32_t)rows + dd) * 16u;
}

// kFull: the FP32 [B][C][L] output mode of the training path is compiled only
// into its own instantiation, so the inference kernel's epilogue is unchanged.
template <bool kFull>
__global__ void __launch_bounds__(kThreads, kMaxCtasPerSm) conv_tc_kernel(const TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  const int na = p.na;                 // input stages (the A ring)
  const uint32_t sA = smem_u32(smem);  // na stages of a_bytes
  const uint32_t sW = sA + (uint32_t)na * (uint32_t)p.a_bytes;
  const uint32_t stage_bytes = (uint32_t)(p.sps * p.wstep);
  const uint32_t w_bytes = p.resident ? (uint32_t)(p.n_steps * p.step_bytes) : (uint32_t)p.nst * stage_bytes;
  const int planes = p.G * p.in_P;
  uint64_t* bars = (uint64_t*)(smem + (size_t)na * p.a_bytes + ((w_bytes + 127u) & ~127u));
  // barrier slots: a_full[na], a_empty[na], acc_full[2], acc_empty[2], drain, w_full[nst], w_empty[nst]
  // then, 16-byte aligned, [n_steps] {A descriptor (stage 0, sub-tile 0), B descriptor (stage 0)}
  uint64_t* s_desc = bars + ((2 * na + 5 + 2 * p.nst + 1) & ~1);
  int64_t* s_poff = reinterpret_cast<int64_t*>(s_desc + 2 * p.n_steps);  // [planes] byte offset of each plane
  volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(s_poff + planes);
  uint32_t* tslot = (uint32_t*)(abort_flag + 1);
  // [npad] bias, then [npad] FP8 scales; 16-byte aligned for vector loads
  float* s_bias = reinterpret_cast<float*>(((uintptr_t)(tslot + 2) + 15) & ~(uintptr_t)15);
  float* s_scale = s_bias + p.npad;
  int* s_plen = reinterpret_cast<int*>(s_scale + p.npad);  // [planes] valid rows of each plane
  auto bar = [&](int i) { return smem_u32(&bars[i]); };
  const int a_full = 0, a_empty = na, acc_full = 2 * na, acc_empty = 2 * na + 2, drain = 2 * na + 4,
            w_full = 2 * na + 5, w_empty = 2 * na + 5 + p.nst;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < na; ++i) {
      mbar_init(bar(a_full + i), 1);
      mbar_init(bar(a_empty + i), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(bar(acc_full + i), 1);
      mbar_init(bar(acc_empty + i), kEpiWarps);  // one arrival per epilogue warp
    }
    mbar_init(bar(drain), 1);
    for (int i = 0; i < p.nst; ++i) {
      mbar_init(bar(w_full + i), 1);
      mbar_init(bar(w_empty + i), 1);
    }
    *abort_flag = 0u;
    fence_barrier_init();
  }
  // per-CTA tables: MMA descriptors of every K-step (so the issue loop only
  // adds stage offsets), plane offsets and lengths, bias and scales
  const uint32_t stage_b = p.resident ? 0u : (uint32_t)p.sps;
  for (int i = tid; i < p.n_steps; i += kThreads) {
    const uint32_t o0 = slice_off(p.table[2 * i], p.in_P, p.rows), o1 = slice_off(p.table[2 * i + 1], p.in_P, p.rows);
    s_desc[2 * i] = make_desc(sA + o0, o1 - o0, 128u);
    const uint32_t pos = p.resident ? (uint32_t)i : (uint32_t)i % stage_b;
    s_desc[2 * i + 1] = make_desc(sW + pos * (uint32_t)p.wstep, (uint32_t)p.npad * 16u, 128u);
  }
  for (int i = tid; i < planes; i += kThreads) {
    const int g = i / p.in_P, phi = i % p.in_P;
    s_poff[i] = (int64_t)g * p.in_g + (int64_t)phi * p.in_p;
    s_plen[i] = (p.in_L - phi + p.in_P - 1) / p.in_P;
  }
  for (int i = tid; i < p.npad; i += kThreads) {
    s_bias[i] = i < p.cout ? p.bias[i] : 0.f;
    s_scale[i] = (p.wscale && i < p.cout) ? p.wscale[i] : 1.f;
  }
  if (warp == 1) tmem_alloc(smem_u32(tslot), (uint32_t)p.ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int n_chunks = p.resident ? 1 : (p.n_steps + p.sps - 1) / p.sps;
  // Programmatic dependent launch: the next kernel in the stream may start its
  // own set-up now; everything above (barriers, tables, TMEM) and the resident
  // weight load below touch only this launch's constant data and run while
  // the previous kernel finishes.  griddep_wait() blocks until the previous
  // kernel has completed and its writes are visible (a no-op for a launch
  // without the attribute).
  griddep_launch_dependents();

  if (warp == 0 || warp >= 2 + kEpiWarps) {
    // ---------------- producers: input tiles (and weights) by bulk TMA ----------------
    const int pw = warp == 0 ? 0 : warp - 1 - kEpiWarps;  // producer index
    // Resident weights: the producers take alternate tiles' inputs.  The input
    // ring is safe with two: each producer issues its tiles in order, and its
    // previous wait implies every older use of the stage was consumed, so no
    // producer gets more than one phase ahead.  Streamed weights: producer 0
    // loads every input tile, and the weight chunks alternate between the
    // p.wprod producers by chunk parity.  With an even number of stages every
    // weight stage then belongs to one producer, which re-arms it only after
    // its own wait for the previous use; taking alternate tiles instead, two
    // producers could re-arm a stage two phases ahead of its consumer, which a
    // parity wait cannot tell apart.
    const int nprod = p.resident ? kProdWarps : 1;
    if (p.resident && lane == 0 && pw == 0) {
      mbar_expect_tx(bar(w_full), (uint32_t)(p.n_steps * p.step_bytes));
      bulk_g2s(sW, p.wimg, (uint32_t)(p.n_steps * p.step_bytes), bar(w_full));
    }
    griddep_wait();
    int i = 0;
    int s = 0, k = 0;  // ring stage and its use count, advanced without divisions
    for (int t = blockIdx.x; t < p.n_tiles; t += gridDim.x, ++i, k += (++s == na), s = s == na ? 0 : s) {
      const bool do_a = i % nprod == pw, do_w = !p.resident && pw < p.wprod;
      if (!do_a && !do_w) continue;
      if (p.stall_test && blockIdx.x == 0 && i == 0) continue;  // no arrival and no copy: nothing in flight
      int b, m0, sl;
      tile_coords(p, t, b, m0, sl);
      if (do_a) {
        if (k >= 1 && !mbar_wait(bar(a_empty + s), (uint32_t)(k - 1) & 1u, abort_flag, p.err, kErrWaitEmpty)) break;
        const int base = m0 + p.dmin;
        const uint32_t sAs = sA + (uint32_t)s * (uint32_t)p.a_bytes;
        const char* src0 = p.item_ptr
                               ? p.item_ptr[b] + (int64_t)base * 16
                               : p.in + p.in_off0 + (int64_t)b * p.in_b + ((int64_t)base + (int64_t)b * p.in_boff) * 16;
        if (base >= 0 && base + p.rows <= p.min_plen) {
          // interior tile: every plane is one full run of rows
          if (lane == 0) mbar_expect_tx(bar(a_full + s), (uint32_t)(planes * p.rows) * 16u);
          __syncwarp();
          for (int plane = lane; plane < planes; plane += 32)
            bulk_g2s(sAs + (uint32_t)(plane * p.rows) * 16u, src0 + s_poff[plane], (uint32_t)p.rows * 16u,
                     bar(a_full + s));
        } else {
          // edge tile: rows outside a plane are the layer's zero padding; they
          // are copied from a zero buffer by the same bulk engine, so every row
          // of the stage arrives through the async proxy (no fence, no serial
          // zero stores) and the stage expects the same bytes as an interior one
          if (lane == 0) mbar_expect_tx(bar(a_full + s), (uint32_t)(planes * p.rows) * 16u);
          __syncwarp();
          for (int plane = lane; plane < planes; plane += 32) {
            const int r0 = min(p.rows, max(0, -base)), r1 = max(r0, min(p.rows, s_plen[plane] - base));
            const uint32_t dst = sAs + (uint32_t)(plane * p.rows) * 16u;
            if (r0 > 0) bulk_g2s(dst, g_zero_rows, (uint32_t)r0 * 16u, bar(a_full + s));
            if (r1 > r0)
              bulk_g2s(dst + (uint32_t)r0 * 16u, src0 + s_poff[plane] + (int64_t)r0 * 16, (uint32_t)(r1 - r0) * 16u,
                       bar(a_full + s));
            if (p.rows > r1) bulk_g2s(dst + (uint32_t)r1 * 16u, g_zero_rows, (uint32_t)(p.rows - r1) * 16u, bar(a_full + s));
          }
        }
      }
      if (lane == 0) {
        if (do_w) {
          for (int c = 0; c < n_chunks; ++c) {
            const int gc = i * n_chunks + c, st = gc % p.nst, use = gc / p.nst;
            if (gc % p.wprod != pw) continue;
            if (use >= 1 && !mbar_wait(bar(w_empty + st), (uint32_t)(use - 1) & 1u, abort_flag, p.err, kErrWaitEmpty))
              break;
            const int s0 = c * p.sps, s1 = min(p.n_steps, s0 + p.sps);
            if (p.nsplit == 1) {
              const uint32_t bytes = (uint32_t)((s1 - s0) * p.step_bytes);
              mbar_expect_tx(bar(w_full + st), bytes);
              bulk_g2s(sW + (uint32_t)st * stage_bytes, p.wimg + (int64_t)s0 * p.step_bytes, bytes, bar(w_full + st));
            } else {
              // only this slice's rows of both K-halves of every step, each
              // at its place in the full step layout, or packed (wcompact)
              const uint32_t rows_bytes = (uint32_t)p.ncol * 16u, half = (uint32_t)p.npad * 16u;
              const uint32_t off = (uint32_t)sl * rows_bytes;
              const uint32_t dhalf = p.wcompact ? rows_bytes : half, doff = p.wcompact ? 0u : off;
              mbar_expect_tx(bar(w_full + st), (uint32_t)(2 * (s1 - s0)) * rows_bytes);
              for (int sx = s0; sx < s1; ++sx)
                for (uint32_t hh = 0; hh < 2; ++hh) {
                  const uint32_t o = (uint32_t)(sx - s0) * (uint32_t)p.wstep + hh * dhalf + doff;
                  bulk_g2s(sW + (uint32_t)st * stage_bytes + o,
                           p.wimg + (int64_t)sx * p.step_bytes + hh * half + off, rows_bytes, bar(w_full + st));
                }
            }
          }
        }
      }
      __syncwarp();
      if (*abort_flag) break;
    }
  } else if (warp == 1) {
    // ---------------- MMA issue: one thread ----------------
    if (lane == 0) {
      bool ok = !p.resident || mbar_wait(bar(w_full), 0u, abort_flag, p.err, kErrWaitW);
      const bool fp8 = p.fp8 != 0;
      const int MT = p.MT, npad = p.ncol;  // accumulator columns of one tile (its slice)
      const uint32_t idesc = p.idesc;
      int i = 0;
      int sa = 0, ka = 0;  // input stage and its use count, advanced without divisions
      for (int t = blockIdx.x; ok && t < p.n_tiles; t += gridDim.x, ++i, ka += (++sa == na), sa = sa == na ? 0 : sa) {
        const int s = i & 1, k = i >> 1;     // accumulator buffer
        const int sl = t & (p.nsplit - 1);   // column slice (nsplit is a power of two)
        if (!mbar_wait(bar(a_full + sa), (uint32_t)ka & 1u, abort_flag, p.err, kErrWaitA)) break;
        if (k >= 1 && !mbar_wait(bar(acc_empty + s), (uint32_t)(k - 1) & 1u, abort_flag, p.err, kErrWaitAcc)) break;
        tc_fence_after();
        // descriptor start addresses count 16-byte units in their low bits
        const uint64_t a_stage = (uint64_t)(((uint32_t)sa * (uint32_t)p.a_bytes) >> 4);
        const uint32_t d0 = tmem + (uint32_t)(s * MT * npad);
        // the slice's B rows start sl * ncol rows into each K-half (at the
        // stage's start when the slice is packed)
        const uint64_t b_slice = p.wcompact ? 0ull : (uint64_t)(sl * p.ncol);
        for (int c = 0; c < n_chunks; ++c) {
          uint64_t b_stage = b_slice;
          int st = 0;
          if (!p.resident) {
            const int gc = i * n_chunks + c, use = gc / p.nst;
            st = gc - use * p.nst;
            if (!mbar_wait(bar(w_full + st), (uint32_t)use & 1u, abort_flag, p.err, kErrWaitW)) {
              ok = false;
              break;
            }
            tc_fence_after();
            b_stage = b_slice + (uint64_t)(((uint32_t)st * stage_bytes) >> 4);
          }
          const int s0 = p.resident ? 0 : c * p.sps, s1 = p.resident ? p.n_steps : min(p.n_steps, s0 + p.sps);
          // The issue rate of this one thread bounds the tensor pipe for small
          // N, so the loop is kept lean: one 16-byte descriptor pair per step,
          // the next pair loaded while the current MMAs issue.
          const ulonglong2* tab = reinterpret_cast<const ulonglong2*>(s_desc);
          if (MT == 1 && p.param_desc) {
            // descriptors from the parameter table: A start and LBO packed per
            // step, B at a fixed stride from the stage's first step
            const uint64_t hi = ((uint64_t)(128u >> 4) << 32) | (1ull << 46);
            const uint32_t a_base = (sA >> 4) + (uint32_t)a_stage;
            const uint32_t b_rows = p.wcompact ? (uint32_t)p.ncol : (uint32_t)p.npad;  // K-half distance
            const uint64_t b_hi = hi | ((uint64_t)((b_rows * 16u) >> 4) << 16);
            const uint32_t b_base = (sW >> 4) + (uint32_t)b_stage, b_step = (uint32_t)p.wstep >> 4;
            if (fp8) {
              for (int sidx = s0; sidx < s1; ++sidx) {
                const uint32_t e = p.apack[sidx];
                mma_f8(d0, hi | (uint64_t)((a_base + (e & 0xFFFFu)) & 0x3FFFu) | ((uint64_t)(e >> 16) << 16),
                       b_hi | (uint64_t)((b_base + (uint32_t)(sidx - s0) * b_step) & 0x3FFFu), idesc,
                       sidx == 0 ? 0u : 1u);
              }
            } else {
#pragma unroll 4
              for (int sidx = s0; sidx < s1; ++sidx) {
                const uint32_t e = p.apack[sidx];
                mma_f16(d0, hi | (uint64_t)((a_base + (e & 0xFFFFu)) & 0x3FFFu) | ((uint64_t)(e >> 16) << 16),
                        b_hi | (uint64_t)((b_base + (uint32_t)(sidx - s0) * b_step) & 0x3FFFu), idesc,
                        sidx == 0 ? 0u : 1u);
              }
            }
            if (!p.resident) mma_commit(bar(w_empty + st));
            continue;
          }
          ulonglong2 cur = tab[s0];
          if (fp8) {
            for (int sidx = s0; sidx < s1; ++sidx) {
              const ulonglong2 nxt = tab[sidx + 1 < s1 ? sidx + 1 : sidx];
              const uint32_t acc = sidx == 0 ? 0u : 1u;
              for (int mt = 0; mt < MT; ++mt)  // M sub-tile mt starts 128 rows (2048 bytes) further
                mma_f8(d0 + (uint32_t)(mt * npad), cur.x + a_stage + (uint64_t)(mt * 128), cur.y + b_stage, idesc,
                       acc);
              cur = nxt;
            }
          } else if (MT == 1) {
            // Under load (bulk copies landing, operand reads, epilogue
            // traffic) a shared-memory read takes longer than issuing several
            // MMAs, so the descriptor pairs are read four steps ahead.
            const int last = s1 - 1;
            ulonglong2 q1 = tab[min(s0 + 1, last)], q2 = tab[min(s0 + 2, last)], q3 = tab[min(s0 + 3, last)];
            int sidx = s0;
            for (; sidx + 4 <= s1; sidx += 4) {
              mma_f16(d0, cur.x + a_stage, cur.y + b_stage, idesc, sidx == 0 ? 0u : 1u);
              cur = tab[min(sidx + 4, last)];
              mma_f16(d0, q1.x + a_stage, q1.y + b_stage, idesc, 1u);
              q1 = tab[min(sidx + 5, last)];
              mma_f16(d0, q2.x + a_stage, q2.y + b_stage, idesc, 1u);
              q2 = tab[min(sidx + 6, last)];
              mma_f16(d0, q3.x + a_stage, q3.y + b_stage, idesc, 1u);
              q3 = tab[min(sidx + 7, last)];
            }
            // fewer than four steps left: they are in cur, q1, q2
            if (sidx < s1) mma_f16(d0, cur.x + a_stage, cur.y + b_stage, idesc, sidx == 0 ? 0u : 1u);
            if (sidx + 1 < s1) mma_f16(d0, q1.x + a_stage, q1.y + b_stage, idesc, 1u);
            if (sidx + 2 < s1) mma_f16(d0, q2.x + a_stage, q2.y + b_stage, idesc, 1u);
          } else {
            for (int sidx = s0; sidx < s1; ++sidx) {
              const ulonglong2 nxt = tab[sidx + 1 < s1 ? sidx + 1 : sidx];
              const uint32_t acc = sidx == 0 ? 0u : 1u;
              for (int mt = 0; mt < MT; ++mt)
                mma_f16(d0 + (uint32_t)(mt * npad), cur.x + a_stage + (uint64_t)(mt * 128), cur.y + b_stage, idesc,
                        acc);
              cur = nxt;
            }
          }
          if (!p.resident) mma_commit(bar(w_empty + st));
        }
        if (!ok) break;
        mma_commit(bar(a_empty + sa));
        mma_commit(bar(acc_full + s));
      }
      // all MMAs issued by this thread complete before TMEM is released
      mma_commit(bar(drain));
      mbar_wait(bar(drain), 0u, abort_flag, p.err, kErrDrain);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue (warps 2 .. 1 + kEpiWarps): TMEM -> bias/residual/activation -> global ----------------
    const int quarter = warp & 3;          // TMEM lanes this warp may access
    const int col_half = (warp - 2) >> 2;  // first 32-column chunk it drains (then every kEpiWarps / 4-th)
    const int row = quarter * 32 + lane;
    const bool plain = !kFull && !p.fp32_single && !p.fp32_d2s && !p.fp8_out && !p.res && !p.wscale;
    griddep_wait();  // outputs and residuals are shared with the previous kernels
    int i = 0;
    for (int t = blockIdx.x; t < p.n_tiles; t += gridDim.x, ++i) {
      const int s = i & 1, k = i >> 1;
      // One warp polls the accumulator barrier; the other seven sleep in the
      // named barrier instead of spinning on issue slots that the MMA thread,
      // the producer and the other CTA on the SM need.
      bool ok = true;
      if (warp == 2) ok = mbar_wait(bar(acc_full + s), (uint32_t)k & 1u, abort_flag, p.err, kErrWaitAcc);
      if (!epi_bar_and(ok)) break;
      tc_fence_after();
      int b, m0, sl;
      tile_coords(p, t, b, m0, sl);
      char* const outb = p.out + (int64_t)b * p.out_b;
      const char* const resb = p.res ? p.res + (int64_t)b * p.res_b : nullptr;
      const int out_mask = p.out_P - 1, res_mask = p.res_P - 1;
      for (int mt = 0; mt < p.MT; ++mt) {
        const int m = m0 + mt * 128 + row;
        const bool valid = m < p.mout;
        for (int j = col_half; j < p.ncol / 32; j += kEpiWarps / 4) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((s * p.MT + mt) * p.ncol + j * 32), v);
          if (!valid) continue;
          const int jg = sl * (p.ncol / 32) + j;  // chunk index among all npad columns
          if (plain) {
            // bf16 out, no residual, no FP8 scale: 4 groups of 8 channels,
            // straight-line, bias as float4 pairs, no per-group branches
            // (the common DeepClean / BBHnet case; invalid groups are those
            // past Q, C_out or the output length, known per column / row)
            const int n_base = jg * 32;
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const int n0 = n_base + h * 8;
              const int sg = n0 >> p.coutp_log, o0 = n0 & (p.coutp - 1);
              const int u = p.Q * m + sg;
              const float4 b0 = *reinterpret_cast<const float4*>(s_bias + o0);
              const float4 b1 = *reinterpret_cast<const float4*>(s_bias + o0 + 4);
              const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
              __align__(16) __nv_bfloat162 o16[4];
#pragma unroll
              for (int e = 0; e < 4; ++e)
                o16[e] = __floats2bfloat162_rn(act_fn(v[h * 8 + 2 * e] + bb[2 * e], p.act),
                                               act_fn(v[h * 8 + 2 * e + 1] + bb[2 * e + 1], p.act));
              if (sg < p.Q && o0 < p.cout && u < p.lout) {
                char* op = outb + (int64_t)(o0 >> 3) * p.out_g + (int64_t)(u & out_mask) * p.out_p +
                           (int64_t)(u >> p.out_P_log) * 16;
                *reinterpret_cast<uint4*>(op) = *reinterpret_cast<const uint4*>(o16);
              }
            }
            continue;
          }
          if (kFull) {
            // FP32 [B][C][L] (training): bias, activation, optionally times the
            // derivative of the activation whose output is gy
            const float* gyb = p.gy ? p.gy + (int64_t)b * p.gy_b : nullptr;
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              const int n = jg * 32 + e;
              const int sg = n >> p.coutp_log, o = n & (p.coutp - 1);
              const int u = p.Q * m + sg;
              if (sg >= p.Q || o >= p.cout || u >= p.lout) continue;
              float val = act_fn(v[e] + s_bias[o], p.act);
              if (gyb) {
                const float a = gyb[(int64_t)o * p.gy_c + u];
                val *= p.gact == ACT_TANH ? 1.f - a * a : (a > 0.f ? 1.f : 0.f);
              }
              reinterpret_cast<float*>(outb + (int64_t)o * p.out_g)[u] = val;
              if (p.blk)
                *reinterpret_cast<__nv_bfloat16*>(p.blk + (int64_t)b * p.blk_b + (int64_t)(o >> 3) * p.blk_g +
                                                  (int64_t)(u & ((1 << p.blk_P_log) - 1)) * p.blk_p +
                                                  (int64_t)(u >> p.blk_P_log) * 16 + (o & 7) * 2) =
                    __float2bfloat16_rn(val);
            }
            continue;
          }
          if (p.fp32_single) {
            // column n = sigma: output position Q m + sigma, channel 0
            float* y = reinterpret_cast<float*>(outb);
            const float bias = s_bias[0];
            const int u0 = p.Q * m + jg * 32;
            if (jg * 32 + 32 <= p.Q && u0 + 32 <= p.lout && ((uintptr_t)(y + u0) & 15) == 0) {
              // 32 consecutive samples of this row: eight 16-byte stores
              float4* y4 = reinterpret_cast<float4*>(y + u0);
#pragma unroll
              for (int e = 0; e < 8; ++e)
                y4[e] = make_float4(act_fn(v[4 * e] + bias, p.act), act_fn(v[4 * e + 1] + bias, p.act),
                                    act_fn(v[4 * e + 2] + bias, p.act), act_fn(v[4 * e + 3] + bias, p.act));
            } else {
#pragma unroll
              for (int e = 0; e < 32; ++e) {
                const int sg = jg * 32 + e;
                const int u = p.Q * m + sg;
                if (sg < p.Q && u < p.lout) y[u] = act_fn(v[e] + bias, p.act);
              }
            }
            continue;
          }
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const int n0 = jg * 32 + h * 8;
            const int sg = n0 >> p.coutp_log, o0 = n0 & (p.coutp - 1);
            const int u = p.Q * m + sg;
            if (sg >= p.Q || o0 >= p.cout || u >= p.lout) continue;
            float x[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int o = o0 + e;
              x[e] = o < p.cout ? fmaf(v[h * 8 + e], s_scale[o], s_bias[o]) : 0.f;
            }
            if (resb) {
              if (p.res_fp8) {
                const char* rp = resb + (int64_t)(o0 >> 4) * p.res_g + (int64_t)(u & res_mask) * p.res_p +
                                 (int64_t)(u >> p.res_P_log) * 16 + (o0 & 15);
                const uint2 rv = *reinterpret_cast<const uint2*>(rp);
                const __nv_fp8_e4m3* r8 = reinterpret_cast<const __nv_fp8_e4m3*>(&rv);
#pragma unroll
                for (int e = 0; e < 8; ++e) x[e] += float(r8[e]) * p.res_scale;
              } else {
                const char* rp = resb + (int64_t)(o0 >> 3) * p.res_g + (int64_t)(u & res_mask) * p.res_p +
                                 (int64_t)(u >> p.res_P_log) * 16;
                const uint4 rv = *reinterpret_cast<const uint4*>(rp);
                const __nv_bfloat16* r16 = reinterpret_cast<const __nv_bfloat16*>(&rv);
#pragma unroll
                for (int e = 0; e < 8; ++e) x[e] += __bfloat162float(r16[e]);
              }
            }
#pragma unroll
            for (int e = 0; e < 8; ++e) x[e] = act_fn(x[e], p.act);
            if (p.fp32_d2s) {
              // depth-to-space: channel o of position u is output sample 8 u + o
              float4* op = reinterpret_cast<float4*>(outb + (int64_t)u * 32);
              op[0] = make_float4(x[0], x[1], x[2], x[3]);
              op[1] = make_float4(x[4], x[5], x[6], x[7]);
            } else if (p.fp8_out) {
              __align__(8) __nv_fp8_e4m3 o8[8];
#pragma unroll
              for (int e = 0; e < 8; ++e) o8[e] = __nv_fp8_e4m3(x[e] * p.out_scale);
              char* op = outb + (int64_t)(o0 >> 4) * p.out_g + (int64_t)(u & out_mask) * p.out_p +
                         (int64_t)(u >> p.out_P_log) * 16 + (o0 & 15);
              *reinterpret_cast<uint2*>(op) = *reinterpret_cast<const uint2*>(o8);
            } else {
              __align__(16) __nv_bfloat16 o16[8];
#pragma unroll
              for (int e = 0; e < 8; ++e) o16[e] = __float2bfloat16_rn(x[e]);
              char* op = outb + (int64_t)(o0 >> 3) * p.out_g + (int64_t)(u & out_mask) * p.out_p +
                         (int64_t)(u >> p.out_P_log) * 16;
              *reinterpret_cast<uint4*>(op) = *reinterpret_cast<const uint4*>(o16);
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(acc_empty + s));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, (uint32_t)p.ncols);
}

// FP32 element (b, c, t) at x[b xb + c xc + t ts] -> blocked layout (bf16 rows
// of 8 channels, or e4m3 rows of 16).  ts = 8, xc = 1 turns one signal into 8
// "channels" of consecutive samples (space-to-depth).  Optionally the
// (standardised) FP32 values also go to y[b yb + c yc + t].
__global__ void to_blocked_kernel(const float* __restrict__ x, int64_t xb, int64_t xc, int64_t ts, int B, int C,
                                  int L, const float* __restrict__ mean, const float* __restrict__ istd, float scale,
                                  char* __restrict__ out, int64_t ob, int64_t og, int64_t op, int P, int fp8,
                                  float* __restrict__ y, int64_t yb, int64_t yc) {
  const int cg = fp8 ? 16 : 8;
  const int G = (C + cg - 1) / cg;
  const int64_t total = (int64_t)B * G * L;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(e % L);
    const int g = (int)((e / L) % G);
    const int b = (int)(e / ((int64_t)L * G));
    float v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int c = g * cg + i;
      float a = 0.f;
      if (i < cg && c < C) {
        a = x[(int64_t)b * xb + (int64_t)c * xc + (int64_t)t * ts];
        if (mean) a = (a - mean[c]) * istd[c];
        if (y) y[(int64_t)b * yb + (int64_t)c * yc + t] = a;
      }
      v[i] = a;
    }
    char* dst = out + (int64_t)b * ob + (int64_t)g * og + (int64_t)(t % P) * op + (int64_t)(t / P) * 16;
    if (fp8) {
      __align__(16) __nv_fp8_e4m3 o8[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) o8[i] = __nv_fp8_e4m3(v[i] * scale);
      *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(o8);
    } else {
      __align__(16) __nv_bfloat16 o16[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) o16[i] = __float2bfloat16_rn(v[i]);
      *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(o16);
    }
  }
}

// Global average pool of a blocked activation + linear head; one CTA per
// item.  A warp takes one phase plane of one channel group at a time (its
// lanes consecutive 16-byte rows, so that the loads coalesce), sums each
// channel over its rows in registers, reduces across the warp and adds the
// plane's sums to per-channel totals in shared memory; then every channel's
// mean is weighted and the products reduced.
constexpr int kGapMaxC = 1024;
__global__ void gap_linear_blocked_kernel(const char* __restrict__ in, int64_t ib, int64_t ig, int64_t ip, int P,
                                          int L, int C, int fp8, float in_scale, const float* __restrict__ w,
                                          const float* __restrict__ bias, float* __restrict__ out) {
  __shared__ float acc[kGapMaxC];
  __shared__ float red[32];
  const int b = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int cg = fp8 ? 16 : 8;
  const int G = (C + cg - 1) / cg, R = (L + P - 1) / P;
  for (int c = threadIdx.x; c < G * cg; c += blockDim.x) acc[c] = 0.f;
  __syncthreads();
  for (int plane = warp; plane < G * P; plane += nwarps) {
    const int g = plane / P, phase = plane - g * P;
    const char* base = in + (int64_t)b * ib + (int64_t)g * ig + (int64_t)phase * ip;
    float v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = 0.f;
    for (int r = lane; r < R && r * P + phase < L; r += 32) {
      const uint4 q = *reinterpret_cast<const uint4*>(base + (int64_t)r * 16);
      if (fp8) {
        const __nv_fp8_e4m3* e = reinterpret_cast<const __nv_fp8_e4m3*>(&q);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] += float(e[i]);
      } else {
        const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&q);
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] += __bfloat162float(e[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < 16; ++i)
      for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    if (lane == 0)
      for (int i = 0; i < cg; ++i) atomicAdd(&acc[g * cg + i], v[i]);
  }
  __syncthreads();
  float part = 0.f;
  for (int c = threadIdx.x; c < C; c += blockDim.x) part = fmaf(acc[c] * in_scale / (float)L, w[c], part);
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if (lane == 0) red[warp] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < nwarps; ++i) t += red[i];
    out[b] = t + bias[0];
  }
}

inline int pmod_i(int a, int m) { return ((a % m) + m) % m; }
inline int floordiv_i(int a, int b) { return (a - pmod_i(a, b)) / b; }


}  // namespace

int tc_supported() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3;
}

// Output positions folded into one M row (J): enough to make N reach 64
// columns for small channel counts, bounded so the tap halo stays small.
//
// Every tcgen05.mma with M = 128, K = 16 occupies the tensor pipe for the same
// time whatever its N (up to 256), so the number of (row tile, K-step) pairs
// sets the cost: folding more positions into N cuts the rows, at the price of
// more K-steps (the tap halo) and a larger input tile and weight image.
// Measured on GB300: an M=128, K=16 BF16 MMA costs about 100 cycles at N=64,
// 112 at N=128 and 143 at N=256 (the last at the dense peak), but layers
// folded to N=128 ran slower end to end than at N=64 (larger input tiles and
// weight images, fewer tiles per SM to pipeline).  Target N = 64 and halve J
// until two input stages plus the resident weights fit in shared memory.
static int choose_j(const LayerSpec& s) {
  const int coutp = s.cout == 1 ? 1 : (s.cout + 7) / 8 * 8;
  const int per_j = s.transposed ? 2 * coutp : coutp;
  int J = s.cout == 1 ? 16 : std::max(1, 64 / per_j);
  const int G = (s.cin + 7) / 8;
  for (; J > 1; J /= 2) {
    const int Q = s.transposed ? 2 * J : J, P = s.transposed ? J : s.stride * J;
    std::set<int> qs;
    for (int sg = 0; sg < Q; ++sg)
      for (int k = 0; k < s.k; ++k) {
        if (!s.transposed) {
          qs.insert(s.stride * sg + k - s.pad_l);
        } else if (pmod_i(sg % 2 + s.pad_l - k, 2) == 0) {
          qs.insert(sg / 2 + (sg % 2 + s.pad_l - k) / 2);
        }
      }
    const int dspan = floordiv_i(*qs.rbegin(), P) - floordiv_i(*qs.begin(), P);
    const size_t steps = ((size_t)qs.size() * G + 1) / 2;
    const size_t npad = std::max(32, (Q * coutp + 31) / 32 * 32);
    const size_t a_stage = (size_t)G * P * (128 + dspan) * 16;
    if (P <= 32 && npad <= 256 && 2 * a_stage + steps * 32 * npad <= 200 * 1024) break;
  }
  return J;
}

// Lowers one folded layer: K slices, K-steps and the packed B image (per step
// [2 K-halves][npad rows][16 bytes]: LBO = npad * 16 bytes, SBO = 128 bytes).
// map (optional, BF16 only): for every bf16 element of the image, the index
// (o C_in + c) K + k of the weight it holds, or -1; wf may then be empty.
static void lower_layer(LayerDev& L, const std::vector<double>& wf, bool fp8, std::vector<uint8_t>& img,
                        std::vector<uint32_t>& table, std::vector<float>& wscale,
                        std::vector<int32_t>* map = nullptr) {
  const LayerSpec& s = L.s;
  const int cg = fp8 ? 16 : 8;
  const int G = (s.cin + cg - 1) / cg;
  const int J = L.J > 0 ? L.J : choose_j(s);
  const int Q = s.transposed ? 2 * J : J;
  const int P = s.transposed ? J : s.stride * J;
  const int coutp = s.cout == 1 ? 1 : (s.cout + 7) / 8 * 8;
  // N padded to a multiple of 32 (the epilogue drains 32 columns per load)
  const int npad = std::max(32, (Q * coutp + 31) / 32 * 32);
  GW_CHECK_ARG(npad <= 256, "output columns above 256 are not supported by the tensor-core path");
  GW_CHECK_ARG(G <= 255 && P <= 63, "layer too wide for the tensor-core path");  // 8-bit group, 6-bit phase
  if (s.transposed)
    GW_CHECK_ARG(s.stride == 2 && s.pad_l == s.pad_r, "transposed conv must have stride 2 and symmetric padding");
  // contributions (sigma, tap) -> input (phi, d)
  struct Contrib { int sigma, k, phi, d; };
  std::vector<Contrib> cons;
  for (int sg = 0; sg < Q; ++sg)
    for (int k = 0; k < s.k; ++k) {
      int q;
      if (!s.transposed) {
        q = s.stride * sg + k - s.pad_l;
      } else {
        const int j = sg / 2, psi = sg % 2;
        if (pmod_i(psi + s.pad_l - k, 2) != 0) continue;
        q = j + (psi + s.pad_l - k) / 2;
      }
      cons.push_back({sg, k, pmod_i(q, P), floordiv_i(q, P)});
    }
  int dmin = 1 << 30, dmax = -(1 << 30);
  std::set<std::pair<int, int>> pos;
  for (auto& c : cons) {
    dmin = std::min(dmin, c.d);
    dmax = std::max(dmax, c.d);
    pos.insert({c.phi, c.d});
  }
  GW_CHECK_ARG(dmax - dmin < 2048, "tap span too large");
  struct Slice { int g, phi, dd; bool dummy; };
  auto key = [](const Slice& a) { return ((int64_t)a.g * 64 + a.phi) * 4096 + a.dd; };
  std::vector<std::pair<Slice, Slice>> steps;
  std::vector<Slice> left;
  for (auto& ps : pos) {
    int g = 0;
    for (; g + 1 < G; g += 2)
      steps.push_back({{g, ps.first, ps.second - dmin, false}, {g + 1, ps.first, ps.second - dmin, false}});
    if (g < G) left.push_back({g, ps.first, ps.second - dmin, false});
  }
  std::sort(left.begin(), left.end(), [&](const Slice& a, const Slice& b) { return key(a) < key(b); });
  for (size_t i = 0; i < left.size(); i += 2) {
    if (i + 1 < left.size()) {
      steps.push_back({left[i], left[i + 1]});
    } else {
      Slice d = left[i];
      d.dummy = true;
      steps.push_back({left[i], d});
    }
  }
  for (auto& st : steps)
    if (key(st.second) < key(st.first)) std::swap(st.first, st.second);
  GW_CHECK_ARG(steps.size() <= 4096, "too many K-steps");
  const int n_steps = (int)steps.size();
  const size_t step_bytes = 32 * (size_t)npad;
  img.assign(n_steps * step_bytes, 0);
  table.assign(2 * n_steps, 0u);
  GW_CHECK_ARG(!map || !fp8, "weight maps are for BF16 images");
  if (map) map->assign(img.size() / 2, -1);
  // FP8: per-output-channel weight scale so that max |w| maps to 448
  wscale.assign(s.cout, 1.f);
  if (fp8) {
    for (int o = 0; o < s.cout; ++o) {
      double mx = 0;
      for (size_t e = 0; e < (size_t)s.cin * s.k; ++e) mx = std::max(mx, std::fabs(wf[(size_t)o * s.cin * s.k + e]));
      wscale[o] = mx > 0 ? (float)(mx / 448.0) : 1.f;
    }
  }
  // weight of column (sigma, o), slice (g, phi, d), channel c: the tap k
  // that maps (sigma, k) to (phi, d), if any
  const size_t nd = (size_t)(dmax - dmin + 1);
  std::vector<int> tap_of((size_t)Q * P * nd, -1);
  for (auto& c : cons) tap_of[((size_t)c.sigma * P + c.phi) * nd + (c.d - dmin)] = c.k;
  for (int si = 0; si < n_steps; ++si) {
    for (int half = 0; half < 2; ++half) {
      const Slice& sl = half ? steps[si].second : steps[si].first;
      for (int n = 0; n < npad; ++n) {
        const int sg = n / coutp, o = n % coutp;
        if (sl.dummy || sg >= Q || o >= s.cout) continue;
        const int k = tap_of[((size_t)sg * P + sl.phi) * nd + sl.dd];
        if (k < 0) continue;
        uint8_t* dst = img.data() + si * step_bytes + ((size_t)half * npad + n) * 16;
        for (int kk = 0; kk < cg; ++kk) {
          const int c = sl.g * cg + kk;
          if (c >= s.cin) continue;
          const size_t wi = ((size_t)o * s.cin + c) * s.k + k;
          if (map) (*map)[((size_t)(dst - img.data()) >> 1) + kk] = (int32_t)wi;
          const double v = wf.empty() ? 0.0 : wf[wi];
          if (fp8) {
            __nv_fp8_e4m3 q((float)(v / wscale[o]));
            memcpy(dst + kk, &q, 1);
          } else {
            __nv_bfloat16 q = __float2bfloat16_rn((float)v);
            memcpy(dst + kk * 2, &q, 2);
          }
        }
      }
    }
    // one 32-bit code per slice: group (8 bits) | phase (6 bits) << 8 | row shift << 14
    auto code = [](const Slice& a) { return (uint32_t)a.g | ((uint32_t)a.phi << 8) | ((uint32_t)a.dd << 14); };
    table[2 * si] = code(steps[si].first);
    table[2 * si + 1] = code(steps[si].second);
  }
  L.n_steps = n_steps;
  L.npad = npad;
  L.gin = G;
  L.pin = P;
  L.n_chains = Q;      // output positions per M row
  L.dspan = dmax - dmin;
  L.dmin = dmin;
  L.J = J;
  L.coutp = coutp;
}

void tc_lower_layer(LayerDev& L, const std::vector<double>& wf, std::vector<uint8_t>& img,
                    std::vector<uint32_t>& table) {
  std::vector<float> wscale;
  lower_layer(L, wf, false, img, table, wscale);
  L.table_h = table;
}

uint32_t tc_slice_offset(uint32_t code, int P, int rows) { return slice_off(code, P, rows); }

namespace {
__global__ void tc_pack_kernel(const float* __restrict__ w, const int32_t* __restrict__ map, int64_t n,
                               __nv_bfloat16* __restrict__ img) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = map[e];
    img[e] = __float2bfloat16_rn(i >= 0 ? w[i] : 0.f);
  }
}
struct TcPackList {
  TcPackSeg s[kTcPackMax];
};
__global__ void tc_pack_many_kernel(const __grid_constant__ TcPackList l) {
  const TcPackSeg& g = l.s[blockIdx.y];
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  __nv_bfloat16* img = (__nv_bfloat16*)g.img;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < g.n; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = g.map[e];
    img[e] = i >= 0 ? __float2bfloat16_rn(g.w[i]) : zero;
  }
}
}  // namespace

void launch_tc_pack_many(const TcPackSeg* segs, int n_segs, cudaStream_t st) {
  GW_CHECK_ARG(n_segs >= 1 && n_segs <= kTcPackMax, "pack list size");
  TcPackList l{};
  int64_t mx = 0;
  for (int i = 0; i < n_segs; ++i) {
    l.s[i] = segs[i];
    mx = std::max(mx, segs[i].n);
  }
  tc_pack_many_kernel<<<dim3((unsigned)std::min<int64_t>((mx + 255) / 256, 512), n_segs), 256, 0, st>>>(l);
  GW_LAUNCH_CHECK();
}

void tc_prepare_trainable(LayerDev& L, gw_ctx* ctx, size_t* counter, std::vector<void*>& allocs,
                          const std::vector<int32_t>& src_of, const int32_t** d_map, int64_t* n_map) {
  std::vector<uint8_t> img;
  std::vector<uint32_t> table;
  std::vector<float> wscale;
  std::vector<int32_t> map;
  lower_layer(L, {}, false, img, table, wscale, &map);
  for (auto& m : map)
    if (m >= 0) {
      GW_CHECK_ARG((size_t)m < src_of.size(), "weight map out of range");
      m = src_of[m];
    }
  void* d_img = dev_alloc(ctx, img.size(), counter);
  allocs.push_back(d_img);
  GW_CUDA(cudaMemset(d_img, 0, img.size()));
  uint32_t* d_tab = (uint32_t*)dev_alloc(ctx, table.size() * 4, counter);
  allocs.push_back(d_tab);
  GW_CUDA(cudaMemcpy(d_tab, table.data(), table.size() * 4, cudaMemcpyHostToDevice));
  int32_t* dm = (int32_t*)dev_alloc(ctx, map.size() * 4, counter);
  allocs.push_back(dm);
  GW_CUDA(cudaMemcpy(dm, map.data(), map.size() * 4, cudaMemcpyHostToDevice));
  L.wq = d_img;
  L.table = d_tab;
  L.table_h = table;
  *d_map = dm;
  *n_map = (int64_t)map.size();
}

void launch_tc_pack(const float* w, const int32_t* map, int64_t n, void* img, cudaStream_t st) {
  tc_pack_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(w, map, n,
                                                                                  (__nv_bfloat16*)img);
  GW_LAUNCH_CHECK();
}

void tc_pack_layer(LayerDev& L, const std::vector<double>& wf, int precision, gw_ctx* ctx, size_t* counter,
                   std::vector<void*>& allocs, std::vector<float>* wscale_out) {
  const LayerSpec& s = L.s;
  const bool fp8 = precision == GW_FP8;
  std::vector<uint8_t> img;
  std::vector<uint32_t> table;
  std::vector<float> wscale;
  lower_layer(L, wf, fp8, img, table, wscale);
  void* d_img = dev_alloc(ctx, img.size(), counter);
  allocs.push_back(d_img);
  GW_CUDA(cudaMemcpy(d_img, img.data(), img.size(), cudaMemcpyHostToDevice));
  uint32_t* d_tab = (uint32_t*)dev_alloc(ctx, table.size() * 4, counter);
  allocs.push_back(d_tab);
  GW_CUDA(cudaMemcpy(d_tab, table.data(), table.size() * 4, cudaMemcpyHostToDevice));
  if (fp8) {
    // dequantisation per output channel: weight scale / scale of the input activations
    std::vector<float> deq(s.cout);
    for (int o = 0; o < s.cout; ++o) deq[o] = wscale[o] / L.act_scale;
    float* d_sc = (float*)dev_alloc(ctx, deq.size() * 4, counter);
    allocs.push_back(d_sc);
    GW_CUDA(cudaMemcpy(d_sc, deq.data(), deq.size() * 4, cudaMemcpyHostToDevice));
    L.wscale = d_sc;
    if (wscale_out) *wscale_out = wscale;
  }
  L.wq = d_img;
  L.table = d_tab;
  L.table_h = table;
}

// Host-side launch plan: tile size, weight residency or staging, TMEM columns,
// persistent grid, instruction descriptor.
static void plan_conv_tc(TcParams& q, const LayerDev& L, bool fp8, const TcIn& in, int lout, const TcOut& out,
                         int* err, size_t* smem_out, dim3* grid_out, int B, int sms) {
  const LayerSpec& s = L.s;
  const int esz = fp8 ? 1 : 2;
  GW_CHECK_ARG(in.P == L.pin, "input phase count does not match the layer");
  GW_CHECK_ARG(out.fp32_single == (s.cout == 1 ? 1 : 0), "single-channel layers write FP32 predictions");
  q = TcParams{};
  q.in = (const char*)in.p;
  q.in_off0 = in.off0 * esz;
  q.in_b = in.bstride * esz;
  q.in_boff = in.boff;
  q.item_ptr = reinterpret_cast<const char* const*>(in.item_ptr);
  q.in_g = in.gstride * esz;
  q.in_p = in.pstride * esz;
  q.in_P = in.P;
  q.in_L = in.L;
  q.G = L.gin;
  q.Q = L.n_chains;
  q.coutp = L.coutp;
  q.lout = lout;
  q.mout = (lout + q.Q - 1) / q.Q;
  q.dmin = L.dmin;
  q.step_bytes = 32 * L.npad;
  q.n_steps = L.n_steps;
  q.npad = L.npad;
  const size_t wbytes = (size_t)L.n_steps * q.step_bytes;
  // rows per stage plane rounded up to 8: every plane (and so every 8-row
  // core matrix of a slice with d = 0) starts on a 128-byte boundary
  auto rows_for = [&](int mt) { return (128 * mt + L.dspan + 7) / 8 * 8; };
  auto a_bytes_for = [&](int mt) { return (size_t)L.gin * L.pin * rows_for(mt) * 16; };
  const size_t budget = 220 * 1024;
  const size_t planes = (size_t)L.gin * L.pin;
  const size_t fixed = 128 + 8 * 32 + 16 + 16 * (size_t)L.n_steps + 12 * planes + 8 * (size_t)L.npad + 16;
  int MT = 4;
  const int tiles_needed = (q.mout + 127) / 128;
  // prefer small tiles while there are fewer than 8 tiles per SM: the
  // persistent pipeline overlaps tiles, and more tiles balance the SMs
  while (MT > 1 && (2 * MT * L.npad > 512 || MT > tiles_needed ||
                    (int64_t)((q.mout + 128 * MT - 1) / (128 * MT)) * B < (int64_t)kTilesPerSm * sms))
    MT /= 2;
  q.resident = 0;
  q.sps = 1;
  q.nst = 1;
  for (;; MT /= 2) {
    const size_t a2 = 2 * a_bytes_for(MT);
    if (a2 + wbytes + fixed <= budget) {
      q.resident = 1;
      q.sps = L.n_steps;
      q.nst = 1;
      break;
    }
    const int sps = std::max(1, (int)(kWStage / q.step_bytes));
    int nst = std::min(3, (L.n_steps + sps - 1) / sps);
    while (nst > 1 && a2 + (size_t)nst * sps * q.step_bytes + fixed > budget) --nst;
    if (a2 + (size_t)nst * sps * q.step_bytes + fixed <= budget) {
      q.sps = sps;
      q.nst = std::max(1, nst);
      break;
    }
    GW_CHECK_ARG(MT > 1, "shared memory plan too large");
  }
  q.MT = MT;
  q.rows = rows_for(MT);
  GW_CHECK_ARG(q.rows <= kZeroRows, "input tile taller than the zero-row buffer");
  q.a_bytes = (int)a_bytes_for(MT);
  q.tiles_per_item = (q.mout + 128 * MT - 1) / (128 * MT);
  // output-channel split while a layer has fewer tiles than SMs (small batches
  // of the deep BBHnet layers): slices of >= 32 columns, each CTA streaming
  // only its slice of the weights
  q.nsplit = 1;
  {
    const int64_t tiles_m = (int64_t)q.tiles_per_item * B;
    while (q.nsplit < 8 && L.npad / (2 * q.nsplit) >= 32 && (L.npad / (2 * q.nsplit)) % 32 == 0 &&
           tiles_m * 2 * q.nsplit <= sms)
      q.nsplit *= 2;
  }
  q.ncol = L.npad / q.nsplit;
  // streamed weights of a split layer: stages hold only the slice's rows,
  // packed, so that a 16 KB stage carries nsplit times as many K-steps (the
  // packed layout is addressed by the parameter-table MMA path only)
  q.wstep = q.step_bytes;
  q.wcompact = 0;
  if (q.nsplit > 1 && !q.resident && MT == 1 && L.n_steps <= kParamSteps && (int)L.table_h.size() >= 2 * L.n_steps) {
    q.wcompact = 1;
    q.wstep = q.step_bytes / q.nsplit;
    q.sps = std::min(L.n_steps, std::max(1, kWStagePacked / q.wstep));
    q.nst = 1;
  }
  int ncols = 32;
  while (ncols < 2 * MT * q.ncol) ncols *= 2;
  GW_CHECK_ARG(ncols <= 512, "accumulators exceed tensor memory");
  q.ncols = ncols;
  // input stages: as many as fit (up to kMaxA), keeping two CTAs per SM where
  // the two-stage plan allowed it; more tiles in flight hide the input latency
  {
    auto smem_for = [&](int na, int nst) {
      const size_t wsm0 = q.resident ? wbytes : (size_t)nst * q.sps * q.wstep;
      return 128 + (size_t)na * q.a_bytes + (wsm0 + 127) / 128 * 128 + 8 * (size_t)(2 * na + 6 + 2 * nst) +
             16 * (size_t)L.n_steps + 12 * planes + 32 + 8 * (size_t)L.npad + 16;
    };
    // shared memory per SM is 228 KB, of which 1 KB per CTA is reserved
    int per = kMaxCtasPerSm;
    while (per > 1 && (smem_for(2, q.nst) > (size_t)(228 / per - 1) * 1024 || ncols * per > 512)) --per;
    const size_t cap = (size_t)(228 / per - 1) * 1024;
    // streamed weights first get a deeper ring (every tile streams the whole
    // weight image, several times the bytes of its input tile), then the
    // input ring takes what is left
    q.wprod = 1;
    int na_min = 2;
    if (!q.resident) {
      const int chunks = (L.n_steps + q.sps - 1) / q.sps;
      while (q.nst < kMaxW && q.nst < chunks && smem_for(2, q.nst + 1) <= cap) ++q.nst;
      // a second weight stage before a second input stage: the weights are
      // the larger stream, and the loads of one stage then overlap the MMAs
      // of the other
      if (q.nst < 2 && chunks >= 2 && smem_for(1, 2) <= cap) {
        q.nst = 2;
        na_min = 1;
      }
      // two weight producers need an even ring (each owns every other stage)
      if (kWProd == 2 && q.nst >= 2) {
        q.nst &= ~1;
        q.wprod = 2;
      }
    }
    int na = na_min;
    while (na < kMaxA && smem_for(na + 1, q.nst) <= cap) ++na;
    q.na = na;
    q.per_sm = per;
  }
  q.n_tiles = q.tiles_per_item * B * q.nsplit;
  // instruction descriptor: D = F32, A/B = BF16 (kind::f16) or E4M3 (kind::f8f6f4),
  // both K-major, N >> 3 at bit 17, M >> 4 at bit 24 (N = the slice's columns)
  q.idesc = (1u << 4) | (fp8 ? 0u : ((1u << 7) | (1u << 10))) | ((uint32_t)(q.ncol >> 3) << 17) |
            ((uint32_t)(128 >> 4) << 24);
  q.fp8 = fp8;
  q.bias = L.b;
  q.wscale = L.wscale;
  q.cout = s.cout;
  q.act = s.act;
  q.out = (char*)out.p;
  GW_CHECK_ARG(!out.fp32_d2s || s.cout == 8, "depth-to-space output needs 8 channels");
  q.fp32_d2s = out.fp32_d2s;
  GW_CHECK_ARG(!out.fp32_full || (!fp8 && !out.res && !out.fp32_d2s && !out.fp32_single && s.cout > 1),
               "FP32 [B][C][L] output: BF16 layer, no residual");
  q.fp32_full = out.fp32_full;
  q.gy = out.gy;
  q.gy_b = out.gy_b;
  q.gy_c = out.gy_c;
  q.gact = out.gact;
  q.blk = (char*)out.blk;
  q.blk_b = out.blk_b * 2;
  q.blk_g = out.blk_g * 2;
  q.blk_p = out.blk_p * 2;
  {
    int lg = 0;
    while ((1 << lg) < std::max(1, out.blk_P)) ++lg;
    GW_CHECK_ARG(!out.blk || (1 << lg) == out.blk_P, "blocked copy: phase count must be a power of two");
    q.blk_P_log = lg;
  }
  const int oesz = (out.fp32_single || out.fp32_d2s || out.fp32_full) ? 4 : (out.fp8_out ? 1 : 2);
  q.out_b = out.bstride * oesz;
  q.out_g = out.gstride * oesz;
  q.out_p = out.pstride * oesz;
  q.out_P = out.P;
  q.fp32_single = out.fp32_single;
  q.fp8_out = out.fp8_out;
  q.out_scale = L.out_scale;
  q.res = (const char*)out.res;
  const int resz = fp8 ? 1 : 2;
  q.res_b = out.rbstride * resz;
  q.res_g = out.rgstride * resz;
  q.res_p = out.rpstride * resz;
  q.res_P = out.rP ? out.rP : 1;
  q.res_fp8 = fp8 ? 1 : 0;
  q.res_scale = fp8 ? 1.0f / L.out_scale : 1.0f;
  q.err = err;
  auto log2_exact = [](int v, const char* what) {
    int l = 0;
    while ((1 << l) < v) ++l;
    GW_CHECK_ARG((1 << l) == v, std::string(what) + " must be a power of two");
    return l;
  };
  q.coutp_log = log2_exact(q.coutp, "channels per output position");
  q.out_P_log = log2_exact(std::max(1, out.P), "output phase count");
  q.res_P_log = log2_exact(q.res_P, "residual phase count");
  q.min_plen = in.L / in.P;
  q.param_desc = 0;
  if (L.n_steps <= kParamSteps && (int)L.table_h.size() >= 2 * L.n_steps) {
    q.param_desc = 1;
    for (int i = 0; i < L.n_steps; ++i) {
      const uint32_t o0 = slice_off(L.table_h[2 * i], q.in_P, q.rows), o1 = slice_off(L.table_h[2 * i + 1], q.in_P, q.rows);
      q.apack[i] = (o0 >> 4) | (((o1 - o0) >> 4) << 16);
    }
  }
  GW_CHECK_ARG(!q.wcompact || (q.param_desc && q.MT == 1), "packed weight stages need the parameter-table MMA path");
  q.wimg = (const char*)L.wq;
  q.table = L.table;
  const size_t wsm = q.resident ? wbytes : (size_t)q.nst * q.sps * q.wstep;
  const size_t smem = 128 + (size_t)q.na * q.a_bytes + (wsm + 127) / 128 * 128 + 8 * (size_t)(2 * q.na + 6 + 2 * q.nst) +
                      16 * (size_t)L.n_steps + 12 * planes + 32 + 8 * (size_t)L.npad + 16;
  GW_CHECK_ARG(smem <= 227 * 1024, "shared memory plan too large");
  *smem_out = smem;
  *grid_out = dim3(std::min(q.n_tiles, sms * q.per_sm));
}

// Armed by the failure-path test on its own thread and taken by that
// thread's next tensor-core launch (the per-layer or the fused kernel).
static thread_local bool g_stall_next = false;
void conv_tc_arm_stall_test() { g_stall_next = true; }
bool tc_take_stall_test() {
  const bool s = g_stall_next;
  g_stall_next = false;
  return s;
}

void launch_conv_tc(const LayerDev& L, const TcIn& in, int lout, const TcOut& out, int B, int* err, cudaStream_t st) {
  TcParams q;
  size_t smem = 0;
  dim3 grid;
  plan_conv_tc(q, L, L.wscale != nullptr, in, lout, out, err, &smem, &grid, B, current_sm_count());
  q.stall_test = tc_take_stall_test() ? 1 : 0;
  set_smem_limit_once(conv_tc_kernel<false>, 227 * 1024);
  set_smem_limit_once(conv_tc_kernel<true>, 227 * 1024);
  // programmatic stream serialisation: this launch may begin (set-up, weight
  // loads) while the previous kernel in the stream runs; the kernel waits on
  // griddepcontrol before touching the previous kernels' data
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (q.fp32_full)
    GW_CUDA(cudaLaunchKernelEx(&cfg, conv_tc_kernel<true>, q));
  else
    GW_CUDA(cudaLaunchKernelEx(&cfg, conv_tc_kernel<false>, q));
}

void launch_to_blocked(const float* x, int64_t xb, int64_t xc, int B, int C, int L, const float* mean,
                       const float* istd, float scale, const TcOut& out, int fp8, cudaStream_t st, int64_t ts,
                       float* y, int64_t yb, int64_t yc) {
  const int esz = fp8 ? 1 : 2;
  const int cg = fp8 ? 16 : 8;
  const int64_t total = (int64_t)B * ((C + cg - 1) / cg) * L;
  const int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 32);
  to_blocked_kernel<<<grid, 256, 0, st>>>(x, xb, xc, ts, B, C, L, mean, istd, scale, (char*)out.p, out.bstride * esz,
                                          out.gstride * esz, out.pstride * esz, out.P, fp8, y, yb, yc);
  GW_LAUNCH_CHECK();
}

void launch_gap_linear_blocked(const TcIn& in, int C, int fp8, float in_scale, const float* w, const float* b,
                               float* out, int B, cudaStream_t st) {
  const int esz = fp8 ? 1 : 2;
  GW_CHECK_ARG((C + 15) / 16 * 16 <= kGapMaxC, "too many channels for the pooling head");
  gap_linear_blocked_kernel<<<B, 256, 0, st>>>((const char*)in.p + in.off0 * esz, in.bstride * esz, in.gstride * esz,
                                               in.pstride * esz, in.P, in.L, C, fp8, in_scale, w, b, out);
  GW_LAUNCH_CHECK();
}

}  // namespace gw

// Host-only inspection of the lowering and launch plan of one layer (no GPU).
extern "C" int gw_tc_inspect(const int* spec, int precision, const double* wfold, int lin, int in_P, int out_P, int batch,
                             void* img_out, size_t img_cap, uint32_t* table_out, int table_cap, int* meta_out) {
  using namespace gw;
  try {
    GW_CHECK_ARG(spec && wfold && img_out && table_out && meta_out, "NULL argument");
    GW_CHECK_ARG(precision == GW_BF16 || precision == GW_FP8, "precision must be BF16 or FP8");
    LayerDev L;
    L.s = LayerSpec{spec[0] != 0, spec[1], spec[2], spec[3], spec[4], spec[5], spec[6], spec[7], true, ACT_NONE};
    const LayerSpec& s = L.s;
    GW_CHECK_ARG(s.cin >= 1 && s.cout >= 1 && s.k >= 1 && s.stride >= 1 && lin >= 1, "bad layer spec");
    std::vector<double> wf(wfold, wfold + (size_t)s.cout * s.cin * s.k);
    std::vector<uint8_t> img;
    std::vector<uint32_t> table;
    std::vector<float> wscale;
    const bool fp8 = precision == GW_FP8;
    lower_layer(L, wf, fp8, img, table, wscale);
    L.table_h = table;  // as on the device path: the plan may use the parameter-table MMA path
    GW_CHECK_ARG(img.size() <= img_cap && (int)table.size() <= table_cap, "output buffers too small");
    memcpy(img_out, img.data(), img.size());
    memcpy(table_out, table.data(), table.size() * 4);
    const int lout = s.lout(lin);
    TcIn in{};
    in.P = in_P > 0 ? in_P : L.pin;
    in.L = lin;
    TcOut out{};
    out.P = out_P;
    out.fp32_single = s.cout == 1 ? 1 : 0;
    TcParams q;
    size_t smem = 0;
    dim3 grid;
    plan_conv_tc(q, L, fp8, in, lout, out, nullptr, &smem, &grid, batch > 0 ? batch : 1, 152);
    const int meta[26] = {L.n_steps, L.npad,   L.gin,   L.pin,        L.n_chains,   L.dspan, L.dmin,
                          q.MT,      q.rows,   q.a_bytes, q.resident ? L.n_steps : q.sps, q.nst, q.step_bytes,
                          q.ncols,   q.tiles_per_item, q.mout, L.coutp, (int)q.idesc, (int)smem, lout, q.nsplit,
                          q.wstep,   q.wcompact, q.wprod, q.na, q.per_sm};
    memcpy(meta_out, meta, sizeof(meta));
    return GW_OK;
  } catch (const gw::Error& e) {
    gw::set_last_error(e.what());
    return e.code;
  }
}
