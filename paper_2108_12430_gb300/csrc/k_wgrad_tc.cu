// Weight gradient of a conv / transposed-conv layer on the tensor cores (BF16
// operands, FP32 accumulation in TMEM), for the training step's backward.
//
// The weight gradient is one contraction over all (item, position) pairs:
//   dW[a][c][k] = sum_{b, t} A[b][a][t] Bm[b][c][s t + k - p]
// (conv: A = the output gradient, Bm = the layer input; transposed conv: A =
// the layer input, Bm = the output gradient), zero outside [0, LB).  As a
// GEMM, D[a][n] = sum_t A[a][t] B[n][t] with n = k NC + c and
// B[n][t] = Bm[c][s t + k - p]: M = the A channels (zero-padded to 128 MMA
// rows), N = K NC columns, and the reduction runs over positions, which is
// the dimension the tensor core's K steps walk.
//
// Each CTA (512 threads, one per SM) takes chunks of 128 positions of one
// item in turn.  All its threads stage a chunk: FP32 values are read from
// global memory once (the A rows and each B channel's raw span), rounded to
// BF16, and the shifted, strided tap rows of B are built from shared memory,
// all in the canonical K-major layout (core matrices of 8 rows x 16 bytes);
// one thread then issues the chunk's eight MMAs into the CTA's TMEM
// accumulator.  Two stages let the threads fill one while the MMAs read the
// other.  At the end the
// accumulator (D, NA x N) goes to the CTA's partial slot, and a second
// kernel sums the partials in CTA order (deterministic).
#include <cuda_bf16.h>

#include <algorithm>

#include "gw_internal.h"
#include "gw_train.h"
#include "tc_ptx.h"

namespace gw {

namespace {

using namespace ptx;

constexpr int kWgChunk = 128;    // positions per chunk (eight MMA K steps)
constexpr int kWgSegs = kWgChunk / 8, kWgLgSegs = 4;  // 16-byte segments of a chunk row
static_assert((1 << kWgLgSegs) == kWgSegs, "segments per row");
constexpr int kWgThreads = 512, kWgWarps = kWgThreads / 32;
constexpr int kWgRowsA = 128;    // MMA M: the A channels, zero-padded
constexpr int kWgGroup = 6;      // a thread's 16-byte segments of a chunk (all its pass-1 tasks)
constexpr int kWgMaxCtasPerSm = 1;

struct WgTcParams {
  const float* A;
  int64_t ab, aa;  // A[b][a][t] at A + b ab + a aa + t, t < LA
  int NA, LA;
  const float* Bm;
  int64_t bb, bc;  // Bm[b][c][u] at Bm + b bb + c bc + u, u < LB
  int NC, LB;
  int K, s, p;
  int N, Npad;     // N = K NC columns n = k NC + c; Npad: the D columns (N, + 1 for bias 1) rounded up to 32
  int bias;        // 1: B row N all ones (D[a][N] = sum_t A[a][t]); 2: A row NA all ones
  int NAr;         // D rows kept: NA, + 1 for bias 2
  int span_pad;    // raw B row of a chunk: 63 s + K values, rounded up to 8
  int a_vec;       // A rows 16-byte aligned at every chunk start
  int chunks_per_b, n_chunks;
  float* partial;  // [gridDim.x][NAr][Npad]
  int* err;
};

// Byte offset of 16-byte segment q (K elements 8q .. 8q + 7) of row r in a
// K-major tile of R rows: core matrices of 8 rows x 16 bytes, K-adjacent core
// matrices R / 8 x 128 bytes apart (the descriptor's LBO), row-adjacent ones
// 128 bytes apart (SBO).
__device__ __forceinline__ uint32_t seg_off(int r, int q, int R) {
  return (uint32_t)((((q * (R >> 3)) + (r >> 3)) << 7) + ((r & 7) << 4));
}

// A chunk cid (item b, positions t0 .. t0 + kWgChunk - 1) is staged by the
// CTA's warps, each owning the A rows a = w, w + 16, ... and the B channels
// c = w, w + 16, ... (w its warp index), in two passes that need no
// synchronisation beyond the warp.  Pass 1 reads global memory once per value:
// the warp's A rows (task = row, 16-byte segment; 16-byte loads when the row
// is aligned) and, for each of its B channels c, the raw span u0 .. u0 +
// span - 1 (u0 = s t0 - p, span = (kWgChunk - 1) s + K) of Bm[c].  Each thread
// holds its (at most kWgGroup) tasks' 8 values in registers: the loads of
// chunk i + 1 are issued right after chunk i's values are stored, so that
// they are in flight while chunk i's tap rows are built and its MMAs issued.
// The stores round to BF16 into the A tile and raw[c][.].  Pass 2 builds the
// warp's tap rows B[k NC + c][t] = raw[c][s (t - t0) + k] from shared memory.
// A task's addresses relative to the chunk are the same for every chunk: each
// thread works them out once (Pass1Task, tap_task).
struct Pass1Task {
  int goff;       // element offset from the chunk's row start (A: row aa + 8 q; B: c bc + j0)
  int pos;        // position offset: 8 q (A) or j0 (B); -1: no task
  uint32_t soff;  // A: byte offset in the A tile; B: byte offset in raw
  bool is_b;
};

// Rows (or channels) r < n with r = w (mod kWgWarps): how many.
__host__ __device__ __forceinline__ int owned(int n, int w) { return n > w ? (n - w + kWgWarps - 1) / kWgWarps : 0; }

__device__ __forceinline__ Pass1Task pass1_task(const WgTcParams& p, int w, int task) {
  Pass1Task t{0, -1, 0u, false};
  const int span8 = p.span_pad / 8;
  const int n_a = owned(p.NA, w) * kWgSegs, n_tasks = n_a + owned(p.NC, w) * span8;
  if (task >= n_tasks) return t;
  if (task < n_a) {
    const int row = w + kWgWarps * (task >> kWgLgSegs), q = task & (kWgSegs - 1);
    t.goff = row * (int)p.aa + 8 * q;
    t.pos = 8 * q;
    t.soff = seg_off(row, q, kWgRowsA);
  } else {
    const int r = task - n_a, m = r / span8, j0 = (r - m * span8) * 8, c = w + kWgWarps * m;
    t.goff = c * (int)p.bc + j0;
    t.pos = j0;
    t.soff = (uint32_t)(c * p.span_pad + j0) * 2u;
    t.is_b = true;
  }
  return t;
}

__device__ __forceinline__ void load_chunk(const WgTcParams& p, int cid, const Pass1Task (&tk)[kWgGroup],
                                           float (&v)[kWgGroup][8]) {
  const int b = cid / p.chunks_per_b;
  const int t0 = (cid - b * p.chunks_per_b) * kWgChunk;
  const int u0 = p.s * t0 - p.p;
  const float* Ab = p.A + (int64_t)b * p.ab + t0;
  const float* Bb = p.Bm + (int64_t)b * p.bb + u0;
#pragma unroll
  for (int gi = 0; gi < kWgGroup; ++gi) {
#pragma unroll
    for (int e = 0; e < 8; ++e) v[gi][e] = 0.f;
    if (tk[gi].pos < 0) continue;
    if (!tk[gi].is_b) {
      const int t = t0 + tk[gi].pos;
      const float* src = Ab + tk[gi].goff;
      if (p.a_vec && t + 8 <= p.LA) {
        const float4 x0 = reinterpret_cast<const float4*>(src)[0], x1 = reinterpret_cast<const float4*>(src)[1];
        v[gi][0] = x0.x, v[gi][1] = x0.y, v[gi][2] = x0.z, v[gi][3] = x0.w;
        v[gi][4] = x1.x, v[gi][5] = x1.y, v[gi][6] = x1.z, v[gi][7] = x1.w;
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e)
          if (t + e < p.LA) v[gi][e] = src[e];
      }
    } else {
      const int u = u0 + tk[gi].pos;
      const float* src = Bb + tk[gi].goff;
      if (u >= 0 && u + 8 <= p.LB) {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[gi][e] = src[e];
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e)
          if (u + e >= 0 && u + e < p.LB) v[gi][e] = src[e];
      }
    }
  }
}

__device__ __forceinline__ void store_chunk(const Pass1Task (&tk)[kWgGroup], const float (&v)[kWgGroup][8],
                                            uint8_t* a_smem, uint8_t* raw) {
#pragma unroll
  for (int gi = 0; gi < kWgGroup; ++gi) {
    if (tk[gi].pos < 0) continue;
    __nv_bfloat162 h[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) h[e] = __floats2bfloat162_rn(v[gi][2 * e], v[gi][2 * e + 1]);
    uint8_t* dst = (tk[gi].is_b ? raw : a_smem) + tk[gi].soff;
    *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(h);
  }
}

// Pass 2 task (tap row n = k NC + c of one of the warp's channels c, segment
// q): source element offset in raw (low 16 bits) and offset in the B tile in
// 16-byte units (high 16 bits); ~0u: no task.
constexpr int kWgTaps = 12;
__device__ __forceinline__ uint32_t tap_task(const WgTcParams& p, int w, int task) {
  const int per_c = p.K * kWgSegs;
  if (task >= owned(p.NC, w) * per_c) return ~0u;
  const int m = task / per_c, r = task - m * per_c, k = r >> kWgLgSegs, q = r & (kWgSegs - 1);
  const int c = w + kWgWarps * m, n = k * p.NC + c;
  return (uint32_t)(c * p.span_pad + p.s * 8 * q + k) | ((seg_off(n, q, p.Npad) >> 4) << 16);
}

__device__ __forceinline__ void build_taps(const WgTcParams& p, const uint32_t (&tt)[kWgTaps], uint8_t* b_smem,
                                           const __nv_bfloat16* raw) {
#pragma unroll
  for (int it = 0; it < kWgTaps; ++it) {
    if (tt[it] == ~0u) continue;
    const __nv_bfloat16* src = raw + (tt[it] & 0xffffu);
    __align__(16) __nv_bfloat16 h[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) h[e] = src[p.s * e];
    *reinterpret_cast<uint4*>(b_smem + ((tt[it] >> 16) << 4)) = *reinterpret_cast<const uint4*>(h);
  }
}

__global__ void __launch_bounds__(kWgThreads, kWgMaxCtasPerSm) wgrad_tc_kernel(const WgTcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t base = smem_u32(smem);
  const uint32_t a_bytes = kWgRowsA * kWgChunk * 2, b_bytes = (uint32_t)p.Npad * kWgChunk * 2;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  // [0..1] stage free (its MMAs done), [2] all MMAs done, [3..4] stage staged (one arrival per warp)
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * stage_bytes);
  volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(bars + 5);
  uint32_t* tslot = (uint32_t*)(abort_flag + 1);
  __nv_bfloat16* raw = reinterpret_cast<__nv_bfloat16*>(smem + 2 * stage_bytes + 64);  // [NC][span_pad]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // both stages start at zero: the A rows >= NA and B rows >= N are never
  // written and contribute zeros
  {
    uint4* z = reinterpret_cast<uint4*>(smem);
    for (uint32_t i = tid; i < 2 * stage_bytes / 16; i += kWgThreads) z[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  if (tid == 0) {
    for (int i = 0; i < 3; ++i) mbar_init(smem_u32(&bars[i]), 1);
    for (int i = 3; i < 5; ++i) mbar_init(smem_u32(&bars[i]), kWgWarps);
    *abort_flag = 0u;
    fence_barrier_init();
  }
  __syncthreads();
  if (p.bias) {
    // the bias row of ones (BF16 1.0) in both stages: staging never writes it
    const uint4 ones = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
    if (tid < 2 * kWgSegs) {
      const int st = tid >> kWgLgSegs, q = tid & (kWgSegs - 1);
      uint8_t* tile = smem + st * stage_bytes + (p.bias == 1 ? a_bytes : 0u);
      *reinterpret_cast<uint4*>(tile + (p.bias == 1 ? seg_off(p.N, q, p.Npad) : seg_off(p.NA, q, kWgRowsA))) = ones;
    }
  }
  fence_proxy_async_smem();
  const uint32_t tcols = p.Npad <= 128 ? 128u : 256u;
  if (warp == 0) tmem_alloc(smem_u32(tslot), tcols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  // D = F32, A = B = BF16, both K-major, N >> 3 at bit 17, M >> 4 at bit 24
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(p.Npad >> 3) << 17) |
                         ((uint32_t)(kWgRowsA >> 4) << 24);
  const uint32_t lbo_a = (kWgRowsA / 8) * 128, lbo_b = (uint32_t)(p.Npad / 8) * 128;

  int i = 0;
  Pass1Task tk[kWgGroup];
#pragma unroll
  for (int gi = 0; gi < kWgGroup; ++gi) tk[gi] = pass1_task(p, warp, lane + 32 * gi);
  uint32_t tt[kWgTaps];
#pragma unroll
  for (int it = 0; it < kWgTaps; ++it) tt[it] = tap_task(p, warp, lane + 32 * it);
  float v[kWgGroup][8];
  if ((int)blockIdx.x < p.n_chunks) load_chunk(p, blockIdx.x, tk, v);
  for (int cid = blockIdx.x; cid < p.n_chunks; cid += gridDim.x, ++i) {
    const int st = i & 1;
    // the stage's previous MMAs (chunk i - 2) have read it
    bool ok = true;
    if (i >= 2 && lane == 0) ok = mbar_wait(smem_u32(&bars[st]), (uint32_t)((i - 2) >> 1) & 1u, abort_flag, p.err, 1);
    if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) break;
    uint8_t* a_s = smem + st * stage_bytes;
    store_chunk(tk, v, a_s, reinterpret_cast<uint8_t*>(raw));
    if (cid + (int)gridDim.x < p.n_chunks) load_chunk(p, cid + gridDim.x, tk, v);
    __syncwarp();  // the warp's raw rows are complete
    build_taps(p, tt, a_s + a_bytes, raw);
    fence_proxy_async_smem();  // the stores above are read by the tensor core (async proxy)
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_u32(&bars[3 + st]));
    if (tid == 0) {
      // every warp has staged its part of the chunk
      ok = mbar_wait(smem_u32(&bars[3 + st]), (uint32_t)(i >> 1) & 1u, abort_flag, p.err, 4);
      if (ok) {
        tc_fence_after();
        const uint32_t a0 = base + st * stage_bytes, b0 = a0 + a_bytes;
#pragma unroll
        for (int j = 0; j < kWgChunk / 16; ++j)
          mma_f16(tmem, make_desc(a0 + 2 * j * lbo_a, lbo_a, 128), make_desc(b0 + 2 * j * lbo_b, lbo_b, 128), idesc,
                  (i > 0 || j > 0) ? 1u : 0u);
        mma_commit(smem_u32(&bars[st]));
      }
    }
    if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) break;
  }
  __syncthreads();
  // every MMA of this CTA has completed before the accumulator is read
  if (tid == 0) mma_commit(smem_u32(&bars[2]));
  mbar_wait_landed(smem_u32(&bars[2]), 0u, p.err, 2);
  tc_fence_after();
  if (warp < 4) {
    const int r = warp * 32 + lane;  // TMEM lane = MMA row = A channel
    float* dst = p.partial + ((int64_t)blockIdx.x * p.NAr + r) * p.Npad;
    for (int c0 = 0; c0 < p.Npad; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (r < p.NAr) {
#pragma unroll
        for (int q = 0; q < 32; ++q) dst[c0 + q] = i > 0 ? v[q] : 0.f;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, tcols);
}

// out[a][c][k] = sum over CTAs g of partial[g][a][k NC + c].  A block takes
// 32 consecutive (a, n) columns of the partials; warp w sums g = w, w + 8, ...
// in order (lanes on consecutive n: coalesced), then the eight warp sums are
// added in warp order, so the result does not depend on the schedule.  The
// bias gradient: bias 1, db[a] = the sum of column N; bias 2, db[c] = the
// sum of row NA's columns k NC + c for k = p .. p + s - 1 (the taps that put
// every output position u = s t + k - p of channel c in exactly one (t, k)).
constexpr int kWgRedWarps = 8;
struct WgRedParams {
  const float* partial;
  int G, NA, NAr, NC, K, N, Npad, bias, s, p;
  float* out;
  float* db;
};
__global__ void __launch_bounds__(32 * kWgRedWarps) wgrad_tc_reduce_kernel(const WgRedParams q) {
  __shared__ float red[kWgRedWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * 32 + lane;  // index into [NAr][Npad]
  const int64_t stride = (int64_t)q.NAr * q.Npad;
  const int a = (int)(e / q.Npad), n = (int)(e - (int64_t)a * q.Npad);
  // the partial columns this lane adds (cnt of them, NC apart)
  int cnt = 0;
  if (e < stride) {
    if (a < q.NA)
      cnt = (n < q.N || (q.bias == 1 && n == q.N)) ? 1 : 0;
    else if (n < q.N && n / q.NC == q.p)
      cnt = q.s;
  }
  float acc = 0.f;
  for (int j = 0; j < cnt; ++j) {
    // four CTAs' partials in flight per step
    const float* src = q.partial + e + j * q.NC;
    int g = warp;
    for (; g + 3 * kWgRedWarps < q.G; g += 4 * kWgRedWarps) {
      const float v0 = src[(int64_t)g * stride], v1 = src[(int64_t)(g + kWgRedWarps) * stride];
      const float v2 = src[(int64_t)(g + 2 * kWgRedWarps) * stride], v3 = src[(int64_t)(g + 3 * kWgRedWarps) * stride];
      acc += v0;
      acc += v1;
      acc += v2;
      acc += v3;
    }
    for (; g < q.G; g += kWgRedWarps) acc += src[(int64_t)g * stride];
  }
  red[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && cnt > 0) {
    float t = 0.f;
    for (int w = 0; w < kWgRedWarps; ++w) t += red[w][lane];
    if (a < q.NA && n < q.N) {
      const int k = n / q.NC, c = n - k * q.NC;
      q.out[((int64_t)a * q.NC + c) * q.K + k] = t;
    } else if (a < q.NA) {
      q.db[a] = t;
    } else {
      q.db[n - q.p * q.NC] = t;
    }
  }
}

int wgrad_tc_grid(const WgradArgs& w, int B) {
  const int chunks = B * ((w.LA + kWgChunk - 1) / kWgChunk);
  return std::max(1, std::min(chunks, kWgMaxCtasPerSm * current_sm_count()));
}

}  // namespace

namespace {
// D's columns (N, + 1 for the ones row of bias 1) rounded up to 32, and rows
// (NA, + 1 for bias 2).
int wg_npad(const WgradArgs& w) { return (w.K * w.NC + (w.bias == 1 ? 1 : 0) + 31) / 32 * 32; }
int wg_rows(const WgradArgs& w) { return w.NA + (w.bias == 2 ? 1 : 0); }
}  // namespace

bool wgrad_tc_supported(const WgradArgs& w) {
  const int span_pad = ((kWgChunk - 1) * w.s + w.K + 7) / 8 * 8;
  // bias 2 sums taps p .. p + s - 1 of every t < LA: each output position
  // u < LB exactly once when LB = s LA
  const bool bias_ok = w.bias == 0 || w.bias == 1 || (w.bias == 2 && w.LB == w.s * w.LA && w.p + w.s <= w.K);
  return tc_supported() && bias_ok && w.NA >= 1 && wg_rows(w) <= kWgRowsA && w.NC >= 1 && wg_npad(w) <= 256 &&
         owned(w.NA, 0) * kWgSegs + owned(w.NC, 0) * (span_pad / 8) <= 32 * kWgGroup &&
         owned(w.NC, 0) * w.K * kWgSegs <= 32 * kWgTaps && w.NC * span_pad < 65536 &&
         (int64_t)w.NA * w.aa < (1LL << 31) && (int64_t)w.NC * w.bc < (1LL << 31);
}

size_t wgrad_tc_partial_floats(const WgradArgs& w, int B) {
  return (size_t)wgrad_tc_grid(w, B) * wg_rows(w) * wg_npad(w);
}

void launch_wgrad_tc(const WgradArgs& w, int B, float* partial, float* out, float* db, int* err, cudaStream_t st) {
  GW_CHECK_ARG(wgrad_tc_supported(w), "layer shape outside the tensor-core weight-gradient kernel");
  GW_CHECK_ARG(!w.bias || db, "bias gradient requested without an output");
  WgTcParams p{};
  p.A = w.A;
  p.ab = w.ab;
  p.aa = w.aa;
  p.NA = w.NA;
  p.LA = w.LA;
  p.Bm = w.Bm;
  p.bb = w.bb;
  p.bc = w.bc;
  p.NC = w.NC;
  p.LB = w.LB;
  p.K = w.K;
  p.s = w.s;
  p.p = w.p;
  p.N = w.K * w.NC;
  p.Npad = wg_npad(w);
  p.bias = w.bias;
  p.NAr = wg_rows(w);
  p.span_pad = ((kWgChunk - 1) * w.s + w.K + 7) / 8 * 8;
  p.a_vec = (w.aa % 4 == 0 && w.ab % 4 == 0 && ((uintptr_t)w.A & 15) == 0) ? 1 : 0;
  p.chunks_per_b = (w.LA + kWgChunk - 1) / kWgChunk;
  p.n_chunks = B * p.chunks_per_b;
  p.partial = partial;
  p.err = err;
  const int grid = wgrad_tc_grid(w, B);
  // at least 80 KB of shared memory per CTA, so that at most two CTAs share an
  // SM and their TMEM allocations (up to 256 columns each) always fit
  const size_t raw_bytes = (size_t)w.NC * p.span_pad * 2;
  const size_t smem = std::max<size_t>(kWgMaxCtasPerSm == 2 ? 80 * 1024 : 0,
                                       1024 + 2 * (size_t)(kWgRowsA + p.Npad) * kWgChunk * 2 + 64 + raw_bytes);
  GW_CHECK_ARG(smem <= 227 * 1024, "weight-gradient tile exceeds shared memory");
  // the limit is set once per device, to the most any layer may ask for
  set_smem_limit_once(wgrad_tc_kernel, 227 * 1024);
  wgrad_tc_kernel<<<grid, kWgThreads, smem, st>>>(p);
  GW_LAUNCH_CHECK();
  WgRedParams q{partial, grid, w.NA, p.NAr, w.NC, w.K, p.N, p.Npad, w.bias, w.s, w.p, out, db};
  const int64_t cols = (int64_t)p.NAr * p.Npad;
  wgrad_tc_reduce_kernel<<<(unsigned)((cols + 31) / 32), 32 * kWgRedWarps, 0, st>>>(q);
  GW_LAUNCH_CHECK();
}

}  // namespace gw
