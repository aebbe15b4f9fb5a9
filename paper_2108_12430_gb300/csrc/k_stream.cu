// Streaming kernels: snapshot-state update (device rings) and the fused
// subtract + aggregate step.
//
// Snapshot state (Methods, "Streaming IaaS"): the last samples of every
// channel live in a device ring of capacity R >= W + (max_batch - 1) S.  The
// witness ring is double-mapped -- sample t is stored at t mod R and at
// t mod R + R -- so every window [t - W, t) is one contiguous run starting at
// (t - W) mod R, which the first conv layer reads in place.
#include <algorithm>

#include "gw_internal.h"

namespace gw {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int64_t pmod(int64_t a, int64_t m) {
  int64_t r = a % m;
  return r < 0 ? r + m : r;
}

__device__ __forceinline__ int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }
__device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ int64_t floordiv64(int64_t a, int64_t b) {
  return (a >= 0) ? a / b : -((-a + b - 1) / b);
}

// The ring position of new sample i is (h0 + i) mod R with h0 = head mod R
// reduced on the host; i < n <= R, so one conditional subtraction suffices and
// all ring arithmetic stays in 32 bits.
__device__ __forceinline__ uint32_t ring_pos(int h0, int i, int R) {
  uint32_t q = (uint32_t)h0 + (uint32_t)i;
  return q >= (uint32_t)R ? q - (uint32_t)R : q;
}

// src [C][src_ld] (n new samples per channel) -> ring [C][2R], standardised.
// Grid: (samples, channel).
__global__ void ring_push_f32_kernel(const float* __restrict__ src, int64_t src_ld, int n,
                                     float* __restrict__ ring, int R, int h0, const float* __restrict__ mean,
                                     const float* __restrict__ istd, int* status, const int* skip) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y;
  if (i >= n || (skip && *skip)) return;
  float v = __ldg(src + (int64_t)c * src_ld + i);
  if (!isfinite(v)) atomicExch(status, GW_ENONFINITE);
  if (mean) v = (v - mean[c]) * istd[c];
  const uint32_t q = ring_pos(h0, i, R);
  float* row = ring + (int64_t)c * 2 * R;
  row[q] = v;
  row[q + (uint32_t)R] = v;
}

// src [C][src_ld] -> ring [G][P][2R / P][8] bf16 (channel-group blocked,
// P phase planes), standardised.  One thread writes the 8 channels of one
// (group, time) as a 16-byte store; R is a multiple of P.  Grid: (samples, group).
__global__ void ring_push_bf16_kernel(const float* __restrict__ src, int64_t src_ld, int C, int n,
                                      __nv_bfloat16* __restrict__ ring, int R, int h0, int P,
                                      const float* __restrict__ mean, const float* __restrict__ istd,
                                      int* status, const int* skip) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, g = blockIdx.y;
  if (i >= n || (skip && *skip)) return;
  __align__(16) __nv_bfloat16 v8[8];
  bool bad = false;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int c = g * 8 + j;
    float v = 0.f;
    if (c < C) {
      v = __ldg(src + (int64_t)c * src_ld + i);
      bad |= !isfinite(v);
      if (mean) v = (v - mean[c]) * istd[c];
    }
    v8[j] = __float2bfloat16_rn(v);
  }
  if (bad) atomicExch(status, GW_ENONFINITE);
  const uint32_t q = ring_pos(h0, i, R), q2 = q + (uint32_t)R, up = (uint32_t)P;
  const uint32_t plane_rows = 2u * (uint32_t)R / up;
  const uint4 val = *reinterpret_cast<const uint4*>(v8);
  uint4* grp = reinterpret_cast<uint4*>(ring + (int64_t)g * 2 * R * 8);
  grp[(q % up) * plane_rows + q / up] = val;
  grp[(q2 % up) * plane_rows + q2 / up] = val;
}
// One snapshot update of a BF16 stream in one launch: blockIdx.y < G writes
// the witness ring's channel group blockIdx.y (as ring_push_bf16_kernel),
// blockIdx.y == G the strain ring.  Launched as a programmatic dependent of
// the previous push's aggregation kernel, whose strain reads share ring slots
// with these writes: it waits for that kernel before touching memory.
__global__ void stream_push_bf16_kernel(const float* __restrict__ src, int64_t src_ld, int C, int G, int n,
                                        __nv_bfloat16* __restrict__ ring, int R, int h0, int P,
                                        const float* __restrict__ mean, const float* __restrict__ istd,
                                        const float* __restrict__ strain_src, float* __restrict__ strain_ring,
                                        int* status, const int* skip) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int i = blockIdx.x * blockDim.x + threadIdx.x, g = blockIdx.y;
  if (i >= n || (skip && *skip)) return;
  if (g == G) {
    const float v = __ldg(strain_src + i);
    if (!isfinite(v)) atomicExch(status, GW_ENONFINITE);
    strain_ring[ring_pos(h0, i, R)] = v;
    return;
  }
  __align__(16) __nv_bfloat16 v8[8];
  bool bad = false;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int c = g * 8 + j;
    float v = 0.f;
    if (c < C) {
      v = __ldg(src + (int64_t)c * src_ld + i);
      bad |= !isfinite(v);
      if (mean) v = (v - mean[c]) * istd[c];
    }
    v8[j] = __float2bfloat16_rn(v);
  }
  if (bad) atomicExch(status, GW_ENONFINITE);
  const uint32_t q = ring_pos(h0, i, R), q2 = q + (uint32_t)R, up = (uint32_t)P;
  const uint32_t plane_rows = 2u * (uint32_t)R / up;
  const uint4 val = *reinterpret_cast<const uint4*>(v8);
  uint4* grp = reinterpret_cast<uint4*>(ring + (int64_t)g * 2 * R * 8);
  grp[(q % up) * plane_rows + q / up] = val;
  grp[(q2 % up) * plane_rows + q2 / up] = val;
}

__global__ void strain_push_kernel(const float* __restrict__ src, int n, float* __restrict__ ring, int R, int h0,
                                   int* status, const int* skip) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || (skip && *skip)) return;
  const float v = __ldg(src + i);
  if (!isfinite(v)) atomicExch(status, GW_ENONFINITE);
  ring[ring_pos(h0, i, R)] = v;
}

// Fused subtract + aggregate over one batch of n windows (Methods, "Data
// aggregation", "Aggregation latency"); LATEST mode (AVERAGE: below).  Window j of the batch covers times
// [head + (j+1) S - W, head + (j+1) S).  One thread per time tau of the
// union of the batch's windows:
//   AVERAGE: sum = acc[tau] (windows of earlier batches, zero for new times)
//            + pred_j(tau) for covering j in ascending order; the emitted
//            value of snapshot k(tau) = floor((tau + delta) / S) is the
//            partial sum up to window k(tau) over the number of windows
//            (j >= 0) it contains; acc[tau] keeps the full sum.
//   LATEST:  the emitted value is pred_{k(tau)}(tau).
// cleaned = strain(tau) - value, written to out[tau - head + delta].
__global__ void sub_ola_kernel(const float* __restrict__ pred, int64_t pred_ld, int n, int S, int W,
                               int64_t R, int64_t head, int mode, int delta, float* __restrict__ acc,
                               const float* __restrict__ strain_ring, float* __restrict__ out, const int* skip,
                               float* __restrict__ pring, int64_t Rp, int* skip_copy) {
  // a programmatic dependent of the DeepClean kernel that writes pred (a no-op
  // when launched without the attribute)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (skip_copy && blockIdx.x == 0 && threadIdx.x == 0) *skip_copy = skip ? *skip : 0;
  if (skip && *skip) return;
  const int64_t lo = head + S - W;
  const int64_t count = (int64_t)W + (int64_t)(n - 1) * S;
  const int64_t k0 = head / S;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t tau = lo + e;
    const int64_t r = tau - head;
    const int64_t k_emit = floordiv64(tau + delta, S);         // global snapshot emitting tau
    const bool emits = (tau >= head - delta) && (tau < head + (int64_t)n * S - delta);
    const int jlo = (int)imax64(0, floordiv64(r, S));
    const int jhi = (int)imin64(n - 1, floordiv64(r + W, S) - 1);
    const float s_tau = (tau >= 0) ? strain_ring[pmod(tau, R)] : 0.f;
    // an emitted time gets strain - prediction, or with post-processing its
    // prediction goes to the ring that the post-processing FIR reads
    auto emit = [&](float value) {
      if (pring) {
        if (tau >= 0) pring[pmod(tau, Rp)] = value;
      } else {
        out[tau - head + delta] = s_tau - value;
      }
    };
    if (mode == GW_AGG_LATEST) {
      if (!emits) continue;
      const int j = (int)(k_emit - k0);
      const int64_t start = head + (int64_t)(j + 1) * S - W;
      emit(pred[(int64_t)j * pred_ld + (tau - start)]);
      continue;
    }
    float sum = (tau < head) ? acc[pmod(tau, R)] : 0.f;
    const int j_emit = emits ? (int)(k_emit - k0) : -1;
    const int64_t first = imax64(0, floordiv64(tau, S));
    const float cnt = (float)(k_emit - first + 1);
    // window j holds tau at offset tau - (head + (j+1) S - W) of its prediction
    const float* pj = pred + (tau - head - S + W);
    int j = jlo;
    // eight windows' values are loaded before they are added (in window order),
    // so each thread keeps eight loads in flight
    for (; j + 7 <= jhi; j += 8) {
      float val[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) val[q] = pj[(int64_t)(j + q) * (pred_ld - S)];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        sum += val[q];
        if (j + q == j_emit) emit(sum / cnt);
      }
    }
    for (; j <= jhi; ++j) {
      sum += pj[(int64_t)j * (pred_ld - S)];
      if (j == j_emit) emit(sum / cnt);
    }
    acc[pmod(tau, R)] = sum;
  }
}

// AVERAGE aggregation with the windows of a batch split over the 8 warps of
// a block: the block handles 32 V consecutive times (V per lane); warp q sums,
// in window order, its contiguous block of windows [q b, q b + b), b =
// ceil(n / 8), and keeps its running sum at the emitting window.  Warp 0 then
// adds, per time, the accumulator (earlier batches) and the eight block sums
// in block order: the emitted value is the sum up to the emitting window, the
// accumulator keeps the full sum (warp v does this for the lanes' times
// tau + v).  Every load of a warp reads 32 V consecutive floats of one
// window's prediction.  V = 4 (16-byte loads) needs S, W, delta,
// head, R and the prediction stride to be multiples of 4, so that a lane's four
// times share their window range and emitting snapshot; the sums are the same
// (same order) for either V.
constexpr int kOlaWarps = 8;
template <int V>
__global__ void __launch_bounds__(32 * kOlaWarps) sub_ola_avg_kernel(
    const float* __restrict__ pred, int64_t pred_ld, int n, int S, int W, int64_t R, int64_t head, int delta,
    float* __restrict__ acc, const float* __restrict__ strain_ring, float* __restrict__ out, const int* skip,
    float* __restrict__ pring, int64_t Rp, int* skip_copy) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (skip_copy && blockIdx.x == 0 && threadIdx.x == 0) *skip_copy = skip ? *skip : 0;
  if (skip && *skip) return;
  __shared__ float part[kOlaWarps][32 * V + 1], upto[kOlaWarps][32 * V + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t count = (int64_t)W + (int64_t)(n - 1) * S;
  const int64_t e = ((int64_t)blockIdx.x * 32 + lane) * V;
  const bool valid = e < count;
  const int64_t tau = head + S - W + e, r = tau - head;
  const int64_t k_emit = floordiv64(tau + delta, S);
  const bool emits = valid && (tau >= head - delta) && (tau < head + (int64_t)n * S - delta);
  const int j_emit = emits ? (int)(k_emit - head / S) : -1;
  const int jlo = (int)imax64(0, floordiv64(r, S));
  const int jhi = (int)imin64(n - 1, floordiv64(r + W, S) - 1);
  const int blk = (n + kOlaWarps - 1) / kOlaWarps;
  const int ja = max(jlo, warp * blk), jb = valid ? min(jhi, warp * blk + blk - 1) : -1;
  // window j holds tau at offset tau - (head + (j+1) S - W) = e - j S of its prediction
  const float* pj = pred + e;
  const int64_t wstep = pred_ld - S;
  float sum[V], at_emit[V];
#pragma unroll
  for (int v = 0; v < V; ++v) sum[v] = at_emit[v] = 0.f;
  auto load = [&](int jj, float (&x)[V]) {
    if constexpr (V == 4) {
      const float4 q4 = *reinterpret_cast<const float4*>(pj + (int64_t)jj * wstep);
      x[0] = q4.x;
      x[1] = q4.y;
      x[2] = q4.z;
      x[3] = q4.w;
    } else {
      x[0] = pj[(int64_t)jj * wstep];
    }
  };
  int j = ja;
  for (; j + 7 <= jb; j += 8) {
    float val[8][V];
#pragma unroll
    for (int q = 0; q < 8; ++q) load(j + q, val[q]);
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int v = 0; v < V; ++v) {
        sum[v] += val[q][v];
        if (j + q == j_emit) at_emit[v] = sum[v];
      }
  }
  for (; j <= jb; ++j) {
    float val[V];
    load(j, val);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      sum[v] += val[v];
      if (j == j_emit) at_emit[v] = sum[v];
    }
  }
#pragma unroll
  for (int v = 0; v < V; ++v) {
    part[warp][lane * V + v] = sum[v];
    upto[warp][lane * V + v] = at_emit[v];
  }
  __syncthreads();
  // warp v < V finishes time tau + v of every lane
  if (warp >= V || !valid) return;
  const int v = warp;
  const int q_emit = j_emit >= 0 ? j_emit / blk : -1;
  const int64_t first = imax64(0, floordiv64(tau, S));
  const int64_t tv = tau + v;
  float total = (tv < head) ? acc[pmod(tv, R)] : 0.f, value = 0.f;
#pragma unroll
  for (int q = 0; q < kOlaWarps; ++q) {
    if (q == q_emit) value = total + upto[q][lane * V + v];
    total += part[q][lane * V + v];
  }
  if (emits) {
    value /= (float)(k_emit - first + 1);
    if (pring) {
      if (tv >= 0) pring[pmod(tv, Rp)] = value;
    } else {
      out[tv - head + delta] = ((tv >= 0) ? strain_ring[pmod(tv, R)] : 0.f) - value;
    }
  }
  acc[pmod(tv, R)] = total;
}

int grid_for(int64_t n) {
  int64_t g = (n + kThreads - 1) / kThreads;
  return (int)std::min<int64_t>(std::max<int64_t>(g, 1), 152 * 16);
}

// Every position of a witness ring set to the standardised value of a zero
// sample, (0 - mean_c) / std_c (0 in padding channels): the stream's missing
// past counts as zero input, which the model's standardisation maps here.
// bf16: rows of 8 channels, G groups x R2 rows (the phase-plane order does
// not matter, every row of a group holds the same value); fp32: [C][R2].
__global__ void ring_fill_kernel(void* __restrict__ ring, int bf16, int C, int G, int64_t R2,
                                 const float* __restrict__ mean, const float* __restrict__ istd) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (bf16) {
    uint4* rows = reinterpret_cast<uint4*>(ring);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)G * R2; e += stride) {
      const int grp = (int)(e / R2);
      __align__(16) __nv_bfloat16 v8[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = grp * 8 + j;
        v8[j] = __float2bfloat16_rn(c < C ? -mean[c] * istd[c] : 0.f);
      }
      rows[e] = *reinterpret_cast<const uint4*>(v8);
    }
  } else {
    float* r = reinterpret_cast<float*>(ring);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)C * R2; e += stride) {
      const int c = (int)(e / R2);
      r[e] = -mean[c] * istd[c];
    }
  }
}

// Post-processing of the aggregated prediction: one CTA per kPostBlock
// outputs stages the taps and the prediction segment it needs in shared
// memory; each thread computes one output.
constexpr int kPostBlock = 256;
__global__ void post_sub_kernel(const float* __restrict__ pring, int64_t Rp, const float* __restrict__ h, int K,
                                const float* __restrict__ strain_ring, int64_t R, int64_t t0, int count,
                                float* __restrict__ out, const int* skip) {
  if (skip && *skip) return;
  extern __shared__ float sh[];
  float* hs = sh;      // [K]
  float* ps = sh + K;  // p[t_blk - c + i], i < kPostBlock + K - 1
  const int c = (K - 1) / 2;
  const int64_t t_blk = t0 + (int64_t)blockIdx.x * kPostBlock;
  for (int k = threadIdx.x; k < K; k += blockDim.x) hs[k] = h[k];
  for (int i = threadIdx.x; i < kPostBlock + K - 1; i += blockDim.x) {
    const int64_t t = t_blk - c + i;
    ps[i] = t >= 0 ? pring[pmod(t, Rp)] : 0.f;
  }
  __syncthreads();
  const int i = blockIdx.x * kPostBlock + threadIdx.x;
  if (threadIdx.x >= kPostBlock || i >= count) return;
  float q = 0.f;
  for (int k = 0; k < K; ++k) q = fmaf(hs[k], ps[threadIdx.x + k], q);
  const int64_t t = t_blk + threadIdx.x;
  out[i] = (t >= 0 ? strain_ring[pmod(t, R)] : 0.f) - q;
}

// Any non-finite value among n floats (16-byte aligned, n a multiple of 4
// handled by vector loads, the tail one by one) sets *flag.
__global__ void check_finite_kernel(const float* __restrict__ x, int64_t n, int* flag) {
  bool bad = false;
  const int64_t n4 = n / 4, stride = (int64_t)gridDim.x * blockDim.x;
  const float4* x4 = reinterpret_cast<const float4*>(x);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n4; e += stride) {
    const float4 v = __ldg(x4 + e);
    bad |= !isfinite(v.x) || !isfinite(v.y) || !isfinite(v.z) || !isfinite(v.w);
  }
  for (int64_t e = 4 * n4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += stride) bad |= !isfinite(x[e]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(flag, 1);
}

}  // namespace

void launch_check_finite(const float* x, int64_t n, int* flag, cudaStream_t st) {
  GW_CHECK_ARG(((uintptr_t)x & 15) == 0, "finiteness check needs a 16-byte aligned buffer");
  if (n <= 0) return;
  const int64_t blocks = std::min<int64_t>((n / 4 + kThreads - 1) / kThreads + 1, 4 * 152);
  check_finite_kernel<<<(int)blocks, kThreads, 0, st>>>(x, n, flag);
  GW_LAUNCH_CHECK();
}

void launch_ring_fill(void* ring, int bf16, int C, int G, int64_t R2, const float* mean, const float* istd,
                      cudaStream_t st) {
  if (!mean) {
    GW_CUDA(cudaMemsetAsync(ring, 0, (size_t)(bf16 ? (int64_t)G * R2 * 16 : (int64_t)C * R2 * 4), st));
    return;
  }
  ring_fill_kernel<<<304, 256, 0, st>>>(ring, bf16, C, G, R2, mean, istd);
  GW_LAUNCH_CHECK();
}

// head reduced to [0, R) on the host; the kernels index the ring in 32 bits
static int ring_head(int64_t head, int64_t R, int n) {
  GW_CHECK_ARG(R >= 1 && 2 * R < (int64_t)1 << 31, "ring capacity out of range");
  GW_CHECK_ARG(n >= 0 && n <= R, "more new samples than the ring holds");
  const int64_t h = head % R;
  return (int)(h < 0 ? h + R : h);
}

void launch_ring_push_f32(const float* src, int64_t src_ld, int C, int n, float* ring, int64_t R,
                          int64_t head, const float* mean, const float* istd, int* status, cudaStream_t st,
                          const int* skip) {
  const int h0 = ring_head(head, R, n);
  if (n == 0 || C == 0) return;
  ring_push_f32_kernel<<<dim3((n + kThreads - 1) / kThreads, C), kThreads, 0, st>>>(src, src_ld, n, ring, (int)R, h0,
                                                                                     mean, istd, status, skip);
  GW_LAUNCH_CHECK();
}

void launch_ring_push_bf16(const float* src, int64_t src_ld, int C, int G, int n, __nv_bfloat16* ring,
                           int64_t R, int64_t head, int P, const float* mean, const float* istd, int* status,
                           cudaStream_t st, const int* skip) {
  GW_CHECK_ARG(P >= 1 && R % P == 0, "ring capacity must be a multiple of the phase count");
  const int h0 = ring_head(head, R, n);
  if (n == 0 || G == 0) return;
  ring_push_bf16_kernel<<<dim3((n + kThreads - 1) / kThreads, G), kThreads, 0, st>>>(src, src_ld, C, n, ring, (int)R,
                                                                                      h0, P, mean, istd, status,
                                                                                      skip);
  GW_LAUNCH_CHECK();
}

void launch_strain_push(const float* src, int n, float* ring, int64_t R, int64_t head, int* status,
                        cudaStream_t st, const int* skip) {
  const int h0 = ring_head(head, R, n);
  if (n == 0) return;
  strain_push_kernel<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(src, n, ring, (int)R, h0, status, skip);
  GW_LAUNCH_CHECK();
}

// Launch with programmatic stream serialization: the kernel may be scheduled
// while the previous kernel of the stream finishes; it waits (griddepcontrol)
// for that kernel before touching memory, so only the launch latency overlaps.
template <typename... KArgs, typename... Args>
static void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  GW_CUDA(cudaLaunchKernelEx(&cfg, kernel, args...));
}

void launch_sub_ola(const float* pred, int64_t pred_ld, int n, int S, int W, int64_t R, int64_t head, int mode,
                    int delta, float* acc, const float* strain_ring, float* out, cudaStream_t st,
                    const int* skip, float* pring, int64_t Rp, int* skip_copy) {
  GW_CHECK_ARG(!pring || Rp >= (int64_t)n * S, "prediction ring too small");
  const int64_t count = (int64_t)W + (int64_t)(n - 1) * S;
  if (mode == GW_AGG_AVERAGE) {
    const bool vec = S % 4 == 0 && W % 4 == 0 && delta % 4 == 0 && head % 4 == 0 && R % 4 == 0 && pred_ld % 4 == 0 &&
                     ((uintptr_t)pred & 15) == 0;
    if (vec)
      launch_pdl(sub_ola_avg_kernel<4>, dim3((unsigned)((count + 127) / 128)), dim3(32 * kOlaWarps), st, pred,
                 pred_ld, n, S, W, R, head, delta, acc, strain_ring, out, skip, pring, Rp, skip_copy);
    else
      launch_pdl(sub_ola_avg_kernel<1>, dim3((unsigned)((count + 31) / 32)), dim3(32 * kOlaWarps), st, pred,
                 pred_ld, n, S, W, R, head, delta, acc, strain_ring, out, skip, pring, Rp, skip_copy);
    return;
  }
  launch_pdl(sub_ola_kernel, dim3(grid_for(count)), dim3(kThreads), st, pred, pred_ld, n, S, W, R, head, mode, delta,
             acc, strain_ring, out, skip, pring, Rp, skip_copy);
}

void launch_stream_push_bf16(const float* src, int64_t src_ld, int C, int G, int n, __nv_bfloat16* ring, int64_t R,
                             int64_t head, int P, const float* mean, const float* istd, const float* strain_src,
                             float* strain_ring, int* status, cudaStream_t st, const int* skip) {
  GW_CHECK_ARG(P >= 1 && R % P == 0, "ring capacity must be a multiple of the phase count");
  const int h0 = ring_head(head, R, n);
  if (n == 0) return;
  launch_pdl(stream_push_bf16_kernel, dim3((n + kThreads - 1) / kThreads, G + 1), dim3(kThreads), st, src, src_ld, C,
             G, n, ring, (int)R, h0, P, mean, istd, strain_src, strain_ring, status, skip);
}

void launch_post_sub(const float* pring, int64_t Rp, const float* h, int K, const float* strain_ring, int64_t R,
                     int64_t t0, int count, float* out, cudaStream_t st, const int* skip) {
  GW_CHECK_ARG(K >= 1 && (K & 1), "post-processing FIR needs an odd number of taps");
  if (count <= 0) return;
  const size_t smem = (size_t)(2 * K + kPostBlock - 1) * sizeof(float);
  GW_CHECK_ARG(smem <= 200 * 1024, "post-processing FIR too long");
  set_smem_limit_once(post_sub_kernel, 200 * 1024);
  post_sub_kernel<<<(count + kPostBlock - 1) / kPostBlock, kPostBlock, smem, st>>>(pring, Rp, h, K, strain_ring, R, t0,
                                                                                 count, out, skip);
  GW_LAUNCH_CHECK();
}

}  // namespace gw
