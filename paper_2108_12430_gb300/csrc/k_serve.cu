// Batched kernels of the serving loop: one tick processes one snapshot of
// each of up to max_batch streams, each stream with its own stride and state
// (Methods, "Streaming IaaS": the snapshot state stays on the GPU and each
// request brings only the new samples).
//
// Sample timing (per item; the resampler and the alignment are readings):
//   cleaned   c[tau] emitted for tau in [head - delta, head + S - delta);
//   decimated d[m] = sum_j f[j] c[2m + j - (Kf-1)/2]       (c[tau < 0] = 0);
//   whitened  w[n] = sum_j h[j] d[n + j - (Kh-1)/2]        (d[m < 0] = 0);
//   BBHnet input: w[n1 - Lb, n1) of every detector          (w[n < 0] = 0).
#include "gw_serve.h"

namespace gw {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int64_t floordiv64(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
// Ring residue of an absolute sample index (int64, may be negative): one
// 64-bit reduction per thread; the element loops then step through the ring
// in 32 bits with wrap(), which needs 0 <= b < m and 0 <= d < m.
__device__ __forceinline__ uint32_t ring_mod(int64_t a, int64_t m) {
  const int64_t r = a % m;
  return (uint32_t)(r < 0 ? r + m : r);
}
__device__ __forceinline__ uint32_t wrap(uint32_t b, uint32_t d, uint32_t m) {
  const uint32_t q = b + d;
  return q >= m ? q - m : q;
}

// Witness ring update (standardised on write) and strain ring update.
// Blocked BF16 ring: channel group g, ring position q (0 <= q < 2R) is the
// 16-byte row at g * 2R * 8 + (q % P) * (2R / P) * 8 + (q / P) * 8 elements;
// both copies q and q + R are written, so every window is contiguous.
__global__ void serve_push_kernel(const ServeItem* __restrict__ items, ServeGeom g, const float* __restrict__ mean,
                                  const float* __restrict__ istd) {
  // the network kernel after this one may start now: it reads only older
  // samples of the rings until it waits for this kernel to finish
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const ServeItem it = items[blockIdx.y];
  if (!it.active) return;
  const int S = it.S;
  const float* src = it.in;
  const uint32_t R = (uint32_t)g.R, h0 = ring_mod(it.head, g.R);
  if (g.bf16) {
    __nv_bfloat16* ring = reinterpret_cast<__nv_bfloat16*>(it.wring);
    const uint32_t P = (uint32_t)g.P, plane_rows = 2u * R / P;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < g.G * S; e += gridDim.x * blockDim.x) {
      const int grp = e / S, t = e - grp * S;
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = grp * 8 + j;
        v[j] = c < g.C ? src[c * S + t] : 0.f;  // all loads in flight before the first use
      }
      __align__(16) __nv_bfloat16 v8[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = grp * 8 + j;
        v8[j] = __float2bfloat16_rn(c < g.C ? (v[j] - mean[c]) * istd[c] : 0.f);
      }
      const uint32_t q = wrap(h0, (uint32_t)t, R), q2 = q + R;
      uint4* base = reinterpret_cast<uint4*>(ring + (int64_t)grp * 2 * R * 8);
      const uint4 val = *reinterpret_cast<const uint4*>(v8);
      base[(q % P) * plane_rows + q / P] = val;
      base[(q2 % P) * plane_rows + q2 / P] = val;
    }
  } else {
    float* ring = reinterpret_cast<float*>(it.wring);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < g.C * S; e += gridDim.x * blockDim.x) {
      const int c = e / S, t = e - c * S;
      const float v = (src[c * S + t] - mean[c]) * istd[c];
      const uint32_t q = wrap(h0, (uint32_t)t, R);
      ring[(int64_t)c * 2 * R + q] = v;
      ring[(int64_t)c * 2 * R + q + R] = v;
    }
  }
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < S; t += gridDim.x * blockDim.x)
    it.strain[wrap(h0, (uint32_t)t, R)] = src[g.C * S + t];
}

// Subtraction and aggregation of one new window per item (the window ends at
// head + S).  AVERAGE: sums per time in window order, divided by the number
// of windows so far covering the time; LATEST: the newest window alone.
__global__ void serve_sub_ola_kernel(const ServeItem* __restrict__ items, ServeGeom g, const float* __restrict__ pred) {
  const ServeItem it = items[blockIdx.y];
  if (!it.active) return;
  const int S = it.S, W = g.W;
  const int64_t head = it.head, k = head / S;
  const float* pr = pred + (int64_t)blockIdx.y * W;
  // window sample e is time tau = head + S - W + e; it is emitted as cleaned
  // sample o = e - (W - S - delta) when 0 <= o < S
  const uint32_t R = (uint32_t)g.R, qb = ring_mod(head + S - W, g.R);
  const uint32_t cb = ring_mod(head - g.delta, g.Rc);
  const int o_shift = W - S - g.delta;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < W; e += gridDim.x * blockDim.x) {
    const int64_t tau = head + S - W + e;
    const int o = e - o_shift;
    const bool emits = o >= 0 && o < S;
    const uint32_t q = wrap(qb, (uint32_t)e, R);
    float value;
    if (g.mode == GW_AGG_LATEST) {
      if (!emits) continue;
      value = pr[e];
    } else {
      const float sum = (tau < head ? it.acc[q] : 0.f) + pr[e];
      it.acc[q] = sum;
      if (!emits) continue;
      const int64_t first = tau >= 0 ? floordiv64(tau, S) : 0;
      value = sum / (float)(k - first + 1);
    }
    if (g.post) {
      // the post-processing FIR reads the aggregated prediction from its ring
      if (tau >= 0) it.pring[ring_mod(tau, g.Rp)] = value;
      continue;
    }
    const float c = (tau >= 0 ? it.strain[q] : 0.f) - value;
    it.out[o] = c;
    if (tau >= 0) it.clean[wrap(cb, (uint32_t)o, (uint32_t)g.Rc)] = c;
  }
}

// Post-processing: cleaned[t] = strain[t] - sum_k h[k] p[t + k - c] for the
// times t = head - delta - c + o, o < S (the prediction at negative times is
// zero: there is no data before the stream start).  One CTA per kServePost
// outputs of an item stages the taps and the prediction segment it reads.
constexpr int kServePost = 256;
__global__ void serve_post_kernel(const ServeItem* __restrict__ items, ServeGeom g, const float* __restrict__ h,
                                  int K) {
  const ServeItem it = items[blockIdx.y];
  if (!it.active) return;
  const int o0 = blockIdx.x * kServePost;
  if (o0 >= it.S) return;
  extern __shared__ float sh[];
  float* hs = sh;      // [K]
  float* ps = sh + K;  // p[t(o0) - c + i], i < kServePost + K - 1
  const int c = g.post_c;
  const int64_t t0 = it.head - g.delta - c + o0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) hs[k] = h[k];
  for (int i = threadIdx.x; i < kServePost + K - 1; i += blockDim.x) {
    const int64_t u = t0 - c + i;
    ps[i] = u >= 0 ? it.pring[ring_mod(u, g.Rp)] : 0.f;
  }
  __syncthreads();
  const int o = o0 + threadIdx.x;
  if (threadIdx.x >= kServePost || o >= it.S) return;
  float q = 0.f;
  for (int k = 0; k < K; ++k) q = fmaf(hs[k], ps[threadIdx.x + k], q);
  const int64_t t = t0 + threadIdx.x;
  const float v = (t >= 0 ? it.strain[ring_mod(t, g.R)] : 0.f) - q;
  it.out[o] = v;
  if (t >= 0) it.clean[ring_mod(t, g.Rc)] = v;
}

// New decimated samples d[m], m in [m0, m1).
__global__ void serve_decimate_kernel(const ServeItem* __restrict__ items, ServeGeom g, const float* __restrict__ f,
                                      int K) {
  const ServeItem it = items[blockIdx.y];
  if (!it.active) return;
  const int c = (K - 1) / 2;
  const uint32_t Rc = (uint32_t)g.Rc;
  for (int64_t m = it.m0 + blockIdx.x * blockDim.x + threadIdx.x; m < it.m1; m += gridDim.x * blockDim.x) {
    // taps j with 2m + j - c < 0 read the zeros before the stream start
    const int64_t jz = c - 2 * m;
    const int j0 = jz <= 0 ? 0 : (jz > K ? K : (int)jz);
    uint32_t q = ring_mod(2 * m - c + j0, g.Rc);
    float a = 0.f;
    for (int j = j0; j < K; ++j) {
      a = fmaf(f[j], it.clean[q], a);
      q = q + 1 == Rc ? 0u : q + 1;
    }
    it.dec[ring_mod(m, g.Rd)] = a;
  }
}

// New whitened samples w[n], n in [n0, n1): one CTA per item; the taps and
// the decimated segment are staged in shared memory, each warp computes one
// output at a time with its lanes splitting the taps.
__global__ void serve_whiten_kernel(const ServeItem* __restrict__ items, ServeGeom g, const float* __restrict__ h,
                                    int K) {
  extern __shared__ float sh[];
  const ServeItem it = items[blockIdx.y];
  if (!it.active || it.n1 <= it.n0) return;
  const int c = (K - 1) / 2;
  const int nn = (int)(it.n1 - it.n0);
  float* hs = sh;
  float* ds = sh + K;  // d[n0 - c + i], i < nn + K - 1 (< Rd)
  for (int j = threadIdx.x; j < K; j += blockDim.x) hs[j] = h[j];
  const uint32_t Rd = (uint32_t)g.Rd, db = ring_mod(it.n0 - c, g.Rd);
  for (int i = threadIdx.x; i < nn + K - 1; i += blockDim.x)
    ds[i] = it.n0 - c + i >= 0 ? it.dec[wrap(db, (uint32_t)i, Rd)] : 0.f;
  __syncthreads();
  const uint32_t Rw = (uint32_t)g.Rw, wb = ring_mod(it.n0, g.Rw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i < nn; i += blockDim.x >> 5) {
    float a = 0.f;
    for (int j = lane; j < K; j += 32) a = fmaf(hs[j], ds[i + j], a);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) it.white[wrap(wb, (uint32_t)i, Rw)] = a;
  }
}

// BBHnet input x[r][d][t] = w_d[n1 - Lb + t] of request r (zero for n < 0
// and for padding requests).
__global__ void serve_gather_kernel(const ServeItem* __restrict__ items, int Bb, int n_det, int Lb, ServeGeom g,
                                    float* __restrict__ x) {
  const int r = blockIdx.y;
  const ServeItem it0 = items[r];
  float* dst = x + (int64_t)r * n_det * Lb;
  const uint32_t Rw = (uint32_t)g.Rw, wb = ring_mod(it0.n1 - Lb, g.Rw);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_det * Lb; e += gridDim.x * blockDim.x) {
    const int d = e / Lb, t = e - d * Lb;
    float v = 0.f;
    if (it0.active && it0.n1 - Lb + t >= 0) v = items[d * Bb + r].white[wrap(wb, (uint32_t)t, Rw)];
    dst[e] = v;
  }
}

// Scores to the requests' host slots (NaN without a BBHnet), and the tick's
// device status: nonzero when a tensor-core kernel gave up a bounded wait.
__global__ void serve_scores_kernel(const ServeItem* __restrict__ items, int Bb, const float* __restrict__ logits,
                                    const int* e0, const int* e1, int* status) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r == 0) *status = ((e0 && *e0) || (e1 && *e1)) ? 1 : 0;
  if (r >= Bb) return;
  const ServeItem& it = items[r];
  if (it.active && it.score) *it.score = logits ? logits[r] : __int_as_float(0x7fc00000);
}

int grid_x(int64_t work) {
  const int64_t b = (work + kThreads - 1) / kThreads;
  return (int)(b < 1 ? 1 : (b > 64 ? 64 : b));
}

}  // namespace

void launch_serve_push(const ServeItem* items, int n, const ServeGeom& g, int S_max, const float* mean,
                       const float* istd, cudaStream_t st) {
  const int64_t work = (int64_t)(g.bf16 ? g.G : g.C) * S_max;
  serve_push_kernel<<<dim3(grid_x(work), n), kThreads, 0, st>>>(items, g, mean, istd);
  GW_LAUNCH_CHECK();
}

void launch_serve_sub_ola(const ServeItem* items, int n, const ServeGeom& g, const float* pred, cudaStream_t st) {
  serve_sub_ola_kernel<<<dim3(grid_x(g.W), n), kThreads, 0, st>>>(items, g, pred);
  GW_LAUNCH_CHECK();
}

void launch_serve_post(const ServeItem* items, int n, const ServeGeom& g, const float* h, int K, int S_max,
                       cudaStream_t st) {
  const size_t smem = (size_t)(2 * K + kServePost) * sizeof(float);
  GW_CHECK_ARG(smem <= 200 * 1024, "post-processing FIR too long for the serving kernel");
  set_smem_limit_once(serve_post_kernel, 200 * 1024);
  serve_post_kernel<<<dim3((S_max + kServePost - 1) / kServePost, n), kServePost, smem, st>>>(items, g, h, K);
  GW_LAUNCH_CHECK();
}

void launch_serve_decimate(const ServeItem* items, int n, const ServeGeom& g, const float* taps, int K, int max_new,
                           cudaStream_t st) {
  serve_decimate_kernel<<<dim3((max_new + 127) / 128, n), 128, 0, st>>>(items, g, taps, K);
  GW_LAUNCH_CHECK();
}

size_t serve_whiten_smem(int K, int max_new) { return (size_t)(2 * K + max_new) * sizeof(float); }

void launch_serve_whiten(const ServeItem* items, int n, const ServeGeom& g, const float* taps, int K, int max_new,
                         cudaStream_t st) {
  const size_t smem = serve_whiten_smem(K, max_new);
  GW_CHECK_ARG(smem <= 200 * 1024, "whitening FIR too long for the streaming kernel");
  set_smem_limit_once(serve_whiten_kernel, 200 * 1024);
  serve_whiten_kernel<<<dim3(1, n), kThreads, smem, st>>>(items, g, taps, K);
  GW_LAUNCH_CHECK();
}

void launch_serve_gather(const ServeItem* items, int Bb, int n_det, int Lb, const ServeGeom& g, float* x,
                         cudaStream_t st) {
  serve_gather_kernel<<<dim3(grid_x((int64_t)n_det * Lb), Bb), kThreads, 0, st>>>(items, Bb, n_det, Lb, g, x);
  GW_LAUNCH_CHECK();
}

void launch_serve_scores(const ServeItem* items, int Bb, const float* logits, const int* e0, const int* e1,
                         int* status, cudaStream_t st) {
  serve_scores_kernel<<<(Bb + 127) / 128, 128, 0, st>>>(items, Bb, logits, e0, e1, status);
  GW_LAUNCH_CHECK();
}

}  // namespace gw
