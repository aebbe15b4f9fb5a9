// FP32 SIMT kernels: the plain-FP32 path (conv, transposed conv, FIR, pool+head).
//
// These run every layer in FP32 FMA (no TF32, which could not meet a 1e-5
// relative error): they are the accuracy reference path on the GPU and the
// baseline that the BF16 tensor-core path is measured against.
#include "gw_internal.h"

namespace gw {

namespace {

constexpr int kThreads = 256;
constexpr int kCPT = 8;  // output channels per thread
constexpr int kPPT = 4;  // output positions per thread (strided by the thread count)

__device__ __forceinline__ int floordiv(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }

__device__ __forceinline__ float apply_act(float v, int act) {
  if (act == ACT_TANH) return tanhf(v);
  if (act == ACT_RELU) return fmaxf(v, 0.f);
  return v;
}

// One CTA: TL output positions x CB output channels of one batch item.
// Conv:  y[o,u] = b[o] + sum_{i,k} w[o,i,k] x[i, s u + k - p]
// ConvT: y[o,u] = b[o] + sum_{i,k : s | (u + p - k)} w[o,i,k] x[i, (u + p - k) / s]
__global__ void __launch_bounds__(kThreads) conv_f32_kernel(ConvF32Args a, int CB, int CI) {
  extern __shared__ float smem[];
  const LayerSpec& s = a.s;
  const int ng = CB / kCPT, np = kThreads / ng, TL = np * kPPT;
  const int tid = threadIdx.x, cg = tid / np, pt = tid % np;
  const int t0 = blockIdx.x * TL, co0 = blockIdx.y * CB, b = blockIdx.z;
  const int K = s.k, st = s.stride, pad = s.pad_l;

  int lo, span;
  if (!s.transposed) {
    lo = t0 * st - pad;
    span = (TL - 1) * st + K;
  } else {
    lo = floordiv(t0 + pad - (K - 1), st);
    span = floordiv(t0 + TL - 1 + pad, st) - lo + 1;
  }
  float* xs = smem;                 // [CI][span]
  float* ws = smem + CI * span;     // [CB][CI][K]

  float acc[kCPT][kPPT];
#pragma unroll
  for (int c = 0; c < kCPT; ++c)
#pragma unroll
    for (int j = 0; j < kPPT; ++j) acc[c][j] = 0.f;

  const float* xb = a.item_ptr ? a.item_ptr[b] : a.x + (int64_t)b * a.xb;
  for (int ci0 = 0; ci0 < s.cin; ci0 += CI) {
    __syncthreads();
    for (int e = tid; e < CI * span; e += kThreads) {
      int ci = e / span, j = e % span, t = lo + j, c = ci0 + ci;
      float v = 0.f;
      if (c < s.cin && t >= 0 && t < a.lin) {
        v = xb[(int64_t)c * a.xc + t];
        if (a.in_mean) v = (v - a.in_mean[c]) * a.in_istd[c];
      }
      xs[e] = v;
    }
    for (int e = tid; e < CB * CI * K; e += kThreads) {
      int co = e / (CI * K), r = e % (CI * K), ci = r / K, k = r % K;
      int o = co0 + co, c = ci0 + ci;
      ws[e] = (o < s.cout && c < s.cin) ? a.w[((int64_t)o * s.cin + c) * K + k] : 0.f;
    }
    __syncthreads();
    const float* wrow = ws + (cg * kCPT) * CI * K;
    if (!s.transposed) {
      for (int ci = 0; ci < CI; ++ci) {
        const float* xr = xs + ci * span;
        for (int k = 0; k < K; ++k) {
          float xv[kPPT];
#pragma unroll
          for (int j = 0; j < kPPT; ++j) xv[j] = xr[(pt + j * np) * st + k];
#pragma unroll
          for (int c = 0; c < kCPT; ++c) {
            float wv = wrow[(c * CI + ci) * K + k];
#pragma unroll
            for (int j = 0; j < kPPT; ++j) acc[c][j] = fmaf(wv, xv[j], acc[c][j]);
          }
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < kPPT; ++j) {
        const int u = t0 + pt + j * np;
        const int k0 = (u + pad) % st;
        for (int k = k0; k < K; k += st) {
          const int tt = (u + pad - k) / st - lo;
          for (int ci = 0; ci < CI; ++ci) {
            float xv = xs[ci * span + tt];
#pragma unroll
            for (int c = 0; c < kCPT; ++c) acc[c][j] = fmaf(wrow[(c * CI + ci) * K + k], xv, acc[c][j]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < kCPT; ++c) {
    const int o = co0 + cg * kCPT + c;
    if (o >= s.cout) continue;
    const float bias = a.bias[o];
#pragma unroll
    for (int j = 0; j < kPPT; ++j) {
      const int u = t0 + pt + j * np;
      if (u >= a.lout) continue;
      float v = acc[c][j] + bias;
      if (a.res) v += a.res[(int64_t)b * a.rb + (int64_t)o * a.rc + u];
      if (a.gy) {
        // backward: times the derivative of the activation whose output is gy
        const float yv = a.gy[(int64_t)b * a.gyb + (int64_t)o * a.gyc + u];
        v *= a.gact == ACT_TANH ? 1.f - yv * yv : (a.gact == ACT_RELU ? (yv > 0.f ? 1.f : 0.f) : 1.f);
      }
      a.y[(int64_t)b * a.yb + (int64_t)o * a.yc + u] = apply_act(v, s.act);
    }
  }
}

// FIR over one row, CTA = 1024 outputs:
//   y[r][n] = scale * sum_k h'[k] x[r][n + k + x_off],  x zero outside [0, x_len),
// h' = h (rev = 0) or h reversed (rev = 1).  Valid mode: x_off = 0,
// x_len = lout + ntaps - 1.  Its adjoint (dx[m] = sum_k h[k] dy[m - k]) is
// x_off = -(ntaps - 1), rev = 1.
constexpr int kFirTile = 1024;
__global__ void __launch_bounds__(kThreads) fir_f32_kernel(const float* __restrict__ x, int64_t x_row,
                                                           float* __restrict__ y, int64_t y_row,
                                                           const float* __restrict__ h, int ntaps, int lout,
                                                           int x_off, int x_len, int rev, float scale) {
  extern __shared__ float smem[];
  float* hs = smem;
  float* xs = smem + ntaps;
  const int r = blockIdx.y, n0 = blockIdx.x * kFirTile;
  const float* xr = x + (int64_t)r * x_row;
  const int span = kFirTile + ntaps - 1;
  for (int e = threadIdx.x; e < ntaps; e += kThreads) hs[e] = h[rev ? ntaps - 1 - e : e];
  for (int e = threadIdx.x; e < span; e += kThreads) {
    const int q = n0 + e + x_off;
    xs[e] = (q >= 0 && q < x_len) ? xr[q] : 0.f;
  }
  __syncthreads();
  float acc[kFirTile / kThreads];
#pragma unroll
  for (int j = 0; j < kFirTile / kThreads; ++j) acc[j] = 0.f;
  for (int k = 0; k < ntaps; ++k) {
    const float hv = hs[k];
#pragma unroll
    for (int j = 0; j < kFirTile / kThreads; ++j) acc[j] = fmaf(hv, xs[threadIdx.x + j * kThreads + k], acc[j]);
  }
#pragma unroll
  for (int j = 0; j < kFirTile / kThreads; ++j) {
    const int n = n0 + threadIdx.x + j * kThreads;
    if (n < lout) y[(int64_t)r * y_row + n] = scale * acc[j];
  }
}

// Global average pool over time followed by the linear head; one CTA per item.
__global__ void __launch_bounds__(kThreads) gap_linear_f32_kernel(const float* __restrict__ h, int64_t hb,
                                                                  int64_t hc, int C, int L,
                                                                  const float* __restrict__ w,
                                                                  const float* __restrict__ bias,
                                                                  float* __restrict__ out) {
  __shared__ float red[kThreads / 32];
  const int b = blockIdx.x;
  float part = 0.f;
  for (int c = threadIdx.x; c < C; c += kThreads) {
    const float* row = h + (int64_t)b * hb + (int64_t)c * hc;
    float sum = 0.f;
    for (int t = 0; t < L; ++t) sum += row[t];
    part = fmaf(sum / (float)L, w[c], part);
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    float v = 0.f;
    for (int i = 0; i < kThreads / 32; ++i) v += red[i];
    out[b] = v + bias[0];
  }
}

// *amax = max(*amax, max_i |x[i]|): block maximum, then an atomic max on the
// bit pattern (non-negative floats order like their bits as integers, and a
// maximum does not depend on the order it is taken in).
__global__ void __launch_bounds__(kThreads) absmax_kernel(const float* __restrict__ x, int64_t n,
                                                         float* __restrict__ amax) {
  __shared__ float red[kThreads / 32];
  float m = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
    m = fmaxf(m, fabsf(x[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < kThreads / 32; ++i) m = fmaxf(m, red[i]);
    atomicMax(reinterpret_cast<int*>(amax), __float_as_int(m));
  }
}

}  // namespace

void launch_absmax(const float* x, int64_t n, float* amax, cudaStream_t st) {
  const int64_t blocks = std::min<int64_t>((n + kThreads - 1) / kThreads, 1216);
  absmax_kernel<<<(int)std::max<int64_t>(blocks, 1), kThreads, 0, st>>>(x, n, amax);
  GW_LAUNCH_CHECK();
}

void launch_conv_f32(const ConvF32Args& a, cudaStream_t st) {
  const LayerSpec& s = a.s;
  const int CB = std::min(64, (s.cout + 7) / 8 * 8);
  const int ng = CB / kCPT, np = kThreads / ng, TL = np * kPPT;
  const int span_max = s.transposed ? TL / s.stride + s.k / s.stride + 3 : (TL - 1) * s.stride + s.k;
  int CI = 16;
  while (CI > 1 && (size_t)(CI * span_max + CB * CI * s.k) * 4 > 96 * 1024) CI /= 2;
  if (CI > s.cin) CI = s.cin;
  const size_t smem = (size_t)(CI * span_max + CB * CI * s.k) * 4;
  set_smem_limit_once(conv_f32_kernel, 96 * 1024);
  dim3 grid((a.lout + TL - 1) / TL, (s.cout + CB - 1) / CB, a.B);
  conv_f32_kernel<<<grid, kThreads, smem, st>>>(a, CB, CI);
  GW_LAUNCH_CHECK();
}

void launch_fir_f32(const float* x, int64_t x_row, float* y, int64_t y_row, int rows, const float* taps,
                    int ntaps, int lout, cudaStream_t st, int x_off, int x_len, int rev, float scale) {
  if (x_len < 0) x_len = lout + ntaps - 1;
  const size_t smem = (size_t)(ntaps + kFirTile + ntaps - 1) * 4;
  GW_CHECK_ARG(smem <= 200 * 1024, "FIR too long for the FP32 kernel");
  set_smem_limit_once(fir_f32_kernel, 200 * 1024);
  dim3 grid((lout + kFirTile - 1) / kFirTile, rows);
  fir_f32_kernel<<<grid, kThreads, smem, st>>>(x, x_row, y, y_row, taps, ntaps, lout, x_off, x_len, rev, scale);
  GW_LAUNCH_CHECK();
}

void launch_gap_linear_f32(const float* h, int64_t hb, int64_t hc, int B, int C, int L, const float* w,
                           const float* b, float* out, cudaStream_t st) {
  gap_linear_f32_kernel<<<B, kThreads, 0, st>>>(h, hb, hc, C, L, w, b, out);
  GW_LAUNCH_CHECK();
}

}  // namespace gw
