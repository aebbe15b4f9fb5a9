// FP32 SIMT kernels: the plain-FP32 path (conv, transposed conv, FIR, pool+head).
//
// These run every layer in FP32 FMA (no TF32, which could not meet a 1e-5
// relative error): they are the accuracy reference path on the GPU and the
// baseline that the BF16 tensor-core path is measured against.
#include "gw_internal.h"

namespace gw {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int floordiv(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }

__device__ __forceinline__ float apply_act(float v, int act) {
  if (act == ACT_TANH) return tanhf(v);
  if (act == ACT_RELU) return fmaxf(v, 0.f);
  return v;
}

// Conv:  y[o,u] = b[o] + sum_{i,k} w[o,i,k] x[i, s u + k - p]
// ConvT: y[o,u] = b[o] + sum_{i,k : s | (u + p - k)} w[o,i,k] x[i, (u + p - k) / s]
// (w here in [C_out][C_in][K] for both; the host passes a transposed conv's
// weights rearranged to that layout).
//
// Register-blocked FP32 conv for the shapes of DeepClean and BBHnet (K taps,
// stride S, transposed or not, known at compile time).  A thread computes CPT
// output channels x 4 consecutive positions.  For each input channel it loads
// the x values that its 4 positions and K taps read once, as 16- or 8-byte
// vectors from shared memory, and per tap its CPT weights as float4 vectors
// (weights staged [ci][k][CB]), so that every loaded value feeds several FMAs.
// A transposed conv of stride 1 is the conv with the taps reversed and the
// padding K - 1 - p.  Every output is an FP32 FMA chain over (ci, k), input
// channels in order and taps in order within each.
template <int K, int CPT>
__device__ __forceinline__ void rb_load_w(const float* wr, int CB, int k, float (&wv)[CPT]) {
  if constexpr (CPT % 4 == 0) {
#pragma unroll
    for (int q = 0; q < CPT / 4; ++q) {
      const float4 v = reinterpret_cast<const float4*>(wr + k * CB)[q];
      wv[4 * q] = v.x;
      wv[4 * q + 1] = v.y;
      wv[4 * q + 2] = v.z;
      wv[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int c = 0; c < CPT; ++c) wv[c] = wr[k * CB + c];
  }
}

// Transposed stride 2: output u = t0 + 4 pt + j takes tap k when
// u + p - k is even; with A = t0 + p - (K - 1), lo = floor(A / 2), par = A & 1
// and d = j - k + K - 1, that is when d + par is even, and it reads
// x[lo + 2 pt + (d + par) / 2].
template <int K, int CPT, int PAR>
__device__ __forceinline__ void rb_accum_tr2(const float* xr, const float* wr, int CB, int pt,
                                             float (&acc)[CPT][4]) {
  constexpr int NV2 = ((K + 3) / 2 + 2) / 2;
  float xv[NV2 * 2];
  const float2* x2 = reinterpret_cast<const float2*>(xr + 2 * pt);
#pragma unroll
  for (int q = 0; q < NV2; ++q) {
    const float2 v = x2[q];
    xv[2 * q] = v.x;
    xv[2 * q + 1] = v.y;
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    float wv[CPT];
    rb_load_w<K, CPT>(wr, CB, k, wv);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int d = j - k + K - 1;
      if (((d + PAR) & 1) == 0) {
#pragma unroll
        for (int c = 0; c < CPT; ++c) acc[c][j] = fmaf(wv[c], xv[(d + PAR) >> 1], acc[c][j]);
      }
    }
  }
}

template <int K, int S, bool TR, int CPT>
__global__ void __launch_bounds__(kThreads) conv_f32_rb_kernel(ConvF32Args a, int CB, int CI, int spanp) {
  static_assert(!TR || S == 1 || S == 2, "transposed convs of stride 1 or 2");
  constexpr bool kTr2 = TR && S == 2;   // transposed, stride 2
  constexpr bool kFlip = TR && S == 1;  // transposed, stride 1: reversed taps
  extern __shared__ __align__(16) float smem[];
  const LayerSpec& s = a.s;
  const int ng = CB / CPT, np = kThreads / ng, TL = np * 4;
  const int tid = threadIdx.x, cg = tid / np, pt = tid % np;
  const int t0 = blockIdx.x * TL, co0 = blockIdx.y * CB, b = blockIdx.z;
  const int pad = kFlip ? K - 1 - s.pad_l : s.pad_l;
  int lo, span;
  if constexpr (!kTr2) {
    lo = t0 * S - pad;
    span = (TL - 1) * S + K;
  } else {
    lo = floordiv(t0 + pad - (K - 1), 2);
    span = floordiv(t0 + TL - 1 + pad, 2) - lo + 1;
  }
  const int par = (t0 + pad - (K - 1)) & 1;  // used by kTr2 only
  float* xs = smem;               // [CI][spanp]
  float* ws = smem + CI * spanp;  // [CI][K][CB]
  float acc[CPT][4];
#pragma unroll
  for (int c = 0; c < CPT; ++c)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[c][j] = 0.f;
  const float* xb = a.item_ptr ? a.item_ptr[b] : a.x + (int64_t)b * a.xb;
  for (int ci0 = 0; ci0 < s.cin; ci0 += CI) {
    __syncthreads();
    for (int e = tid; e < CI * spanp; e += kThreads) {
      const int ci = e / spanp, j = e - ci * spanp, t = lo + j, c = ci0 + ci;
      float v = 0.f;
      if (c < s.cin && j < span && t >= 0 && t < a.lin) {
        v = xb[(int64_t)c * a.xc + t];
        if (a.in_mean) v = (v - a.in_mean[c]) * a.in_istd[c];
      }
      xs[e] = v;
    }
    for (int e = tid; e < CI * K * CB; e += kThreads) {
      const int co = e % CB, r = e / CB, k = r % K, ci = r / K;
      const int o = co0 + co, c = ci0 + ci, kk = kFlip ? K - 1 - k : k;
      ws[e] = (o < s.cout && c < s.cin) ? a.w[((int64_t)o * s.cin + c) * K + kk] : 0.f;
    }
    __syncthreads();
    for (int ci = 0; ci < CI; ++ci) {
      const float* xr = xs + ci * spanp;
      const float* wr = ws + ci * K * CB + cg * CPT;
      if constexpr (!kTr2) {
        // output u = t0 + 4 pt + j reads x[lo + (4 pt + j) S + k]
        constexpr int NV = (3 * S + K + 3) / 4 * 4;
        float xv[NV];
        const float4* x4 = reinterpret_cast<const float4*>(xr + 4 * pt * S);
#pragma unroll
        for (int q = 0; q < NV / 4; ++q) {
          const float4 v = x4[q];
          xv[4 * q] = v.x;
          xv[4 * q + 1] = v.y;
          xv[4 * q + 2] = v.z;
          xv[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
          float wv[CPT];
          rb_load_w<K, CPT>(wr, CB, k, wv);
#pragma unroll
          for (int c = 0; c < CPT; ++c)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[c][j] = fmaf(wv[c], xv[j * S + k], acc[c][j]);
        }
      } else {
        if (par == 0)
          rb_accum_tr2<K, CPT, 0>(xr, wr, CB, pt, acc);
        else
          rb_accum_tr2<K, CPT, 1>(xr, wr, CB, pt, acc);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < CPT; ++c) {
    const int o = co0 + cg * CPT + c;
    if (o >= s.cout) continue;
    const float bias = a.bias[o];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int u = t0 + 4 * pt + j;
      if (u >= a.lout) continue;
      float v = acc[c][j] + bias;
      if (a.res) v += a.res[(int64_t)b * a.rb + (int64_t)o * a.rc + u];
      if (a.gy) {
        const float yv = a.gy[(int64_t)b * a.gyb + (int64_t)o * a.gyc + u];
        v *= a.gact == ACT_TANH ? 1.f - yv * yv : (a.gact == ACT_RELU ? (yv > 0.f ? 1.f : 0.f) : 1.f);
      }
      a.y[(int64_t)b * a.yb + (int64_t)o * a.yc + u] = apply_act(v, s.act);
    }
  }
}

// FIR over one row:
//   y[r][n] = scale * sum_k h'[k] x[r][n + k + x_off],  x zero outside [0, x_len),
// h' = h (rev = 0) or h reversed (rev = 1).  Valid mode: x_off = 0,
// x_len = lout + ntaps - 1.  Its adjoint (dx[m] = sum_k h[k] dy[m - k]) is
// x_off = -(ntaps - 1), rev = 1.
// CTA: kFirTile outputs, kFirThreads threads of kFirOut consecutive outputs
// each.  Taps go in blocks of 8 (zero-padded): per block a thread loads the 8
// taps and the 16 inputs its outputs read as float4 vectors from shared
// memory, so that every loaded value feeds 4-8 FMAs.  Each output's sum runs
// over the taps in order.
constexpr int kFirThreads = 128, kFirOut = 8, kFirTile = kFirThreads * kFirOut;
__global__ void __launch_bounds__(kFirThreads) fir_f32_kernel(const float* __restrict__ x, int64_t x_row,
                                                              float* __restrict__ y, int64_t y_row,
                                                              const float* __restrict__ h, int ntaps, int lout,
                                                              int x_off, int x_len, int rev, float scale) {
  extern __shared__ __align__(16) float smem[];
  const int npad = (ntaps + 7) / 8 * 8;
  float* hs = smem;         // [npad]
  float* xs = smem + npad;  // [kFirTile + npad + 8]
  const int r = blockIdx.y, n0 = blockIdx.x * kFirTile;
  const float* xr = x + (int64_t)r * x_row;
  const int span = kFirTile + npad + 8;
  for (int e = threadIdx.x; e < npad; e += kFirThreads) hs[e] = e < ntaps ? h[rev ? ntaps - 1 - e : e] : 0.f;
  for (int e = threadIdx.x; e < span; e += kFirThreads) {
    const int q = n0 + e + x_off;
    xs[e] = (q >= 0 && q < x_len) ? xr[q] : 0.f;
  }
  __syncthreads();
  float acc[kFirOut];
#pragma unroll
  for (int j = 0; j < kFirOut; ++j) acc[j] = 0.f;
  const float* xt = xs + threadIdx.x * kFirOut;
  for (int kb = 0; kb < npad; kb += 8) {
    float hv[8], xv[16];
    const float4 h0 = *reinterpret_cast<const float4*>(hs + kb), h1 = *reinterpret_cast<const float4*>(hs + kb + 4);
    hv[0] = h0.x, hv[1] = h0.y, hv[2] = h0.z, hv[3] = h0.w, hv[4] = h1.x, hv[5] = h1.y, hv[6] = h1.z, hv[7] = h1.w;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 v = *reinterpret_cast<const float4*>(xt + kb + 4 * q);
      xv[4 * q] = v.x, xv[4 * q + 1] = v.y, xv[4 * q + 2] = v.z, xv[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int kk = 0; kk < 8; ++kk)
#pragma unroll
      for (int j = 0; j < kFirOut; ++j) acc[j] = fmaf(hv[kk], xv[j + kk], acc[j]);
  }
#pragma unroll
  for (int j = 0; j < kFirOut; ++j) {
    const int n = n0 + threadIdx.x * kFirOut + j;
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

// Geometry of one register-blocked launch: CB channels x TL positions per CTA,
// CI input channels per shared-memory chunk, x rows padded to spanp floats (a
// multiple of 4, wide enough for the vector loads past the last position).
template <int K, int S, bool TR, int CPT>
bool launch_conv_f32_rb(const ConvF32Args& a, cudaStream_t st) {
  const LayerSpec& s = a.s;
  const int CB = CPT == 1 ? 1 : std::min(64, (s.cout + CPT - 1) / CPT * CPT);
  const int ng = CB / CPT, np = kThreads / ng, TL = np * 4;
  int span_max, need;
  if (TR && S == 2) {
    span_max = TL / 2 + K / 2 + 3;
    need = 2 * (np - 1) + ((K + 3) / 2 + 2) / 2 * 2;
  } else {
    span_max = (TL - 1) * S + K;
    need = 4 * (np - 1) * S + (3 * S + K + 3) / 4 * 4;
  }
  const int spanp = (std::max(span_max, need) + 3) / 4 * 4;
  int CI = 16;
  while (CI > 1 && (size_t)CI * (spanp + K * CB) * 4 > 96 * 1024) CI /= 2;
  const int chunks = (s.cin + CI - 1) / CI;
  CI = (s.cin + chunks - 1) / chunks;
  const size_t smem = (size_t)CI * (spanp + K * CB) * 4;
  if (smem > 96 * 1024) return false;
  set_smem_limit_once(conv_f32_rb_kernel<K, S, TR, CPT>, 96 * 1024);
  dim3 grid((a.lout + TL - 1) / TL, (s.cout + CB - 1) / CB, a.B);
  conv_f32_rb_kernel<K, S, TR, CPT><<<grid, kThreads, smem, st>>>(a, CB, CI, spanp);
  GW_LAUNCH_CHECK();
  return true;
}

void launch_conv_f32(const ConvF32Args& a, cudaStream_t st) {
  const LayerSpec& s = a.s;
  const bool tr = s.transposed;
  bool done = false;
  if (s.k == 7 && s.stride == 1 && !tr)
    done = s.cout == 1 ? launch_conv_f32_rb<7, 1, false, 1>(a, st) : launch_conv_f32_rb<7, 1, false, 8>(a, st);
  else if (s.k == 7 && s.stride == 1 && tr)
    done = s.cout == 1 ? launch_conv_f32_rb<7, 1, true, 1>(a, st) : launch_conv_f32_rb<7, 1, true, 8>(a, st);
  else if (s.k == 7 && s.stride == 2 && !tr)
    done = launch_conv_f32_rb<7, 2, false, 8>(a, st);
  else if (s.k == 7 && s.stride == 2 && tr)
    done = launch_conv_f32_rb<7, 2, true, 8>(a, st);
  else if (s.k == 16 && s.stride == 1 && !tr)
    done = launch_conv_f32_rb<16, 1, false, 8>(a, st);
  else if (s.k == 1 && s.stride == 2 && !tr)
    done = launch_conv_f32_rb<1, 2, false, 8>(a, st);
  GW_CHECK_ARG(done, "layer shape has no FP32 conv kernel (DeepClean and BBHnet shapes only)");
}

void launch_fir_f32(const float* x, int64_t x_row, float* y, int64_t y_row, int rows, const float* taps,
                    int ntaps, int lout, cudaStream_t st, int x_off, int x_len, int rev, float scale) {
  if (x_len < 0) x_len = lout + ntaps - 1;
  const int npad = (ntaps + 7) / 8 * 8;
  const size_t smem = (size_t)(npad + kFirTile + npad + 8) * 4;
  GW_CHECK_ARG(smem <= 200 * 1024, "FIR too long for the FP32 kernel");
  set_smem_limit_once(fir_f32_kernel, 200 * 1024);
  dim3 grid((lout + kFirTile - 1) / kFirTile, rows);
  fir_f32_kernel<<<grid, kFirThreads, smem, st>>>(x, x_row, y, y_row, taps, ntaps, lout, x_off, x_len, rev, scale);
  GW_LAUNCH_CHECK();
}

void launch_gap_linear_f32(const float* h, int64_t hb, int64_t hc, int B, int C, int L, const float* w,
                           const float* b, float* out, cudaStream_t st) {
  gap_linear_f32_kernel<<<B, kThreads, 0, st>>>(h, hb, hc, C, L, w, b, out);
  GW_LAUNCH_CHECK();
}

}  // namespace gw
