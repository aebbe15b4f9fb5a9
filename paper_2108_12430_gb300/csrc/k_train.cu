// Training kernels (FP32): BatchNorm fold and its chain rule, weight and bias
// gradients of conv / transposed-conv layers, the band-limited loss and Adam.
//
// Data gradients reuse the forward conv kernel (a conv's data gradient is a
// transposed conv with the transposed weights and vice versa), with the
// activation derivative fused into its epilogue.  Every reduction here runs
// in a fixed order (per-chunk partials, then a sum over chunks), so a
// gradient is bitwise reproducible.
#include "gw_train.h"

namespace gw {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxJ = 32;  // weight-gradient outputs per thread

__device__ __forceinline__ float block_sum(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x == 0)
    for (int i = 0; i < nw; ++i) t += red[i];
  return t;  // valid in thread 0
}

// Folded weights of one layer in the device layout [C_out][C_in][K] (wf),
// the same values transposed to [C_in][C_out][K] (wT, the data-gradient
// kernel's weights) and the folded bias (bf):
//   sc[o] = gamma[o] / sqrt(var[o] + eps),  w' = w sc[o],  b' = (b - mean) sc + beta.
__device__ __forceinline__ void fold_body(const FoldArgs& f) {
  const int n = f.cout * f.cin * f.K;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int k = e % f.K, oi = e / f.K, i = oi % f.cin, o = oi / f.cin;
    const int64_t raw = f.transposed ? ((int64_t)i * f.cout + o) * f.K + k : e;
    double sc = 1.0;
    if (f.bn) sc = (double)f.p[f.off_g + o] / sqrt((double)f.p[f.off_var + o] + (double)kBnEps);
    const float w = (float)((double)f.p[f.off_w + raw] * sc);
    f.wf[e] = w;
    f.wT[((int64_t)i * f.cout + o) * f.K + k] = w;
  }
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < f.cout; o += gridDim.x * blockDim.x) {
    const double b = f.p[f.off_b + o];
    if (f.bn) {
      const double sc = (double)f.p[f.off_g + o] / sqrt((double)f.p[f.off_var + o] + (double)kBnEps);
      f.bf[o] = (float)((b - (double)f.p[f.off_mu + o]) * sc + (double)f.p[f.off_be + o]);
    } else {
      f.bf[o] = (float)b;
    }
  }
}
__global__ void fold_kernel(FoldArgs f) { fold_body(f); }
// Every layer's fold in one launch (blockIdx.y = layer).
struct FoldList {
  FoldArgs f[kFoldMax];
};
__global__ void fold_many_kernel(const __grid_constant__ FoldList l) { fold_body(l.f[blockIdx.y]); }

// Chain rule from the folded parameters' gradients (dWf in the layer's
// gradient layout, dbf) to the raw ones; one CTA per output channel o:
//   dw = dWf sc,  db = dbf sc,  dbeta = dbf,
//   dgamma = a (sum_{i,k} w dWf + dbf (b - mean)),  a = 1 / sqrt(var + eps);
// running mean and variance are not trained (gradient 0).
__device__ __forceinline__ void unfold_body(const FoldArgs& f, const float* __restrict__ dWf, int dw_in_major,
                                            const float* __restrict__ dbf, float* __restrict__ dp, int o) {
  __shared__ float red[kThreads / 32];
  const double a = f.bn ? 1.0 / sqrt((double)f.p[f.off_var + o] + (double)kBnEps) : 1.0;
  const double sc = f.bn ? (double)f.p[f.off_g + o] * a : 1.0;
  float dot = 0.f;
  for (int j = threadIdx.x; j < f.cin * f.K; j += blockDim.x) {
    const int i = j / f.K, k = j % f.K;
    const int64_t g = dw_in_major ? ((int64_t)i * f.cout + o) * f.K + k : ((int64_t)o * f.cin + i) * f.K + k;
    const int64_t raw = f.transposed ? ((int64_t)i * f.cout + o) * f.K + k : ((int64_t)o * f.cin + i) * f.K + k;
    const float d = dWf[g];
    dp[f.off_w + raw] = (float)((double)d * sc);
    dot = fmaf(f.p[f.off_w + raw], d, dot);
  }
  dot = block_sum(dot, red);
  if (threadIdx.x == 0) {
    const double db = dbf[o];
    dp[f.off_b + o] = (float)(db * sc);
    if (f.bn) {
      dp[f.off_g + o] = (float)(a * ((double)dot + db * ((double)f.p[f.off_b + o] - (double)f.p[f.off_mu + o])));
      dp[f.off_be + o] = (float)db;
      dp[f.off_mu + o] = 0.f;
      dp[f.off_var + o] = 0.f;
    }
  }
}

__global__ void unfold_kernel(FoldArgs f, const float* __restrict__ dWf, int dw_in_major,
                              const float* __restrict__ dbf, float* __restrict__ dp) {
  unfold_body(f, dWf, dw_in_major, dbf, dp, blockIdx.x);
}

// Several layers' unfolds in one launch: block (o, i) is output channel o of
// layer i.
struct UnfoldList {
  UnfoldItem u[kFoldMax];
};
__global__ void unfold_many_kernel(const __grid_constant__ UnfoldList l, float* __restrict__ dp) {
  const UnfoldItem& u = l.u[blockIdx.y];
  if ((int)blockIdx.x >= u.f.cout) return;
  unfold_body(u.f, u.dWf, u.dw_in_major, u.dbf, dp, blockIdx.x);
}

// Weight-gradient partials of one chunk of (item, positions):
//   P[chunk][a][c][k] = sum_{t in chunk} A[b][a][t] Bv(b, c, s t + k - p),
// Bv = Bm inside [0, LB), 0 outside.  Conv: A = output gradient, Bm = input;
// transposed conv: A = input, Bm = output gradient.  CTA: AB values of a (a
// power of two), all (c, k), T positions; the A tile (rows padded by one
// float against bank conflicts) and the B span sit in shared memory.  Thread:
// one a (AB groups of 256 / AB threads) and NJ of the (c, k) outputs, so one
// A value feeds NJ multiply-adds per position.  NJ is a compile-time bound
// (>= w.nj) so that the inner loop has no idle slots.
template <int NJ>
__global__ void __launch_bounds__(kThreads) wgrad_partial_kernel(WgradArgs w) {
  extern __shared__ float sm[];
  const int chunk = blockIdx.x, b = chunk / w.chunks_per_b, t0 = (chunk % w.chunks_per_b) * w.T;
  const int a0 = blockIdx.y * w.AB;
  const int span = w.s * (w.T - 1) + w.K;
  const int as = w.T + 1;
  float* As = sm;                 // [AB][T + 1]
  float* Bs = sm + w.AB * as;     // [NC][span]
  const int q0 = w.s * t0 - w.p;
  for (int e = threadIdx.x; e < w.AB * w.T; e += blockDim.x) {
    const int al = e / w.T, t = e % w.T;
    const int a = a0 + al, tt = t0 + t;
    As[al * as + t] = (a < w.NA && tt < w.LA) ? w.A[(int64_t)b * w.ab + (int64_t)a * w.aa + tt] : 0.f;
  }
  for (int e = threadIdx.x; e < w.NC * span; e += blockDim.x) {
    const int c = e / span, q = q0 + e % span;
    Bs[e] = (q >= 0 && q < w.LB) ? w.Bm[(int64_t)b * w.bb + (int64_t)c * w.bc + q] : 0.f;
  }
  __syncthreads();
  const int tpa = kThreads / w.AB;          // threads per a
  const int al = threadIdx.x / tpa, ck0 = threadIdx.x % tpa;
  const int nck = w.NC * w.K;
  float acc[NJ];
  int boff[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    acc[j] = 0.f;
    const int ck = ck0 + j * tpa;
    boff[j] = ck < nck ? (ck / w.K) * span + ck % w.K : 0;
  }
  const float* arow = As + al * as;
  const int tmax = min(w.T, w.LA - t0);
  const int s = w.s;
  for (int t = 0; t < tmax; ++t) {
    const float av = arow[t];
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[j] = fmaf(av, Bs[boff[j] + s * t], acc[j]);
  }
  if (a0 + al < w.NA) {
    float* out = w.partial + (int64_t)chunk * w.NA * nck + (int64_t)(a0 + al) * nck;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int ck = ck0 + j * tpa;
      if (ck < nck) out[ck] = acc[j];
    }
  }
}

// out[e] = sum_{ch < n_chunks} P[ch][e] in chunk order.
__global__ void reduce_chunks_kernel(const float* __restrict__ P, int64_t n, int n_chunks, float* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int c = 0; c < n_chunks; ++c) s += P[(int64_t)c * n + e];
    out[e] = s;
  }
}

// part[b][n] = sum_t G[b][n][t] (one CTA per (n, b)).
__global__ void rowsum_kernel(const float* __restrict__ G, int64_t gb, int64_t gn, int L, int N,
                              float* __restrict__ part) {
  __shared__ float red[kThreads / 32];
  const int n = blockIdx.x, b = blockIdx.y;
  const float* row = G + (int64_t)b * gb + (int64_t)n * gn;
  float s = 0.f;
  for (int t = threadIdx.x; t < L; t += blockDim.x) s += row[t];
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[(int64_t)b * N + n] = s;
}

// x_std[b][c][t] = (x[b][c][t] - mean[c]) / std[c]
__global__ void standardise_kernel(const float* __restrict__ x, int64_t n, int C, int L, const float* __restrict__ mean,
                                   const float* __restrict__ istd, float* __restrict__ y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)((e / L) % C);
    y[e] = (x[e] - mean[c]) * istd[c];
  }
}

__global__ void diff_kernel(const float* __restrict__ s, const float* __restrict__ y, int64_t n, float* __restrict__ e) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    e[i] = s[i] - y[i];
}

// part[b] = sum_n r[b][n]^2 (one CTA per row)
__global__ void sumsq_rows_kernel(const float* __restrict__ r, int Lr, float* __restrict__ part) {
  __shared__ float red[kThreads / 32];
  const float* row = r + (int64_t)blockIdx.x * Lr;
  float s = 0.f;
  for (int t = threadIdx.x; t < Lr; t += blockDim.x) s = fmaf(row[t], row[t], s);
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void loss_final_kernel(const float* __restrict__ part, int B, float inv_n, float* __restrict__ loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += part[b];
    *loss = s * inv_n;
  }
}

__global__ void scale_by_kernel(float* __restrict__ x, int64_t n, const float* __restrict__ s) {
  const float v = *s;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= v;
}

// Adam with bias correction (Kingma & Ba, Algorithm 1), FP32 state.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// The same update with the step count t read from device memory (bias
// corrections 1 - b1^t, 1 - b2^t worked out per thread), after
// adam_count_kernel has incremented it.
__global__ void adam_dev_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                                const int* __restrict__ step) {
  const float t = (float)*step;
  const float c1 = 1.f - powf(b1, t), c2 = 1.f - powf(b2, t);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}
__global__ void adam_count_kernel(int* step) { *step += 1; }

int grid_for(int64_t n) {
  const int64_t b = (n + kThreads - 1) / kThreads;
  return (int)std::min<int64_t>(std::max<int64_t>(b, 1), 1216);
}

}  // namespace

void launch_fold(const FoldArgs& f, cudaStream_t st) {
  fold_kernel<<<grid_for((int64_t)f.cout * f.cin * f.K), kThreads, 0, st>>>(f);
  GW_LAUNCH_CHECK();
}

void launch_fold_many(const FoldArgs* f, int n, cudaStream_t st) {
  GW_CHECK_ARG(n >= 1 && n <= kFoldMax, "fold list size");
  FoldList l{};
  int64_t mx = 0;
  for (int i = 0; i < n; ++i) {
    l.f[i] = f[i];
    mx = std::max<int64_t>(mx, (int64_t)f[i].cout * f[i].cin * f[i].K);
  }
  fold_many_kernel<<<dim3(grid_for(mx), n), kThreads, 0, st>>>(l);
  GW_LAUNCH_CHECK();
}

void launch_unfold(const FoldArgs& f, const float* dWf, int dw_in_major, const float* dbf, float* dp, cudaStream_t st) {
  unfold_kernel<<<f.cout, kThreads, 0, st>>>(f, dWf, dw_in_major, dbf, dp);
  GW_LAUNCH_CHECK();
}

void launch_unfold_many(const UnfoldItem* u, int n, float* dp, cudaStream_t st) {
  GW_CHECK_ARG(n >= 1 && n <= kFoldMax, "unfold list size");
  UnfoldList l{};
  int mx = 1;
  for (int i = 0; i < n; ++i) {
    l.u[i] = u[i];
    mx = std::max(mx, u[i].f.cout);
  }
  unfold_many_kernel<<<dim3(mx, n), kThreads, 0, st>>>(l, dp);
  GW_LAUNCH_CHECK();
}

WgradArgs plan_wgrad(int NA, int NC, int K, int s, int LA) {
  WgradArgs w{};
  w.NA = NA;
  w.NC = NC;
  w.K = K;
  w.s = s;
  w.LA = LA;
  // AB: the largest power of two <= min(16, NA) whose thread groups still
  // cover the (c, k) outputs with at most kMaxJ per thread
  w.AB = 1;
  while (w.AB * 2 <= std::min(16, NA) && (NC * K + kThreads / (w.AB * 2) - 1) / (kThreads / (w.AB * 2)) <= kMaxJ)
    w.AB *= 2;
  w.T = 256;
  while (w.T > 32 && wgrad_smem(w) > 160 * 1024) w.T /= 2;
  w.chunks_per_b = (LA + w.T - 1) / w.T;
  const int tpa = kThreads / w.AB;
  w.nj = (NC * K + tpa - 1) / tpa;
  return w;
}

size_t wgrad_smem(const WgradArgs& w) {
  return ((size_t)w.AB * (w.T + 1) + (size_t)w.NC * (w.s * (w.T - 1) + w.K)) * sizeof(float);
}

void launch_wgrad_partial(const WgradArgs& w, int B, cudaStream_t st) {
  GW_CHECK_ARG(w.nj <= kMaxJ, "weight gradient tile too large");
  const size_t smem = wgrad_smem(w);
  GW_CHECK_ARG(smem <= 200 * 1024, "weight gradient tile exceeds shared memory");
  set_smem_limit_once(wgrad_partial_kernel<1>, 200 * 1024);
  set_smem_limit_once(wgrad_partial_kernel<2>, 200 * 1024);
  set_smem_limit_once(wgrad_partial_kernel<4>, 200 * 1024);
  set_smem_limit_once(wgrad_partial_kernel<8>, 200 * 1024);
  set_smem_limit_once(wgrad_partial_kernel<16>, 200 * 1024);
  set_smem_limit_once(wgrad_partial_kernel<32>, 200 * 1024);
  const int n_chunks = B * w.chunks_per_b;
  dim3 grid(n_chunks, (w.NA + w.AB - 1) / w.AB);
  if (w.nj <= 1)
    wgrad_partial_kernel<1><<<grid, kThreads, smem, st>>>(w);
  else if (w.nj <= 2)
    wgrad_partial_kernel<2><<<grid, kThreads, smem, st>>>(w);
  else if (w.nj <= 4)
    wgrad_partial_kernel<4><<<grid, kThreads, smem, st>>>(w);
  else if (w.nj <= 8)
    wgrad_partial_kernel<8><<<grid, kThreads, smem, st>>>(w);
  else if (w.nj <= 16)
    wgrad_partial_kernel<16><<<grid, kThreads, smem, st>>>(w);
  else
    wgrad_partial_kernel<32><<<grid, kThreads, smem, st>>>(w);
  GW_LAUNCH_CHECK();
}

void launch_wgrad_reduce(const WgradArgs& w, int B, float* out, cudaStream_t st) {
  const int n_chunks = B * w.chunks_per_b;
  const int64_t n = (int64_t)w.NA * w.NC * w.K;
  reduce_chunks_kernel<<<grid_for(n), kThreads, 0, st>>>(w.partial, n, n_chunks, out);
  GW_LAUNCH_CHECK();
}

void launch_bias_grad(const float* G, int64_t gb, int64_t gn, int B, int N, int L, float* part, float* out,
                      cudaStream_t st) {
  rowsum_kernel<<<dim3(N, B), kThreads, 0, st>>>(G, gb, gn, L, N, part);
  GW_LAUNCH_CHECK();
  reduce_chunks_kernel<<<grid_for(N), kThreads, 0, st>>>(part, N, B, out);
  GW_LAUNCH_CHECK();
}

void launch_standardise(const float* x, int B, int C, int L, const float* mean, const float* istd, float* y,
                        cudaStream_t st) {
  const int64_t n = (int64_t)B * C * L;
  standardise_kernel<<<grid_for(n), kThreads, 0, st>>>(x, n, C, L, mean, istd, y);
  GW_LAUNCH_CHECK();
}

void launch_band_loss(const float* strain, const float* y_hat, int B, int L, const float* taps, int K, float* e,
                      float* r, float* part, float* loss, cudaStream_t st) {
  const int64_t n = (int64_t)B * L;
  diff_kernel<<<grid_for(n), kThreads, 0, st>>>(strain, y_hat, n, e);
  GW_LAUNCH_CHECK();
  const int Lr = L - K + 1;
  launch_fir_f32(e, L, r, Lr, B, taps, K, Lr, st);
  sumsq_rows_kernel<<<B, kThreads, 0, st>>>(r, Lr, part);
  GW_LAUNCH_CHECK();
  loss_final_kernel<<<1, 32, 0, st>>>(part, B, 1.f / ((float)B * (float)Lr), loss);
  GW_LAUNCH_CHECK();
}

void launch_band_loss_backward(const float* r, int B, int L, const float* taps, int K, const float* dloss,
                               float* dy_hat, cudaStream_t st) {
  const int Lr = L - K + 1;
  // dL/dy_hat[m] = -(2 / N) sum_k g[k] r[m - k]: the FIR's adjoint of r
  launch_fir_f32(r, Lr, dy_hat, L, B, taps, K, L, st, -(K - 1), Lr, 1, -2.f / ((float)B * (float)Lr));
  if (dloss) {
    const int64_t n = (int64_t)B * L;
    scale_by_kernel<<<grid_for(n), kThreads, 0, st>>>(dy_hat, n, dloss);
    GW_LAUNCH_CHECK();
  }
}

void launch_adam_dev(float* p, const float* g, float* m, float* v, int64_t n, int* step, float lr, float b1,
                     float b2, float eps, cudaStream_t st) {
  adam_count_kernel<<<1, 1, 0, st>>>(step);
  GW_LAUNCH_CHECK();
  adam_dev_kernel<<<grid_for(n), kThreads, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, step);
  GW_LAUNCH_CHECK();
}

void launch_adam(float* p, const float* g, float* m, float* v, int64_t n, int step, float lr, float b1, float b2,
                 float eps, cudaStream_t st) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<grid_for(n), kThreads, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
  GW_LAUNCH_CHECK();
}

}  // namespace gw
