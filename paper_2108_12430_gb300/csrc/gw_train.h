// Internal declarations of the training path (train.cu, k_train.cu).
#pragma once

#include <algorithm>

#include "gw_internal.h"

namespace gw {

constexpr float kBnEps = 1e-5f;

// One layer's raw parameters inside the flat parameter vector (offsets in
// floats; the BatchNorm ones only when bn) and its folded device copies.
struct FoldArgs {
  const float* p;             // raw parameters (device)
  int64_t off_w, off_b, off_g, off_be, off_mu, off_var;
  int cin, cout, K, transposed, bn;
  float* wf;                  // folded [C_out][C_in][K]
  float* wT;                  // folded, transposed [C_in][C_out][K]
  float* bf;                  // folded bias [C_out]
};

// Weight-gradient GEMM: P[chunk][a][c][k] = sum_t A[b][a][t] Bv(b, c, s t + k - p).
struct WgradArgs {
  const float* A; int64_t ab, aa; int NA, LA;
  const float* Bm; int64_t bb, bc; int NC, LB;
  int K, s, p;
  int AB, T, chunks_per_b, nj;
  float* partial;
  // tensor-core kernel only: also the bias gradient, 1 = sum_t A[a][t] (conv:
  // A is the output gradient), 2 = sum_u Bm[c][u] (transposed conv: Bm is the
  // output gradient; needs LB = s LA and p + s <= K)
  int bias = 0;
};

void launch_fold(const FoldArgs& f, cudaStream_t st);
// Several layers' folds in one launch (at most kFoldMax).
constexpr int kFoldMax = 16;
void launch_fold_many(const FoldArgs* f, int n, cudaStream_t st);
// dw_in_major: dWf is [C_in][C_out][K] (transposed conv) instead of [C_out][C_in][K].
void launch_unfold(const FoldArgs& f, const float* dWf, int dw_in_major, const float* dbf, float* dp,
                   cudaStream_t st);
// Several layers' unfolds in one launch (at most kFoldMax).
struct UnfoldItem {
  FoldArgs f;
  const float* dWf;
  int dw_in_major;
  const float* dbf;
};
void launch_unfold_many(const UnfoldItem* u, int n, float* dp, cudaStream_t st);
WgradArgs plan_wgrad(int NA, int NC, int K, int s, int LA);
size_t wgrad_smem(const WgradArgs& w);
// w.partial must hold B * w.chunks_per_b * NA * NC * K floats; out gets NA * NC * K.
void launch_wgrad_partial(const WgradArgs& w, int B, cudaStream_t st);
void launch_wgrad_reduce(const WgradArgs& w, int B, float* out, cudaStream_t st);
// The same weight gradient on the tensor cores (BF16 operands, FP32
// accumulation; k_wgrad_tc.cu): out gets NA * NC * K floats and, with
// w.bias, db the bias gradient (NA floats for bias 1, NC for bias 2); partial
// must hold wgrad_tc_partial_floats(w, B); err receives a bounded wait's give-up.
bool wgrad_tc_supported(const WgradArgs& w);
size_t wgrad_tc_partial_floats(const WgradArgs& w, int B);
void launch_wgrad_tc(const WgradArgs& w, int B, float* partial, float* out, float* db, int* err, cudaStream_t st);
// out[n] = sum_{b, t} G[b][n][t]; part holds B * N floats.
void launch_bias_grad(const float* G, int64_t gb, int64_t gn, int B, int N, int L, float* part, float* out,
                      cudaStream_t st);
void launch_standardise(const float* x, int B, int C, int L, const float* mean, const float* istd, float* y,
                        cudaStream_t st);
// loss = (1 / (B Lr)) sum r^2 with r = g (*) (strain - y_hat) valid (Lr = L - K + 1);
// e holds B * L floats, r B * Lr, part B.
void launch_band_loss(const float* strain, const float* y_hat, int B, int L, const float* taps, int K, float* e,
                      float* r, float* part, float* loss, cudaStream_t st);
// dy_hat = dloss * d loss / d y_hat (dloss: device scalar, or null for 1).
void launch_band_loss_backward(const float* r, int B, int L, const float* taps, int K, const float* dloss,
                               float* dy_hat, cudaStream_t st);
void launch_adam(float* p, const float* g, float* m, float* v, int64_t n, int step, float lr, float b1, float b2,
                 float eps, cudaStream_t st);
// Adam with the step count in device memory (incremented by the first of two launches).
void launch_adam_dev(float* p, const float* g, float* m, float* v, int64_t n, int* step, float lr, float b1,
                     float b2, float eps, cudaStream_t st);

}  // namespace gw
