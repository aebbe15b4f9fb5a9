// Internal declarations of the serving loop (serve.cu, k_serve.cu).
#pragma once

#include "gw_internal.h"

namespace gw {

// One (snapshot, detector) of a tick.  Items are detector-major: item
// d * Bb + r is detector d of the tick's request r (Bb = the graph's batch
// bucket), so each detector's DeepClean batch is one contiguous run.  The
// state pointers are device memory of the stream; `in`, `out` and `score`
// point into host-mapped pinned request slots.
struct ServeItem {
  int active;         // 0: padding up to the bucket (no state is touched)
  int S;              // stride of the stream
  int64_t head;       // samples pushed before this snapshot
  int64_t m0, m1;     // decimated samples that become computable with it
  int64_t n0, n1;     // whitened samples that become computable (0 <= n0)
  void* wring;        // witness ring (blocked BF16 in P planes, or FP32 [C][2R])
  float* strain;      // strain ring [R]
  float* acc;         // aggregation sums [R]
  float* clean;       // cleaned ring [Rc] (input rate)
  float* dec;         // decimated ring [Rd]
  float* white;       // whitened ring [Rw]
  float* pring;       // with post-processing: aggregated prediction ring [Rp]
  const float* in;    // [C + 1][S]: witness rows, then the strain row
  float* out;         // [S] cleaned samples
  float* score;       // detector 0 only: the request's logit
};

struct ServeGeom {
  int C, G, P, W;     // witness channels, their 8-channel groups, phase planes, window
  int64_t R, Rc, Rd, Rw;
  int bf16;
  int mode, delta;
  int post, post_c;   // post-processing FIR present; its half length c = (K - 1) / 2
  int64_t Rp;
};

void launch_serve_push(const ServeItem* items, int n, const ServeGeom& g, int S_max, const float* mean,
                       const float* istd, cudaStream_t st);
void launch_serve_sub_ola(const ServeItem* items, int n, const ServeGeom& g, const float* pred, cudaStream_t st);
// With post-processing: cleaned samples of the times [head - delta - c,
// head - delta - c + S) from the prediction ring, h the FIR's K taps.
void launch_serve_post(const ServeItem* items, int n, const ServeGeom& g, const float* h, int K, int S_max,
                       cudaStream_t st);
void launch_serve_decimate(const ServeItem* items, int n, const ServeGeom& g, const float* taps, int K,
                           int max_new, cudaStream_t st);
size_t serve_whiten_smem(int K, int max_new);
void launch_serve_whiten(const ServeItem* items, int n, const ServeGeom& g, const float* taps, int K,
                         int max_new, cudaStream_t st);
// BBHnet input [Bb][n_det][Lb] from the whitened rings of items r, Bb + r, ...
void launch_serve_gather(const ServeItem* items, int Bb, int n_det, int Lb, const ServeGeom& g, float* x,
                         cudaStream_t st);
// Logits to the requests' score slots (NaN when logits is null) and the
// tick status (nonzero if *e0 or *e1, the tensor-core error flags, is set).
void launch_serve_scores(const ServeItem* items, int Bb, const float* logits, const int* e0, const int* e1,
                         int* status, cudaStream_t st);

}  // namespace gw
