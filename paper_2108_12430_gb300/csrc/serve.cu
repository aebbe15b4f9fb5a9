// Serving loop: continuous batching of snapshots from many streams.
//
// The paper's inference service keeps each stream's snapshot state on the
// GPU and answers many concurrent clients whose requests carry only the new
// samples (Methods, "Streaming IaaS", "Online Deployment"); its end-to-end
// ensemble cleans both detectors with DeepClean, resamples, whitens and
// scores with BBHnet ("Offline Deployment").  Here one host loop thread forms
// ticks: it takes the oldest pending snapshot of each stream (at most one per
// stream, so a stream's snapshots run in order), up to max_batch, fills a tick
// table and launches the tick as one CUDA graph for the batch rounded up to a
// bucket.  A completion thread waits for ticks in order, hands results to the
// callers and records latency.  While tick k runs on the device the loop
// already forms tick k+1 from the requests that arrived meanwhile.
//
// Memory: request inputs and outputs live in pinned, device-mapped host
// slots that the kernels read and write directly (no per-request copies);
// each open stream owns one device block with its rings; the tick workspace
// (activations, predictions, BBHnet buffers, tables) is allocated at create.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <set>
#include <thread>

#include "gw_serve.h"

namespace gw {

namespace {

constexpr int kMaxInflight = 4;

double now_us() {
  return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

struct Req {
  int stream = -1;
  uint64_t ticket = 0;
  double t_arrival = 0;   // submit time (or the scheduled arrival of a replay)
  float* in = nullptr;    // pinned: [n_det][C + 1][S]
  float* out = nullptr;   // pinned: [n_det][S], then the score at n_det * S_max
  float* in_dev = nullptr;   // the same slots as device addresses
  float* out_dev = nullptr;
  float* clean_out = nullptr;
  float* score_out = nullptr;
  double* lat_out = nullptr;
};

struct Stream {
  bool open = false;
  int S = 0;
  int64_t k_sched = 0;   // snapshots placed in ticks
  int64_t me = 0;        // decimated samples computable after the last scheduled snapshot
  int64_t ne = 0;        // whitened samples computable (may be negative)
  int pending = 0;       // submitted, not yet scheduled
  int64_t mark = -1;     // last tick this stream was placed in
  int inflight = 0;      // scheduled, not yet completed
  char* block = nullptr;
  size_t bytes = 0;
  void* wring[2] = {};
  float* strain[2] = {};
  float* acc[2] = {};
  float* clean[2] = {};
  float* dec[2] = {};
  float* white[2] = {};
  float* pring[2] = {};
};

struct Tick {
  int slot = 0, n = 0, bucket = 0, bi = 0;
  int64_t kernels = 0;
  double t_launch = 0;  // host time of the launch
  double t_a_end = 0;   // expected end of the first stage (it starts after the previous tick's first stage)
  double t_expect = 0;  // expected completion (its second stage starts after the previous tick's)
  std::vector<int> reqs;
};

}  // namespace
}  // namespace gw

struct gw_server {
  gw_ctx* ctx = nullptr;
  gw_server_desc d{};
  gw_model* dc[2] = {nullptr, nullptr};
  gw_model* bbh = nullptr;
  gw_fir* fdec = nullptr;
  gw_fir* fwht = nullptr;
  gw_fir* fpost = nullptr;
  gw::ServeGeom geom{};
  int prec = 0, Kf = 0, Kh = 0, Lb = 0, max_new = 0, n_slots = 0;
  std::vector<int> buckets;

  // device workspace
  std::vector<std::pair<void*, size_t>> allocs;
  size_t bytes = 0;
  float* pred = nullptr;
  void* act[2][2] = {};
  float* bbh_x = nullptr;
  float* logits = nullptr;
  char* bbh_ws = nullptr;
  int* d_err = nullptr;
  char* dummy = nullptr;
  gw::ServeItem* d_items[gw::kMaxInflight] = {};
  void** d_ptrs[gw::kMaxInflight] = {};
  // pinned host
  std::vector<void*> host_allocs;
  gw::ServeItem* h_items[gw::kMaxInflight] = {};
  void** h_ptrs[gw::kMaxInflight] = {};
  int* h_status = nullptr;
  int* d_status = nullptr;
  float* req_in = nullptr;
  float* req_out = nullptr;
  size_t req_in_elems = 0, req_out_elems = 0;

  cudaStream_t st = nullptr, side = nullptr, st2 = nullptr;  // st2: the ticks' second stage
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  cudaEvent_t done_ev[gw::kMaxInflight] = {};
  // per slot: first stage starts / ends, second stage starts (done_ev: ends)
  cudaEvent_t start_ev[gw::kMaxInflight] = {}, mid_ev[gw::kMaxInflight] = {}, bstart_ev[gw::kMaxInflight] = {};
  std::vector<cudaGraphExec_t> graphs;    // [bucket][slot]: first stage
  std::vector<cudaGraphExec_t> graphs_b;  // [bucket][slot]: second stage
  std::vector<int64_t> graph_kernels;   // per bucket

  // host state (guarded by mu)
  std::mutex mu;
  std::condition_variable cv_loop, cv_done, cv_free, cv_complete;
  std::vector<gw::Stream> streams;
  std::vector<gw::Req> reqs;
  std::vector<int> free_reqs;
  std::deque<int> queue;
  std::set<uint64_t> active;
  uint64_t next_ticket = 1;
  std::deque<gw::Tick> inflight;
  int64_t tick_seq = 0;
  std::vector<double> dur_us;    // per bucket: running estimate of a tick's first-stage device time (0 = none yet)
  std::vector<double> dur_b_us;  // ... and of its second stage
  bool stop = false, loop_done = false;
  int sticky = 0;
  std::string sticky_msg;
  // statistics
  std::vector<double> lat;
  size_t lat_next = 0;
  int64_t st_snap = 0, st_ticks = 0, st_kernels = 0;
  double st_batch_sum = 0, t_first = -1, t_last = 0;
  double st_max_dev = 0, st_max_wait = 0, st_max_late = 0, st_max_call = 0;  // gw_server_stats' maxima

  std::thread loop_th, done_th;
};

namespace gw {

namespace {

constexpr size_t kLatKeep = 1 << 20;

template <typename T>
T* walloc(gw_server* s, size_t count) {
  const size_t b = std::max<size_t>(count * sizeof(T), 256);
  T* p = (T*)dev_alloc(s->ctx, b, &s->bytes);
  s->allocs.push_back({p, b});
  GW_CUDA(cudaMemset(p, 0, b));
  return p;
}

template <typename T>
T* halloc(gw_server* s, size_t count) {
  void* p = nullptr;
  GW_CUDA(cudaHostAlloc(&p, std::max<size_t>(count * sizeof(T), 64), cudaHostAllocMapped | cudaHostAllocPortable));
  s->host_allocs.push_back(p);
  memset(p, 0, std::max<size_t>(count * sizeof(T), 64));
  return (T*)p;
}

template <typename T>
T* dptr(T* host) {
  void* p = nullptr;
  GW_CUDA(cudaHostGetDevicePointer(&p, host, 0));
  return (T*)p;
}

// Bytes of one detector's state, each part 256-byte aligned.
struct StateLayout {
  size_t wring, strain, acc, clean, dec, white, pring, det;
};
StateLayout state_layout(const gw_server* s) {
  const ServeGeom& g = s->geom;
  StateLayout L{};
  L.wring = round_up(g.bf16 ? (int64_t)g.G * 2 * g.R * 8 * 2 : (int64_t)g.C * 2 * g.R * 4, 256);
  L.strain = round_up(g.R * 4, 256);
  L.acc = round_up(g.R * 4, 256);
  L.clean = round_up(g.Rc * 4, 256);
  L.dec = round_up(g.Rd * 4, 256);
  L.white = round_up(g.Rw * 4, 256);
  L.pring = g.post ? round_up(g.Rp * 4, 256) : 0;
  L.det = L.wring + L.strain + L.acc + L.clean + L.dec + L.white + L.pring;
  return L;
}

// Decimated samples computable once the cleaned series is known below c_end.
int64_t m_end(int64_t c_end, int Kf) {
  const int64_t hf = (Kf - 1) / 2;
  return c_end >= hf + 1 ? (c_end - hf - 1) / 2 + 1 : 0;
}

// Address of the first row of a window starting at ring position p0.
void* window_ptr(const gw_server* s, void* ring, int64_t p0) {
  const ServeGeom& g = s->geom;
  if (g.bf16) return (char*)ring + (p0 / g.P) * 16;
  return (float*)ring + p0;
}

// Enqueues the first stage of one tick of bucket Bb using table slot `slot`
// (the tick table upload and both detectors' branches: ring update,
// DeepClean, subtraction, resampling, whitening) on streams a (main) and b
// (second detector's branch, joined back into a).
void record_tick_a(gw_server* s, int Bb, int slot, cudaStream_t a, cudaStream_t b) {
  const ServeGeom& g = s->geom;
  const int nd = s->d.n_det, Bmax = s->d.max_batch, W = s->d.window;
  ServeItem* items = s->d_items[slot];
  void** ptrs = s->d_ptrs[slot];
  GW_CUDA(cudaMemcpyAsync(s->d_items[slot], s->h_items[slot], sizeof(ServeItem) * nd * Bb, cudaMemcpyHostToDevice, a));
  GW_CUDA(cudaMemcpyAsync(s->d_ptrs[slot], s->h_ptrs[slot], sizeof(void*) * nd * Bb, cudaMemcpyHostToDevice, a));
  if (nd == 2) {
    GW_CUDA(cudaEventRecord(s->fork_ev, a));
    GW_CUDA(cudaStreamWaitEvent(b, s->fork_ev, 0));
  }
  for (int det = 0; det < nd; ++det) {
    cudaStream_t sd = det == 0 ? a : b;
    gw_model* m = s->dc[det];
    const ServeItem* it = items + det * Bb;
    float* pred = s->pred + (size_t)det * Bmax * W;
    {
      Prof p("serve_push", sd);
      launch_serve_push(it, Bb, g, s->d.max_stride, m->in_mean, m->in_istd, sd);
    }
    if (s->prec == GW_FP32) {
      deepclean_f32(m, nullptr, 0, 2 * g.R, false, Bb, W, pred, W, (float*)s->act[det][0], (float*)s->act[det][1],
                    sd, (const float* const*)(ptrs + det * Bb));
    } else {
      TcIn in{};
      in.p = s->dummy;
      in.gstride = 2 * g.R * 8;
      in.pstride = (2 * g.R / g.P) * 8;
      in.P = g.P;
      in.L = W;
      in.item_ptr = (const void* const*)(ptrs + det * Bb);
      // the ring update before this launch writes each window's newest S <=
      // max_stride samples: tiles that read only older ones start under it
      deepclean_tc(m, in, Bb, W, pred, W, s->act[det][0], s->act[det][1], s->d_err, sd, W - s->d.max_stride, 0);
    }
    {
      Prof p("serve_sub_ola", sd);
      launch_serve_sub_ola(it, Bb, g, pred, sd);
    }
    if (g.post) {
      Prof p("serve_post", sd);
      launch_serve_post(it, Bb, g, s->fpost->d_taps, s->fpost->ntaps, s->d.max_stride, sd);
    }
    {
      Prof p("serve_decimate", sd);
      launch_serve_decimate(it, Bb, g, s->fdec->d_taps, s->Kf, s->max_new, sd);
    }
    {
      Prof p("serve_whiten", sd);
      launch_serve_whiten(it, Bb, g, s->fwht->d_taps, s->Kh, s->max_new, sd);
    }
  }
  if (nd == 2) {
    GW_CUDA(cudaEventRecord(s->join_ev, b));
    GW_CUDA(cudaStreamWaitEvent(a, s->join_ev, 0));
  }
}

// Enqueues the second stage of the tick (BBHnet on the newest whitened
// samples and the scores) on stream a.  It reads only the whitened rings' last
// bbh_len samples and the slot's table, so the next tick's first stage (which
// writes newer whitened samples) may run beside it.
void record_tick_b(gw_server* s, int Bb, int slot, cudaStream_t a) {
  const ServeGeom& g = s->geom;
  const int nd = s->d.n_det;
  ServeItem* items = s->d_items[slot];
  if (s->bbh) {
    {
      Prof p("serve_gather", a);
      launch_serve_gather(items, Bb, nd, s->Lb, g, s->bbh_x, a);
    }
    if (s->bbh->precision == GW_FP32)
      bbhnet_f32(s->bbh, s->bbh_x, Bb, s->Lb, s->logits, (float*)s->bbh_ws, a);
    else if (s->bbh->precision == GW_BF16)
      bbhnet_tc(s->bbh, s->bbh_x, Bb, s->Lb, s->logits, s->bbh_ws, a);
    else
      bbhnet_fp8(s->bbh, s->bbh_x, Bb, s->Lb, s->logits, s->bbh_ws, a);
  }
  Prof p("serve_scores", a);
  launch_serve_scores(items, Bb, s->bbh ? s->logits : nullptr, s->d_err, s->bbh ? s->bbh->err : nullptr,
                      s->d_status + slot, a);
}

int64_t graph_kernel_count(cudaGraph_t g) {
  size_t n = 0;
  GW_CUDA(cudaGraphGetNodes(g, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  GW_CUDA(cudaGraphGetNodes(g, nodes.data(), &n));
  int64_t k = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    GW_CUDA(cudaGraphNodeGetType(nd, &t));
    if (t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

void capture_graphs(gw_server* s) {
  const int nb = (int)s->buckets.size();
  s->graphs.assign((size_t)nb * s->n_slots, nullptr);
  s->graphs_b.assign((size_t)nb * s->n_slots, nullptr);
  s->graph_kernels.assign(nb, 0);
  cudaStream_t cs = nullptr, cb = nullptr;
  GW_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  GW_CUDA(cudaStreamCreateWithFlags(&cb, cudaStreamNonBlocking));
  struct Guard {
    cudaStream_t a, b;
    ~Guard() {
      prof_set_capturing(false);
      cudaStreamDestroy(a);
      cudaStreamDestroy(b);
    }
  } guard{cs, cb};
  auto capture = [&](int bi, int slot, bool second) {
    cudaGraph_t graph = nullptr;
    prof_set_capturing(true);
    GW_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    try {
      if (second)
        record_tick_b(s, s->buckets[bi], slot, cs);
      else
        record_tick_a(s, s->buckets[bi], slot, cs, cb);
    } catch (...) {
      cudaStreamEndCapture(cs, &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
    GW_CUDA(cudaStreamEndCapture(cs, &graph));
    prof_set_capturing(false);
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    const int64_t kern = e == cudaSuccess ? graph_kernel_count(graph) : 0;
    cudaGraphDestroy(graph);
    GW_CUDA(e);
    (second ? s->graphs_b : s->graphs)[(size_t)bi * s->n_slots + slot] = exec;
    return kern;
  };
  for (int bi = 0; bi < nb; ++bi)
    for (int slot = 0; slot < s->n_slots; ++slot)  // every slot's graphs hold the same kernels
      s->graph_kernels[bi] = capture(bi, slot, false) + capture(bi, slot, true);
}

int bucket_index(const gw_server* s, int n) {
  for (size_t i = 0; i < s->buckets.size(); ++i)
    if (s->buckets[i] >= n) return (int)i;
  return (int)s->buckets.size() - 1;
}

// Fills the pinned tick table of `t` (called without the lock; the stream
// fields it reads were fixed when the tick was formed).
void fill_table(gw_server* s, const Tick& t, const std::vector<ServeItem>& proto) {
  const int nd = s->d.n_det, Bb = t.bucket;
  ServeItem* items = s->h_items[t.slot];
  void** ptrs = s->h_ptrs[t.slot];
  for (int det = 0; det < nd; ++det)
    for (int r = 0; r < Bb; ++r) {
      const int i = det * Bb + r;
      if (r < t.n) {
        items[i] = proto[(size_t)det * t.n + r];
        const int64_t p0 = ((items[i].head + items[i].S - s->d.window) % s->geom.R + s->geom.R) % s->geom.R;
        ptrs[i] = window_ptr(s, items[i].wring, p0);
      } else {
        items[i] = ServeItem{};
        ptrs[i] = s->dummy;
      }
    }
}

void fail_all_locked(gw_server* s, int code, const std::string& msg) {
  if (!s->sticky) {
    s->sticky = code;
    s->sticky_msg = msg;
  }
}

void loop_main(gw_server* s) {
  cudaSetDevice(s->ctx->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv_loop.wait(lk, [&] {
      return (s->stop && s->queue.empty()) ||
             (!s->queue.empty() && (int)s->inflight.size() < s->n_slots);
    });
    if (s->queue.empty()) break;  // stopping and drained
    // just-in-time formation: while a tick runs, wait until the next one can
    // start within form_lead_us - its first stage once the running tick's
    // first stage has ended, timed so that it ends when the running tick's
    // second stage does - (or a full batch is queued), so that snapshots
    // arriving meanwhile join the next tick instead of the one after it
    if (s->d.form_lead_us > 0) {
      while (!s->stop && !s->inflight.empty() && (int)s->queue.size() < s->d.max_batch) {
        const Tick& last = s->inflight.back();
        const double ready = std::max(last.t_a_end, last.t_expect - s->dur_us[last.bi]) - s->d.form_lead_us;
        const double now = now_us();
        if (now >= ready) break;
        s->cv_loop.wait_for(lk, std::chrono::microseconds((int64_t)std::max(1.0, ready - now)));
      }
      if (s->queue.empty()) continue;
    }
    if (s->d.max_wait_us > 0 && (int)s->queue.size() < s->d.max_batch && !s->stop) {
      const double deadline = s->reqs[s->queue.front()].t_arrival + s->d.max_wait_us;
      while (!s->stop && (int)s->queue.size() < s->d.max_batch && now_us() < deadline)
        s->cv_loop.wait_for(lk, std::chrono::microseconds((int64_t)std::max(1.0, deadline - now_us())));
    }
    // form the tick: oldest first, one snapshot per stream
    Tick t;
    t.slot = (int)(s->tick_seq % s->n_slots);
    std::vector<ServeItem> proto;
    for (auto q = s->queue.begin(); q != s->queue.end() && (int)t.reqs.size() < s->d.max_batch;) {
      Stream& sm = s->streams[s->reqs[*q].stream];
      if (sm.mark == s->tick_seq) {
        ++q;
        continue;
      }
      sm.mark = s->tick_seq;
      t.reqs.push_back(*q);
      q = s->queue.erase(q);
    }
    t.n = (int)t.reqs.size();
    t.bi = bucket_index(s, t.n);
    t.bucket = s->buckets[t.bi];
    {
      const double now = now_us();
      const double a_start = s->inflight.empty() ? now : std::max(now, s->inflight.back().t_a_end);
      t.t_launch = now;
      for (int rid : t.reqs) s->st_max_wait = std::max(s->st_max_wait, now - s->reqs[rid].t_arrival);
      t.t_a_end = a_start + s->dur_us[t.bi];
      t.t_expect = (s->inflight.empty() ? t.t_a_end : std::max(t.t_a_end, s->inflight.back().t_expect)) +
                   s->dur_b_us[t.bi];
    }
    proto.resize((size_t)s->d.n_det * t.n);
    for (int r = 0; r < t.n; ++r) {
      Req& rq = s->reqs[t.reqs[r]];
      Stream& sm = s->streams[rq.stream];
      const int64_t k = sm.k_sched++;
      const int64_t S = sm.S;
      const int64_t me = m_end((k + 1) * S - s->d.agg_delay - s->geom.post_c, s->Kf);
      const int64_t ne = me - (s->Kh - 1) / 2;
      for (int det = 0; det < s->d.n_det; ++det) {
        ServeItem& it = proto[(size_t)det * t.n + r];
        it.active = 1;
        it.S = (int)S;
        it.head = k * S;
        it.m0 = sm.me;
        it.m1 = me;
        it.n0 = std::max<int64_t>(sm.ne, 0);
        it.n1 = ne;
        it.wring = sm.wring[det];
        it.strain = sm.strain[det];
        it.acc = sm.acc[det];
        it.clean = sm.clean[det];
        it.dec = sm.dec[det];
        it.white = sm.white[det];
        it.pring = sm.pring[det];
        it.in = rq.in_dev + (size_t)det * (s->d.n_witness + 1) * S;
        it.out = rq.out_dev + (size_t)det * S;
        it.score = det == 0 ? rq.out_dev + (size_t)s->d.n_det * s->d.max_stride : nullptr;
      }
      sm.me = me;
      sm.ne = ne;
      sm.pending--;
      sm.inflight++;
    }
    s->tick_seq++;
    lk.unlock();
    bool ok = true;
    std::string err;
    const double t_call0 = now_us();
    try {
      fill_table(s, t, proto);
      const int bi = bucket_index(s, t.n);
      // first stage on st, second stage on st2 after it: the next tick's
      // first stage runs beside this tick's second stage
      GW_CUDA(cudaEventRecord(s->start_ev[t.slot], s->st));
      const int64_t before = gw_launch_count();
      if (s->d.use_graphs)
        GW_CUDA(cudaGraphLaunch(s->graphs[(size_t)bi * s->n_slots + t.slot], s->st));
      else
        record_tick_a(s, t.bucket, t.slot, s->st, s->side);
      GW_CUDA(cudaEventRecord(s->mid_ev[t.slot], s->st));
      GW_CUDA(cudaStreamWaitEvent(s->st2, s->mid_ev[t.slot], 0));
      GW_CUDA(cudaEventRecord(s->bstart_ev[t.slot], s->st2));
      if (s->d.use_graphs) {
        GW_CUDA(cudaGraphLaunch(s->graphs_b[(size_t)bi * s->n_slots + t.slot], s->st2));
        add_launches(s->graph_kernels[bi]);
        t.kernels = s->graph_kernels[bi];
      } else {
        record_tick_b(s, t.bucket, t.slot, s->st2);
        t.kernels = gw_launch_count() - before;
      }
      GW_CUDA(cudaEventRecord(s->done_ev[t.slot], s->st2));
    } catch (const std::exception& e) {
      ok = false;
      err = e.what();
    }
    const double t_call = now_us() - t_call0;
    lk.lock();
    s->st_max_call = std::max(s->st_max_call, t_call);
    if (!ok) fail_all_locked(s, GW_ECUDA, "tick launch failed: " + err);
    s->inflight.push_back(std::move(t));
    s->cv_complete.notify_one();
  }
  s->loop_done = true;
  s->cv_complete.notify_one();
}

void done_main(gw_server* s) {
  cudaSetDevice(s->ctx->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv_complete.wait(lk, [&] { return !s->inflight.empty() || s->loop_done; });
    if (s->inflight.empty()) break;
    Tick& t = s->inflight.front();
    const int slot = t.slot;
    lk.unlock();
    const cudaError_t e = cudaEventSynchronize(s->done_ev[slot]);
    // the slot's stage timings, read before the slot can be reused
    float a_ms = 0.f, b_ms = 0.f;
    const bool timed = e == cudaSuccess &&
                       cudaEventElapsedTime(&a_ms, s->start_ev[slot], s->mid_ev[slot]) == cudaSuccess &&
                       cudaEventElapsedTime(&b_ms, s->bstart_ev[slot], s->done_ev[slot]) == cudaSuccess;
    const int dev_status = s->h_status[slot];
    lk.lock();
    if (e != cudaSuccess) fail_all_locked(s, GW_ECUDA, std::string("tick failed: ") + cudaGetErrorString(e));
    if (dev_status) fail_all_locked(s, GW_ETIMEOUT, "a tensor-core kernel gave up a bounded wait");
    Tick done = std::move(s->inflight.front());
    s->inflight.pop_front();
    // results are copied without the lock: the request slots stay owned by
    // their tickets until released below
    lk.unlock();
    const double t_now = now_us();
    for (int rid : done.reqs) {
      Req& rq = s->reqs[rid];
      const int S = s->streams[rq.stream].S;
      if (rq.clean_out) memcpy(rq.clean_out, rq.out, sizeof(float) * s->d.n_det * S);
      if (rq.score_out) *rq.score_out = rq.out[(size_t)s->d.n_det * s->d.max_stride];
      if (rq.lat_out) *rq.lat_out = t_now - rq.t_arrival;
    }
    lk.lock();
    for (int rid : done.reqs) {
      Req& rq = s->reqs[rid];
      const double l = t_now - rq.t_arrival;
      if (s->lat.size() < kLatKeep)
        s->lat.push_back(l);
      else
        s->lat[s->lat_next++ % kLatKeep] = l;
      s->active.erase(rq.ticket);
      s->streams[rq.stream].inflight--;
      rq.stream = -1;
      s->free_reqs.push_back(rid);
    }
    s->st_snap += done.n;
    s->st_ticks += 1;
    s->st_batch_sum += done.n;
    if (timed) {
      // running estimates of the bucket's two stage times (events around each
      // stage), read by the loop's tick formation under the same lock
      double& ea = s->dur_us[done.bi];
      double& eb = s->dur_b_us[done.bi];
      ea = ea > 0 ? 0.8 * ea + 0.2 * 1e3 * a_ms : 1e3 * a_ms;
      eb = eb > 0 ? 0.8 * eb + 0.2 * 1e3 * b_ms : 1e3 * b_ms;
      s->st_max_dev = std::max(s->st_max_dev, 1e3 * ((double)a_ms + (double)b_ms));
    }
    s->st_kernels += done.kernels;
    s->t_last = t_now;
    s->cv_done.notify_all();
    s->cv_free.notify_all();
    s->cv_loop.notify_one();
  }
}

void server_free(gw_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_loop.notify_all();
  if (s->loop_th.joinable()) s->loop_th.join();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->loop_done = true;
  }
  s->cv_complete.notify_all();
  if (s->done_th.joinable()) s->done_th.join();
  // nothing of the server may still run on any of its streams before the
  // graphs, workspace and events go
  for (cudaStream_t q : {s->st, s->side, s->st2})
    if (q) cudaStreamSynchronize(q);
  for (auto g : s->graphs_b)
    if (g) cudaGraphExecDestroy(g);
  for (auto g : s->graphs)
    if (g) cudaGraphExecDestroy(g);
  for (auto& sm : s->streams)
    if (sm.open && sm.block) dev_free(s->ctx, sm.block, sm.bytes, nullptr);
  for (auto& a : s->allocs) dev_free(s->ctx, a.first, a.second, nullptr);
  for (void* p : s->host_allocs) cudaFreeHost(p);
  for (int i = 0; i < kMaxInflight; ++i)
    for (cudaEvent_t ev : {s->done_ev[i], s->start_ev[i], s->mid_ev[i], s->bstart_ev[i]})
      if (ev) cudaEventDestroy(ev);
  if (s->fork_ev) cudaEventDestroy(s->fork_ev);
  if (s->join_ev) cudaEventDestroy(s->join_ev);
  if (s->st) cudaStreamDestroy(s->st);
  if (s->side) cudaStreamDestroy(s->side);
  if (s->st2) cudaStreamDestroy(s->st2);
  delete s;
}

int submit_impl(gw_server* s, int sid, const float* witness, const float* strain, float* clean_out, float* score_out,
                uint64_t* ticket, double t_arrival, double* lat_out) {
  const int nd = s->d.n_det, C = s->d.n_witness;
  std::unique_lock<std::mutex> lk(s->mu);
  GW_CHECK_ARG(sid >= 0 && sid < (int)s->streams.size() && s->streams[sid].open, "stream id is not open");
  if (s->sticky) throw Error(s->sticky, s->sticky_msg);
  const int S = s->streams[sid].S;
  if (s->free_reqs.empty()) {
    if (!s->cv_free.wait_for(lk, std::chrono::seconds(10), [&] { return !s->free_reqs.empty() || s->stop; }))
      throw Error(GW_ETIMEOUT, "no request slot became free within 10 s");
    if (s->stop) throw Error(GW_ESTATE, "server is stopping");
  }
  const int rid = s->free_reqs.back();
  s->free_reqs.pop_back();
  Req& rq = s->reqs[rid];
  rq.stream = sid;
  s->streams[sid].pending++;  // keeps the stream from closing while its inputs are copied
  lk.unlock();
  // copy into the pinned slot; a sample is NaN or Inf iff its exponent bits
  // are all set, checked as an integer OR-reduction (vectorisable)
  uint32_t bad = 0;
  auto copy_check = [&bad](uint32_t* dst, const uint32_t* src, size_t n) {
    uint32_t b = 0;
    for (size_t i = 0; i < n; ++i) {
      const uint32_t u = src[i];
      dst[i] = u;
      b |= (uint32_t)((u & 0x7f800000u) == 0x7f800000u);
    }
    bad |= b;
  };
  for (int det = 0; det < nd; ++det) {
    uint32_t* dst = reinterpret_cast<uint32_t*>(rq.in + (size_t)det * (C + 1) * S);
    copy_check(dst, reinterpret_cast<const uint32_t*>(witness + (size_t)det * C * S), (size_t)C * S);
    copy_check(dst + (size_t)C * S, reinterpret_cast<const uint32_t*>(strain + (size_t)det * S), (size_t)S);
  }
  const bool finite = bad == 0;
  lk.lock();
  if (!finite) {
    rq.stream = -1;
    s->streams[sid].pending--;
    s->free_reqs.push_back(rid);
    s->cv_free.notify_one();
    throw Error(GW_ENONFINITE, "non-finite sample in the submitted snapshot");
  }
  rq.ticket = s->next_ticket++;
  rq.t_arrival = t_arrival > 0 ? t_arrival : now_us();
  rq.clean_out = clean_out;
  rq.score_out = score_out;
  rq.lat_out = lat_out;
  s->active.insert(rq.ticket);
  s->queue.push_back(rid);
  if (s->t_first < 0) s->t_first = rq.t_arrival;
  if (ticket) *ticket = rq.ticket;
  s->cv_loop.notify_one();
  return GW_OK;
}

int wait_impl(gw_server* s, uint64_t ticket, int64_t timeout_us) {
  std::unique_lock<std::mutex> lk(s->mu);
  GW_CHECK_ARG(ticket >= 1 && ticket < s->next_ticket, "ticket was never issued");
  auto done = [&] { return s->active.count(ticket) == 0 || s->sticky != 0; };
  if (timeout_us < 0) {
    s->cv_done.wait(lk, done);
  } else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done)) {
    throw Error(GW_ETIMEOUT, "ticket not completed within the timeout");
  }
  if (s->sticky) throw Error(s->sticky, s->sticky_msg);
  return GW_OK;
}

}  // namespace
}  // namespace gw

using namespace gw;

extern "C" {

int gw_server_create(gw_ctx_t ctx, const gw_server_desc* d, const gw_model_t* deepclean, gw_model_t bbhnet,
                     gw_fir_t decimator, gw_fir_t whitening, gw_server_t* out) {
  gw_server* s = nullptr;
  GW_API_BEGIN
  GW_CHECK_ARG(ctx && d && deepclean && decimator && whitening && out, "NULL argument");
  *out = nullptr;
  GW_CHECK_ARG(d->n_det == 1 || d->n_det == 2, "n_det must be 1 or 2");
  GW_CHECK_ARG(d->max_stride >= 8 && d->max_stride % 8 == 0, "max_stride must be a positive multiple of 8");
  GW_CHECK_ARG(d->window >= d->max_stride && d->window % 8 == 0, "window must be a multiple of 8 and >= max_stride");
  GW_CHECK_ARG(d->max_streams >= 1 && d->max_streams <= 65536, "max_streams out of range");
  GW_CHECK_ARG(d->max_batch >= 1 && d->max_batch <= d->max_streams && d->max_batch <= 1024, "max_batch out of range");
  GW_CHECK_ARG(d->max_pending >= d->max_batch && d->max_pending <= (1 << 20), "max_pending must be >= max_batch");
  GW_CHECK_ARG(d->agg_mode == GW_AGG_LATEST || d->agg_mode == GW_AGG_AVERAGE, "unknown aggregation mode");
  GW_CHECK_ARG(d->agg_delay >= 0 && d->agg_delay <= d->window - d->max_stride, "agg_delay out of range");
  GW_CHECK_ARG(d->bbh_len >= 16 && d->bbh_len % 16 == 0, "bbh_len must be a positive multiple of 16");
  GW_CHECK_ARG(d->max_wait_us >= 0, "max_wait_us must be >= 0");
  GW_CHECK_ARG(d->max_inflight >= 1 && d->max_inflight <= kMaxInflight, "max_inflight must be 1..4");
  GW_CHECK_ARG(d->form_lead_us >= 0, "form_lead_us must be >= 0");
  for (int i = 0; i < d->n_det; ++i) {
    GW_CHECK_ARG(deepclean[i] && deepclean[i]->kind == GW_MODEL_DEEPCLEAN, "need one DeepClean model per detector");
    GW_CHECK_ARG(deepclean[i]->n_in == d->n_witness, "DeepClean n_in != n_witness");
    GW_CHECK_ARG(deepclean[i]->precision == deepclean[0]->precision, "detectors must share a precision");
  }
  GW_CHECK_ARG(deepclean[0]->precision == GW_FP32 || deepclean[0]->precision == GW_BF16,
               "DeepClean precision must be FP32 or BF16");
  if (bbhnet) {
    GW_CHECK_ARG(bbhnet->kind == GW_MODEL_BBHNET && bbhnet->n_in == d->n_det, "BBHnet must have n_in = n_det");
    GW_CHECK_ARG(bbhnet->precision != GW_FP8 || bbhnet->fp8_scaled,
                 "FP8 BBHnet needs activation scales (act_scales or gw_model_calibrate)");
  }
  GW_CHECK_ARG((decimator->ntaps & 1) && (whitening->ntaps & 1), "FIR tap counts must be odd");
  GW_CHECK_ARG(!d->post || (d->post->precision == GW_FP32 && (d->post->ntaps & 1) && d->post->ntaps <= 16385),
               "post-processing FIR must be FP32 with an odd number of taps (<= 16385)");
  GW_CUDA(cudaSetDevice(ctx->device));
  s = new gw_server();
  try {
    s->ctx = ctx;
    s->d = *d;
    for (int i = 0; i < d->n_det; ++i) s->dc[i] = deepclean[i];
    s->bbh = bbhnet;
    s->fdec = decimator;
    s->fwht = whitening;
    s->fpost = d->post;
    s->prec = deepclean[0]->precision;
    s->Kf = decimator->ntaps;
    s->Kh = whitening->ntaps;
    s->Lb = d->bbh_len;
    s->max_new = d->max_stride / 2 + 2;
    s->n_slots = d->max_inflight;
    GW_CHECK_ARG(serve_whiten_smem(s->Kh, s->max_new) <= 200 * 1024, "whitening FIR too long");
    ServeGeom& g = s->geom;
    g.C = d->n_witness;
    g.G = (d->n_witness + 7) / 8;
    g.P = s->prec == GW_FP32 ? 1 : s->dc[0]->layers[0].pin;
    g.W = d->window;
    // with post-processing the strain ring also serves outputs c samples older
    g.post = d->post ? 1 : 0;
    g.post_c = d->post ? (d->post->ntaps - 1) / 2 : 0;
    g.R = round_up(d->window + g.post_c, 64);
    g.Rp = d->post ? round_up(d->max_stride + 2 * g.post_c + 64, 64) : 0;
    GW_CHECK_ARG(g.R % g.P == 0 && d->window % g.P == 0, "window must be a multiple of the first layer's phase count");
    g.Rc = round_up(d->max_stride + 2 * s->Kf + 64, 64);
    g.Rd = round_up(d->max_stride / 2 + 2 * s->Kh + 64, 64);
    g.Rw = round_up(s->Lb + d->max_stride, 64);
    g.bf16 = s->prec == GW_BF16;
    g.mode = d->agg_mode;
    g.delta = d->agg_delay;
    for (int b : {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024})
      if (b < d->max_batch) s->buckets.push_back(b);
    s->buckets.push_back(d->max_batch);
    s->dur_us.assign(s->buckets.size(), 0.0);
    s->dur_b_us.assign(s->buckets.size(), 0.0);

    // device workspace
    const int Bmax = d->max_batch, nd = d->n_det, W = d->window;
    const size_t esz = s->prec == GW_FP32 ? 4 : 2;
    s->pred = walloc<float>(s, (size_t)nd * Bmax * W);
    for (int det = 0; det < nd; ++det)
      for (int j = 0; j < 2; ++j) s->act[det][j] = walloc<char>(s, (size_t)Bmax * deepclean_tc_act_elems(W) * esz);
    if (bbhnet) {
      s->bbh_x = walloc<float>(s, (size_t)Bmax * nd * s->Lb);
      s->logits = walloc<float>(s, (size_t)Bmax);
      s->bbh_ws = walloc<char>(s, bbhnet->precision == GW_FP32 ? bbhnet_f32_ws_bytes(Bmax, s->Lb)
                                                               : bbhnet_tc_ws_bytes(Bmax, s->Lb));
    }
    s->d_err = walloc<int>(s, 1);
    s->dummy = walloc<char>(s, state_layout(s).wring);
    for (int i = 0; i < s->n_slots; ++i) {
      s->d_items[i] = walloc<ServeItem>(s, (size_t)nd * Bmax);
      s->d_ptrs[i] = walloc<void*>(s, (size_t)nd * Bmax);
      s->h_items[i] = halloc<ServeItem>(s, (size_t)nd * Bmax);
      s->h_ptrs[i] = halloc<void*>(s, (size_t)nd * Bmax);
    }
    s->h_status = halloc<int>(s, kMaxInflight);
    s->d_status = dptr(s->h_status);
    s->req_in_elems = (size_t)nd * (d->n_witness + 1) * d->max_stride;
    s->req_out_elems = round_up((int64_t)nd * d->max_stride + 1, 64);
    s->req_in = halloc<float>(s, s->req_in_elems * d->max_pending);
    s->req_out = halloc<float>(s, s->req_out_elems * d->max_pending);
    s->reqs.resize(d->max_pending);
    float* in_dev = dptr(s->req_in);
    float* out_dev = dptr(s->req_out);
    for (int i = 0; i < d->max_pending; ++i) {
      s->reqs[i].in = s->req_in + s->req_in_elems * i;
      s->reqs[i].out = s->req_out + s->req_out_elems * i;
      s->reqs[i].in_dev = in_dev + s->req_in_elems * i;
      s->reqs[i].out_dev = out_dev + s->req_out_elems * i;
      s->free_reqs.push_back(d->max_pending - 1 - i);
    }
    s->streams.resize(d->max_streams);

    GW_CUDA(cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking));
    GW_CUDA(cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking));
    GW_CUDA(cudaEventCreateWithFlags(&s->fork_ev, cudaEventDisableTiming));
    GW_CUDA(cudaEventCreateWithFlags(&s->join_ev, cudaEventDisableTiming));
    GW_CUDA(cudaStreamCreateWithFlags(&s->st2, cudaStreamNonBlocking));
    for (int i = 0; i < kMaxInflight; ++i) {
      GW_CUDA(cudaEventCreate(&s->done_ev[i]));
      GW_CUDA(cudaEventCreate(&s->start_ev[i]));
      GW_CUDA(cudaEventCreate(&s->mid_ev[i]));
      GW_CUDA(cudaEventCreate(&s->bstart_ev[i]));
    }
    GW_CUDA(cudaDeviceSynchronize());
    // one eager all-padding tick of the largest bucket sets the kernels' lazy
    // attributes before capture
    {
      Tick t;
      t.slot = 0;
      t.n = 0;
      t.bucket = s->buckets.back();
      fill_table(s, t, {});
      record_tick_a(s, t.bucket, 0, s->st, s->side);
      record_tick_b(s, t.bucket, 0, s->st);
      GW_CUDA(cudaStreamSynchronize(s->st));
      int e = 0;
      GW_CUDA(cudaMemcpy(&e, s->d_err, sizeof(int), cudaMemcpyDeviceToHost));
      if (e) throw Error(GW_ETIMEOUT, "warm-up tick: a tensor-core kernel gave up a bounded wait");
    }
    if (d->use_graphs) capture_graphs(s);
    s->loop_th = std::thread(loop_main, s);
    s->done_th = std::thread(done_main, s);
  } catch (...) {
    server_free(s);
    throw;
  }
  *out = s;
  GW_API_END
}

int64_t gw_server_stream_bytes(gw_server_t s, int stride) {
  if (!s) return GW_EINVAL;
  (void)stride;  // the rings are sized for max_stride and the window
  return (int64_t)state_layout(s).det * s->d.n_det;
}

int gw_server_open(gw_server_t s, int stride, int* stream_id) {
  GW_API_BEGIN
  GW_CHECK_ARG(s && stream_id, "NULL argument");
  *stream_id = -1;
  GW_CHECK_ARG(stride >= 8 && stride % 8 == 0 && stride <= s->d.max_stride, "stride must be a multiple of 8, <= max_stride");
  GW_CHECK_ARG(s->d.window % stride == 0, "stride must divide the window");
  GW_CHECK_ARG(stride % s->geom.P == 0, "stride must be a multiple of the first DeepClean layer's phase count");
  GW_CHECK_ARG(s->d.agg_delay <= s->d.window - stride, "agg_delay > window - stride");
  int sid = -1;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->sticky) throw Error(s->sticky, s->sticky_msg);
    for (int i = 0; i < (int)s->streams.size(); ++i)
      if (!s->streams[i].open && !s->streams[i].block) {
        sid = i;
        break;
      }
    if (sid < 0) throw Error(GW_ESTATE, "every stream slot is taken");
    s->streams[sid].block = (char*)1;  // reserved while allocating
  }
  const StateLayout L = state_layout(s);
  const size_t bytes = L.det * s->d.n_det;
  char* block = nullptr;
  try {
    GW_CUDA(cudaSetDevice(s->ctx->device));
    block = (char*)dev_alloc(s->ctx, bytes, nullptr);
    GW_CUDA(cudaMemsetAsync(block, 0, bytes, s->st));
    for (int det = 0; det < s->d.n_det; ++det)
      launch_ring_fill(block + L.det * det, s->geom.bf16, s->geom.C, s->geom.G, 2 * s->geom.R, s->dc[det]->in_mean,
                       s->dc[det]->in_istd, s->st);
  } catch (...) {
    if (block) dev_free(s->ctx, block, bytes, nullptr);
    std::lock_guard<std::mutex> lk(s->mu);
    s->streams[sid].block = nullptr;
    throw;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  Stream& sm = s->streams[sid];
  sm = Stream{};
  sm.block = block;
  sm.bytes = bytes;
  sm.S = stride;
  for (int det = 0; det < s->d.n_det; ++det) {
    char* p = block + L.det * det;
    sm.wring[det] = p;
    p += L.wring;
    sm.strain[det] = (float*)p;
    p += L.strain;
    sm.acc[det] = (float*)p;
    p += L.acc;
    sm.clean[det] = (float*)p;
    p += L.clean;
    sm.dec[det] = (float*)p;
    p += L.dec;
    sm.white[det] = (float*)p;
    p += L.white;
    sm.pring[det] = L.pring ? (float*)p : nullptr;
  }
  sm.open = true;
  *stream_id = sid;
  GW_API_END
}

int gw_server_close(gw_server_t s, int stream_id) {
  GW_API_BEGIN
  GW_CHECK_ARG(s, "server is NULL");
  char* block = nullptr;
  size_t bytes = 0;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    GW_CHECK_ARG(stream_id >= 0 && stream_id < (int)s->streams.size() && s->streams[stream_id].open,
                 "stream id is not open");
    Stream& sm = s->streams[stream_id];
    if (sm.pending) throw Error(GW_ESTATE, "stream has pending snapshots");
    sm.open = false;
    if (!s->cv_done.wait_for(lk, std::chrono::seconds(30), [&] { return sm.inflight == 0 || s->sticky; }))
      throw Error(GW_ETIMEOUT, "stream's snapshots did not complete within 30 s");
    block = sm.block;
    bytes = sm.bytes;
    sm = Stream{};
    sm.block = (char*)1;  // slot reserved until the memory is freed
  }
  dev_free(s->ctx, block, bytes, nullptr);
  std::lock_guard<std::mutex> lk(s->mu);
  s->streams[stream_id].block = nullptr;
  GW_API_END
}

int gw_server_submit(gw_server_t s, int stream_id, const float* witness, const float* strain, float* clean_out,
                     float* score_out, uint64_t* ticket) {
  GW_API_BEGIN
  GW_CHECK_ARG(s && witness && strain && clean_out, "NULL argument");
  submit_impl(s, stream_id, witness, strain, clean_out, score_out, ticket, 0.0, nullptr);
  GW_API_END
}

int gw_server_wait(gw_server_t s, uint64_t ticket, int64_t timeout_us) {
  GW_API_BEGIN
  GW_CHECK_ARG(s, "server is NULL");
  wait_impl(s, ticket, timeout_us);
  GW_API_END
}

int gw_server_stats_read(gw_server_t s, int reset, gw_server_stats* out) {
  GW_API_BEGIN
  GW_CHECK_ARG(s && out, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  gw_server_stats r{};
  r.snapshots = s->st_snap;
  r.ticks = s->st_ticks;
  r.kernels = s->st_kernels;
  r.mean_batch = s->st_ticks ? s->st_batch_sum / s->st_ticks : 0.0;
  if (!s->lat.empty()) {
    std::vector<double> v = s->lat;
    auto pct = [&](double q) {
      const size_t i = std::min(v.size() - 1, (size_t)std::floor(q * (v.size() - 1) + 0.5));
      std::nth_element(v.begin(), v.begin() + i, v.end());
      return v[i];
    };
    r.p50_us = pct(0.50);
    r.p99_us = pct(0.99);
    double sum = 0, mx = 0;
    for (double x : s->lat) {
      sum += x;
      mx = std::max(mx, x);
    }
    r.mean_us = sum / s->lat.size();
    r.max_us = mx;
  }
  r.busy_s = s->t_first >= 0 ? (s->t_last - s->t_first) * 1e-6 : 0.0;
  r.max_tick_device_us = s->st_max_dev;
  r.max_launch_wait_us = s->st_max_wait;
  r.max_submit_late_us = s->st_max_late;
  r.max_launch_call_us = s->st_max_call;
  *out = r;
  if (reset) {
    s->lat.clear();
    s->lat_next = 0;
    s->st_snap = s->st_ticks = s->st_kernels = 0;
    s->st_batch_sum = 0;
    s->st_max_dev = s->st_max_wait = s->st_max_late = s->st_max_call = 0;
    s->t_first = -1;
    s->t_last = 0;
  }
  GW_API_END
}

int gw_server_replay(gw_server_t s, int n, const int* ids, const double* t_us, const float* const* witness,
                     const float* const* strain, float* const* clean, float* score, double* latency_us) {
  GW_API_BEGIN
  GW_CHECK_ARG(s && ids && t_us && witness && strain && clean && n >= 0, "NULL argument");
  for (int i = 1; i < n; ++i) GW_CHECK_ARG(t_us[i] >= t_us[i - 1], "arrival times must be non-decreasing");
  std::vector<uint64_t> tickets(n);
  const double t0 = now_us();
  double late = 0;
  for (int i = 0; i < n; ++i) {
    const double due = t0 + t_us[i];
    while (now_us() < due) {
      if (due - now_us() > 200) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    submit_impl(s, ids[i], witness[i], strain[i], clean[i], score ? score + i : nullptr, &tickets[i], due,
                latency_us ? latency_us + i : nullptr);
    late = std::max(late, now_us() - due);  // queued this long after its time (copy, a full request pool)
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->st_max_late = std::max(s->st_max_late, late);
  }
  for (int i = 0; i < n; ++i) wait_impl(s, tickets[i], 60 * 1000000LL);
  GW_API_END
}

int gw_server_destroy(gw_server_t s) {
  GW_API_BEGIN
  GW_CHECK_ARG(s, "server is NULL");
  server_free(s);
  GW_API_END
}

// ---- one scored stream (the problem statement's call shape) ---------------------
// A one-slot server holding one open stream: push = submit, wait = wait.
struct gw_scored_stream {
  gw_server_t srv = nullptr;
  int id = -1;
};

int gw_scored_stream_create(gw_ctx_t ctx, const gw_model_t* deepclean, gw_model_t bbhnet, gw_fir_t decimator,
                            gw_fir_t whitening, int n_det, int n_witness, int window, int stride, int agg_mode,
                            int agg_delay, int bbh_len, int max_pending, gw_scored_stream_t* out) {
  gw_scored_stream* ss = nullptr;
  GW_API_BEGIN
  GW_CHECK_ARG(out, "NULL argument");
  *out = nullptr;
  GW_CHECK_ARG(max_pending >= 1 && max_pending <= 4096, "max_pending out of range [1, 4096]");
  gw_server_desc d{};
  d.n_det = n_det;
  d.n_witness = n_witness;
  d.window = window;
  d.max_stride = stride;
  d.max_streams = 1;
  d.max_batch = 1;
  d.max_pending = max_pending;
  d.agg_mode = agg_mode;
  d.agg_delay = agg_delay;
  d.bbh_len = bbh_len;
  d.max_wait_us = 0;
  d.max_inflight = 2;
  d.use_graphs = 1;
  d.form_lead_us = 0;
  ss = new gw_scored_stream();
  int rc = gw_server_create(ctx, &d, deepclean, bbhnet, decimator, whitening, &ss->srv);
  if (rc == GW_OK) {
    rc = gw_server_open(ss->srv, stride, &ss->id);
    if (rc != GW_OK) {
      const std::string msg = gw_last_error();
      gw_server_destroy(ss->srv);
      gw::set_last_error(msg);
    }
  }
  if (rc != GW_OK) {
    delete ss;
    return rc;  // the message was set by the failing call
  }
  *out = ss;
  GW_API_END
}

int gw_scored_stream_push(gw_scored_stream_t s, const float* witness, const float* strain, float* clean_out,
                          float* score_out, uint64_t* ticket) {
  if (!s) {
    gw::set_last_error("scored stream is NULL");
    return GW_EINVAL;
  }
  return gw_server_submit(s->srv, s->id, witness, strain, clean_out, score_out, ticket);
}

int gw_scored_stream_wait(gw_scored_stream_t s, uint64_t ticket, int64_t timeout_us) {
  if (!s) {
    gw::set_last_error("scored stream is NULL");
    return GW_EINVAL;
  }
  return gw_server_wait(s->srv, ticket, timeout_us);
}

int gw_scored_stream_destroy(gw_scored_stream_t s) {
  if (!s) {
    gw::set_last_error("scored stream is NULL");
    return GW_EINVAL;
  }
  gw_server_close(s->srv, s->id);
  const int rc = gw_server_destroy(s->srv);
  delete s;
  return rc;
}

}  // extern "C"
