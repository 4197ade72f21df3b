// Batched form: many ciphertext pairs of mixed ring dimension and level, each
// multiplied (tensor, relinearisation, one prime dropped) and optionally
// reduced to its digits (Algorithm 3), run as one unit.
//
// Items are grouped by (context, level); a group is joined into one batch and
// split into chunks of `chunk` ciphertexts, and every result is copied back to
// the item's own output. Two execution modes:
//  * streams: chunks are dealt round-robin to `nstreams` streams forked from
//    the caller's stream, each issuing its own launches;
//  * merged lanes: every chunk is a lane (a host thread with its own stream)
//    and the lanes meet at every transform they issue: the transforms of all
//    lanes, of any ring dimension and level, run as one persistent launch per
//    phase over all their tiles (k_ntt16_multi), and so do their key-switch
//    inner products (k_ks_ip_multi), so the many small launches of a mixed
//    batch fill the GPU together.
// The whole run can be captured once into a CUDA graph and replayed. The
// autotuner times the eager run for a few (mode, chunk, streams, NTT tile)
// settings on the actual work list and keeps the fastest. Results do not
// depend on any of these settings.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <map>
#include <mutex>
#include <thread>

#include "ss_internal.h"

namespace ss {
Context& context_of(ss_ctx* c);
void set_error(const std::string& m);
}  // namespace ss

struct ss_batch {
  struct Group {
    int ctx, level, t_exp;
    bool reduce;
    std::vector<int> items;
  };
  std::vector<ss::Context*> ctxs;
  std::vector<ss_batch_item> items;
  std::vector<Group> groups;
  int chunk = 64, nstreams = 1, tile_log = SS_NTT_TILE_LOG;
  int merged = 0;  // 1: lanes with merged transforms
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int skipped = 0;
};

namespace ss {

static void ensure_streams(ss_batch& b, int n) {
  while ((int)b.streams.size() < n) {
    cudaStream_t s;
    SS_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    b.streams.push_back(s);
    cudaEvent_t e;
    SS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    b.events.push_back(e);
  }
  if (b.events.size() < b.streams.size() + 1) {
    cudaEvent_t e;
    SS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    b.events.push_back(e);
  }
}

static void scatter(Context& C, const BufP& src, int j, ss_ct* dst, cudaStream_t st) {
  if (dst->capacity < src->level) throw Error(SS_ERR_SHAPE, "output capacity below the result level");
  size_t row = (size_t)src->level * C.N * 8;
  SS_CUDA(cudaMemcpy2DAsync(dst->data, (size_t)dst->capacity * C.N * 8, src->limb(j, 0, 0, C.N),
                            (size_t)src->cap * C.N * 8, row, src->ncomp, cudaMemcpyDeviceToDevice, st));
  dst->ncomp = src->ncomp;
  dst->level = src->level;
  dst->t_exp = src->t_exp;
}

// One chunk of one group on one stream.
static void run_chunk(ss_batch& b, const ss_batch::Group& g, int i0, int i1, cudaStream_t st) {
  Context& C = *b.ctxs[g.ctx];
  std::vector<std::pair<BufP, int>> pa, pb;
  for (int i = i0; i < i1; ++i) {
    const ss_batch_item& it = b.items[g.items[i]];
    pa.push_back({view_buf(it.a), 1});
    pb.push_back({view_buf(it.b), 1});
  }
  BufP A = ev_concat(C, pa, st), B = ev_concat(C, pb, st);
  BufP P = ev_mul(C, A, B, st);
  for (int i = i0; i < i1; ++i) scatter(C, P, i - i0, b.items[g.items[i]].prod, st);
  if (g.reduce) {
    std::vector<BufP> d = ev_reduce(C, P, st);
    for (int i = i0; i < i1; ++i)
      for (size_t k = 0; k < d.size(); ++k) scatter(C, d[k], i - i0, &b.items[g.items[i]].digits[k], st);
  }
}

// The lanes' meeting point: every active lane submits its next transform or
// inner product (or leaves); when all active lanes have one pending, the last
// to arrive enqueues them as merged persistent launches on the merge stream,
// which waits for each lane's stream and which each lane's stream then waits
// for. Only the lane holding `run` issues CUDA calls: it is released while a
// lane waits for its round and taken back afterwards, so no two threads ever
// add work at the same time (a stream capture builds one graph, which must not
// be modified from two threads at once).
struct LaneMerger : NttMerger, KsMerger {
  std::mutex run;
  std::mutex mu;
  std::condition_variable cv;
  int active = 0;
  uint64_t round = 0;
  struct Req {
    bool ks;  // inner product (else transform)
    NttReq r;
    bool fwd;
    KsReq k;
    cudaStream_t st;
    int lane;
  };
  std::vector<Req> pending;
  cudaStream_t mst = nullptr;
  cudaEvent_t done = nullptr;
  std::vector<cudaEvent_t> lane_ev;
  int tile_log = SS_NTT_TILE_LOG;
  bool failed = false;
  std::string error;

  static thread_local int t_lane;

  void flush_locked() {
    try {
      std::vector<NttReq> fw, iv;
      std::vector<KsReq> ks;
      for (auto& q : pending) {
        SS_CUDA(cudaEventRecord(lane_ev[q.lane], q.st));
        SS_CUDA(cudaStreamWaitEvent(mst, lane_ev[q.lane], 0));
        if (q.ks) ks.push_back(q.k);
        else (q.fwd ? fw : iv).push_back(q.r);
      }
      ntt_multi(fw, true, tile_log, mst);
      ntt_multi(iv, false, tile_log, mst);
      ks_multi(ks, mst);
      SS_CUDA(cudaEventRecord(done, mst));
      for (auto& q : pending) SS_CUDA(cudaStreamWaitEvent(q.st, done, 0));
    } catch (const std::exception& e) {
      if (!failed) error = e.what();
      failed = true;
    }
    pending.clear();
    ++round;
    cv.notify_all();
  }

  // called holding `run` and `mu`; returns holding both
  void wait_round(std::unique_lock<std::mutex>& lk) {
    const uint64_t my = round;
    if ((int)pending.size() == active) {
      flush_locked();
    } else {
      run.unlock();
      cv.wait(lk, [&] { return round != my; });
      lk.unlock();
      run.lock();
      lk.lock();
    }
    if (failed) throw Error(SS_ERR_CUDA, "merged launch failed: " + error);
  }

  void submit(const NttReq& r, bool fwd, cudaStream_t st) override {
    std::unique_lock<std::mutex> lk(mu);
    if (failed) throw Error(SS_ERR_CUDA, "merged launch failed: " + error);
    Req q;
    q.ks = false;
    q.r = r;
    q.fwd = fwd;
    q.st = st;
    q.lane = t_lane;
    pending.push_back(q);
    wait_round(lk);
  }

  void submit_ks(const KsReq& k, cudaStream_t st) override {
    std::unique_lock<std::mutex> lk(mu);
    if (failed) throw Error(SS_ERR_CUDA, "merged launch failed: " + error);
    Req q;
    q.ks = true;
    q.k = k;
    q.st = st;
    q.lane = t_lane;
    pending.push_back(q);
    wait_round(lk);
  }

  // called holding `run`, which it releases
  void leave() {
    {
      std::lock_guard<std::mutex> lk(mu);
      --active;
      if (active > 0 && (int)pending.size() == active) flush_locked();
    }
    run.unlock();
  }
};
thread_local int LaneMerger::t_lane = -1;

// Every chunk as a lane on its own stream, transforms merged across lanes.
static void run_lanes(ss_batch& b, cudaStream_t st) {
  std::vector<std::pair<int, std::pair<int, int>>> lanes;  // (group, [i0, i1))
  for (int gi = 0; gi < (int)b.groups.size(); ++gi)
    for (int i0 = 0; i0 < (int)b.groups[gi].items.size(); i0 += b.chunk)
      lanes.push_back({gi, {i0, std::min((int)b.groups[gi].items.size(), i0 + b.chunk)}});
  const int n = (int)lanes.size();
  ensure_streams(b, n + 1);  // lanes, then the merge stream
  for (auto* c : b.ctxs) c->ntt_tile_log = b.tile_log;
  LaneMerger M;
  M.active = n;
  M.mst = b.streams[n];
  M.tile_log = b.tile_log;
  M.done = b.events[n + 1];
  for (int k = 0; k < n; ++k) M.lane_ev.push_back(b.events[k]);
  cudaEvent_t fork = b.events[n];
  SS_CUDA(cudaEventRecord(fork, st));
  for (int k = 0; k <= n; ++k) SS_CUDA(cudaStreamWaitEvent(b.streams[k], fork, 0));
  std::vector<std::string> errs(n);
  std::vector<ss_status> codes(n, SS_OK);
  std::vector<std::thread> th;
  int dev = 0;
  SS_CUDA(cudaGetDevice(&dev));
  for (int k = 0; k < n; ++k)
    th.emplace_back([&, k] {
      cudaSetDevice(dev);
      LaneMerger::t_lane = k;
      ntt_merger() = &M;
      ks_merger() = &M;
      M.run.lock();
      try {
        run_chunk(b, b.groups[lanes[k].first], lanes[k].second.first, lanes[k].second.second, b.streams[k]);
      } catch (const Error& e) {
        codes[k] = e.code;
        errs[k] = e.what();
      } catch (const std::exception& e) {
        codes[k] = SS_ERR_PARAM;
        errs[k] = e.what();
      }
      ntt_merger() = nullptr;
      ks_merger() = nullptr;
      M.leave();
    });
  for (auto& t : th) t.join();
  for (int k = 0; k <= n; ++k) {
    SS_CUDA(cudaEventRecord(b.events[k], b.streams[k]));
    SS_CUDA(cudaStreamWaitEvent(st, b.events[k], 0));
  }
  if (M.failed) throw Error(SS_ERR_CUDA, M.error);
  for (int k = 0; k < n; ++k)
    if (codes[k] != SS_OK) throw Error(codes[k], errs[k]);
}

// Fork chunks over the streams and join them back into `st`.
static void run_all(ss_batch& b, cudaStream_t st) {
  if (b.merged) return run_lanes(b, st);
  ensure_streams(b, b.nstreams);
  for (auto* c : b.ctxs) c->ntt_tile_log = b.tile_log;
  cudaEvent_t fork = b.events[b.nstreams];
  SS_CUDA(cudaEventRecord(fork, st));
  for (int k = 0; k < b.nstreams; ++k) SS_CUDA(cudaStreamWaitEvent(b.streams[k], fork, 0));
  int rr = 0;
  for (auto& g : b.groups)
    for (int i0 = 0; i0 < (int)g.items.size(); i0 += b.chunk) {
      int i1 = std::min((int)g.items.size(), i0 + b.chunk);
      run_chunk(b, g, i0, i1, b.streams[rr++ % b.nstreams]);
    }
  for (int k = 0; k < b.nstreams; ++k) {
    SS_CUDA(cudaEventRecord(b.events[k], b.streams[k]));
    SS_CUDA(cudaStreamWaitEvent(st, b.events[k], 0));
  }
}

// Whether Algorithm 3 fits on a product at `level` (a plan-only run).
static bool reduce_fits(Context& C, int level) {
  if (level < 2) return false;
  PlanScope ps(C);
  bool ok = true;
  try {
    auto x = std::make_shared<Buf>();
    x->count = 1;
    x->ncomp = 2;
    x->level = level;
    x->cap = level;
    x->t_exp = C.r;
    ev_reduce(C, x, nullptr);
  } catch (const Error&) {
    ok = false;
  }
  return ok;
}

static void drop_graph(ss_batch& b) {
  if (b.exec) cudaGraphExecDestroy(b.exec);
  if (b.graph) cudaGraphDestroy(b.graph);
  b.exec = nullptr;
  b.graph = nullptr;
}

}  // namespace ss

extern "C" {

ss_status ss_batch_create(ss_ctx* const* ctxs, int32_t nctx, const ss_batch_item* items, int32_t n, ss_batch** out) {
  try {
    if (!ctxs || nctx < 1 || !items || n < 1 || !out) throw ss::Error(SS_ERR_PARAM, "bad argument");
    auto* b = new ss_batch();
    for (int i = 0; i < nctx; ++i) {
      ss::Context& C = ss::context_of(ctxs[i]);
      if (!C.have_keys) {
        delete b;
        throw ss::Error(SS_ERR_PARAM, "context without keys");
      }
      b->ctxs.push_back(&C);
    }
    std::map<std::tuple<int, int, int, int>, int> gi;
    for (int i = 0; i < n; ++i) {
      const ss_batch_item& it = items[i];
      if (it.ctx < 0 || it.ctx >= nctx || !it.prod) {
        delete b;
        throw ss::Error(SS_ERR_PARAM, "bad item");
      }
      const ss::Context& C = *b->ctxs[it.ctx];
      if (it.a.count != 1 || it.b.count != 1 || it.a.ncomp != 2 || it.b.ncomp != 2 || it.a.level != it.b.level ||
          it.a.t_exp != it.b.t_exp || it.a.level < 2 || it.a.level > C.L || it.a.t_exp != C.r) {
        delete b;
        throw ss::Error(SS_ERR_SHAPE, "each item needs two single ciphertexts at one level and t = p^r");
      }
      bool reduce = it.reduce != 0 && it.digits != nullptr;
      if (reduce && !ss::reduce_fits(*b->ctxs[it.ctx], it.a.level - 1)) {
        reduce = false;
        ++b->skipped;
      }
      auto key = std::make_tuple(it.ctx, it.a.level, it.a.t_exp, reduce ? 1 : 0);
      auto f = gi.find(key);
      if (f == gi.end()) {
        gi[key] = (int)b->groups.size();
        b->groups.push_back({it.ctx, it.a.level, it.a.t_exp, reduce, {i}});
      } else {
        b->groups[f->second].items.push_back(i);
      }
      b->items.push_back(it);
    }
    *out = b;
    return SS_OK;
  } catch (const ss::Error& e) {
    ss::set_error(e.what());
    return e.code;
  }
}

ss_status ss_batch_config(ss_batch* b, int32_t chunk, int32_t nstreams, int32_t ntt_tile_log) {
  if (!b || chunk < 1 || nstreams < 0 || nstreams > 8 || (ntt_tile_log != 11 && ntt_tile_log != 12)) {
    ss::set_error("bad batch configuration");
    return SS_ERR_PARAM;
  }
  b->chunk = chunk;
  b->merged = nstreams == 0 ? 1 : 0;
  b->nstreams = nstreams == 0 ? 1 : nstreams;
  b->tile_log = ntt_tile_log;
  ss::drop_graph(*b);
  return SS_OK;
}

ss_status ss_batch_get_config(const ss_batch* b, int32_t* chunk, int32_t* nstreams, int32_t* ntt_tile_log,
                              int32_t* groups, int32_t* skipped) {
  if (!b) return SS_ERR_PARAM;
  if (groups) *groups = (int32_t)b->groups.size();
  if (skipped) *skipped = b->skipped;
  if (chunk) *chunk = b->chunk;
  if (nstreams) *nstreams = b->merged ? 0 : b->nstreams;
  if (ntt_tile_log) *ntt_tile_log = b->tile_log;
  return SS_OK;
}

ss_status ss_batch_run(ss_batch* b, ss_stream stream) {
  try {
    if (!b) throw ss::Error(SS_ERR_PARAM, "null batch");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (b->exec) SS_CUDA(cudaGraphLaunch(b->exec, st));
    else ss::run_all(*b, st);
    return SS_OK;
  } catch (const ss::Error& e) {
    ss::set_error(e.what());
    return e.code;
  }
}

ss_status ss_batch_capture(ss_batch* b, ss_stream stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  try {
    if (!b) throw ss::Error(SS_ERR_PARAM, "null batch");
    if (!st) throw ss::Error(SS_ERR_PARAM, "capture needs a non-default stream");
    ss::drop_graph(*b);
    ss::ensure_streams(*b, b->nstreams);
    SS_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    try {
      ss::run_all(*b, st);
    } catch (...) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(st, &g);
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      throw;
    }
    SS_CUDA(cudaStreamEndCapture(st, &b->graph));
    SS_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
    return SS_OK;
  } catch (const ss::Error& e) {
    ss::set_error(e.what());
    return e.code;
  }
}

ss_status ss_batch_tune(ss_batch* b, ss_stream stream, int32_t* best_chunk, int32_t* best_streams,
                        int32_t* best_tile_log) {
  try {
    if (!b) throw ss::Error(SS_ERR_PARAM, "null batch");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ss::drop_graph(*b);
    const int chunks[] = {8, 32, 64};
    const int nstr[] = {1, 3, 0};  // 0: merged lanes
    const int tiles[] = {11, 12};
    double best = 1e300;
    int bc = b->chunk, bs = b->merged ? 0 : b->nstreams, bt = b->tile_log;
    cudaEvent_t e0, e1;
    SS_CUDA(cudaEventCreate(&e0));
    SS_CUDA(cudaEventCreate(&e1));
    for (int tl : tiles)
      for (int c : chunks)
        for (int s : nstr) {
          b->chunk = c;
          b->merged = s == 0 ? 1 : 0;
          b->nstreams = s == 0 ? 1 : s;
          b->tile_log = tl;
          ss::run_all(*b, st);  // warm the pool for this shape
          SS_CUDA(cudaEventRecord(e0, st));
          ss::run_all(*b, st);
          SS_CUDA(cudaEventRecord(e1, st));
          SS_CUDA(cudaEventSynchronize(e1));
          float ms = 0;
          SS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          if (ms < best) { best = ms; bc = c; bs = s; bt = tl; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->chunk = bc;
    b->merged = bs == 0 ? 1 : 0;
    b->nstreams = bs == 0 ? 1 : bs;
    b->tile_log = bt;
    if (best_chunk) *best_chunk = bc;
    if (best_streams) *best_streams = bs;
    if (best_tile_log) *best_tile_log = bt;
    return SS_OK;
  } catch (const ss::Error& e) {
    ss::set_error(e.what());
    return e.code;
  }
}

void ss_batch_destroy(ss_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  ss::drop_graph(*b);
  for (auto s : b->streams) cudaStreamDestroy(s);
  for (auto e : b->events) cudaEventDestroy(e);
  for (auto* c : b->ctxs) c->ntt_tile_log = SS_NTT_TILE_LOG;
  delete b;
}

}  // extern "C"
