// Served form: a request loop over one or several contexts (parameter sets,
// e.g. N = 2^15 with 257^2 and N = 2^16 with 257^3) with continuous batching.
//
// Queries arrive through ss_server_submit(_to) at any time, each for one of
// the server's contexts. `workers` host threads each own a CUDA stream. A
// worker that is free takes the oldest pending query and every other pending
// query of the same context and shape (level, plaintext modulus) that still
// fits the one HBM budget shared by all contexts, up to `max_merge`, joins
// them into one batch (ev_query_multi) and runs it on its stream while the
// other workers run theirs, so queries of any ring dimension that arrive while
// others are on the GPU are admitted as soon as a worker and memory free up and
// their work overlaps on the device. Keys and tables of every context stay
// resident. Every result equals the same query run alone (the schedule is per
// ciphertext).
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "ss_internal.h"

namespace ss {

typedef std::chrono::steady_clock Clock;

struct Request {
  uint64_t id;
  int ctx = 0;
  QueryCols cols;
  ss_ct* out;
  size_t bytes;
  Clock::time_point t_submit, t_start, t_done;
  ss_status status = SS_OK;
  std::string error;
  bool done = false;
};

struct Server {
  std::vector<Context*> ctxs;
  int max_merge = 1;
  size_t budget = 0, inflight = 0, peak_inflight = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> pending;
  std::map<uint64_t, std::shared_ptr<Request>> all;
  uint64_t next_id = 1, completed = 0, batches = 0;
  bool stop = false;
  std::vector<std::thread> threads;
  std::vector<cudaStream_t> streams;

  static bool same_shape(const Request& a, const Request& b) {
    return a.ctx == b.ctx && a.cols.A->level == b.cols.A->level && a.cols.A->t_exp == b.cols.A->t_exp;
  }

  void worker(int w) {
    cudaStream_t st = streams[w];
    for (;;) {
      std::vector<std::shared_ptr<Request>> group;
      size_t bytes = 0;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] {
          return stop || (!pending.empty() && (inflight == 0 || inflight + pending.front()->bytes <= budget));
        });
        if (stop && pending.empty()) return;
        if (!pending.empty() && inflight > 0 && inflight + pending.front()->bytes > budget) {
          cv_work.wait_for(lk, std::chrono::milliseconds(1));  // shutting down: wait for memory to free up
          continue;
        }
        // oldest first; merge compatible requests while they fit
        auto it = pending.begin();
        while (it != pending.end() && (int)group.size() < max_merge) {
          const auto& r = *it;
          bool fits = inflight + bytes + r->bytes <= budget || (inflight == 0 && group.empty());
          if ((group.empty() || same_shape(*group[0], *r)) && fits) {
            group.push_back(r);
            bytes += r->bytes;
            it = pending.erase(it);
          } else {
            ++it;
          }
        }
        inflight += bytes;
        peak_inflight = std::max(peak_inflight, inflight);
        ++batches;
      }
      auto t0 = Clock::now();
      ss_status status = SS_OK;
      std::string err;
      try {
        Context* C = ctxs[group[0]->ctx];
        std::vector<QueryCols> qs;
        for (auto& r : group) qs.push_back(r->cols);
        auto res = ev_query_multi(*C, qs, st);
        for (size_t i = 0; i < group.size(); ++i) {
          ss_ct* o = group[i]->out;
          const BufP& r = res[i];
          if (o->capacity < r->level || o->count != 1) throw Error(SS_ERR_SHAPE, "result buffer too small");
          size_t row = (size_t)r->level * C->N * 8;
          SS_CUDA(cudaMemcpy2DAsync(o->data, (size_t)o->capacity * C->N * 8, r->data, (size_t)r->cap * C->N * 8, row,
                                    2, cudaMemcpyDeviceToDevice, st));
          o->ncomp = 2;
          o->level = r->level;
          o->t_exp = r->t_exp;
        }
        res.clear();
        SS_CUDA(cudaStreamSynchronize(st));
      } catch (const Error& e) {
        status = e.code;
        err = e.what();
        cudaStreamSynchronize(st);
      } catch (const std::exception& e) {
        status = SS_ERR_PARAM;
        err = e.what();
        cudaStreamSynchronize(st);
      }
      auto t1 = Clock::now();
      {
        std::lock_guard<std::mutex> lk(mu);
        for (auto& r : group) {
          r->t_start = t0;
          r->t_done = t1;
          r->status = status;
          r->error = err;
          r->done = true;
          ++completed;
        }
        inflight -= bytes;
      }
      cv_done.notify_all();
      cv_work.notify_all();
    }
  }
};

}  // namespace ss

struct ss_server {
  ss::Server S;
};

namespace ss {
Context& context_of(ss_ctx* c);  // defined in capi.cpp
void set_error(const std::string& m);
}

extern "C" {

ss_status ss_server_create_multi(ss_ctx* const* ctxs, int32_t nctx, int32_t workers, int32_t max_merge,
                                 uint64_t hbm_budget, ss_server** out) {
  try {
    if (!ctxs || nctx < 1 || !out || workers < 1 || workers > 16 || max_merge < 1)
      throw ss::Error(SS_ERR_PARAM, "bad argument");
    for (int i = 0; i < nctx; ++i) {
      if (!ctxs[i]) throw ss::Error(SS_ERR_PARAM, "null context");
      if (!ss::context_of(ctxs[i]).have_keys) throw ss::Error(SS_ERR_PARAM, "no keys");
    }
    if (hbm_budget == 0) {
      size_t fr = 0, tot = 0;
      SS_CUDA(cudaMemGetInfo(&fr, &tot));
      hbm_budget = fr / 10 * 8;
    }
    auto* s = new ss_server();
    for (int i = 0; i < nctx; ++i) s->S.ctxs.push_back(&ss::context_of(ctxs[i]));
    s->S.max_merge = max_merge;
    s->S.budget = hbm_budget;
    int dev = 0;
    SS_CUDA(cudaGetDevice(&dev));
    for (int w = 0; w < workers; ++w) {
      cudaStream_t st;
      SS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      s->S.streams.push_back(st);
    }
    for (int w = 0; w < workers; ++w)
      s->S.threads.emplace_back([s, w, dev] {
        cudaSetDevice(dev);
        s->S.worker(w);
      });
    *out = s;
    return SS_OK;
  } catch (const ss::Error& e) {
    ss::set_error(e.what());
    return e.code;
  }
}

ss_status ss_server_create(ss_ctx* ctx, int32_t workers, int32_t max_merge, uint64_t hbm_budget, ss_server** out) {
  return ss_server_create_multi(&ctx, 1, workers, max_merge, hbm_budget, out);
}

ss_status ss_server_submit_to(ss_server* s, int32_t ctx_index, const ss_ct* A, const ss_ct* B, const ss_ct* C1,
                              const ss_ct* C2, ss_ct* out, uint64_t* ticket) {
  try {
    if (!s || !A || !B || !C1 || !C2 || !out || !ticket) throw ss::Error(SS_ERR_PARAM, "null argument");
    if (ctx_index < 0 || ctx_index >= (int)s->S.ctxs.size()) throw ss::Error(SS_ERR_PARAM, "context index out of range");
    ss::Context& C = *s->S.ctxs[ctx_index];
    for (const ss_ct* c : {A, B, C1, C2})
      if (!c->data || c->level < 2 || c->level > C.L || c->t_exp != C.r || c->ncomp != 2)
        throw ss::Error(SS_ERR_PARAM, "columns must be 2-component ciphertexts at t = p^r");
    if (A->level != B->level || A->level != C1->level || A->level != C2->level)
      throw ss::Error(SS_ERR_LEVEL, "columns at different levels");
    if (B->count != A->count || C1->count != A->count || (C2->count != A->count && C2->count != 1))
      throw ss::Error(SS_ERR_SHAPE, "column batch sizes differ");
    if (out->count != 1 || !out->data) throw ss::Error(SS_ERR_SHAPE, "result buffer must hold one ciphertext");
    // the plan first: a chain too short for the query is rejected at submission
    ss::plan_query_depth(C, A->level);
    auto r = std::make_shared<ss::Request>();
    r->ctx = ctx_index;
    r->cols = {ss::view_buf(*A), ss::view_buf(*B), ss::view_buf(*C1), ss::view_buf(*C2)};
    r->out = out;
    r->bytes = ss::query_bytes_estimate(C, A->count, A->level);
    r->t_submit = ss::Clock::now();
    {
      std::lock_guard<std::mutex> lk(s->S.mu);
      r->id = s->S.next_id++;
      s->S.pending.push_back(r);
      s->S.all[r->id] = r;
      *ticket = r->id;
    }
    s->S.cv_work.notify_all();
    return SS_OK;
  } catch (const ss::Error& e) {
    ss::set_error(e.what());
    return e.code;
  }
}

ss_status ss_server_submit(ss_server* s, const ss_ct* A, const ss_ct* B, const ss_ct* C1, const ss_ct* C2, ss_ct* out,
                           uint64_t* ticket) {
  return ss_server_submit_to(s, 0, A, B, C1, C2, out, ticket);
}

// Bounded wait: SS_ERR_TIMEOUT if the ticket is not done within timeout_ms
// (a negative timeout waits without bound). On completion the ticket is
// released and its queueing and run times are returned.
ss_status ss_server_wait(ss_server* s, uint64_t ticket, int32_t timeout_ms, double* queued_ms, double* run_ms) {
  if (!s) return SS_ERR_PARAM;
  std::unique_lock<std::mutex> lk(s->S.mu);
  auto it = s->S.all.find(ticket);
  if (it == s->S.all.end()) {
    ss::set_error("unknown ticket");
    return SS_ERR_PARAM;
  }
  auto r = it->second;
  auto ready = [&] { return r->done; };
  if (timeout_ms < 0) s->S.cv_done.wait(lk, ready);
  else if (!s->S.cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    ss::set_error("ticket not done within the timeout");
    return SS_ERR_TIMEOUT;
  }
  s->S.all.erase(it);
  if (queued_ms) *queued_ms = std::chrono::duration<double, std::milli>(r->t_start - r->t_submit).count();
  if (run_ms) *run_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_start).count();
  if (r->status != SS_OK) ss::set_error(r->error);
  return r->status;
}

ss_status ss_server_stats(ss_server* s, uint64_t* completed, uint64_t* batches, uint64_t* peak_inflight_bytes) {
  if (!s) return SS_ERR_PARAM;
  std::lock_guard<std::mutex> lk(s->S.mu);
  if (completed) *completed = s->S.completed;
  if (batches) *batches = s->S.batches;
  if (peak_inflight_bytes) *peak_inflight_bytes = s->S.peak_inflight;
  return SS_OK;
}

void ss_server_destroy(ss_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->S.mu);
    s->S.stop = true;
  }
  s->S.cv_work.notify_all();
  for (auto& t : s->S.threads) t.join();
  for (auto st : s->S.streams) cudaStreamDestroy(st);
  delete s;
}

}  // extern "C"
