// extern "C" entry points declared in include/ss.h. Every entry point catches
// library errors and returns them as ss_status; the message is kept per thread.
#include <cstring>
#include <string>

#include "ss_internal.h"

struct ss_ctx {
  ss::Context C;
};

namespace {

thread_local std::string g_err;

template <class F>
ss_status guard(F f) {
  try {
    f();
    return SS_OK;
  } catch (const ss::Error& e) {
    g_err = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    g_err = "host allocation failed";
    return SS_ERR_OOM;
  } catch (const std::exception& e) {
    g_err = e.what();
    return SS_ERR_PARAM;
  }
}

cudaStream_t S(ss_stream s) { return static_cast<cudaStream_t>(s); }

void need(bool ok, ss_status code, const char* msg) {
  if (!ok) throw ss::Error(code, msg);
}

void check_ct(const ss::Context& C, const ss_ct* c, const char* what) {
  need(c != nullptr && c->data != nullptr, SS_ERR_PARAM, what);
  need(c->count >= 1 && (c->ncomp == 2 || c->ncomp == 3), SS_ERR_SHAPE, "bad ciphertext shape");
  need(c->level >= 1 && c->level <= C.L && c->capacity >= c->level, SS_ERR_LEVEL, "bad ciphertext level");
  need(c->t_exp >= 1 && c->t_exp <= C.r, SS_ERR_TMOD, "bad plaintext modulus exponent");
}

void check_out(const ss_ct* o, int count, int ncomp, int level) {
  need(o != nullptr && o->data != nullptr, SS_ERR_PARAM, "null output");
  need(o->count == count, SS_ERR_SHAPE, "output batch size differs");
  need(o->capacity >= level, SS_ERR_SHAPE, "output capacity too small");
  (void)ncomp;
}

// copy a pool result into caller memory and describe it
void deliver(ss::Context& C, const ss::BufP& r, ss_ct* out, cudaStream_t st) {
  check_out(out, r->count, r->ncomp, r->level);
  size_t row = (size_t)r->level * C.N * 8;
  if (r->data)
    SS_CUDA(cudaMemcpy2DAsync(out->data, (size_t)out->capacity * C.N * 8, r->data, (size_t)r->cap * C.N * 8, row,
                              (size_t)r->count * r->ncomp, cudaMemcpyDeviceToDevice, st));
  out->ncomp = r->ncomp;
  out->level = r->level;
  out->t_exp = r->t_exp;
}

ss::Buf as_out(ss_ct* o) {
  ss::Buf b;
  b.data = o->data;
  b.count = o->count;
  b.ncomp = o->ncomp;
  b.level = o->level;
  b.t_exp = o->t_exp;
  b.cap = o->capacity;
  return b;
}

void write_back(const ss::Buf& b, ss_ct* o) {
  o->ncomp = b.ncomp;
  o->level = b.level;
  o->t_exp = b.t_exp;
}

}  // namespace

namespace ss {
Context& context_of(ss_ctx* c) { return c->C; }
void set_error(const std::string& m) { g_err = m; }
}  // namespace ss

extern "C" {

const char* ss_last_error(void) { return g_err.c_str(); }

ss_status ss_params_preset(int id, ss_params* out) {
  return guard([&] {
    need(out != nullptr, SS_ERR_PARAM, "null params");
    ss_params p;
    std::memset(&p, 0, sizeof(p));
    p.h = 120;
    p.seed = 0x5EED0000ULL + (uint64_t)id;
    switch (id) {
      case 0: p.logN = 13; p.bits = 36; p.alpha = 2; p.p = 17; p.r = 2; p.L = 18; break;
      case 1: p.logN = 15; p.bits = 55; p.alpha = 2; p.p = 257; p.r = 2; p.L = 30; break;
      case 2: p.logN = 16; p.bits = 55; p.alpha = 3; p.p = 257; p.r = 3; p.L = 41; break;
      // N = 2^16 on the ring m = 3N: 256 slots for 257^3 (128 on X^N + 1)
      case 3: p.logN = 16; p.bits = 55; p.alpha = 3; p.p = 257; p.r = 3; p.L = 41; p.m_odd = 3; break;
      // the same on the ring m = 5N/2: 512 slots
      case 4: p.logN = 16; p.bits = 55; p.alpha = 3; p.p = 257; p.r = 3; p.L = 41; p.m_odd = 5; break;
      default: throw ss::Error(SS_ERR_PARAM, "unknown preset");
    }
    *out = p;
  });
}

ss_status ss_context_create(const ss_params* prm, ss_ctx** out) {
  return guard([&] {
    need(prm && out, SS_ERR_PARAM, "null argument");
    *out = nullptr;
    auto* h = new ss_ctx();
    try {
      ss::build_context(h->C, *prm);
      // keep freed pool memory cached for reuse instead of returning it to the driver
      int dev = 0;
      SS_CUDA(cudaGetDevice(&dev));
      cudaMemPool_t pool;
      SS_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
      uint64_t thr = UINT64_MAX;
      SS_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    } catch (...) {
      delete h;
      throw;
    }
    *out = h;
  });
}

void ss_context_destroy(ss_ctx* ctx) {
  if (ctx) {
    cudaDeviceSynchronize();
    delete ctx;
  }
}

ss_status ss_context_info(const ss_ctx* ctx, int32_t* N, int32_t* L, int32_t* alpha, int32_t* slots, int32_t* d,
                          uint64_t* primes) {
  return guard([&] {
    need(ctx != nullptr, SS_ERR_PARAM, "null context");
    const ss::Context& C = ctx->C;
    if (N) *N = C.N;
    if (L) *L = C.L;
    if (alpha) *alpha = C.alpha;
    if (slots) *slots = C.slots;
    if (d) *d = C.d;
    if (primes)
      for (int i = 0; i < C.ntot; ++i) primes[i] = C.primes[i];
  });
}

ss_status ss_keygen(ss_ctx* ctx, const int32_t* galois, int32_t ng) {
  return guard([&] {
    need(ctx != nullptr && (ng == 0 || galois != nullptr) && ng >= 0, SS_ERR_PARAM, "bad argument");
    ss::op_keygen(ctx->C, std::vector<int>(galois, galois + ng));
  });
}

int32_t ss_rotate_sum_elements(const ss_ctx* ctx, int32_t* out, int32_t cap) {
  if (!ctx) return -1;
  auto g = ss::rotate_sum_elements(ctx->C);
  for (int i = 0; i < (int)g.size() && i < cap; ++i) out[i] = g[i];
  return (int32_t)g.size();
}

ss_status ss_encode(const ss_ctx* ctx, int32_t t_exp, const uint64_t* slots, uint64_t* coeffs) {
  return guard([&] {
    need(ctx && slots && coeffs, SS_ERR_PARAM, "null argument");
    auto m = ss::encode(ctx->C, t_exp, slots);
    std::memcpy(coeffs, m.data(), m.size() * 8);
  });
}

ss_status ss_decode(const ss_ctx* ctx, int32_t t_exp, const uint64_t* coeffs, uint64_t* slots) {
  return guard([&] {
    need(ctx && slots && coeffs, SS_ERR_PARAM, "null argument");
    auto v = ss::decode(ctx->C, t_exp, coeffs);
    std::memcpy(slots, v.data(), v.size() * 8);
  });
}

ss_status ss_encrypt(ss_ctx* ctx, const uint64_t* coeffs, int32_t count, uint32_t nonce0, int32_t t_exp, ss_ct* out,
                     ss_stream stream) {
  return guard([&] {
    need(ctx && coeffs && out && count >= 1, SS_ERR_PARAM, "bad argument");
    check_out(out, count, 2, ctx->C.L);
    ss::Buf o = as_out(out);
    ss::op_encrypt(ctx->C, coeffs, count, nonce0, t_exp, o, S(stream));
    write_back(o, out);
  });
}

ss_status ss_decrypt(ss_ctx* ctx, const ss_ct* in, uint64_t* coeffs, ss_stream stream) {
  return guard([&] {
    need(ctx && coeffs, SS_ERR_PARAM, "bad argument");
    check_ct(ctx->C, in, "null input");
    ss::op_decrypt(ctx->C, *ss::view_buf(*in), coeffs, S(stream));
  });
}

static ss_status binary_op(ss_ctx* ctx, int op, const ss_ct* a, const ss_ct* b, ss_ct* out, ss_stream stream) {
  return guard([&] {
    need(ctx != nullptr, SS_ERR_PARAM, "null context");
    check_ct(ctx->C, a, "null a");
    check_ct(ctx->C, b, "null b");
    need(a->level == b->level, SS_ERR_LEVEL, "levels differ");
    need(a->t_exp == b->t_exp, SS_ERR_TMOD, "plaintext moduli differ");
    need(a->ncomp == b->ncomp, SS_ERR_SHAPE, "component counts differ");
    need(a->count == b->count || b->count == 1, SS_ERR_SHAPE, "batch sizes differ");
    check_out(out, a->count, a->ncomp, a->level);
    ss::Buf o = as_out(out);
    o.ncomp = a->ncomp;
    o.level = a->level;
    o.t_exp = a->t_exp;
    ss::k_binary(ctx->C, op, *ss::view_buf(*a), *ss::view_buf(*b), o, S(stream));
    write_back(o, out);
  });
}

ss_status ss_add(ss_ctx* ctx, const ss_ct* a, const ss_ct* b, ss_ct* out, ss_stream s) { return binary_op(ctx, 0, a, b, out, s); }
ss_status ss_sub(ss_ctx* ctx, const ss_ct* a, const ss_ct* b, ss_ct* out, ss_stream s) { return binary_op(ctx, 1, a, b, out, s); }

static ss_status scalar_op(ss_ctx* ctx, int op, const ss_ct* a, int64_t c, ss_ct* out, ss_stream stream) {
  return guard([&] {
    need(ctx != nullptr, SS_ERR_PARAM, "null context");
    check_ct(ctx->C, a, "null a");
    if (op == 2) need(a->t_exp >= 2, SS_ERR_TMOD, "DivideByP needs t = p^e with e >= 2");
    check_out(out, a->count, a->ncomp, a->level);
    ss::Buf o = as_out(out);
    o.ncomp = a->ncomp;
    o.level = a->level;
    o.t_exp = op == 2 ? a->t_exp - 1 : a->t_exp;
    ss::k_scalar(ctx->C, op, *ss::view_buf(*a), c, o, S(stream));
    write_back(o, out);
  });
}

ss_status ss_mul_scalar(ss_ctx* ctx, const ss_ct* a, int64_t c, ss_ct* out, ss_stream s) { return scalar_op(ctx, 0, a, c, out, s); }
ss_status ss_add_scalar(ss_ctx* ctx, const ss_ct* a, int64_t c, ss_ct* out, ss_stream s) { return scalar_op(ctx, 1, a, c, out, s); }
ss_status ss_divide_by_p(ss_ctx* ctx, const ss_ct* a, ss_ct* out, ss_stream s) { return scalar_op(ctx, 2, a, 0, out, s); }

ss_status ss_linear_combination(ss_ctx* ctx, const ss_ct* terms, const int64_t* coeffs, int32_t nterms, int64_t cst,
                                ss_ct* out, ss_stream stream) {
  return guard([&] {
    need(ctx != nullptr && terms != nullptr && coeffs != nullptr && nterms >= 1, SS_ERR_PARAM, "bad argument");
    std::vector<std::pair<ss::BufP, int64_t>> t;
    for (int i = 0; i < nterms; ++i) {
      check_ct(ctx->C, &terms[i], "null term");
      need(terms[i].level == terms[0].level, SS_ERR_LEVEL, "terms at different levels");
      need(terms[i].count == terms[0].count, SS_ERR_SHAPE, "batch sizes differ");
      t.push_back({ss::view_buf(terms[i]), coeffs[i]});
    }
    auto r = ss::ev_lincomb(ctx->C, t, cst, S(stream));
    deliver(ctx->C, r, out, S(stream));
  });
}

ss_status ss_linear_combinations(ss_ctx* ctx, const ss_ct* terms, int32_t nterms, const int64_t* coeffs,
                                 int32_t nout, ss_ct* outs, ss_stream stream) {
  return guard([&] {
    need(ctx != nullptr && terms != nullptr && coeffs != nullptr && outs != nullptr, SS_ERR_PARAM, "bad argument");
    need(nterms >= 1 && nterms <= 16 && nout >= 1 && nout <= 16, SS_ERR_PARAM, "1..16 terms and outputs");
    std::vector<ss::BufP> keep;
    std::vector<const ss::Buf*> ys;
    for (int i = 0; i < nterms; ++i) {
      check_ct(ctx->C, &terms[i], "null term");
      need(terms[i].ncomp == 2, SS_ERR_SHAPE, "2-component terms");
      need(terms[i].level == terms[0].level, SS_ERR_LEVEL, "terms at different levels");
      need(terms[i].t_exp == terms[0].t_exp, SS_ERR_TMOD, "plaintext moduli differ");
      need(terms[i].count == terms[0].count, SS_ERR_SHAPE, "batch sizes differ");
      keep.push_back(ss::view_buf(terms[i]));
      ys.push_back(keep.back().get());
    }
    std::vector<std::vector<int64_t>> cs(nout);
    std::vector<ss::Buf> ob(nout);
    std::vector<ss::Buf*> op;
    for (int k = 0; k < nout; ++k) {
      cs[k].assign(coeffs + (size_t)k * nterms, coeffs + (size_t)(k + 1) * nterms);
      check_out(&outs[k], terms[0].count, 2, terms[0].level);
      ob[k] = as_out(&outs[k]);
      ob[k].ncomp = 2;
      ob[k].level = terms[0].level;
      ob[k].t_exp = terms[0].t_exp;
      op.push_back(&ob[k]);
    }
    ss::k_lincomb_multi(ctx->C, ys, cs, op, S(stream));
    for (int k = 0; k < nout; ++k) write_back(ob[k], &outs[k]);
  });
}

ss_status ss_mul(ss_ctx* ctx, const ss_ct* a, const ss_ct* b, ss_ct* out, ss_stream stream) {
  return guard([&] {
    need(ctx != nullptr, SS_ERR_PARAM, "null context");
    check_ct(ctx->C, a, "null a");
    check_ct(ctx->C, b, "null b");
    need(a->ncomp == 2 && b->ncomp == 2, SS_ERR_SHAPE, "tensor needs 2-component inputs");
    need(a->level == b->level, SS_ERR_LEVEL, "levels differ");
    need(a->t_exp == b->t_exp, SS_ERR_TMOD, "plaintext moduli differ");
    need(a->count == b->count, SS_ERR_SHAPE, "batch sizes differ");
    check_out(out, a->count, 3, a->level);
    ss::Buf o = as_out(out);
    o.ncomp = 3;
    o.level = a->level;
    o.t_exp = a->t_exp;
    ss::k_tensor(ctx->C, *ss::view_buf(*a), *ss::view_buf(*b), o, S(stream));
    write_back(o, out);
  });
}

ss_status ss_relin(ss_ctx* ctx, const ss_ct* a, ss_ct* out, ss_stream stream) {
  return guard([&] {
    need(ctx != nullptr, SS_ERR_PARAM, "null context");
    check_ct(ctx->C, a, "null a");
    check_out(out, a->count, 2, a->level);
    need(out->data != a->data, SS_ERR_PARAM, "relinearisation output must not alias its input");
    ss::Buf o = as_out(out);
    ss::op_relin(ctx->C, *ss::view_buf(*a), o, S(stream));
    write_back(o, out);
  });
}

ss_status ss_mul_relin(ss_ctx* ctx, const ss_ct* a, const ss_ct* b, ss_ct* out, ss_stream stream) {
  return guard([&] {
    need(ctx != nullptr, SS_ERR_PARAM, "null context");
    check_ct(ctx->C, a, "null a");
    check_ct(ctx->C, b, "null b");
    need(a->count == b->count, SS_ERR_SHAPE, "batch sizes differ");
    auto r = ss::plan_then_run(ctx->C, [&] {
      return ss::ev_mul(ctx->C, ss::view_buf(*a), ss::view_buf(*b), S(stream));
    });
    deliver(ctx->C, r, out, S(stream));
  });
}

ss_status ss_relin_noalloc(ss_ctx* ctx, const ss_ct* a, ss_ct* out, ss_stream stream) {
  return guard([&] {
    need(ctx != nullptr, SS_ERR_PARAM, "null context");
    check_ct(ctx->C, a, "null a");
    check_out(out, a->count, 2, a->level);
    need(out->data != a->data, SS_ERR_PARAM, "relinearisation output must not alias its input");
    ss::Buf o = as_out(out);
    ss::op_relin_noalloc(ctx->C, *ss::view_buf(*a), o, S(stream));
    write_back(o, out);
  });
}

ss_status ss_modswitch(ss_ctx* ctx, const ss_ct* a, int32_t drop, ss_ct* out, ss_stream stream) {
  return guard([&] {
    need(ctx != nullptr, SS_ERR_PARAM, "null context");
    check_ct(ctx->C, a, "null a");
    need(drop >= 1 && drop < a->level, SS_ERR_LEVEL, "drop must leave at least one prime");
    check_out(out, a->count, a->ncomp, a->level - drop);
    ss::Buf o = as_out(out);
    ss::op_modswitch(ctx->C, *ss::view_buf(*a), drop, o, S(stream));
    write_back(o, out);
  });
}

ss_status ss_rotate(ss_ctx* ctx, const ss_ct* a, int32_t g, ss_ct* out, ss_stream stream) {
  return guard([&] {
    need(ctx != nullptr, SS_ERR_PARAM, "null context");
    check_ct(ctx->C, a, "null a");
    check_out(out, a->count, 2, a->level);
    need(out->data != a->data, SS_ERR_PARAM, "rotation output must not alias its input");
    ss::Buf o = as_out(out);
    ss::op_rotate(ctx->C, *ss::view_buf(*a), g, o, S(stream));
    write_back(o, out);
  });
}

ss_status ss_rotate_sum(ss_ctx* ctx, const ss_ct* a, ss_ct* out, ss_stream stream) {
  return guard([&] {
    need(ctx != nullptr, SS_ERR_PARAM, "null context");
    check_ct(ctx->C, a, "null a");
    auto r = ss::plan_then_run(ctx->C, [&] { return ss::ev_rotate_sum(ctx->C, ss::view_buf(*a), S(stream)); });
    deliver(ctx->C, r, out, S(stream));
  });
}

ss_status ss_eval_g(ss_ctx* ctx, const ss_ct* x, int32_t e, ss_ct* out, ss_stream stream) {
  return guard([&] {
    need(ctx != nullptr, SS_ERR_PARAM, "null context");
    check_ct(ctx->C, x, "null x");
    need(e >= 1 && e <= x->t_exp, SS_ERR_TMOD, "G_{p,e} needs e <= t_exp");
    auto r = ss::plan_then_run(ctx->C, [&] { return ss::ev_eval_g(ctx->C, ss::view_buf(*x), e, S(stream)); });
    deliver(ctx->C, r, out, S(stream));
  });
}

ss_status ss_reduce_to_digits(ss_ctx* ctx, const ss_ct* a, ss_ct* digits, ss_stream stream) {
  return guard([&] {
    need(ctx != nullptr && digits != nullptr, SS_ERR_PARAM, "null argument");
    check_ct(ctx->C, a, "null a");
    auto d = ss::plan_then_run(ctx->C, [&] { return ss::ev_reduce(ctx->C, ss::view_buf(*a), S(stream)); });
    for (size_t i = 0; i < d.size(); ++i) deliver(ctx->C, d[i], &digits[i], S(stream));
  });
}

ss_status ss_compare_lt(ss_ctx* ctx, const ss_ct* a, const ss_ct* b, ss_ct* out, ss_stream stream) {
  return guard([&] {
    need(ctx != nullptr, SS_ERR_PARAM, "null context");
    check_ct(ctx->C, a, "null a");
    check_ct(ctx->C, b, "null b");
    auto r = ss::plan_then_run(ctx->C, [&] {
      return ss::ev_compare_lt(ctx->C, ss::view_buf(*a), ss::view_buf(*b), S(stream));
    });
    deliver(ctx->C, r, out, S(stream));
  });
}

ss_status ss_compare(ss_ctx* ctx, int32_t pred, const ss_ct* a, const ss_ct* b, ss_ct* out, ss_stream stream) {
  return guard([&] {
    need(ctx != nullptr, SS_ERR_PARAM, "null context");
    need(pred >= SS_PRED_LT && pred <= SS_PRED_NEQ, SS_ERR_PARAM, "unknown predicate");
    check_ct(ctx->C, a, "null a");
    check_ct(ctx->C, b, "null b");
    auto r = ss::plan_then_run(ctx->C, [&] {
      return ss::ev_compare(ctx->C, pred, ss::view_buf(*a), ss::view_buf(*b), S(stream));
    });
    deliver(ctx->C, r, out, S(stream));
  });
}

ss_status ss_raise_modulus(ss_ctx* ctx, const ss_ct* in, ss_ct* out, ss_stream stream) {
  return guard([&] {
    need(ctx != nullptr, SS_ERR_PARAM, "null context");
    check_ct(ctx->C, in, "null input");
    auto r = ss::plan_then_run(ctx->C, [&] { return ss::ev_raise(ctx->C, ss::view_buf(*in), S(stream)); });
    deliver(ctx->C, r, out, S(stream));
  });
}

ss_status ss_query_sum_where_lt(ss_ctx* ctx, const ss_ct* A, const ss_ct* B, const ss_ct* C1, const ss_ct* C2,
                                ss_ct* out, ss_stream stream) {
  return guard([&] {
    need(ctx != nullptr, SS_ERR_PARAM, "null context");
    for (const ss_ct* c : {A, B, C1, C2}) check_ct(ctx->C, c, "null column");
    auto r = ss::plan_then_run(ctx->C, [&] {
      return ss::ev_query(ctx->C, ss::view_buf(*A), ss::view_buf(*B), ss::view_buf(*C1), ss::view_buf(*C2),
                          S(stream));
    });
    deliver(ctx->C, r, out, S(stream));
  });
}

ss_status ss_query_sum_where(ss_ctx* ctx, const ss_ct* A, const ss_ct* B, const ss_cond* conds, int32_t n_conds,
                             ss_ct* out, ss_stream stream) {
  return guard([&] {
    need(ctx != nullptr && conds != nullptr && n_conds >= 1, SS_ERR_PARAM, "bad argument");
    check_ct(ctx->C, A, "null column");
    check_ct(ctx->C, B, "null column");
    std::vector<ss::QCond> qc;
    for (int k = 0; k < n_conds; ++k) {
      need(conds[k].pred >= SS_PRED_LT && conds[k].pred <= SS_PRED_NEQ, SS_ERR_PARAM, "unknown predicate");
      check_ct(ctx->C, conds[k].x, "null condition column");
      check_ct(ctx->C, conds[k].y, "null condition column");
      qc.push_back({conds[k].pred, ss::view_buf(*conds[k].x), ss::view_buf(*conds[k].y)});
    }
    auto r = ss::plan_then_run(ctx->C, [&] {
      return ss::ev_query_where(ctx->C, ss::view_buf(*A), ss::view_buf(*B), qc, S(stream));
    });
    deliver(ctx->C, r, out, S(stream));
  });
}

ss_status ss_query_sum_where_lt_host(ss_ctx* ctx, const uint64_t* A, const uint64_t* B, const uint64_t* C1,
                                     const uint64_t* C2, int32_t count, int32_t count2, int32_t level,
                                     uint64_t* host_out, int32_t* out_level, int32_t* out_t_exp, ss_stream stream) {
  return guard([&] {
    need(ctx && A && B && C1 && C2 && host_out && count >= 1 && (count2 == 1 || count2 == count), SS_ERR_PARAM,
         "bad argument");
    ss::Context& C = ctx->C;
    need(level >= 1 && level <= C.L, SS_ERR_LEVEL, "bad level");
    cudaStream_t st = S(stream);
    size_t ct_words = (size_t)2 * level * C.N;
    {  // the plan first: a chain too short for the query fails here, before any copy or launch
      ss::PlanScope ps(C);
      auto col = [&](int n) { return ss::alloc_buf(C, n, 2, level, C.r, st); };
      ss::ev_query_where(C, col(count), col(count), {ss::QCond{SS_PRED_LT, col(count), col(count2)}}, st);
    }
    // Buffers come from the pool on st. The comparison columns are copied on
    // st; A and B on a second stream that starts once the allocations are
    // ordered, so their upload overlaps the comparisons (the first product
    // waits for it). Everything is freed on st after the final synchronise.
    ss::BufP a = ss::alloc_buf(C, count, 2, level, C.r, st), b = ss::alloc_buf(C, count, 2, level, C.r, st);
    ss::BufP c1 = ss::alloc_buf(C, count, 2, level, C.r, st), c2 = ss::alloc_buf(C, count2, 2, level, C.r, st);
    cudaStream_t s2 = nullptr;
    cudaEvent_t allocated = nullptr, ab_ready = nullptr;
    auto cleanup = [&] {
      if (s2) cudaStreamSynchronize(s2);
      if (allocated) cudaEventDestroy(allocated);
      if (ab_ready) cudaEventDestroy(ab_ready);
      if (s2) cudaStreamDestroy(s2);
    };
    try {
      SS_CUDA(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
      SS_CUDA(cudaEventCreateWithFlags(&allocated, cudaEventDisableTiming));
      SS_CUDA(cudaEventCreateWithFlags(&ab_ready, cudaEventDisableTiming));
      SS_CUDA(cudaMemcpyAsync(c1->data, C1, count * ct_words * 8, cudaMemcpyHostToDevice, st));
      SS_CUDA(cudaMemcpyAsync(c2->data, C2, count2 * ct_words * 8, cudaMemcpyHostToDevice, st));
      SS_CUDA(cudaEventRecord(allocated, st));
      SS_CUDA(cudaStreamWaitEvent(s2, allocated, 0));
      SS_CUDA(cudaMemcpyAsync(a->data, A, count * ct_words * 8, cudaMemcpyHostToDevice, s2));
      SS_CUDA(cudaMemcpyAsync(b->data, B, count * ct_words * 8, cudaMemcpyHostToDevice, s2));
      SS_CUDA(cudaEventRecord(ab_ready, s2));
      ss::BufP r = ss::ev_query_where(C, a, b, {ss::QCond{SS_PRED_LT, c1, c2}}, st, ab_ready);
      size_t row = (size_t)r->level * C.N * 8;
      SS_CUDA(cudaMemcpy2DAsync(host_out, row, r->data, (size_t)r->cap * C.N * 8, row, 2, cudaMemcpyDeviceToHost,
                                st));
      SS_CUDA(cudaStreamSynchronize(st));
      if (out_level) *out_level = r->level;
      if (out_t_exp) *out_t_exp = r->t_exp;
    } catch (...) {
      cudaStreamSynchronize(st);
      cleanup();
      throw;
    }
    cleanup();
  });
}

ss_status ss_query_depth(ss_ctx* ctx, int32_t level, int32_t* out_level) {
  return guard([&] {
    need(ctx && out_level, SS_ERR_PARAM, "null argument");
    *out_level = ss::plan_query_depth(ctx->C, level);
  });
}

ss_status ss_query_bytes(const ss_ctx* ctx, int32_t n_ct, int32_t level, uint64_t* bytes) {
  return guard([&] {
    need(ctx && bytes && n_ct >= 1, SS_ERR_PARAM, "bad argument");
    need(level >= 1 && level <= ctx->C.L, SS_ERR_LEVEL, "bad level");
    *bytes = ss::query_bytes_estimate(ctx->C, n_ct, level);
  });
}

ss_status ss_set_g_table(ss_ctx* ctx, int32_t mode) {
  return guard([&] {
    need(ctx && (mode == 0 || mode == 1), SS_ERR_PARAM, "G table mode must be 0 or 1");
    ctx->C.reduced_g = mode == 1;
  });
}

ss_status ss_set_batch(ss_ctx* ctx, int32_t batch) {
  return guard([&] {
    need(ctx && batch >= 1, SS_ERR_PARAM, "bad batch");
    ctx->C.batch = batch;
  });
}

static ss_status raw_ntt(ss_ctx* ctx, bool fwd, uint64_t* data, int32_t npoly, int32_t first, int32_t nprimes,
                         ss_stream stream) {
  return guard([&] {
    need(ctx && data && npoly >= 1 && nprimes >= 1, SS_ERR_PARAM, "bad argument");
    ss::Context& C = ctx->C;
    need(first >= 0 && first + nprimes <= C.L, SS_ERR_PARAM, "prime range outside the data primes");
    need(npoly % nprimes == 0, SS_ERR_SHAPE, "npoly must be a multiple of nprimes");
    ss::PolySet s{data, (long)nprimes * C.N, npoly / nprimes, nprimes, first, nprimes};
    if (fwd) ss::ntt_forward(C, s, S(stream));
    else ss::ntt_inverse(C, s, S(stream));
  });
}

ss_status ss_ntt_forward(ss_ctx* ctx, uint64_t* d, int32_t n, int32_t f, int32_t np, ss_stream s) {
  return raw_ntt(ctx, true, d, n, f, np, s);
}
ss_status ss_ntt_inverse(ss_ctx* ctx, uint64_t* d, int32_t n, int32_t f, int32_t np, ss_stream s) {
  return raw_ntt(ctx, false, d, n, f, np, s);
}

ss_status ss_trace(ss_ctx* ctx, int32_t on) {
  return guard([&] {
    need(ctx != nullptr, SS_ERR_PARAM, "null context");
    ctx->C.trace_on = on != 0;
    ctx->C.trace.clear();
  });
}

int32_t ss_trace_get(ss_ctx* ctx, char* buf, int32_t len) {
  if (!ctx) return -1;
  std::string s;
  for (auto& o : ctx->C.trace) { s += o; s += '\n'; }
  if (buf && len > 0) {
    int n = (int)std::min<size_t>(s.size(), (size_t)len - 1);
    std::memcpy(buf, s.data(), n);
    buf[n] = 0;
  }
  return (int32_t)s.size();
}

ss_status ss_kernel_timing(ss_ctx* ctx, int32_t on) {
  return guard([&] {
    need(ctx != nullptr, SS_ERR_PARAM, "null context");
    ss::Context& C = ctx->C;
    ss::kt_collect(C);
    if (on) {
      for (int k = 0; k < ss::KC_N; ++k) { C.kt.launches[k] = 0; C.kt.ms[k] = 0; C.kt.bytes[k] = 0; }
      C.kt.ntt_products = 0;
      for (int k = 0; k < ss::ST_N; ++k) { C.kt.st_count[k] = 0; C.kt.st_ms[k] = 0; }
    }
    C.kt.on = on != 0;
  });
}

ss_status ss_kernel_stats(ss_ctx* ctx, int32_t cls, uint64_t* launches, double* ms, double* bytes) {
  return guard([&] {
    need(ctx != nullptr && cls >= 0 && cls < ss::KC_N, SS_ERR_PARAM, "bad argument");
    ss::Context& C = ctx->C;
    ss::kt_collect(C);
    if (launches) *launches = C.kt.launches[cls];
    if (ms) *ms = C.kt.ms[cls];
    if (bytes) *bytes = C.kt.bytes[cls];
  });
}

ss_status ss_ntt_products(ss_ctx* ctx, double* products) {
  return guard([&] {
    need(ctx != nullptr && products != nullptr, SS_ERR_PARAM, "null argument");
    *products = ctx->C.kt.ntt_products;
  });
}

ss_status ss_stage_stats(ss_ctx* ctx, int32_t stage, uint64_t* count, double* ms) {
  return guard([&] {
    need(ctx != nullptr && stage >= 0 && stage < ss::ST_N, SS_ERR_PARAM, "bad argument");
    ss::Context& C = ctx->C;
    ss::kt_collect(C);
    if (count) *count = C.kt.st_count[stage];
    if (ms) *ms = C.kt.st_ms[stage];
  });
}

ss_status ss_alu_probe(int32_t kind, int32_t iters, double* per_second) {
  return guard([&] {
    need(kind >= 0 && kind <= 2 && iters >= 1 && iters <= (1 << 20) && per_second, SS_ERR_PARAM, "bad argument");
    *per_second = ss::alu_probe(kind, iters);
  });
}

uint64_t ss_launch_count(const ss_ctx* ctx) { return ctx ? ctx->C.launches.load() : 0; }

}  // extern "C"
