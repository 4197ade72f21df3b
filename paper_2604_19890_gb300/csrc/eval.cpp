// Evaluator for space switching on ciphertext batches. One schedule serves
// every ciphertext of a batch, so each kernel launch covers the whole batch.
//
// Schedule (fixed, so that results are reproducible word for word):
//  * multiplication: align both operands to the lower level by modulus
//    switching the higher one (dropping all extra primes at once), tensor,
//    then relinearise and drop exactly one prime in one ModDown by q_{l-1} P;
//  * linear combinations: a term above the combination's level is scaled at
//    its own level, then switched down; terms already at that level are
//    scaled and summed in one pass;
//  * powers of y: y^e = (y^(e/2))^2 when e is a power of two, otherwise
//    y^(2^floor(log2 e)) * y^(e - 2^floor(log2 e));
//  * Paterson-Stockmeyer (Theorem 2) for H(y) = sum_j h_j y^j:
//    k = 2^ceil(floor(log2(n+1))/2) baby steps y^1..y^(k-1), giant steps
//    y^(k 2^i), coefficient vector padded to k 2^m >= n+1 and split in halves
//    recursively (H = H_lo + H_hi * y^half); empty halves are skipped and a
//    half that is a bare constant multiplies the giant step as a scalar;
//  * G_{p,e}(x) = x * H(x^2) with H the odd coefficients (Section 4.2);
//  * per digit: F_LT(x) = x * H_LT(x^2) + c_(p-1) y^((p-1)/2) and
//    F_EQ(x) = 1 - y^((p-1)/2), sharing y = x^2 (Section 4.3).
#include <algorithm>
#include <functional>
#include <map>

#include "ss_internal.h"

namespace ss {

static std::string L_(int l) { return "L" + std::to_string(l); }

// ------------------------------------------------------------------ primitives
BufP ev_modswitch_to(Context& C, const BufP& a, int level, cudaStream_t st) {
  if (level == a->level) return a;
  if (level > a->level) throw Error(SS_ERR_LEVEL, "cannot raise a level");
  if (level < 1) throw Error(SS_ERR_NOISE, "the plan needs more levels than the chain has");
  BufP out = alloc_buf(C, a->count, a->ncomp, level, a->t_exp, st);
  if (!is_dry(C)) op_modswitch(C, *a, a->level - level, *out, st);
  return out;
}

static void same_t(const BufP& a, const BufP& b) {
  if (a->t_exp != b->t_exp) throw Error(SS_ERR_TMOD, "plaintext moduli differ");
}

static int out_count(const BufP& a, const BufP& b) {
  if (a->count == b->count) return a->count;
  if (b->count == 1) return a->count;
  if (a->count == 1) return b->count;
  throw Error(SS_ERR_SHAPE, "batch sizes differ");
}

static BufP binary(Context& C, int op, const BufP& a0, const BufP& b0, cudaStream_t st) {
  same_t(a0, b0);
  if (a0->ncomp != b0->ncomp) throw Error(SS_ERR_SHAPE, "component counts differ");
  int l = std::min(a0->level, b0->level);
  BufP a = ev_modswitch_to(C, a0, l, st), b = ev_modswitch_to(C, b0, l, st);
  if (a->count == 1 && b->count > 1) {
    // a - b with a broadcast: -(b - a), the same canonical residues word for word
    if (op == 1) return ev_scalar(C, 0, binary(C, 1, b, a, st), -1, st);
    std::swap(a, b);
  }
  BufP out = alloc_buf(C, out_count(a, b), a->ncomp, l, a->t_exp, st);
  if (!is_dry(C)) k_binary(C, op, *a, *b, *out, st);
  return out;
}

BufP ev_add(Context& C, const BufP& a, const BufP& b, cudaStream_t st) { return binary(C, 0, a, b, st); }
BufP ev_sub(Context& C, const BufP& a, const BufP& b, cudaStream_t st) { return binary(C, 1, a, b, st); }

BufP ev_scalar(Context& C, int op, const BufP& a, i64 c, cudaStream_t st) {
  BufP out = alloc_buf(C, a->count, a->ncomp, a->level, op == 2 ? a->t_exp - 1 : a->t_exp, st);
  if (!is_dry(C)) k_scalar(C, op, *a, c, *out, st);
  return out;
}

// sum_t c_t * y_t + cst (cst on component 0), all terms aligned to the lowest
// level; equal word for word to the chain of scalar products and additions.
BufP ev_lincomb(Context& C, const std::vector<std::pair<BufP, i64>>& terms, i64 cst, cudaStream_t st) {
  if (terms.empty()) throw Error(SS_ERR_PARAM, "empty linear combination");
  int l = terms[0].first->level, cnt = terms[0].first->count;
  for (auto& t : terms) {
    same_t(terms[0].first, t.first);
    if (t.first->ncomp != 2) throw Error(SS_ERR_SHAPE, "linear combination of 2-component ciphertexts");
    if (t.first->count != cnt) throw Error(SS_ERR_SHAPE, "batch sizes differ");
    l = std::min(l, t.first->level);
  }
  // A term above the common level is scaled at its own level and then switched
  // down (modulus switching does not commute word for word with scaling, and
  // scaling first keeps the rounding noise unscaled).
  std::vector<BufP> al;
  std::vector<i64> cf;
  for (auto& t : terms) {
    if (t.first->level > l && t.second != 1) {
      al.push_back(ev_modswitch_to(C, ev_scalar(C, 0, t.first, t.second, st), l, st));
      cf.push_back(1);
    } else {
      al.push_back(ev_modswitch_to(C, t.first, l, st));
      cf.push_back(t.second);
    }
  }
  BufP acc;
  size_t i = 0;
  while (i < al.size()) {
    std::vector<const Buf*> ys;
    std::vector<i64> cs;
    if (acc) { ys.push_back(acc.get()); cs.push_back(1); }
    while (i < al.size() && ys.size() < 16) { ys.push_back(al[i].get()); cs.push_back(cf[i]); ++i; }
    BufP out = alloc_buf(C, cnt, 2, l, terms[0].first->t_exp, st);
    if (!is_dry(C)) k_lincomb(C, ys, cs, i == al.size() ? cst : 0, *out, st);
    acc = out;
  }
  return acc;
}

BufP ev_mul(Context& C, const BufP& a0, const BufP& b0, cudaStream_t st) {
  same_t(a0, b0);
  if (a0->ncomp != 2 || b0->ncomp != 2) throw Error(SS_ERR_SHAPE, "multiplication needs 2-component inputs");
  int l = std::min(a0->level, b0->level);
  if (l < 2) throw Error(SS_ERR_NOISE, "the plan needs more levels than the chain has");
  BufP a = ev_modswitch_to(C, a0, l, st), b = ev_modswitch_to(C, b0, l, st);
  if (a->count != b->count) throw Error(SS_ERR_SHAPE, "batch sizes differ");
  BufP t3 = alloc_buf(C, a->count, 3, l, a->t_exp, st);
  BufP out = alloc_buf(C, a->count, 2, l - 1, a->t_exp, st);
  if (!is_dry(C)) {
    k_tensor(C, *a, *b, *t3, st);
    op_relin_drop(C, *t3, *out, st);
  }
  return out;
}

// ------------------------------------------------------------------ powers and BSGS
namespace {

struct Powers {
  Context& C;
  cudaStream_t st;
  std::map<int, BufP> pw;
  std::map<std::pair<int, int>, BufP> aligned;
  Powers(Context& c, const BufP& y, cudaStream_t s) : C(c), st(s) { pw[1] = y; }
  BufP get(int e) {
    auto it = pw.find(e);
    if (it != pw.end()) return it->second;
    int h = 1;
    while (h * 2 <= e) h *= 2;
    BufP r;
    if (h == e) {
      BufP z = get(e / 2);
      r = ev_mul(C, z, z, st);
      note(C, "pow " + std::to_string(e) + " = sq " + std::to_string(e / 2) + " -> " + L_(r->level));
    } else {
      BufP a = get(h);
      BufP b = get(e - h);
      r = ev_mul(C, a, b, st);
      note(C, "pow " + std::to_string(e) + " = " + std::to_string(h) + "*" + std::to_string(e - h) + " -> " +
                  L_(r->level));
    }
    pw[e] = r;
    return r;
  }
  BufP at_level(int e, int level) {
    BufP x = get(e);
    if (x->level == level) return x;
    auto key = std::make_pair(e, level);
    auto it = aligned.find(key);
    if (it != aligned.end()) return it->second;
    BufP r = ev_modswitch_to(C, x, level, st);
    aligned[key] = r;
    return r;
  }
};

struct Term {
  BufP ct;  // null when the value is a bare constant
  i64 cst = 0;
};

Term bsgs(Context& C, const std::vector<i64>& h, Powers& P, cudaStream_t st) {
  int n1 = (int)h.size();
  int lg = 0;
  while ((2 << lg) <= n1) ++lg;
  int k = 1 << ((lg + 1) / 2);
  int len = k;
  while (len < n1) len *= 2;
  std::vector<i64> c(len, 0);
  std::copy(h.begin(), h.end(), c.begin());
  note(C, "bsgs n+1=" + std::to_string(n1) + " k=" + std::to_string(k) + " len=" + std::to_string(len));
  auto nonzero = [&](int lo) {
    std::vector<int> idx;
    for (int i = 1; i < k; ++i)
      if (c[lo + i] != 0) idx.push_back(i);
    return idx;
  };
  // Leaf combinations computed ahead, several per pass over the baby steps
  // (k_lincomb_multi reads each aligned baby step once for up to 16 leaves).
  // A leaf joins when its terms are among the first leaf's and its common
  // level is the first leaf's; each result equals its own linear combination.
  std::map<int, BufP> ahead;
  auto plan_leaves = [&](const std::vector<int>& idx0, int lvl0) {
    if (idx0.size() > 16) return;
    std::vector<int> los;
    for (int lo = 0; lo < len; lo += k) {
      std::vector<int> idx = nonzero(lo);
      if (idx.empty()) continue;
      bool inside = true;
      int lvl = 1 << 30;
      for (int i : idx) {
        if (!std::binary_search(idx0.begin(), idx0.end(), i)) { inside = false; break; }
        lvl = std::min(lvl, P.get(i)->level);
      }
      if (inside && lvl == lvl0) los.push_back(lo);
    }
    if (los.size() < 2) return;
    std::vector<const Buf*> ys;
    for (int i : idx0) ys.push_back(P.at_level(i, lvl0).get());
    const Buf& y0 = *ys[0];
    for (size_t b = 0; b < los.size(); b += 16) {
      std::vector<std::vector<i64>> cs;
      std::vector<Buf*> outs;
      for (size_t j = b; j < los.size() && j < b + 16; ++j) {
        std::vector<i64> row;
        for (int i : idx0) row.push_back(c[los[j] + i]);
        cs.push_back(row);
        BufP o = alloc_buf(C, y0.count, 2, lvl0, y0.t_exp, st);
        ahead[los[j]] = o;
        outs.push_back(o.get());
      }
      if (!is_dry(C)) k_lincomb_multi(C, ys, cs, outs, st);
    }
  };
  std::function<Term(int, int)> rec = [&](int lo, int ln) -> Term {
    Term out;
    if (ln == k) {
      out.cst = c[lo];
      std::vector<int> idx = nonzero(lo);
      if (idx.empty()) return out;
      int lvl = 1 << 30;
      for (int i : idx) lvl = std::min(lvl, P.get(i)->level);
      if (lo == 0) plan_leaves(idx, lvl);
      auto it = ahead.find(lo);
      if (it != ahead.end()) {
        out.ct = it->second;
      } else {
        std::vector<std::pair<BufP, i64>> terms;
        for (int i : idx) terms.push_back({P.at_level(i, lvl), c[lo + i]});
        out.ct = ev_lincomb(C, terms, 0, st);
      }
      note(C, "baby lo=" + std::to_string(lo) + " terms=" + std::to_string(idx.size()) + " " + L_(lvl));
      return out;
    }
    int half = ln / 2;
    Term A = rec(lo, half), B = rec(lo + half, half);
    if (!B.ct && B.cst == 0) return A;
    BufP G = P.get(half);
    out.cst = A.cst;
    if (B.ct) {
      BufP b = B.cst != 0 ? ev_scalar(C, 1, B.ct, B.cst, st) : B.ct;
      BufP prod = ev_mul(C, b, G, st);
      out.ct = A.ct ? ev_add(C, A.ct, prod, st) : prod;
    } else if (A.ct) {
      out.ct = ev_lincomb(C, {{A.ct, 1}, {G, B.cst}}, 0, st);
    } else {
      out.ct = ev_lincomb(C, {{G, B.cst}}, 0, st);
    }
    note(C, "giant lo=" + std::to_string(lo) + " half=" + std::to_string(half) + " -> " + L_(out.ct->level));
    return out;
  };
  return rec(0, len);
}

BufP mul_term(Context& C, const BufP& x, const Term& T, cudaStream_t st) {
  if (!T.ct) return ev_scalar(C, 0, x, T.cst, st);
  BufP b = T.cst != 0 ? ev_scalar(C, 1, T.ct, T.cst, st) : T.ct;
  return ev_mul(C, x, b, st);
}

}  // namespace

// ------------------------------------------------------------------ space switching
BufP ev_eval_g(Context& C, const BufP& x, int e, cudaStream_t st) {
  std::vector<i64> g = C.reduced_g ? nt::g_coeffs_reduced(C.p, e) : nt::g_coeffs(C.p, e);
  std::vector<i64> h;
  for (size_t i = 1; i < g.size(); i += 2) h.push_back(g[i]);
  while (h.size() > 1 && h.back() == 0) h.pop_back();
  note(C, "G p=" + std::to_string(C.p) + " e=" + std::to_string(e) + " in " + L_(x->level));
  BufP y = ev_mul(C, x, x, st);
  Powers P(C, y, st);
  Term H = bsgs(C, h, P, st);
  BufP out = mul_term(C, x, H, st);
  note(C, "G done -> " + L_(out->level));
  return out;
}

// Algorithm 3
std::vector<BufP> ev_reduce(Context& C, const BufP& a, cudaStream_t st) {
  int r = C.r;
  if (a->t_exp != r) throw Error(SS_ERR_TMOD, "reduction input must be at t = p^r");
  std::vector<BufP> digits;
  BufP b = a;
  for (int i = 0; i + 1 < r; ++i) {
    BufP ai = ev_eval_g(C, b, r - i, st);
    BufP diff = ev_sub(C, ev_modswitch_to(C, b, ai->level, st), ai, st);
    b = ev_scalar(C, 2, diff, 0, st);  // DivideByP
    note(C, "digit " + std::to_string(i) + " " + L_(ai->level));
    digits.push_back(ai);
  }
  digits.push_back(b);
  std::vector<BufP> out;
  for (auto& d : digits) {  // ChangeModToP: same words, t <- p
    auto v = std::make_shared<Buf>(*d);
    v->owned = false;
    v->parent = d;
    v->t_exp = 1;
    out.push_back(v);
  }
  return out;
}

static void compare_digit(Context& C, const BufP& x, BufP& lt, BufP& eq, cudaStream_t st) {
  int p = C.p;
  std::vector<i64> f = nt::flt_coeffs(p);
  std::vector<i64> h;
  for (int i = 1; i <= p - 2; i += 2) h.push_back(f[i]);
  while (h.size() > 1 && h.back() == 0) h.pop_back();
  BufP y = ev_mul(C, x, x, st);
  Powers P(C, y, st);
  Term H = bsgs(C, h, P, st);
  BufP T = P.get((p - 1) / 2);
  lt = ev_lincomb(C, {{mul_term(C, x, H, st), 1}, {T, f[p - 1]}}, 0, st);
  eq = ev_lincomb(C, {{T, -1}}, 1, st);
  note(C, "cmp digit -> LT " + L_(lt->level) + " EQ " + L_(eq->level));
}

// Algorithm 4
BufP ev_compare_lt(Context& C, const BufP& a, const BufP& b, cudaStream_t st) {
  int r = C.r;
  std::vector<BufP> dg;
  {
    StageScope sc(C, ST_REDUCE, st);
    dg = ev_reduce(C, ev_sub(C, a, b, st), st);
  }
  std::vector<BufP> LT(r), EQ(r);
  {
    StageScope sc(C, ST_COMPARE, st);
    for (int i = 0; i < r; ++i) compare_digit(C, dg[i], LT[i], EQ[i], st);
  }
  StageScope sc(C, ST_AGGREGATE, st);
  BufP lt = LT[r - 1], eq = EQ[r - 1];
  for (int i = r - 2; i >= 0; --i) {
    lt = ev_add(C, lt, ev_mul(C, eq, LT[i], st), st);
    if (i > 0) eq = ev_mul(C, eq, EQ[i], st);
  }
  note(C, "LT -> " + L_(lt->level));
  return lt;
}

// Per-digit EQ against zero alone (Section 4.3): F_EQ(x) = 1 - x^(p-1) as
// 1 - y^((p-1)/2), y = x^2, the power built by the Powers rule.
static BufP eq_digit(Context& C, const BufP& x, cudaStream_t st) {
  BufP y = ev_mul(C, x, x, st);
  Powers P(C, y, st);
  BufP eq = ev_lincomb(C, {{P.get((C.p - 1) / 2), -1}}, 1, st);
  note(C, "eq digit -> EQ " + L_(eq->level));
  return eq;
}

// Section 4.3, EQ: Reduce(a - b), F_EQ per digit, product from the most
// significant digit down.
BufP ev_compare_eq(Context& C, const BufP& a, const BufP& b, cudaStream_t st) {
  int r = C.r;
  std::vector<BufP> dg;
  {
    StageScope sc(C, ST_REDUCE, st);
    dg = ev_reduce(C, ev_sub(C, a, b, st), st);
  }
  std::vector<BufP> EQ(r);
  {
    StageScope sc(C, ST_COMPARE, st);
    for (int i = 0; i < r; ++i) EQ[i] = eq_digit(C, dg[i], st);
  }
  StageScope sc(C, ST_AGGREGATE, st);
  BufP eq = EQ[r - 1];
  for (int i = r - 2; i >= 0; --i) eq = ev_mul(C, eq, EQ[i], st);
  note(C, "EQ -> " + L_(eq->level));
  return eq;
}

// 1 - x at t = p
static BufP complement(Context& C, const BufP& x, cudaStream_t st) {
  StageScope sc(C, ST_AGGREGATE, st);
  return ev_lincomb(C, {{x, -1}}, 1, st);
}

// Section 4.3: GT(a, b) = LT(b, a) on the symmetric centred range; NEQ, GE and
// LE are 1 - EQ, 1 - LT and 1 - GT.
BufP ev_compare(Context& C, int pred, const BufP& a, const BufP& b, cudaStream_t st) {
  switch (pred) {
    case SS_PRED_LT: return ev_compare_lt(C, a, b, st);
    case SS_PRED_LE: return complement(C, ev_compare_lt(C, b, a, st), st);
    case SS_PRED_GT: return ev_compare_lt(C, b, a, st);
    case SS_PRED_GE: return complement(C, ev_compare_lt(C, a, b, st), st);
    case SS_PRED_EQ: return ev_compare_eq(C, a, b, st);
    case SS_PRED_NEQ: return complement(C, ev_compare_eq(C, a, b, st), st);
    default: throw Error(SS_ERR_PARAM, "unknown predicate");
  }
}

// Section 4.4
BufP ev_raise(Context& C, const BufP& a, cudaStream_t st) {
  if (a->t_exp != 1) throw Error(SS_ERR_TMOD, "raise input must be at t = p");
  StageScope sc(C, ST_RAISE, st);
  auto k = std::make_shared<Buf>(*a);
  k->owned = false;
  k->parent = a;
  k->t_exp = C.r;
  BufP out = ev_eval_g(C, k, C.r, st);
  note(C, "raise -> " + L_(out->level));
  return out;
}

BufP ev_rotate_sum(Context& C, const BufP& a, cudaStream_t st) {
  StageScope sc(C, ST_SUM, st);
  BufP s = a;
  for (int g : rotate_sum_elements(C)) {
    BufP r = alloc_buf(C, s->count, 2, s->level, s->t_exp, st);
    if (!is_dry(C)) op_rotate(C, *s, g, *r, st);
    s = ev_add(C, s, r, st);
    note(C, "rot " + std::to_string(g));
  }
  return s;
}

static BufP batch_total(Context& C, const BufP& R, cudaStream_t st) {
  if (R->count == 1) return R;
  StageScope sc(C, ST_SUM, st);
  BufP out = alloc_buf(C, 1, R->ncomp, R->level, R->t_exp, st);
  if (!is_dry(C)) k_batch_sum(C, *R, *out, st);
  return out;
}

// SUM(A*B) over the rows where every condition holds, per ciphertext: the
// conditions' indicators (t = p) are multiplied in order (AND) and raised once,
// ind = Raise(prod_k cond_k), R = ind*(A*B), total = rotate_sum(sum R).
// Ciphertexts are processed C.batch at a time.
BufP ev_query_where(Context& C, const BufP& A, const BufP& B, const std::vector<QCond>& conds, cudaStream_t st,
                    cudaEvent_t ab_ready) {
  int n = A->count;
  if (conds.empty()) throw Error(SS_ERR_PARAM, "a query needs at least one condition");
  if (B->count != n) throw Error(SS_ERR_SHAPE, "column batch sizes differ");
  for (auto& c : conds)
    if (c.X->count != n || (c.Y->count != n && c.Y->count != 1)) throw Error(SS_ERR_SHAPE, "column batch sizes differ");
  BufP total;
  int step = std::max(1, C.batch);
  for (int b0 = 0; b0 < n; b0 += step) {
    int cnt = std::min(step, n - b0);
    BufP a = slice_buf(A, b0, cnt, C.N), b = slice_buf(B, b0, cnt, C.N);
    BufP ind;
    for (size_t k = 0; k < conds.size(); ++k) {
      const QCond& c = conds[k];
      BufP y = c.Y->count == 1 ? c.Y : slice_buf(c.Y, b0, cnt, C.N);
      BufP v = ev_compare(C, c.pred, slice_buf(c.X, b0, cnt, C.N), y, st);
      if (k == 0) {
        ind = v;
      } else {
        StageScope sc(C, ST_AGGREGATE, st);
        ind = ev_mul(C, ind, v, st);
      }
    }
    ind = ev_raise(C, ind, st);
    if (ab_ready && !is_dry(C) && b0 == 0) SS_CUDA(cudaStreamWaitEvent(st, ab_ready, 0));  // A and B still arriving
    BufP R;
    {
      StageScope sc(C, ST_PRODUCT, st);
      R = ev_mul(C, ind, ev_mul(C, a, b, st), st);
    }
    BufP part = batch_total(C, R, st);
    StageScope sc(C, ST_SUM, st);
    total = total ? ev_add(C, total, part, st) : part;
  }
  return ev_rotate_sum(C, total, st);
}

BufP ev_query(Context& C, const BufP& A, const BufP& B, const BufP& C1, const BufP& C2, cudaStream_t st) {
  if (C1->count != A->count || (C2->count != A->count && C2->count != 1))
    throw Error(SS_ERR_SHAPE, "column batch sizes differ");
  return ev_query_where(C, A, B, {QCond{SS_PRED_LT, C1, C2}}, st);
}

static thread_local const Context* t_plan_ctx = nullptr;

bool is_dry(const Context& C) { return t_plan_ctx == &C; }
PlanScope::PlanScope(const Context& C) : prev(t_plan_ctx) { t_plan_ctx = &C; }
PlanScope::~PlanScope() { t_plan_ctx = prev; }

int plan_query_depth(Context& C, int level) {
  PlanScope ps(C);
  auto x = std::make_shared<Buf>();
  x->count = 1;
  x->ncomp = 2;
  x->level = level;
  x->t_exp = C.r;
  x->cap = level;
  return ev_query(C, x, x, x, x, nullptr)->level;
}

}  // namespace ss

namespace ss {

// Batches with one shape, joined along the batch axis (a broadcast part of
// count 1 is repeated `rep` times).
BufP ev_concat(Context& C, const std::vector<std::pair<BufP, int>>& parts, cudaStream_t st) {
  int total = 0;
  for (auto& p : parts) total += p.second;
  const Buf& f = *parts[0].first;
  BufP out = alloc_buf(C, total, f.ncomp, f.level, f.t_exp, st);
  if (is_dry(C)) return out;
  const size_t row = (size_t)f.level * C.N * 8, ct = (size_t)f.ncomp * f.level * C.N;
  size_t off = 0;
  for (auto& p : parts) {
    const Buf& b = *p.first;
    if (b.level != f.level || b.ncomp != f.ncomp || b.t_exp != f.t_exp) throw Error(SS_ERR_SHAPE, "parts differ");
    if (b.count == p.second) {
      SS_CUDA(cudaMemcpy2DAsync(out->data + off * ct, row, b.data, (size_t)b.cap * C.N * 8, row,
                                (size_t)b.count * b.ncomp, cudaMemcpyDeviceToDevice, st));
    } else {
      for (int r = 0; r < p.second; ++r)
        SS_CUDA(cudaMemcpy2DAsync(out->data + (off + r) * ct, row, b.data, (size_t)b.cap * C.N * 8, row, b.ncomp,
                                  cudaMemcpyDeviceToDevice, st));
    }
    off += p.second;
  }
  return out;
}

// Several queries of one shape in one pass: their columns are joined into one
// batch, every ciphertext goes through the same schedule as ev_query, and the
// per-query sums are rotated and summed as one batch. Each result equals
// ev_query on that query alone word for word.
std::vector<BufP> ev_query_multi(Context& C, const std::vector<QueryCols>& qs, cudaStream_t st) {
  if (qs.empty()) return {};
  std::vector<std::pair<BufP, int>> a, b, c1, c2;
  std::vector<int> n;
  for (auto& q : qs) {
    int k = q.A->count;
    if (q.B->count != k || q.C1->count != k || (q.C2->count != k && q.C2->count != 1))
      throw Error(SS_ERR_SHAPE, "column batch sizes differ");
    n.push_back(k);
    a.push_back({q.A, k});
    b.push_back({q.B, k});
    c1.push_back({q.C1, k});
    c2.push_back({q.C2, k});
  }
  BufP A = ev_concat(C, a, st), B = ev_concat(C, b, st), C1 = ev_concat(C, c1, st), C2 = ev_concat(C, c2, st);
  const int total = A->count, step = std::max(1, C.batch);
  std::vector<std::pair<BufP, int>> Rs;
  for (int b0 = 0; b0 < total; b0 += step) {
    int cnt = std::min(step, total - b0);
    BufP ind = ev_raise(C, ev_compare_lt(C, slice_buf(C1, b0, cnt, C.N), slice_buf(C2, b0, cnt, C.N), st), st);
    StageScope sc(C, ST_PRODUCT, st);
    BufP R = ev_mul(C, ind, ev_mul(C, slice_buf(A, b0, cnt, C.N), slice_buf(B, b0, cnt, C.N), st), st);
    Rs.push_back({R, cnt});
  }
  BufP R = Rs.size() == 1 ? Rs[0].first : ev_concat(C, Rs, st);
  std::vector<std::pair<BufP, int>> parts;
  {
    StageScope sc(C, ST_SUM, st);
    int off = 0;
    for (int k : n) {
      BufP s = slice_buf(R, off, k, C.N);
      BufP part = alloc_buf(C, 1, R->ncomp, R->level, R->t_exp, st);
      if (!is_dry(C)) k_batch_sum(C, *s, *part, st);
      parts.push_back({part, 1});
      off += k;
    }
  }
  BufP S = ev_rotate_sum(C, parts.size() == 1 ? parts[0].first : ev_concat(C, parts, st), st);
  std::vector<BufP> out;
  for (size_t i = 0; i < qs.size(); ++i) out.push_back(slice_buf(S, (int)i, 1, C.N));
  return out;
}

// Device bytes a query of n_ct ciphertexts per column at `level` may hold at
// its peak (inputs joined, the live powers of one Paterson-Stockmeyer
// evaluation, key-switch scratch), for admission control.
size_t query_bytes_estimate(const Context& C, int n_ct, int level) {
  const size_t ct = (size_t)2 * level * C.N * 8;
  const int b = std::min(n_ct, std::max(1, C.batch));
  const int dn = (level + C.alpha - 1) / C.alpha, nx = level + C.alpha;
  const size_t ks = (size_t)b * ((size_t)dn * nx + 4 * (size_t)nx + 2 * (size_t)level) * C.N * 8;
  // columns + live intermediates of a pass (powers, up to 16 leaf combinations computed ahead) + key switch
  return 4 * (size_t)n_ct * ct + (size_t)b * ct * (48 + 16) + ks;
}

}  // namespace ss
