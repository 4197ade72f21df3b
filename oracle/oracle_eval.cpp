// Plain CPU reference: interpolation polynomials, the Paterson-Stockmeyer
// evaluation schedule and the space-switching procedures (reduction,
// comparison, modulus raising) plus the compare-then-SUM query.
// TEST INFRASTRUCTURE ONLY (see oracle.hpp).
#include "oracle.hpp"

#include <algorithm>
#include <cstdio>
#include <functional>

namespace orc {

static u64 ipow_u(u64 b, int e) { u64 r = 1; while (e-- > 0) r *= b; return r; }

static int vp_factorial(int k, int p) {
  int s = 0;
  for (long q = p; q <= k; q *= p) s += (int)(k / q);
  return s;
}

// G_{p,e} (Lemma 3): a polynomial of degree D = (e-1)(p-1)+1 with
// G(z0 + p z1) = z0 mod p^e for balanced z0 in (-p/2, p/2].
// Construction: Newton forward differences of f(x) = balanced(x mod p) on
// x = 0..D. Delta^k f(0) / k! is p-integral; the p-part of k! is divided out
// exactly and the unit part inverted mod p^e. The falling factorials are then
// expanded into monomials mod p^e. Finally the odd part (G(x) - G(-x))/2 is
// kept (f is odd for odd p), so G = x * H(x^2) (Section 4.2, Geelen et al.).
std::vector<i64> g_table(int p, int e) {
  int D = (e - 1) * (p - 1) + 1;
  u64 pe = ipow_u((u64)p, e);
  int vmax = vp_factorial(D, p);
  u64 M = pe * ipow_u((u64)p, vmax);  // work modulo p^(e + vmax) before division
  auto bal = [&](long x) -> i64 { long z = x % p; if (z < 0) z += p; return z > p / 2 ? z - p : z; };
  // forward differences: table[k] = Delta^k f(0) mod M, by repeated differencing
  std::vector<u64> row(D + 1);
  for (int x = 0; x <= D; ++x) row[x] = lift(bal(x), M);
  std::vector<u64> delta(D + 1);
  for (int k = 0; k <= D; ++k) {
    delta[k] = row[0];
    for (int x = 0; x + 1 < (int)row.size(); ++x) row[x] = submod(row[x + 1], row[x], M);
    row.pop_back();
  }
  std::vector<u64> coef(D + 1, 0);
  std::vector<u64> ff(1, 1);  // falling factorial x(x-1)...(x-k+1), mod p^e
  for (int k = 0; k <= D; ++k) {
    if (k > 0) {
      std::vector<u64> nf(ff.size() + 1, 0);
      for (size_t j = 0; j < ff.size(); ++j) {
        nf[j + 1] = addmod(nf[j + 1], ff[j], pe);
        nf[j] = submod(nf[j], mulmod(ff[j], (u64)(k - 1) % pe, pe), pe);
      }
      ff = nf;
    }
    int v = vp_factorial(k, p);
    u64 pv = ipow_u((u64)p, v);
    if (delta[k] % pv != 0) throw std::runtime_error("g_table: difference not p-integral");
    u64 num = (delta[k] / pv) % pe;
    // unit part of k!
    u64 unit = 1 % pe;
    for (int i = 1; i <= k; ++i) {
      long x = i;
      while (x % p == 0) x /= p;
      unit = mulmod(unit, (u64)x % pe, pe);
    }
    u64 ck = mulmod(num, invmod(unit, pe), pe);
    if (ck == 0) continue;
    for (size_t j = 0; j < ff.size(); ++j) coef[j] = addmod(coef[j], mulmod(ck, ff[j], pe), pe);
  }
  std::vector<i64> out(D + 1, 0);
  u64 inv2 = invmod(2, pe);
  for (int i = 0; i <= D; ++i) {
    u64 odd = (i % 2 == 1) ? mulmod(addmod(coef[i], coef[i], pe), inv2, pe) : 0;
    out[i] = centre(odd, pe);
  }
  return out;
}

// Lattice-reduced representative of G_{p,e} (Section 4.2: Geelen et al. replace
// G_{p,e} by an equivalent polynomial with smaller integer coefficients, which
// slows noise growth). Two integer polynomials agree on all of Z_{p^e} exactly
// when their difference is null mod p^e; in the falling-factorial basis the
// null polynomials are sum_k a_k (x)_k with p^(e - v_p(k!)) | a_k. Up to the
// degree D = (e-1)(p-1)+1 of G_{p,e}, with (x)_k = (x)_p (x-p)_(k-p) and
// (x)_p = x^p - x (mod p), the odd null polynomials modulo p^e are
//   e = 2:  a p (x^p - x),                          a in Z_p;
//   e = 3:  p^2 * odd part of (x^p - x) R(x),       R in F_p[x], deg R < p.
// Among G + (odd null polynomial) this returns the one whose centred
// coefficients have the least sum of absolute values, by exhaustive search.
// For e = 3, coefficient i (odd) of (x^p - x) R(x) is r_(i-p) - r_(i-1), so
// only the even-indexed r_m enter: coefficient 1 takes -r_0, p takes
// r_0 - r_(p-1), 2p-1 takes r_(p-1), and for even 2 <= m <= p-3 coefficient
// m+1 takes -r_m and p+m takes r_m; the choices of the r_m for 2 <= m <= p-3
// are independent, and (r_0, r_(p-1)) is searched jointly. Ties keep the
// smallest parameter (in [0, p), lexicographic for the joint pair). Other e:
// the canonical table.
std::vector<i64> g_table_reduced(int p, int e) {
  std::vector<i64> g = g_table(p, e);
  if (e != 2 && e != 3) return g;
  const i64 pe = (i64)ipow_u((u64)p, e);
  auto cen = [&](i64 v) {
    i64 z = v % pe;
    if (z < 0) z += pe;
    return z > pe / 2 ? z - pe : z;
  };
  auto mag = [&](int i, i64 delta) { i64 v = cen(g[i] + delta); return v < 0 ? -v : v; };
  std::vector<i64> out = g;
  if (e == 2) {
    const i64 P = p;
    i64 best = -1;
    int ba = 0;
    for (int a = 0; a < p; ++a) {
      i64 c = mag(1, -a * P) + mag(p, a * P);
      if (best < 0 || c < best) { best = c; ba = a; }
    }
    out[1] = cen(g[1] - ba * P);
    out[p] = cen(g[p] + ba * P);
    return out;
  }
  const i64 P2 = (i64)p * p;
  for (int m = 2; m <= p - 3; m += 2) {
    i64 best = -1;
    int br = 0;
    for (int r = 0; r < p; ++r) {
      i64 c = mag(m + 1, -r * P2) + mag(p + m, r * P2);
      if (best < 0 || c < best) { best = c; br = r; }
    }
    out[m + 1] = cen(g[m + 1] - br * P2);
    out[p + m] = cen(g[p + m] + br * P2);
  }
  i64 best = -1;
  int b0 = 0, b1 = 0;
  for (int r0 = 0; r0 < p; ++r0)
    for (int r1 = 0; r1 < p; ++r1) {
      i64 c = mag(1, -r0 * P2) + mag(p, (i64)(r0 - r1) * P2) + mag(2 * p - 1, r1 * P2);
      if (best < 0 || c < best) { best = c; b0 = r0; b1 = r1; }
    }
  out[1] = cen(g[1] - b0 * P2);
  out[p] = cen(g[p] + (i64)(b0 - b1) * P2);
  out[2 * p - 1] = cen(g[2 * p - 1] + b1 * P2);
  return out;
}

// F_LT (Section 4.3): ((p+1)/2) x^(p-1) + sum_{odd i <= p-2} c_i x^i with
// c_i = sum_{j=1}^{(p-1)/2} j^(p-1-i), all mod p.
std::vector<i64> flt_table(int p) {
  std::vector<i64> c(p, 0);
  c[p - 1] = centre((u64)(p + 1) / 2, (u64)p);
  for (int i = 1; i <= p - 2; i += 2) {
    u64 s = 0;
    for (int j = 1; j <= (p - 1) / 2; ++j) s = addmod(s, powmod((u64)j, (u64)(p - 1 - i), (u64)p), (u64)p);
    c[i] = centre(s, (u64)p);
  }
  return c;
}

// ------------------------------------------------------------- evaluation
static void note(Trace* tr, const std::string& s) {
  if (tr && tr->on) tr->ops.push_back(s);
}

// Noise meter (Section 2.1: decryption is correct while |v| < Q/2): records the
// budget of a stage's result when the trace's meter is set.
static void meter(const Context& C, Trace* tr, const std::string& label, const Ct& ct) {
  if (!tr || !tr->meter) return;
  char buf[160];
  std::snprintf(buf, sizeof(buf), "%s L%d %.3f", label.c_str(), ct.level, noise_budget(C, ct));
  tr->noise.push_back(buf);
}

static Ct align_to(const Context& C, const Ct& a, int level) { return modswitch_to(C, a, level); }

static Ct add_aligned(const Context& C, const Ct& a, const Ct& b) {
  int l = std::min(a.level, b.level);
  return add(C, align_to(C, a, l), align_to(C, b, l));
}

// Powers of y, each built from the lowest-depth product: y^e = (y^(e/2))^2 for
// e a power of two, otherwise y^(2^floor(log2 e)) * y^(e - 2^floor(log2 e)).
struct Powers {
  const Context& C;
  Trace* tr;
  std::map<int, Ct> pw;
  Powers(const Context& c, const Ct& y, Trace* t) : C(c), tr(t) { pw[1] = y; }
  const Ct& get(int e) {
    auto it = pw.find(e);
    if (it != pw.end()) return it->second;
    int h = 1;
    while (h * 2 <= e) h *= 2;
    Ct r;
    if (h == e) {
      const Ct& z = get(e / 2);
      r = mul(C, z, z);
      note(tr, "pow " + std::to_string(e) + " = sq " + std::to_string(e / 2) + " -> L" + std::to_string(r.level));
    } else {
      Ct a = get(h);
      const Ct& b = get(e - h);
      r = mul(C, a, b);
      note(tr, "pow " + std::to_string(e) + " = " + std::to_string(h) + "*" + std::to_string(e - h) +
                   " -> L" + std::to_string(r.level));
    }
    return pw[e] = r;
  }
};

struct Term {
  bool has_ct = false;
  Ct ct;
  i64 cst = 0;  // value = ct + cst
};

// Baby-step / giant-step evaluation of H(y) = sum_j h[j] y^j (Theorem 2):
// k = 2^ceil(floor(log2(n+1))/2) baby steps y^1..y^(k-1); giant steps
// y^(k 2^i); the padded coefficient vector (length k 2^m >= n+1) is split in
// halves recursively: H = H_lo + H_hi * y^(half).
static Term bsgs(const Context& C, const std::vector<i64>& h, Powers& P, Trace* tr) {
  int n1 = (int)h.size();
  int lg = 0;
  while ((2 << lg) <= n1) ++lg;           // floor(log2(n+1))
  int k = 1 << ((lg + 1) / 2);
  int len = k;
  while (len < n1) len *= 2;
  std::vector<i64> c(len, 0);
  for (int i = 0; i < n1; ++i) c[i] = h[i];
  note(tr, "bsgs n+1=" + std::to_string(n1) + " k=" + std::to_string(k) + " len=" + std::to_string(len));
  std::function<Term(int, int)> rec = [&](int lo, int ln) -> Term {
    Term out;
    if (ln == k) {
      out.cst = c[lo];
      std::vector<int> idx;
      for (int i = 1; i < k; ++i) if (c[lo + i] != 0) idx.push_back(i);
      if (idx.empty()) return out;
      int lvl = 1 << 30;
      for (int i : idx) lvl = std::min(lvl, P.get(i).level);
      bool first = true;
      for (int i : idx) {
        Ct term = mul_scalar(C, align_to(C, P.get(i), lvl), c[lo + i]);
        out.ct = first ? term : add(C, out.ct, term);
        first = false;
      }
      out.has_ct = true;
      note(tr, "baby lo=" + std::to_string(lo) + " terms=" + std::to_string(idx.size()) + " L" + std::to_string(lvl));
      return out;
    }
    int half = ln / 2;
    Term A = rec(lo, half), B = rec(lo + half, half);
    if (!B.has_ct && B.cst == 0) return A;
    const Ct& G = P.get(half);
    Ct prod;
    if (B.has_ct) {
      Ct b = B.cst != 0 ? add_scalar(C, B.ct, B.cst) : B.ct;
      prod = mul(C, b, G);
    } else {
      prod = mul_scalar(C, G, B.cst);
    }
    out.cst = A.cst;
    out.has_ct = true;
    out.ct = A.has_ct ? add_aligned(C, A.ct, prod) : prod;
    note(tr, "giant lo=" + std::to_string(lo) + " half=" + std::to_string(half) + " -> L" +
                 std::to_string(out.ct.level));
    return out;
  };
  return rec(0, len);
}

// x * T where T = ct + cst
static Ct mul_term(const Context& C, const Ct& x, const Term& T) {
  if (!T.has_ct) return mul_scalar(C, x, T.cst);
  Ct b = T.cst != 0 ? add_scalar(C, T.ct, T.cst) : T.ct;
  return mul(C, x, b);
}

Ct eval_g(const Context& C, const Ct& x, int e, Trace* tr) {
  std::vector<i64> g = C.reduced_g ? g_table_reduced(C.P.p, e) : g_table(C.P.p, e);
  std::vector<i64> h;
  for (size_t i = 1; i < g.size(); i += 2) h.push_back(g[i]);  // G = x * H(x^2)
  while (h.size() > 1 && h.back() == 0) h.pop_back();
  note(tr, "G p=" + std::to_string(C.P.p) + " e=" + std::to_string(e) + " in L" + std::to_string(x.level));
  Ct y = mul(C, x, x);
  Powers P(C, y, tr);
  Term H = bsgs(C, h, P, tr);
  Ct out = mul_term(C, x, H);
  note(tr, "G done -> L" + std::to_string(out.level));
  meter(C, tr, "G_e" + std::to_string(e), out);
  return out;
}

// Algorithm 3: for i = 0..r-2, a_i = G_{p,r-i}(b), b = DivideByP(b - a_i);
// a_{r-1} = b; then ChangeModToP on every digit (t <- p, ciphertext unchanged).
std::vector<Ct> reduce_to_digits(const Context& C, const Ct& a, Trace* tr) {
  int r = C.P.r;
  if (a.t_exp != r) throw std::runtime_error("reduce: input must be at t = p^r");
  std::vector<Ct> digits;
  Ct b = a;
  for (int i = 0; i + 1 < r; ++i) {
    Ct ai = eval_g(C, b, r - i, tr);
    Ct diff = sub(C, align_to(C, b, ai.level), ai);
    b = divide_by_p(C, diff);
    note(tr, "digit " + std::to_string(i) + " L" + std::to_string(ai.level));
    meter(C, tr, "reduce_b" + std::to_string(i + 1), b);
    digits.push_back(ai);
  }
  digits.push_back(b);
  for (auto& d : digits) d.t_exp = 1;  // ChangeModToP
  return digits;
}

// Per-digit LT and EQ against zero (Section 4.3), y = x^2 shared:
// F_LT(x) = x * H_LT(y) + c_{p-1} y^((p-1)/2),  F_EQ(x) = 1 - y^((p-1)/2).
static void compare_digit(const Context& C, const Ct& x, Ct& lt, Ct& eq, Trace* tr) {
  int p = C.P.p;
  std::vector<i64> f = flt_table(p);
  std::vector<i64> h;
  for (int i = 1; i <= p - 2; i += 2) h.push_back(f[i]);
  while (h.size() > 1 && h.back() == 0) h.pop_back();
  Ct y = mul(C, x, x);
  Powers P(C, y, tr);
  Term H = bsgs(C, h, P, tr);
  const Ct& T = P.get((p - 1) / 2);
  lt = add_aligned(C, mul_term(C, x, H), mul_scalar(C, T, f[p - 1]));
  eq = add_scalar(C, mul_scalar(C, T, -1), 1);
  note(tr, "cmp digit -> LT L" + std::to_string(lt.level) + " EQ L" + std::to_string(eq.level));
  meter(C, tr, "cmp_lt_digit", lt);
  meter(C, tr, "cmp_eq_digit", eq);
}

// Algorithm 4: d = a - b, digits = Reduce(d), per-digit LT_i/EQ_i, then fold
// from the most significant digit: LT <- LT + EQ*LT_i, EQ <- EQ*EQ_i. The last
// EQ product (i = 0) does not feed LT and is skipped.
Ct compare_lt(const Context& C, const Ct& a, const Ct& b, Trace* tr) {
  int r = C.P.r;
  Ct d = sub(C, align_to(C, a, std::min(a.level, b.level)), align_to(C, b, std::min(a.level, b.level)));
  std::vector<Ct> dg = reduce_to_digits(C, d, tr);
  std::vector<Ct> LT(r), EQ(r);
  for (int i = 0; i < r; ++i) compare_digit(C, dg[i], LT[i], EQ[i], tr);
  Ct lt = LT[r - 1], eq = EQ[r - 1];
  for (int i = r - 2; i >= 0; --i) {
    lt = add_aligned(C, lt, mul(C, eq, LT[i]));
    if (i > 0) eq = mul(C, eq, EQ[i]);
  }
  note(tr, "LT -> L" + std::to_string(lt.level));
  meter(C, tr, "fold_lt", lt);
  return lt;
}

// Per-digit EQ against zero alone (Section 4.3, Fermat): F_EQ(x) = 1 - x^(p-1),
// taken as 1 - y^((p-1)/2) with y = x^2, the power built by the Powers rule.
static Ct eq_digit(const Context& C, const Ct& x, Trace* tr) {
  Ct y = mul(C, x, x);
  Powers P(C, y, tr);
  Ct eq = add_scalar(C, mul_scalar(C, P.get((C.P.p - 1) / 2), -1), 1);
  note(tr, "eq digit -> EQ L" + std::to_string(eq.level));
  return eq;
}

// Section 4.3, EQ case: d = a - b, digits = Reduce(d), EQ = prod_i F_EQ(d_i),
// multiplied in from the most significant digit down.
Ct compare_eq(const Context& C, const Ct& a, const Ct& b, Trace* tr) {
  int r = C.P.r;
  int l = std::min(a.level, b.level);
  std::vector<Ct> dg = reduce_to_digits(C, sub(C, align_to(C, a, l), align_to(C, b, l)), tr);
  std::vector<Ct> EQ;
  for (int i = 0; i < r; ++i) EQ.push_back(eq_digit(C, dg[i], tr));
  Ct eq = EQ[r - 1];
  for (int i = r - 2; i >= 0; --i) eq = mul(C, eq, EQ[i]);
  note(tr, "EQ -> L" + std::to_string(eq.level));
  return eq;
}

// 1 - x at t = p: complements an indicator
static Ct complement(const Context& C, const Ct& x) { return add_scalar(C, mul_scalar(C, x, -1), 1); }

// Section 4.3: GT(a, b) = LT(b, a) (the centred range is symmetric); NEQ, GE
// and LE are 1 - EQ, 1 - LT and 1 - GT.
Ct compare(const Context& C, int pred, const Ct& a, const Ct& b, Trace* tr) {
  switch (pred) {
    case PRED_LT: return compare_lt(C, a, b, tr);
    case PRED_LE: return complement(C, compare_lt(C, b, a, tr));
    case PRED_GT: return compare_lt(C, b, a, tr);
    case PRED_GE: return complement(C, compare_lt(C, a, b, tr));
    case PRED_EQ: return compare_eq(C, a, b, tr);
    case PRED_NEQ: return complement(C, compare_eq(C, a, b, tr));
    default: throw std::runtime_error("unknown predicate");
  }
}

// Section 4.4: RaiseModToP2R(k) = G_{p,r}(k-bar) after t <- p^r.
Ct raise_modulus(const Context& C, const Ct& lt, Trace* tr) {
  if (lt.t_exp != 1) throw std::runtime_error("raise: input must be at t = p");
  Ct k = lt;
  k.t_exp = C.P.r;
  Ct out = eval_g(C, k, C.P.r, tr);
  note(tr, "raise -> L" + std::to_string(out.level));
  meter(C, tr, "raise", out);
  return out;
}

// Galois elements for a full slot sum: 5^(2^i) for i < log2(slots/2), then -1.
// m = 3N: for each slot-group generator g_i of order n_i (in the order chosen),
// g_i^(2^a) mod 3N for a < log2 n_i. Summing x + sigma(x) over these in turn
// adds up sigma_h(x) over one element h of every slot class, because the
// products g_1^j_1 g_2^j_2 ... (j_i < n_i) are a transversal of (Z/M')^*/<p>.
std::vector<int> rotate_sum_elements(const Context& C) {
  std::vector<int> g;
  if (C.P.m_odd == 3 || C.P.m_odd == 5) {
    const long m = C.m;
    for (auto& gn : C.gens) {
      long e = gn.first % m;
      for (int n = 1; n < gn.second; n *= 2) {
        g.push_back((int)e);
        e = e * e % m;
      }
    }
    return g;
  }
  int twoN = 2 * C.P.N;
  if (C.slots >= 2) {
    long e = 5;
    for (int s = 1; s < C.slots / 2; s *= 2) {
      g.push_back((int)e);
      e = e * e % twoN;
    }
    g.push_back(twoN - 1);
  }
  return g;
}

Ct rotate_sum(const Context& C, const Ct& a, Trace* tr) {
  Ct s = a;
  for (int g : rotate_sum_elements(C)) {
    s = add(C, s, rotate(C, s, g));
    note(tr, "rot " + std::to_string(g));
  }
  return s;
}

// SUM over rows of A*B where every condition holds, per ciphertext: the
// indicators of the conditions (t = p) are multiplied in order (AND), raised
// once, ind = Raise(prod_k cond_k); R = ind * (A*B); total = rotate_sum(sum R).
Ct query_sum_where(const Context& C, const std::vector<Ct>& A, const std::vector<Ct>& B,
                   const std::vector<Cond>& conds, Trace* tr) {
  size_t n = A.size();
  if (B.size() != n || conds.empty()) throw std::runtime_error("query: bad columns");
  for (auto& c : conds)
    if (c.X.size() != n || (c.Y.size() != n && c.Y.size() != 1)) throw std::runtime_error("query: column sizes differ");
  Ct total;
  for (size_t i = 0; i < n; ++i) {
    Ct ind;
    for (size_t k = 0; k < conds.size(); ++k) {
      const Cond& c = conds[k];
      Ct v = compare(C, c.pred, c.X[i], c.Y.size() == 1 ? c.Y[0] : c.Y[i], tr);
      ind = k == 0 ? v : mul(C, ind, v);
    }
    ind = raise_modulus(C, ind, tr);
    Ct prod = mul(C, A[i], B[i]);
    Ct R = mul(C, ind, prod);
    meter(C, tr, "masked_product", R);
    total = (i == 0) ? R : add_aligned(C, total, R);
  }
  Ct out = rotate_sum(C, total, tr);
  meter(C, tr, "sum", out);
  return out;
}

// SUM over rows of A*B where C1 < C2 (Algorithm 4 semantics).
Ct query_sum_where_lt(const Context& C, const std::vector<Ct>& A, const std::vector<Ct>& B,
                      const std::vector<Ct>& C1, const std::vector<Ct>& C2, Trace* tr) {
  if (C2.size() != A.size() && C2.size() != 1) throw std::runtime_error("query: column sizes differ");
  return query_sum_where(C, A, B, {Cond{PRED_LT, C1, C2}}, tr);
}

}  // namespace orc
