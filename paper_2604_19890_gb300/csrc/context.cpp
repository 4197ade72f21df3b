// Host-side number theory and context construction: prime chain, roots of
// unity, transform twiddles, base-conversion constants, CRT constants, slot
// structure and the interpolation coefficient tables.
#include <algorithm>
#include <cstring>

#include "philox.h"
#include "ss_internal.h"

namespace ss {

typedef unsigned __int128 u128;

namespace nt {

u64 mul(u64 a, u64 b, u64 m) { return (u64)(((u128)a * b) % m); }

u64 pow(u64 a, u64 e, u64 m) {
  u64 r = 1 % m, x = a % m;
  for (; e; e >>= 1, x = mul(x, x, m))
    if (e & 1) r = mul(r, x, m);
  return r;
}

u64 inv(u64 a, u64 m) {
  i64 r0 = (i64)m, r1 = (i64)(a % m);
  __int128 s0 = 0, s1 = 1;
  while (r1) {
    i64 q = r0 / r1;
    i64 r2 = r0 - q * r1; r0 = r1; r1 = r2;
    __int128 s2 = s0 - (__int128)q * s1; s0 = s1; s1 = s2;
  }
  if (r0 != 1) throw Error(SS_ERR_PARAM, "modular inverse does not exist");
  __int128 v = s0 % (__int128)m;
  if (v < 0) v += m;
  return (u64)v;
}

u64 lift(i64 c, u64 m) {
  if (c >= 0) return (u64)c % m;
  u64 k = (u64)(-(c + 1)) % m;  // -(c) - 1 without overflow
  return m - 1 - k;
}

bool prime(u64 n) {
  if (n < 4) return n >= 2;
  if (n % 2 == 0) return false;
  u64 d = n - 1;
  int s = 0;
  while (!(d & 1)) { d >>= 1; ++s; }
  const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  for (u64 a : bases) {
    if (a % n == 0) continue;
    u64 x = pow(a, d, n);
    if (x == 1 || x == n - 1) continue;
    int i = 1;
    for (; i < s; ++i) {
      x = mul(x, x, n);
      if (x == n - 1) break;
    }
    if (i == s) return false;
  }
  return true;
}

u64 shoup(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

int brv(int x, int logn) {
  unsigned v = (unsigned)x, r = 0;
  for (int i = 0; i < logn; ++i, v >>= 1) r = (r << 1) | (v & 1u);
  return (int)r;
}

// Largest primes below 2^bits that are 1 mod step, in descending order.
std::vector<u64> chain(int bits, u64 step, int count) {
  std::vector<u64> out;
  u64 hi = (1ULL << bits) - 1;
  u64 q = (hi - 1) / step * step + 1;
  for (; (int)out.size() < count; q -= step) {
    if (q < step || q <= (1ULL << (bits - 1))) throw Error(SS_ERR_PARAM, "prime chain exhausted at this width");
    if (prime(q)) out.push_back(q);
  }
  return out;
}

// Smallest primitive 2N-th root of unity mod q.
u64 root2n(u64 q, int N) {
  u64 g = 0;
  for (u64 x = 2; !g; ++x) {
    u64 c = pow(x, (q - 1) / (2 * (u64)N), q);
    if (pow(c, (u64)N, q) == q - 1) g = c;
  }
  u64 g2 = mul(g, g, q), best = g, cur = g;
  for (int j = 1; j < N; ++j) {
    cur = mul(cur, g2, q);
    best = std::min(best, cur);
  }
  return best;
}

// Smallest primitive 3N-th root of unity mod q (q = 1 mod 3N): some unit
// raised to (q-1)/3N whose N-th and 3N/2-th powers differ from 1, then the
// least of its powers with exponent prime to 6.
u64 root3n(u64 q, int N) {
  const u64 m = 3 * (u64)N;
  u64 g = 0;
  for (u64 x = 2; !g; ++x) {
    u64 c = pow(x, (q - 1) / m, q);
    if (pow(c, (u64)N, q) != 1 && pow(c, m / 2, q) != 1) g = c;
  }
  u64 best = g, cur = 1;
  for (u64 j = 1; j < m; ++j) {
    cur = mul(cur, g, q);
    if (j % 6 == 1 || j % 6 == 5) best = std::min(best, cur);
  }
  return best;
}

// Smallest primitive (5N/2)-th root of unity mod q: a unit raised to
// (q-1)/m whose m/2-th and m/5-th powers differ from 1, then the least of its
// powers with exponent prime to 10.
u64 root5n(u64 q, int N) {
  const u64 m = 5 * (u64)N / 2;
  u64 g = 0;
  for (u64 x = 2; !g; ++x) {
    u64 c = pow(x, (q - 1) / m, q);
    if (pow(c, m / 2, q) != 1 && pow(c, m / 5, q) != 1) g = c;
  }
  u64 best = g, cur = 1;
  for (u64 j = 1; j < m; ++j) {
    cur = mul(cur, g, q);
    if (j % 2 != 0 && j % 5 != 0) best = std::min(best, cur);
  }
  return best;
}

static u64 upow(u64 b, int e) {
  u64 r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

static i64 centred(u64 v, u64 m) { return v > m / 2 ? (i64)v - (i64)m : (i64)v; }

// G_{p,e}: the Newton interpolant of f(x) = balanced(x mod p) through
// x = 0..D, D = (e-1)(p-1)+1, written in monomials mod p^e, odd part kept.
std::vector<i64> g_coeffs(int p, int e) {
  const int D = (e - 1) * (p - 1) + 1;
  const u64 pe = upow((u64)p, e);
  int extra = 0;
  for (long q = p; q <= D; q *= p) extra += (int)(D / q);
  const u64 M = pe * upow((u64)p, extra);
  std::vector<u64> f(D + 1);
  for (int x = 0; x <= D; ++x) {
    int z = x % p;
    f[x] = lift(z > p / 2 ? z - p : z, M);
  }
  // Delta^k f(0) = sum_j (-1)^(k-j) C(k, j) f(j), binomials from Pascal rows mod M
  std::vector<u64> binom(1, 1 % M), dk(D + 1);
  for (int k = 0; k <= D; ++k) {
    if (k > 0) {
      std::vector<u64> nb(k + 1);
      nb[0] = nb[k] = 1 % M;
      for (int j = 1; j < k; ++j) nb[j] = (binom[j - 1] + binom[j]) % M;
      binom.swap(nb);
    }
    u64 s = 0;
    for (int j = 0; j <= k; ++j) {
      u64 term = mul(binom[j], f[j], M);
      s = ((k - j) % 2 == 0) ? (s + term) % M : (s + M - term) % M;
    }
    dk[k] = s;
  }
  std::vector<u64> mono(D + 1, 0), ff(1, 1 % pe);
  u64 unit = 1 % pe;
  int vk = 0;
  for (int k = 0; k <= D; ++k) {
    if (k > 0) {
      long x = k;
      while (x % p == 0) { x /= p; ++vk; }
      unit = mul(unit, (u64)x % pe, pe);
      ff.push_back(0);
      for (int j = k; j >= 1; --j) ff[j] = (ff[j - 1] + pe - mul(ff[j], (u64)(k - 1) % pe, pe)) % pe;
      ff[0] = (pe - mul(ff[0], (u64)(k - 1) % pe, pe)) % pe;
    }
    u64 pv = upow((u64)p, vk);
    if (dk[k] % pv) throw Error(SS_ERR_PARAM, "G table: non-integral difference");
    u64 ck = mul((dk[k] / pv) % pe, inv(unit, pe), pe);
    for (int j = 0; j <= k; ++j) mono[j] = (mono[j] + mul(ck, ff[j], pe)) % pe;
  }
  std::vector<i64> out(D + 1, 0);
  for (int i = 1; i <= D; i += 2) out[i] = centred(mono[i], pe);
  return out;
}

// Lattice-reduced G_{p,e} (Section 4.2, Geelen et al.'s smaller equivalent
// coefficients) for e = 2, 3: the canonical table plus the odd null polynomial
// mod p^e that minimises the sum of |centred coefficients|. The odd null
// polynomials of degree <= (e-1)(p-1)+1 are spanned mod p^e by the generators
//   e = 2:  p (x^p - x);
//   e = 3:  p^2 * odd part of (x^p - x) x^m, m = 0, 2, ..., p-1,
// built here as coefficient vectors. Generators whose supports are disjoint
// from all others are chosen one at a time (exhaustively over their multiplier
// 0..p-1); the two that share coefficient p (m = 0 and m = p-1) are chosen
// jointly. Ties keep the smaller multiplier (the first generator's first). The
// result agrees with G_{p,e} on all of Z_{p^e}. Other e: the canonical table.
std::vector<i64> g_coeffs_reduced(int p, int e) {
  std::vector<i64> g = g_coeffs(p, e);
  if (e != 2 && e != 3) return g;
  const int D = (int)g.size() - 1;
  const i64 pe = (i64)upow((u64)p, e), step = e == 2 ? p : (i64)p * p;
  // generator vectors (coefficients mod p^e of step * odd part of (x^p - x) x^m)
  std::vector<std::vector<i64>> gens;
  for (int m = 0; m <= (e == 2 ? 0 : p - 1); m += 2) {
    std::vector<i64> v(D + 1, 0);
    if (m + p <= D && (m + p) % 2 == 1) v[m + p] += step;
    if (m + 1 <= D && (m + 1) % 2 == 1) v[m + 1] -= step;
    gens.push_back(v);
  }
  auto centre_pe = [&](i64 x) {
    i64 z = x % pe;
    if (z < 0) z += pe;
    return z > pe / 2 ? z - pe : z;
  };
  // cost of the coefficients in `idx` after adding sum_k a[k] * gens[ks[k]]
  auto cost = [&](const std::vector<int>& ks, const std::vector<int>& a, const std::vector<int>& idx) {
    i64 s = 0;
    for (int i : idx) {
      i64 v = g[i];
      for (size_t k = 0; k < ks.size(); ++k) v += (i64)a[k] * gens[ks[k]][i];
      v = centre_pe(v);
      s += v < 0 ? -v : v;
    }
    return s;
  };
  auto support = [&](int k) {
    std::vector<int> s;
    for (int i = 0; i <= D; ++i)
      if (gens[k][i] != 0) s.push_back(i);
    return s;
  };
  std::vector<int> mult(gens.size(), 0);
  std::vector<bool> done(gens.size(), false);
  for (size_t k = 0; k < gens.size(); ++k) {
    if (done[k]) continue;
    // generators sharing a coefficient with k
    std::vector<int> grp{(int)k};
    for (size_t k2 = k + 1; k2 < gens.size(); ++k2)
      for (int i : support((int)k))
        if (gens[k2][i] != 0) { grp.push_back((int)k2); break; }
    if (grp.size() > 2) throw Error(SS_ERR_PARAM, "reduced G: unexpected generator coupling");
    std::vector<int> idx;
    for (int kk : grp)
      for (int i : support(kk))
        if (std::find(idx.begin(), idx.end(), i) == idx.end()) idx.push_back(i);
    i64 best = -1;
    std::vector<int> ba(grp.size(), 0), a(grp.size(), 0);
    for (a[0] = 0; a[0] < p; ++a[0])
      for (int a1 = 0; a1 < (grp.size() > 1 ? p : 1); ++a1) {
        if (grp.size() > 1) a[1] = a1;
        i64 c = cost(grp, a, idx);
        if (best < 0 || c < best) { best = c; ba = a; }
      }
    for (size_t j = 0; j < grp.size(); ++j) {
      mult[grp[j]] = ba[j];
      done[grp[j]] = true;
    }
  }
  std::vector<i64> out(D + 1, 0);
  for (int i = 0; i <= D; ++i) {
    i64 v = g[i];
    for (size_t k = 0; k < gens.size(); ++k) v += (i64)mult[k] * gens[k][i];
    out[i] = centre_pe(v);
  }
  return out;
}

// F_LT over Z_p: coefficient of x^(p-1) is (p+1)/2; odd i <= p-2 carry
// c_i = sum_{j=1}^{(p-1)/2} j^(p-1-i).
std::vector<i64> flt_coeffs(int p) {
  std::vector<i64> c(p, 0);
  c[p - 1] = centred((u64)((p + 1) / 2) % p, (u64)p);
  for (int i = 1; i < p - 1; i += 2) {
    u64 s = 0;
    for (int j = 1; 2 * j <= p - 1; ++j) s = (s + pow((u64)j, (u64)(p - 1 - i), (u64)p)) % (u64)p;
    c[i] = centred(s, (u64)p);
  }
  return c;
}

}  // namespace nt

// ------------------------------------------------------------------ m = 3N slots
// Degree-2 Galois ring GR(p^k, 2) = Z_{p^k}[u]/(u^2 - c): pairs (a0, a1).
namespace {
struct Gr {
  u64 a0, a1;
};
struct GrRing {
  u64 c, t;
  Gr mul(Gr x, Gr y) const {
    return {(nt::mul(x.a0, y.a0, t) + nt::mul(c, nt::mul(x.a1, y.a1, t), t)) % t,
            (nt::mul(x.a0, y.a1, t) + nt::mul(x.a1, y.a0, t)) % t};
  }
  Gr add(Gr x, Gr y) const { return {(x.a0 + y.a0) % t, (x.a1 + y.a1) % t}; }
  Gr sub(Gr x, Gr y) const { return {(x.a0 + t - y.a0) % t, (x.a1 + t - y.a1) % t}; }
  Gr scale(Gr x, u64 k) const { return {nt::mul(x.a0, k, t), nt::mul(x.a1, k, t)}; }
  Gr pow(Gr x, u64 e) const {
    Gr r{1 % t, 0};
    for (; e; e >>= 1, x = mul(x, x))
      if (e & 1) r = mul(r, x);
    return r;
  }
  Gr inv(Gr x) const {  // conjugate over the norm a0^2 - c a1^2
    u64 nrm = (nt::mul(x.a0, x.a0, t) + t - nt::mul(c, nt::mul(x.a1, x.a1, t), t)) % t;
    u64 ni = nt::inv(nrm, t);
    return {nt::mul(x.a0, ni, t), nt::mul((t - x.a1) % t, ni, t)};
  }
  static bool one(Gr x) { return x.a0 == 1 && x.a1 == 0; }
};
}  // namespace

// Slot structure of Phi_3N over Z_{p^r} (Section 2.1 for m = 3N): M' = 3*2^b'
// (2^b || p^2 - 1, b' = min(b, log2 N)), s = 3N/M', Phi_3N(X) = Phi_M'(X^s),
// roots theta^e (e a unit mod M') in GR(p^r, 2); slots = orbits under x p.
static void build_slots_m3(Context& C) {
  const u64 p = (u64)C.p;
  int b = 0;
  for (u64 v = p * p - 1; !(v & 1); v >>= 1) ++b;
  const int bp = std::min(b, C.logN);
  C.Mp = 3 << bp;
  C.s_stride = 3 * C.N / C.Mp;
  C.nprime = C.N / C.s_stride;
  C.gr_c = 0;
  for (u64 c = 2; c < p && !C.gr_c; ++c)
    if (nt::pow(c, (p - 1) / 2, p) == p - 1) C.gr_c = c;
  const u64 Mp = (u64)C.Mp;
  // theta_0: first x0 + x1 u of F_{p^2} (index x0 + p x1) of order exactly M'
  GrRing F{C.gr_c, p};
  Gr th{0, 0};
  for (u64 i = 1; i < p * p && th.a0 == 0 && th.a1 == 0; ++i) {
    Gr x{i % p, i / p};
    if (GrRing::one(F.pow(x, Mp)) && !GrRing::one(F.pow(x, Mp / 2)) && !GrRing::one(F.pow(x, Mp / 3))) th = x;
  }
  if (th.a0 == 0 && th.a1 == 0) throw Error(SS_ERR_PARAM, "no root of unity of order M' in F_{p^2}");
  // Newton's iteration for y^M' = 1 in GR(p^r, 2): y <- y - (y^M' - 1) / (M' y^(M'-1))
  GrRing R{C.gr_c, C.t};
  for (int it = 0; it <= C.r; ++it) {
    Gr f = R.sub(R.pow(th, Mp), Gr{1 % C.t, 0});
    Gr df = R.scale(R.pow(th, Mp - 1), Mp % C.t);
    th = R.sub(th, R.mul(f, R.inv(df)));
  }
  if (!GrRing::one(R.pow(th, Mp))) throw Error(SS_ERR_PARAM, "root lift failed");
  C.theta[0] = th.a0;
  C.theta[1] = th.a1;
  // slot group (Z/M')^* / <p>: generators, smallest residue of largest order first
  std::vector<char> inH(Mp, 0);
  int hsize = 0;
  for (u64 x = 1; !inH[x]; x = x * (p % Mp) % Mp, ++hsize) inH[x] = 1;
  C.slots = C.nprime / hsize;
  C.gens.clear();
  while (hsize < C.nprime) {
    int gbest = 0, nbest = 0;
    for (int g = 1; g < C.Mp; ++g) {
      if (g % 2 == 0 || g % 3 == 0) continue;
      int n = 1;
      for (u64 x = (u64)g; !inH[x]; x = x * (u64)g % Mp) ++n;
      if (n > nbest) { nbest = n; gbest = g; }
    }
    C.gens.push_back({gbest, nbest});
    std::vector<char> nh(Mp, 0);
    for (u64 h = 0; h < Mp; ++h) {
      if (!inH[h]) continue;
      u64 x = h;
      for (int j = 0; j < nbest; ++j, x = x * (u64)gbest % Mp) nh[x] = 1;
    }
    inH.swap(nh);
    hsize = 0;
    for (char v : inH) hsize += v;
  }
  C.slot_exp.assign(C.slots, 1);
  for (int j = 0; j < C.slots; ++j) {
    u64 e = 1;
    int rest = j;
    for (auto& gn : C.gens) {
      e = e * nt::pow((u64)gn.first, (u64)(rest % gn.second), Mp) % Mp;
      rest /= gn.second;
    }
    C.slot_exp[j] = (int)e;
  }
  u64 m = 3 * (u64)C.N, x = p % m;
  int d = 1;
  for (; x != 1; x = x * p % m) ++d;
  C.d = d;
  if ((long)C.slots * d != C.N) throw Error(SS_ERR_PARAM, "slot count does not match the order of p mod 3N");
  C.dec_stride = C.s_stride;
  C.dec_count = C.nprime;
}

// ------------------------------------------------------------------ m = 5N/2 slots
namespace {
// GR(p^k, 4) as GR(p^k, 2)[v]/(v^2 - w): pairs (a, b) of GR(p^k, 2) elements.
struct Gr4 {
  Gr a, b;
};
struct Gr4Ring {
  GrRing R;
  Gr w;
  Gr4 mul(const Gr4& x, const Gr4& y) const {
    return {R.add(R.mul(x.a, y.a), R.mul(R.mul(x.b, y.b), w)), R.add(R.mul(x.a, y.b), R.mul(x.b, y.a))};
  }
  Gr4 add(const Gr4& x, const Gr4& y) const { return {R.add(x.a, y.a), R.add(x.b, y.b)}; }
  Gr4 sub(const Gr4& x, const Gr4& y) const { return {R.sub(x.a, y.a), R.sub(x.b, y.b)}; }
  Gr4 scale(const Gr4& x, u64 k) const { return {R.scale(x.a, k), R.scale(x.b, k)}; }
  Gr4 one() const { return {Gr{1 % R.t, 0}, Gr{0, 0}}; }
  Gr4 pow(Gr4 x, u64 e) const {
    Gr4 r = one();
    for (; e; e >>= 1, x = mul(x, x))
      if (e & 1) r = mul(r, x);
    return r;
  }
  Gr4 inv(const Gr4& x) const {  // (a - b v) / (a^2 - b^2 w)
    Gr ni = R.inv(R.sub(R.mul(x.a, x.a), R.mul(R.mul(x.b, x.b), w)));
    return {R.mul(x.a, ni), R.mul(R.sub(Gr{0, 0}, x.b), ni)};
  }
  static bool is_one(const Gr4& x) { return x.a.a0 == 1 && x.a.a1 == 0 && x.b.a0 == 0 && x.b.a1 == 0; }
};
const int kE5[4] = {1, 3, 7, 9};
}  // namespace

// Slot structure of Phi_m, m = 5N/2 = 5*2^k (Section 2.1): M' = 5*2^b'
// (2^b || p^4 - 1, b' = min(b, k)), s = m/M', Phi_m(X) = Phi_M'(X^s), roots
// theta^e (e a unit mod M') in GR(p^r, 4); theta reduces to the element of
// smallest index x0 + p x1 + p^2 x2 + p^3 x3 of order M' in F_{p^4}.
static void build_slots_m5(Context& C) {
  const u64 p = (u64)C.p, p4 = p * p * p * p;
  int b = 0;
  for (u64 v = p4 - 1; !(v & 1); v >>= 1) ++b;
  const int k = C.logN - 1;
  const int bp = std::min(b, k);
  C.Mp = 5 << bp;
  C.s_stride = (5 << k) / C.Mp;
  C.nprime = C.N / C.s_stride;
  C.gr_c = 0;
  for (u64 c = 2; c < p && !C.gr_c; ++c)
    if (nt::pow(c, (p - 1) / 2, p) == p - 1) C.gr_c = c;
  const GrRing F2{C.gr_c, p};
  Gr w{0, 0};
  for (u64 i = 1; i < p * p && w.a0 == 0 && w.a1 == 0; ++i) {
    Gr x{i % p, i / p};
    if (!GrRing::one(F2.pow(x, (p * p - 1) / 2))) w = x;
  }
  C.gr_w[0] = w.a0;
  C.gr_w[1] = w.a1;
  const Gr4Ring F{F2, w};
  const u64 Mp = (u64)C.Mp;
  auto index = [&](const Gr4& x) { return x.a.a0 + p * (x.a.a1 + p * (x.b.a0 + p * x.b.a1)); };
  Gr4 y{};
  bool found = false;
  for (u64 i = 1; !found; ++i) {
    Gr4 x{Gr{i % p, (i / p) % p}, Gr{(i / (p * p)) % p, (i / (p * p * p)) % p}};
    Gr4 c = F.pow(x, (p4 - 1) / Mp);
    if (!Gr4Ring::is_one(F.pow(c, Mp / 2)) && !Gr4Ring::is_one(F.pow(c, Mp / 5))) { y = c; found = true; }
  }
  Gr4 th = y, cur = F.one();
  u64 best = ~0ULL;
  for (u64 j = 1; j < Mp; ++j) {
    cur = F.mul(cur, y);
    if (j % 2 && j % 5 && index(cur) < best) { best = index(cur); th = cur; }
  }
  // Newton's iteration for y^M' = 1 in GR(p^r, 4)
  const Gr4Ring R{GrRing{C.gr_c, C.t}, w};
  for (int it = 0; it <= C.r; ++it) {
    Gr4 f = R.sub(R.pow(th, Mp), R.one());
    Gr4 df = R.scale(R.pow(th, Mp - 1), Mp % C.t);
    th = R.sub(th, R.mul(f, R.inv(df)));
  }
  if (!Gr4Ring::is_one(R.pow(th, Mp))) throw Error(SS_ERR_PARAM, "root lift failed");
  C.theta4[0] = th.a.a0;
  C.theta4[1] = th.a.a1;
  C.theta4[2] = th.b.a0;
  C.theta4[3] = th.b.a1;
  std::vector<char> inH(Mp, 0);
  int hsize = 0;
  for (u64 x = 1; !inH[x]; x = x * (p % Mp) % Mp, ++hsize) inH[x] = 1;
  C.slots = C.nprime / hsize;
  C.gens.clear();
  while (hsize < C.nprime) {
    int gbest = 0, nbest = 0;
    for (int g = 1; g < C.Mp; ++g) {
      if (g % 2 == 0 || g % 5 == 0) continue;
      int n = 1;
      for (u64 x = (u64)g; !inH[x]; x = x * (u64)g % Mp) ++n;
      if (n > nbest) { nbest = n; gbest = g; }
    }
    C.gens.push_back({gbest, nbest});
    std::vector<char> nh(Mp, 0);
    for (u64 h = 0; h < Mp; ++h) {
      if (!inH[h]) continue;
      u64 x = h;
      for (int j = 0; j < nbest; ++j, x = x * (u64)gbest % Mp) nh[x] = 1;
    }
    inH.swap(nh);
    hsize = 0;
    for (char v : inH) hsize += v;
  }
  C.slot_exp.assign(C.slots, 1);
  for (int j = 0; j < C.slots; ++j) {
    u64 e = 1;
    int rest = j;
    for (auto& gn : C.gens) {
      e = e * nt::pow((u64)gn.first, (u64)(rest % gn.second), Mp) % Mp;
      rest /= gn.second;
    }
    C.slot_exp[j] = (int)e;
  }
  u64 m = 5 * (u64)C.N / 2, x = p % m;
  int d = 1;
  for (; x != 1; x = x * p % m) ++d;
  C.d = d;
  if ((long)C.slots * d != C.N) throw Error(SS_ERR_PARAM, "slot count does not match the order of p mod m");
  C.dec_stride = C.s_stride;
  C.dec_count = C.nprime;
}

// ------------------------------------------------------------------ context
static void upload(void** dst, const void* src, size_t bytes) {
  SS_CUDA(cudaMalloc(dst, bytes));
  SS_CUDA(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
}

Context::~Context() {
  cudaFree(d_mod);
  cudaFree(d_tw);
  cudaFree(d_ninv);
  cudaFree(d_r64);
  cudaFree(d_split);
  cudaFree(d_pinv);
  cudaFree(d_tmod);
  cudaFree(d_tables);
  cudaFree(d_crt);
  cudaFree(d_sk);
  cudaFree(d_sk2);
  cudaFree(rlk.a);
  cudaFree(rlk.b);
  for (auto& kv : gk) { cudaFree(kv.second.a); cudaFree(kv.second.b); }
}

void build_context(Context& C, const ss_params& prm) {
  C.prm = prm;
  if (prm.logN < 3 || prm.logN > 16) throw Error(SS_ERR_PARAM, "logN must be in [3, 16]");
  if (prm.L < 1 || prm.alpha < 1 || prm.L > 200 || prm.alpha > 16) throw Error(SS_ERR_PARAM, "bad L/alpha");
  if (prm.bits < 20 || prm.bits > 58) throw Error(SS_ERR_PARAM, "bits must be in [20, 58]");
  if (prm.m_odd != 0 && prm.m_odd != 1 && prm.m_odd != 3 && prm.m_odd != 5)
    throw Error(SS_ERR_PARAM, "m_odd must be 1 (m = 2N), 3 (m = 3N) or 5 (m = 5N/2)");
  // X^N + 1 splits into binomial slot factors over Z_p only for p = 1 mod 4; the
  // m = 3N and 5N/2 slot algebras (over GR(p^r, 2) and GR(p^r, 4)) take any
  // prime p >= 5 (p != 5 for 5N/2, whose Galois ring needs p^4 < 2^64)
  if (prm.p < 5 || !nt::prime((u64)prm.p) || (prm.m_odd <= 1 && prm.p % 4 != 1))
    throw Error(SS_ERR_PARAM, "p must be a prime >= 5, = 1 mod 4 on the ring X^N + 1");
  if (prm.m_odd == 5 && (prm.p == 5 || prm.p >= 32768 || prm.logN < 5))
    throw Error(SS_ERR_PARAM, "m = 5N/2 needs p != 5, p < 2^15 and N >= 32");
  C.m_odd = prm.m_odd == 3 || prm.m_odd == 5 ? prm.m_odd : 1;
  if (prm.r < 1 || prm.r > 8) throw Error(SS_ERR_PARAM, "bad r");
  C.logN = prm.logN;
  C.N = 1 << prm.logN;
  if (prm.h < 1 || prm.h > C.N) throw Error(SS_ERR_PARAM, "bad Hamming weight");
  int nmax = prm.nmax ? prm.nmax : C.N;
  if (nmax < C.N || (nmax & (nmax - 1))) throw Error(SS_ERR_PARAM, "nmax must be a power of two >= N");
  C.L = prm.L;
  C.alpha = prm.alpha;
  C.ntot = C.L + C.alpha;
  C.dnum = (C.L + C.alpha - 1) / C.alpha;
  C.p = prm.p;
  C.r = prm.r;
  C.tpow.assign(C.r + 1, 1);
  for (int e = 1; e <= C.r; ++e) C.tpow[e] = C.tpow[e - 1] * (u64)C.p;
  C.t = C.tpow[C.r];
  if (C.t >= (1ULL << 40) || C.t >= (1ULL << (prm.bits - 2))) throw Error(SS_ERR_PARAM, "p^r too large for the primes");
  // lazy 128-bit sums in the key-switch inner product need dnum * q^2 < 2^(63+k)
  if ((double)C.dnum * 2.0 >= (double)(1ULL << (63 - prm.bits)))
    throw Error(SS_ERR_PARAM, "too many digits for the lazy inner product at this prime width");

  C.m = C.m_odd == 3 ? 3 * C.N : C.m_odd == 5 ? 5 * C.N / 2 : 2 * C.N;
  // primes = 1 mod (m/N) * nmax * p^r
  const u64 step = C.m_odd == 3 ? 3 * (u64)nmax : C.m_odd == 5 ? 5 * (u64)nmax / 2 : 2 * (u64)nmax;
  C.primes = nt::chain(prm.bits, step * C.t, C.ntot);
  C.psi.resize(C.ntot);
  for (int i = 0; i < C.ntot; ++i)
    C.psi[i] = C.m_odd == 3   ? nt::root3n(C.primes[i], C.N)
               : C.m_odd == 5 ? nt::root5n(C.primes[i], C.N)
                              : nt::root2n(C.primes[i], C.N);

  // slots: d = order of p mod 2N, slots = N/d, X^N+1 = prod (X^d - zeta_j)
  if (C.m_odd == 3) {
    build_slots_m3(C);
  } else if (C.m_odd == 5) {
    build_slots_m5(C);
  } else {
    u64 m2 = 2 * (u64)C.N, x = (u64)C.p % m2;
    int d = 1;
    while (x != 1) { x = x * (u64)C.p % m2; ++d; }
    C.d = d;
    C.slots = C.N / d;
    if (((u64)C.p - 1) % (2 * (u64)C.slots)) throw Error(SS_ERR_PARAM, "slots do not split into linear factors");
    u64 w = 0;
    for (u64 c = 2; c < (u64)C.p && !w; ++c)
      if (nt::pow(c, (u64)C.slots, (u64)C.p) == (u64)C.p - 1) w = c;
    // Newton iteration for w^slots + 1 = 0 mod p^r
    for (int it = 0; it <= C.r; ++it) {
      u64 f = (nt::pow(w, (u64)C.slots, C.t) + 1) % C.t;
      u64 df = nt::mul((u64)C.slots % C.t, nt::pow(w, (u64)C.slots - 1, C.t), C.t);
      w = (w + C.t - nt::mul(f, nt::inv(df, C.t), C.t)) % C.t;
    }
    C.omega = w;
    C.slot_exp.assign(C.slots, 1);
    if (C.slots > 1) {
      int h = C.slots / 2, m = 2 * C.slots;
      long g = 1;
      for (int j = 0; j < h; ++j, g = g * 5 % m) {
        C.slot_exp[j] = (int)g;
        C.slot_exp[j + h] = (int)((m - g) % m);
      }
    }
    C.dec_stride = C.d;
    C.dec_count = C.slots;
  }

  const int N = C.N, T = C.ntot;
  // moduli
  std::vector<ModDesc> md(T);
  for (int i = 0; i < T; ++i) {
    u64 q = C.primes[i];
    int k = 64 - __builtin_clzll(q);
    md[i].q = q;
    md[i].kbits = k;
    md[i].mu = (u64)(((u128)1 << (63 + k)) / q);
    md[i].pad = 0;
    u64 x = q;  // Newton's iteration for q^-1 mod 2^64: 3, 6, 12, 24, 48, 96 correct bits
    for (int it = 0; it < 5; ++it) x *= 2 - q * x;
    md[i].qinv = 0 - x;
  }
  upload((void**)&C.d_mod, md.data(), sizeof(ModDesc) * T);

  // twiddles: psi^brv(i) and psi^-brv(i) with Shoup companions (m = 2N; m = 3N below)
  {
    std::vector<u64> tw((size_t)T * 4 * N);
    std::vector<u64> ninv(4 * T), pinv(2 * T), r64(4 * T, 0);
    std::vector<u64> split(C.m_odd == 5 ? (size_t)T * 24 : 0);
    for (int i = 0; i < T; ++i) {
      u64 q = C.primes[i], ps = C.psi[i], pi = nt::inv(ps, q);
      r64[4 * i] = (UINT64_MAX % q + 1) % q;  // 2^64 mod q
      u64* o = &tw[(size_t)i * 4 * N];
      auto put = [&](int k, u64 f, u64 bk) {
        o[2 * k] = f;
        o[2 * k + 1] = nt::shoup(f, q);
        o[2 * N + 2 * k] = bk;
        o[2 * N + 2 * k + 1] = nt::shoup(bk, q);
      };
      u64 ni = nt::inv((u64)N % q, q);
      ninv[4 * i] = ni;
      ninv[4 * i + 1] = nt::shoup(ni, q);
      if (C.m_odd == 5) {
        // Phi_m = prod_h (X^(N/4) - x_h), x_h = xi^(e_h), xi = omega^(N/4), e =
        // (1, 3, 7, 9): nodes 1..3 are replaced by the four-way split (table
        // d_split); node k >= 4 at depth l in quarter h, index j there, splits
        // with z_k = omega^(((N/4) >> (l-1)) (e_h + 10 bitrev_{l-2}(j))).
        const u64 m = 5 * (u64)N / 2;
        std::vector<u64> pw(m);
        pw[0] = 1;
        for (u64 e = 1; e < m; ++e) pw[e] = nt::mul(pw[e - 1], ps, q);
        for (int k = 0; k < 4; ++k) put(k, 1, 1);
        for (int k = 4; k < N; ++k) {
          const int l = 31 - __builtin_clz((unsigned)k);
          const int h = (k >> (l - 2)) & 3;
          const int j = k - (1 << l) - (h << (l - 2));
          const u64 e = (u64)((N / 4) >> (l - 1)) * (kE5[h] + 10 * (u64)nt::brv(j, l - 2)) % m;
          put(k, pw[e], pw[(m - e) % m]);
        }
        // split constants (the factored four-way split through the quadratics
        // y^2 - c y + 1, c = xi^e + xi^-e): forward c_1, xi, xi^3, xi^7, xi^9;
        // inverse (xi - xi^9)^-1, xi, (xi^3 - xi^7)^-1, xi^3, (1 - 2 c_1)^-1 4/N, 4/N, c_1
        const u64 x1 = pw[N / 4], x3 = pw[(u64)3 * N / 4], x7 = pw[(u64)7 * N / 4 % m], x9 = pw[(u64)9 * N / 4 % m];
        const u64 c1 = (x1 + x9) % q;
        const u64 sigma = nt::mul(4 % q, ni, q);
        const u64 dsig = nt::mul(nt::inv((1 + 2 * q - 2 * c1) % q, q), sigma, q);
        const u64 vals[12] = {c1, x1, x3, x7, x9, nt::inv((x1 + q - x9) % q, q), x1, nt::inv((x3 + q - x7) % q, q), x3,
                              dsig, sigma, c1};
        u64* sp = &split[(size_t)i * 24];
        for (int k2 = 0; k2 < 12; ++k2) {
          sp[2 * k2] = vals[k2];
          sp[2 * k2 + 1] = nt::shoup(vals[k2], q);
        }
        ninv[4 * i + 2] = 0;
        ninv[4 * i + 3] = 0;
      } else if (C.m_odd == 3) {
        // Phi_3N = (X^(N/2) - rho)(X^(N/2) - rho^5), rho = omega^(N/2): node 1
        // is that split (forward twiddle rho; the inverse recovers the high
        // half as (u - v) / (2 rho - 1)). Node k >= 2 at depth l splits
        // X^(2h) - z^2 into X^h -/+ z for the half e = 1 (k's second bit 0)
        // or e = 5: z_k = omega^((N/2 >> l) (e + 6 bitrev_{l-1}(j))), j the
        // index of k within its half at that depth.
        const u64 m = 3 * (u64)N;
        std::vector<u64> pw(m);
        pw[0] = 1;
        for (u64 e = 1; e < m; ++e) pw[e] = nt::mul(pw[e - 1], ps, q);
        const u64 rho = pw[N / 2];
        const u64 wb = nt::inv((2 * rho + q - 1) % q, q);
        put(0, 1, nt::mul(wb, ni, q));  // inverse word 0: (2 rho - 1)^-1 N^-1 for the fused last stage
        put(1, rho, wb);
        for (int k = 2; k < N; ++k) {
          const int l = 31 - __builtin_clz((unsigned)k);
          const int h = (k >> (l - 1)) & 1;
          const int j = k - (1 << l) - (h << (l - 1));
          const u64 e = (u64)((N / 2) >> l) * ((h ? 5 : 1) + 6 * (u64)nt::brv(j, l - 1)) % m;
          put(k, pw[e], pw[(m - e) % m]);
        }
        // the fused last inverse stage's difference output: 2 (2 rho - 1)^-1 N^-1
        const u64 c1 = nt::mul(2 % q, nt::mul(wb, ni, q), q);
        ninv[4 * i + 2] = c1;
        ninv[4 * i + 3] = nt::shoup(c1, q);
      } else {
        std::vector<u64> fw(N), bw(N);
        u64 a = 1, b = 1;
        for (int k = 0; k < N; ++k) { fw[k] = a; bw[k] = b; a = nt::mul(a, ps, q); b = nt::mul(b, pi, q); }
        for (int k = 0; k < N; ++k) {
          int rk = nt::brv(k, C.logN);
          put(k, fw[rk], bw[rk]);
        }
        // 2^64 times the forward node-1 twiddle psi^bitrev(1) = psi^(N/2)
        r64[4 * i + 1] = nt::mul(r64[4 * i], fw[N / 2], q);
        // 2^64 N^-1 and 2^64 N^-1 psi^(-N/2): the inverse's last-stage factors of the lower and upper half
        r64[4 * i + 2] = nt::mul(r64[4 * i], ni, q);
        r64[4 * i + 3] = nt::mul(r64[4 * i + 2], bw[N / 2], q);
        // N^-1 times the last inverse stage's twiddle psi^-bitrev(1) = psi^(-N/2)
        const u64 wni = nt::mul(ni, bw[N / 2], q);
        ninv[4 * i + 2] = wni;
        ninv[4 * i + 3] = nt::shoup(wni, q);
      }
      u64 pv = nt::inv((u64)C.p % q, q);
      pinv[2 * i] = pv;
      pinv[2 * i + 1] = nt::shoup(pv, q);
    }
    upload((void**)&C.d_tw, tw.data(), tw.size() * 8);
    upload((void**)&C.d_ninv, ninv.data(), ninv.size() * 8);
    upload((void**)&C.d_r64, r64.data(), r64.size() * 8);
    if (C.m_odd == 5) upload((void**)&C.d_split, split.data(), split.size() * 8);
    upload((void**)&C.d_pinv, pinv.data(), pinv.size() * 8);
    std::vector<u64> tm((size_t)(C.r + 1) * T * 2);
    for (int e = 0; e <= C.r; ++e)
      for (int i = 0; i < T; ++i) {
        u64 v = C.tpow[e] % C.primes[i];
        tm[((size_t)e * T + i) * 2] = v;
        tm[((size_t)e * T + i) * 2 + 1] = nt::shoup(v, C.primes[i]);
      }
    upload((void**)&C.d_tmod, tm.data(), tm.size() * 8);
  }

  // base-conversion constants
  std::vector<u64> tab;
  auto put2 = [&](u64 v, u64 q) { tab.push_back(v); tab.push_back(nt::shoup(v, q)); };
  // hat(src range [a, b), s) mod q_g = prod_{s' in [a,b), s' != s} q_s' mod q_g
  auto hat = [&](int a, int b, int s, int g) {
    u64 qg = C.primes[g], v = 1 % qg;
    for (int x = a; x < b; ++x)
      if (x != s) v = nt::mul(v, C.primes[x] % qg, qg);
    return v;
  };
  // ModUp: digit j = [j*alpha, e)
  for (int j = 0; j * C.alpha < C.L; ++j) {
    int a = j * C.alpha;
    for (int e = a + 1; e <= std::min(a + C.alpha, C.L); ++e) {
      C.off_modup[{j, e}] = tab.size();
      for (int s = a; s < e; ++s) put2(nt::inv(hat(a, e, s, s), C.primes[s]), C.primes[s]);
      for (int s = a; s < e; ++s)
        for (int g = 0; g < T; ++g) tab.push_back(g >= a && g < e ? 0 : hat(a, e, s, g));
    }
  }
  // ModDown: src = special primes [L, L+alpha)
  C.off_md_c1.assign(C.r + 1, 0);
  for (int te = 1; te <= C.r; ++te) {
    C.off_md_c1[te] = tab.size();
    for (int k = C.L; k < T; ++k) {
      u64 q = C.primes[k];
      put2(nt::mul(nt::inv(C.tpow[te] % q, q), nt::inv(hat(C.L, T, k, k), q), q), q);
    }
  }
  C.off_md_c2 = tab.size();
  for (int k = C.L; k < T; ++k)
    for (int g = 0; g < T; ++g) tab.push_back(g >= C.L ? 0 : hat(C.L, T, k, g));
  C.off_md_pinv = tab.size();
  for (int g = 0; g < T; ++g) {
    u64 q = C.primes[g];
    if (g >= C.L) { tab.push_back(0); tab.push_back(0); continue; }
    u64 P = 1;
    for (int k = C.L; k < T; ++k) P = nt::mul(P, C.primes[k] % q, q);
    put2(nt::inv(P, q), q);
  }
  // relinearise-and-drop: D = {q_{l-1}} and the special primes
  C.off_pmod = tab.size();
  for (int g = 0; g < T; ++g) {
    if (g >= C.L) { tab.push_back(0); tab.push_back(0); continue; }
    u64 q = C.primes[g], P = 1;
    for (int k = C.L; k < T; ++k) P = nt::mul(P, C.primes[k] % q, q);
    put2(P, q);
  }
  auto hatv = [&](const std::vector<int>& D, int s, int g) {
    u64 qg = C.primes[g], v = 1 % qg;
    for (int x : D)
      if (x != s) v = nt::mul(v, C.primes[x] % qg, qg);
    return v;
  };
  C.off_rd.assign(C.L + 1, 0);
  for (int l = 2; l <= C.L; ++l) {
    std::vector<int> D{l - 1};
    for (int k = C.L; k < T; ++k) D.push_back(k);
    C.off_rd[l] = tab.size();
    for (int s : D)
      for (int g = 0; g < T; ++g) tab.push_back(g < l - 1 ? hatv(D, s, g) : 0);
    for (int g = 0; g < T; ++g) {
      if (g >= l - 1) { tab.push_back(0); tab.push_back(0); continue; }
      u64 q = C.primes[g], v = 1;
      for (int x : D) v = nt::mul(v, C.primes[x] % q, q);
      put2(nt::inv(v, q), q);
    }
    for (int te = 1; te <= C.r; ++te) {
      C.off_rd_c1[{l, te}] = tab.size();
      for (int s : D) {
        u64 q = C.primes[s];
        put2(nt::mul(nt::inv(C.tpow[te] % q, q), nt::inv(hatv(D, s, s), q), q), q);
      }
    }
  }
  // modulus switching: level l drops [l-k, l)
  for (int l = 2; l <= C.L; ++l)
    for (int k = 1; k < l; ++k) {
      int a = l - k;
      C.off_ms[{l, k}] = tab.size();
      // c2 rows over the kept primes (row length T, only [0, a) used)
      std::vector<u64> QD(a);
      for (int g = 0; g < a; ++g) {
        u64 q = C.primes[g], v = 1;
        for (int x = a; x < l; ++x) v = nt::mul(v, C.primes[x] % q, q);
        QD[g] = v;
      }
      for (int s = a; s < l; ++s)
        for (int g = 0; g < T; ++g)
          tab.push_back(g < a ? nt::mul(QD[g], nt::inv(C.primes[s] % C.primes[g], C.primes[g]), C.primes[g]) : 0);
      for (int g = 0; g < T; ++g) {
        if (g < a) put2(nt::inv(QD[g], C.primes[g]), C.primes[g]);
        else { tab.push_back(0); tab.push_back(0); }
      }
      for (int te = 1; te <= C.r; ++te) {
        C.off_ms_c1[std::make_tuple(l, k, te)] = tab.size();
        for (int s = a; s < l; ++s) {
          u64 q = C.primes[s];
          put2(nt::mul(nt::inv(C.tpow[te] % q, q), nt::inv(hat(a, l, s, s), q), q), q);
        }
      }
    }
  C.tables_words = tab.size();
  upload((void**)&C.d_tables, tab.data(), tab.size() * 8);

  // decryption CRT (Garner): inverse prefix products, half-Q digits per level,
  // prefix products mod p^e.
  {
    std::vector<u64> crt;
    C.off_crt_pinv = 0;
    for (int i = 0; i < C.L; ++i) {
      u64 q = C.primes[i], v = 1;
      for (int j = 0; j < i; ++j) v = nt::mul(v, C.primes[j] % q, q);
      crt.push_back(i == 0 ? 1 : nt::inv(v, q));
    }
    C.off_crt_half.assign(C.L + 1, 0);
    for (int l = 1; l <= C.L; ++l) {
      C.off_crt_half[l] = crt.size();
      // mixed-radix digits of (Q_l - 1)/2, whose residues are (q_i - 1)/2
      std::vector<u64> v(l);
      for (int i = 0; i < l; ++i) {
        u64 q = C.primes[i], x = (q - 1) / 2;
        u64 acc = 0;
        for (int j = i - 1; j >= 0; --j) acc = (nt::mul(acc, C.primes[j] % q, q) + v[j]) % q;
        v[i] = nt::mul((x + q - acc) % q, crt[i], q);
        crt.push_back(v[i]);
      }
    }
    C.off_crt_qmodt = crt.size();
    // [e][i]: (q_0 ... q_{i-1}) mod p^e, i = 0..L
    for (int e = 0; e <= C.r; ++e) {
      u64 te = C.tpow[e], v = 1 % te;
      for (int i = 0; i <= C.L; ++i) {
        crt.push_back(v);
        if (i < C.L) v = nt::mul(v, C.primes[i] % te, te);
      }
    }
    upload((void**)&C.d_crt, crt.data(), crt.size() * 8);
  }
}

// ------------------------------------------------------------------ slots
static u64 zeta(const Context& C, int j, int power, u64 te) {
  u64 m = 2 * (u64)C.slots;
  u64 e = ((u64)C.slot_exp[j] * (u64)power) % m;
  return nt::pow(C.omega % te, e, te);
}

// m = 3N encoding: the interpolant A (deg < n' = deg Phi_M') with
// A(theta^e) = V_e, split by the two factors y^(n'/2) - rho_h of Phi_M'
// (rho_h = theta^(e_h n'/2), e_0 = 1, e_1 = 5): the roots of factor h are
// theta^(e_h + 6k), so B_h = A mod (y^(n'/2) - rho_h) has the coefficients
// b_i = (n'/2)^-1 theta^(-e_h i) sum_k V_{e_h+6k} theta^(-6ik) (inverse DFT),
// and A = A_lo + y^(n'/2) A_hi with A_hi = (B_0 - B_1) / (rho_0 - rho_1),
// A_lo = B_0 - rho_0 A_hi.
static std::vector<u64> encode_m3(const Context& C, u64 te, const u64* v) {
  const GrRing R{C.gr_c, te};
  const Gr th{C.theta[0] % te, C.theta[1] % te};
  const int Mp = C.Mp, n = C.nprime, n2 = n / 2;
  std::vector<int> slot_of(Mp, -1);
  for (int j = 0; j < C.slots; ++j)
    for (u64 e = (u64)C.slot_exp[j]; slot_of[e] < 0; e = e * ((u64)C.p % Mp) % Mp) slot_of[e] = j;
  std::vector<Gr> tpow(Mp);  // theta^e
  tpow[0] = Gr{1 % te, 0};
  for (int e = 1; e < Mp; ++e) tpow[e] = R.mul(tpow[e - 1], th);
  const u64 n2inv = nt::inv((u64)n2 % te, te);
  std::vector<Gr> B[2];
  for (int h = 0; h < 2; ++h) {
    const int eh = h ? 5 : 1;
    B[h].assign(n2, Gr{0, 0});
    for (int i = 0; i < n2; ++i) {
      Gr acc{0, 0};
      for (int k = 0; k < n2; ++k) {
        const int e = eh + 6 * k;
        if (slot_of[e] < 0) throw Error(SS_ERR_PARAM, "encode: root outside the slots");
        // theta^(-6ik) = theta^(M' - (6ik mod M'))
        const int ex = (int)((u64)6 * i * k % Mp);
        acc = R.add(acc, R.scale(tpow[(Mp - ex) % Mp], v[slot_of[e]] % te));
      }
      const int tex = (int)((u64)eh * i % Mp);
      B[h][i] = R.scale(R.mul(acc, tpow[(Mp - tex) % Mp]), n2inv);
    }
  }
  const Gr rho0 = tpow[(u64)n2 % Mp], rho1 = tpow[(u64)5 * n2 % Mp];
  const Gr dinv = R.inv(R.sub(rho0, rho1));
  std::vector<u64> m(C.N, 0);
  for (int i = 0; i < n2; ++i) {
    const Gr hi = R.mul(R.sub(B[0][i], B[1][i]), dinv);
    const Gr lo = R.sub(B[0][i], R.mul(rho0, hi));
    if (hi.a1 != 0 || lo.a1 != 0) throw Error(SS_ERR_PARAM, "encode: interpolant outside Z_{p^t}");
    m[(size_t)i * C.s_stride] = lo.a0;
    m[(size_t)(i + n2) * C.s_stride] = hi.a0;
  }
  return m;
}

// m = 3N decoding: slot j reads sum_k c[k s] theta^(e_j k), Z_{p^t} coordinate.
static std::vector<u64> decode_m3(const Context& C, u64 te, const u64* c) {
  const GrRing R{C.gr_c, te};
  const Gr th{C.theta[0] % te, C.theta[1] % te};
  std::vector<u64> v(C.slots, 0);
  for (int j = 0; j < C.slots; ++j) {
    const Gr z = R.pow(th, (u64)C.slot_exp[j]);
    Gr zk{1 % te, 0}, acc{0, 0};
    for (int k = 0; k < C.nprime; ++k, zk = R.mul(zk, z)) acc = R.add(acc, R.scale(zk, c[(size_t)k * C.s_stride] % te));
    v[j] = acc.a0;
  }
  return v;
}

// m = 5N/2 encoding: Phi_M'(y) = prod_q (y^h - x_q), h = n'/4, x_q =
// theta^(h e_q), e = (1, 3, 7, 9); factor q has the roots theta^(e_q + 10k),
// so B_q = A mod (y^h - x_q) has b_i = h^-1 theta^(-e_q i) sum_k
// V_{e_q+10k} theta^(-10ik); then A = sum_j y^(jh) A_j with B_q = sum_j x_q^j
// A_j, solved by Gauss-Jordan elimination over GR(p^t, 4).
static std::vector<u64> encode_m5(const Context& C, u64 te, const u64* v) {
  const Gr4Ring R{GrRing{C.gr_c, te}, Gr{C.gr_w[0] % te, C.gr_w[1] % te}};
  const Gr4 th{Gr{C.theta4[0] % te, C.theta4[1] % te}, Gr{C.theta4[2] % te, C.theta4[3] % te}};
  const int Mp = C.Mp, n = C.nprime, h = n / 4;
  std::vector<int> slot_of(Mp, -1);
  for (int j = 0; j < C.slots; ++j)
    for (u64 e = (u64)C.slot_exp[j]; slot_of[e] < 0; e = e * ((u64)C.p % Mp) % Mp) slot_of[e] = j;
  std::vector<Gr4> tp(Mp);
  tp[0] = R.one();
  for (int e = 1; e < Mp; ++e) tp[e] = R.mul(tp[e - 1], th);
  const u64 hinv = nt::inv((u64)h % te, te);
  std::vector<Gr4> B[4];
  for (int qq = 0; qq < 4; ++qq) {
    const int eq = kE5[qq];
    B[qq].assign(h, Gr4{});
    for (int i = 0; i < h; ++i) {
      Gr4 acc{};
      for (int k = 0; k < h; ++k) {
        const int e = eq + 10 * k;
        if (slot_of[e] < 0) throw Error(SS_ERR_PARAM, "encode: root outside the slots");
        const int ex = (int)((u64)10 * i * k % Mp);
        acc = R.add(acc, R.scale(tp[(Mp - ex) % Mp], v[slot_of[e]] % te));
      }
      const int tex = (int)((u64)eq * i % Mp);
      B[qq][i] = R.scale(R.mul(acc, tp[(Mp - tex) % Mp]), hinv);
    }
  }
  // [V | I] -> [I | V^-1], V[q][j] = x_q^j
  Gr4 M[4][8];
  for (int qq = 0; qq < 4; ++qq)
    for (int j = 0; j < 4; ++j) {
      M[qq][j] = tp[(u64)h * kE5[qq] * j % Mp];
      M[qq][4 + j] = qq == j ? R.one() : Gr4{};
    }
  for (int c = 0; c < 4; ++c) {
    const Gr4 iv = R.inv(M[c][c]);  // distinct roots of unity: every pivot is a unit
    for (int j = 0; j < 8; ++j) M[c][j] = R.mul(M[c][j], iv);
    for (int r2 = 0; r2 < 4; ++r2) {
      if (r2 == c) continue;
      const Gr4 f = M[r2][c];
      for (int j = 0; j < 8; ++j) M[r2][j] = R.sub(M[r2][j], R.mul(f, M[c][j]));
    }
  }
  std::vector<u64> m(C.N, 0);
  for (int j = 0; j < 4; ++j)
    for (int i = 0; i < h; ++i) {
      Gr4 a{};
      for (int qq = 0; qq < 4; ++qq) a = R.add(a, R.mul(M[j][4 + qq], B[qq][i]));
      if (a.a.a1 || a.b.a0 || a.b.a1) throw Error(SS_ERR_PARAM, "encode: interpolant outside Z_{p^t}");
      m[(size_t)(j * h + i) * C.s_stride] = a.a.a0;
    }
  return m;
}

static std::vector<u64> decode_m5(const Context& C, u64 te, const u64* c) {
  const Gr4Ring R{GrRing{C.gr_c, te}, Gr{C.gr_w[0] % te, C.gr_w[1] % te}};
  const Gr4 th{Gr{C.theta4[0] % te, C.theta4[1] % te}, Gr{C.theta4[2] % te, C.theta4[3] % te}};
  std::vector<u64> v(C.slots, 0);
  for (int j = 0; j < C.slots; ++j) {
    const Gr4 z = R.pow(th, (u64)C.slot_exp[j]);
    Gr4 zk = R.one(), acc{};
    for (int k = 0; k < C.nprime; ++k, zk = R.mul(zk, z)) acc = R.add(acc, R.scale(zk, c[(size_t)k * C.s_stride] % te));
    v[j] = acc.a.a0;
  }
  return v;
}

std::vector<u64> encode(const Context& C, int t_exp, const u64* v) {
  if (t_exp < 1 || t_exp > C.r) throw Error(SS_ERR_PARAM, "bad t_exp");
  u64 te = C.tpow[t_exp];
  if (C.m_odd == 3) return encode_m3(C, te, v);
  if (C.m_odd == 5) return encode_m5(C, te, v);
  u64 il = nt::inv((u64)C.slots % te, te);
  std::vector<u64> m(C.N, 0);
  for (int k = 0; k < C.slots; ++k) {
    u64 acc = 0;
    for (int j = 0; j < C.slots; ++j)  // zeta_j^(-k) = zeta_j^(2*slots - k)
      acc = (acc + nt::mul(v[j] % te, zeta(C, j, 2 * C.slots - k, te), te)) % te;
    m[(size_t)k * C.d] = nt::mul(acc, il, te);
  }
  return m;
}

std::vector<u64> decode(const Context& C, int t_exp, const u64* m) {
  if (t_exp < 1 || t_exp > C.r) throw Error(SS_ERR_PARAM, "bad t_exp");
  u64 te = C.tpow[t_exp];
  if (C.m_odd == 3) return decode_m3(C, te, m);
  if (C.m_odd == 5) return decode_m5(C, te, m);
  std::vector<u64> v(C.slots, 0);
  for (int j = 0; j < C.slots; ++j) {
    u64 acc = 0;
    for (int k = 0; k < C.slots; ++k) acc = (acc + nt::mul(m[(size_t)k * C.d] % te, zeta(C, j, k, te), te)) % te;
    v[j] = acc;
  }
  return v;
}

std::vector<int> rotate_sum_elements(const Context& C) {
  std::vector<int> g;
  if (C.m_odd == 3 || C.m_odd == 5) {  // g^(2^a) mod m for each slot-group generator of order n, a < log2 n
    for (auto& gn : C.gens) {
      u64 e = (u64)gn.first % (u64)C.m;
      for (int n = 1; n < gn.second; n *= 2, e = e * e % (u64)C.m) g.push_back((int)e);
    }
    return g;
  }
  if (C.slots < 2) return g;
  long m = 2L * C.N, e = 5;
  for (int s = 1; s < C.slots / 2; s *= 2, e = e * e % m) g.push_back((int)e);
  g.push_back((int)(m - 1));
  return g;
}

}  // namespace ss
