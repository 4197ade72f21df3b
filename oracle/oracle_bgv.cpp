// Plain CPU reference: number theory, transforms, slots, keys, encryption and
// the BGV operations. TEST INFRASTRUCTURE ONLY (see oracle.hpp).
#include "oracle.hpp"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <exception>
#include <mutex>
#include <thread>

namespace orc {

// ================================================================ arithmetic
u64 mulmod(u64 a, u64 b, u64 m) { return (u64)((u128)a * b % m); }
u64 addmod(u64 a, u64 b, u64 m) { return (u64)(((u128)a + b) % m); }
u64 submod(u64 a, u64 b, u64 m) { return (u64)(((u128)a + m - b) % m); }

u64 powmod(u64 a, u64 e, u64 m) {
  u64 r = 1 % m;
  a %= m;
  while (e) {
    if (e & 1) r = mulmod(r, a, m);
    a = mulmod(a, a, m);
    e >>= 1;
  }
  return r;
}

u64 invmod(u64 a, u64 m) {
  // extended Euclid over signed 128-bit integers
  __int128 t = 0, nt = 1, r = m, nr = a % m;
  while (nr != 0) {
    __int128 q = r / nr;
    __int128 tmp = t - q * nt; t = nt; nt = tmp;
    tmp = r - q * nr; r = nr; nr = tmp;
  }
  if (r != 1) throw std::runtime_error("invmod: not invertible");
  if (t < 0) t += m;
  return (u64)t;
}

u64 lift(i64 c, u64 m) {
  __int128 v = (__int128)c % (__int128)m;
  if (v < 0) v += m;
  return (u64)v;
}

i64 centre(u64 v, u64 m) {
  v %= m;
  return v > m / 2 ? (i64)v - (i64)m : (i64)v;
}

bool is_prime(u64 n) {
  if (n < 2) return false;
  static const u64 small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  for (u64 s : small) {
    if (n % s == 0) return n == s;
  }
  u64 d = n - 1;
  int s = 0;
  while ((d & 1) == 0) { d >>= 1; ++s; }
  for (u64 a : small) {
    u64 x = powmod(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int i = 1; i < s; ++i) {
      x = mulmod(x, x, n);
      if (x == n - 1) { comp = false; break; }
    }
    if (comp) return false;
  }
  return true;
}

// =================================================================== threads
static int g_threads = 0;  // 0: not set yet (ORC_THREADS or hardware concurrency)
static thread_local bool t_in_worker = false;

void set_threads(int n) { g_threads = n > 0 ? n : (int)std::max(1u, std::thread::hardware_concurrency()); }

int threads() {
  if (g_threads <= 0) {
    const char* e = std::getenv("ORC_THREADS");
    set_threads(e ? std::atoi(e) : 0);
  }
  return g_threads;
}

void parallel_for(int n, const std::function<void(int)>& f) {
  int nt = std::min(threads(), n);
  if (nt <= 1 || t_in_worker) {
    for (int i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<int> next{0};
  std::exception_ptr err;
  std::mutex mu;
  auto work = [&] {
    t_in_worker = true;
    for (int i = next++; i < n; i = next++) {
      try {
        f(i);
      } catch (...) {
        std::lock_guard<std::mutex> g(mu);
        if (!err) err = std::current_exception();
      }
    }
    t_in_worker = false;
  };
  std::vector<std::thread> pool;
  for (int k = 1; k < nt; ++k) pool.emplace_back(work);
  work();
  for (auto& th : pool) th.join();
  if (err) std::rethrow_exception(err);
}

// Splits a loop over limbs (or components) across the workers for rings large
// enough to pay for the threads; small rings run the plain loop.
static void limb_for(const Context& C, int n, const std::function<void(int)>& f) {
  if (C.P.N >= 2048) parallel_for(n, f);
  else for (int i = 0; i < n; ++i) f(i);
}

int bitrev(int x, int logn) {
  int r = 0;
  for (int i = 0; i < logn; ++i) { r = (r << 1) | (x & 1); x >>= 1; }
  return r;
}

// =============================================================== big integer
Big Big::from(u64 x) { Big b; b.w.push_back(x); b.trim(); return b; }
void Big::trim() { while (!w.empty() && w.back() == 0) w.pop_back(); }
bool Big::is_zero() const { return w.empty(); }

Big big_mul_u64(const Big& a, u64 b) {
  Big r;
  u128 carry = 0;
  for (u64 x : a.w) {
    u128 cur = (u128)x * b + carry;
    r.w.push_back((u64)cur);
    carry = cur >> 64;
  }
  if (carry) r.w.push_back((u64)carry);
  r.trim();
  return r;
}

Big big_add(const Big& a, const Big& b) {
  Big r;
  size_t n = std::max(a.w.size(), b.w.size());
  u128 carry = 0;
  for (size_t i = 0; i < n; ++i) {
    u128 cur = carry;
    if (i < a.w.size()) cur += a.w[i];
    if (i < b.w.size()) cur += b.w[i];
    r.w.push_back((u64)cur);
    carry = cur >> 64;
  }
  if (carry) r.w.push_back((u64)carry);
  r.trim();
  return r;
}

int big_cmp(const Big& a, const Big& b) {
  if (a.w.size() != b.w.size()) return a.w.size() < b.w.size() ? -1 : 1;
  for (size_t i = a.w.size(); i-- > 0;) {
    if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1;
  }
  return 0;
}

Big big_sub(const Big& a, const Big& b) {
  if (big_cmp(a, b) < 0) throw std::runtime_error("big_sub: negative");
  Big r;
  u64 borrow = 0;
  for (size_t i = 0; i < a.w.size(); ++i) {
    u64 bi = i < b.w.size() ? b.w[i] : 0;
    u128 sub = (u128)bi + borrow;
    u64 ai = a.w[i];
    if ((u128)ai >= sub) { r.w.push_back((u64)(ai - sub)); borrow = 0; }
    else { r.w.push_back((u64)(((u128)1 << 64) + ai - sub)); borrow = 1; }
  }
  r.trim();
  return r;
}

u64 big_mod_u64(const Big& a, u64 m) {
  u128 rem = 0;
  for (size_t i = a.w.size(); i-- > 0;) rem = ((rem << 64) | a.w[i]) % m;
  return (u64)rem;
}

Big big_shr1(const Big& a) {
  Big r;
  r.w.resize(a.w.size());
  for (size_t i = 0; i < a.w.size(); ++i) {
    u64 hi = (i + 1 < a.w.size()) ? a.w[i + 1] : 0;
    r.w[i] = (a.w[i] >> 1) | (hi << 63);
  }
  r.trim();
  return r;
}

double big_log2(const Big& a) {
  if (a.is_zero()) return -1e300;
  size_t n = a.w.size();
  double top = (double)a.w[n - 1];
  if (n >= 2) top += (double)a.w[n - 2] / 18446744073709551616.0;
  return std::log2(top) + 64.0 * (double)(n - 1);
}

// ==================================================================== philox
void philox4x32_10(const u32 ctr[4], const u32 key[2], u32 out[4]) {
  const u32 M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const u32 W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  u32 c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  u32 k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)M0 * c0;
    uint64_t p1 = (uint64_t)M1 * c2;
    u32 hi0 = (u32)(p0 >> 32), lo0 = (u32)p0;
    u32 hi1 = (u32)(p1 >> 32), lo1 = (u32)p1;
    u32 n0 = hi1 ^ c1 ^ k0;
    u32 n1 = lo1;
    u32 n2 = hi0 ^ c3 ^ k1;
    u32 n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw(const Context& C, u32 a, u32 b, u32 c, u32 d, u32 out[4]) {
  u32 ctr[4] = {a, b, c, d};
  u32 key[2] = {(u32)(C.P.seed & 0xffffffffu), (u32)(C.P.seed >> 32)};
  philox4x32_10(ctr, key, out);
}

// 128 bits of one Philox block, reduced modulo q.
static u64 sample_uniform(const Context& C, u32 n, u32 limb, u32 id, u32 tag, u64 q) {
  u32 x[4];
  draw(C, n, limb, id, tag, x);
  u64 lo = ((u64)x[1] << 32) | x[0];
  u64 hi = ((u64)x[3] << 32) | x[2];
  u128 v = ((u128)hi << 64) | lo;
  return (u64)(v % q);
}

// Centred binomial with eta = 21: popcount of 21 bits minus popcount of 21 bits.
static i64 sample_cbd(const Context& C, u32 n, u32 id, u32 tag) {
  u32 x[4];
  draw(C, n, 0, id, tag, x);
  return (i64)__builtin_popcount(x[0] & 0x1FFFFFu) - (i64)__builtin_popcount(x[1] & 0x1FFFFFu);
}

// ============================================================ construction
std::vector<u64> gen_primes(int bits, u64 M, int count) {
  std::vector<u64> out;
  u64 top = (bits >= 64) ? ~0ULL : ((1ULL << bits) - 2);
  u64 k = top / M;
  u64 low = 1ULL << (bits - 1);
  while ((int)out.size() < count) {
    if (k == 0) throw std::runtime_error("gen_primes: ran out of candidates");
    u64 q = k * M + 1;
    if (q <= low) throw std::runtime_error("gen_primes: not enough primes of this width");
    if (is_prime(q)) out.push_back(q);
    --k;
  }
  return out;
}

u64 find_psi(u64 q, int N) {
  u64 c = 0;
  for (u64 x = 2;; ++x) {
    c = powmod(x, (q - 1) / (2 * (u64)N), q);
    if (powmod(c, (u64)N, q) == q - 1) break;
  }
  // The primitive 2N-th roots are exactly the odd powers of c; take the smallest.
  u64 best = c, w = c, c2 = mulmod(c, c, q);
  for (int j = 1; j < N; ++j) {
    w = mulmod(w, c2, q);
    if (w < best) best = w;
  }
  return best;
}

// Smallest primitive 3N-th root of unity mod q (q = 1 mod 3N). A unit has
// order exactly 3N when its 3N-th power is 1 and its 3N/2-th and N-th powers
// are not (the maximal proper divisors of 3N = 3 * 2^k).
u64 find_root3(u64 q, int N) {
  const u64 m = 3 * (u64)N;
  auto order_m = [&](u64 x) {
    return powmod(x, m, q) == 1 && powmod(x, m / 2, q) != 1 && powmod(x, m / 3, q) != 1;
  };
  u64 c = 0;
  for (u64 x = 2; !c; ++x) {
    u64 y = powmod(x, (q - 1) / m, q);
    if (order_m(y)) c = y;
  }
  // the primitive 3N-th roots are c^j, gcd(j, 6) = 1; take the smallest
  u64 best = c, w = 1;
  for (u64 j = 1; j < m; ++j) {
    w = mulmod(w, c, q);
    if (j % 2 != 0 && j % 3 != 0 && w < best) best = w;
  }
  return best;
}

static u64 ipow(u64 b, int e) { u64 r = 1; while (e-- > 0) r *= b; return r; }

// ------------------------------------------------ Galois ring GR(p^k, 2)
// Z_{p^k}[u] / (u^2 - c) with c a quadratic non-residue mod p: the unramified
// degree-2 extension of Z_{p^k}. An element is x[0] + x[1] u.
struct GR2 {
  u64 x[2];
};
static GR2 gr_mul(const GR2& a, const GR2& b, u64 c, u64 t) {
  u64 r0 = addmod(mulmod(a.x[0], b.x[0], t), mulmod(c, mulmod(a.x[1], b.x[1], t), t), t);
  u64 r1 = addmod(mulmod(a.x[0], b.x[1], t), mulmod(a.x[1], b.x[0], t), t);
  return GR2{{r0, r1}};
}
static GR2 gr_add(const GR2& a, const GR2& b, u64 t) { return GR2{{addmod(a.x[0], b.x[0], t), addmod(a.x[1], b.x[1], t)}}; }
static GR2 gr_sub(const GR2& a, const GR2& b, u64 t) { return GR2{{submod(a.x[0], b.x[0], t), submod(a.x[1], b.x[1], t)}}; }
static GR2 gr_pow(GR2 a, u64 e, u64 c, u64 t) {
  GR2 r{{1 % t, 0}};
  while (e) {
    if (e & 1) r = gr_mul(r, a, c, t);
    a = gr_mul(a, a, c, t);
    e >>= 1;
  }
  return r;
}
// (a0 + a1 u)^-1 = (a0 - a1 u) / (a0^2 - c a1^2); the norm is a unit for units
static GR2 gr_inv(const GR2& a, u64 c, u64 t) {
  u64 nrm = submod(mulmod(a.x[0], a.x[0], t), mulmod(c, mulmod(a.x[1], a.x[1], t), t), t);
  u64 ni = invmod(nrm, t);
  return GR2{{mulmod(a.x[0], ni, t), mulmod(submod(0, a.x[1], t), ni, t)}};
}
static bool gr_is(const GR2& a, u64 v0, u64 v1) { return a.x[0] == v0 && a.x[1] == v1; }

// Slot algebra of Phi_3N mod p^r (Section 2.1 with m = 3N, N = 2^k).
// With 2^b the largest power of two dividing p^2 - 1, b' = min(b, k),
// M' = 3 * 2^b' and s = 3N / M': Phi_3N(X) = Phi_M'(X^s), and Phi_M'(y)
// splits over GR(p^r, 2) into the linear factors y - theta^e, e in (Z/M')^*,
// because M' divides p^2 - 1. Frobenius maps theta^e to theta^(e p), so the
// slots (the factors of Phi_3N over Z_{p^r}) are the orbits of (Z/M')^*
// under multiplication by p. A plaintext with constant slot values is
// A(X^s) with A(theta^e) = value of e's slot for every root.
static void make_slots_m3(Context& C) {
  const Params& P = C.P;
  const u64 p = (u64)P.p;
  int b = 0;
  for (u64 v = p * p - 1; v % 2 == 0; v /= 2) ++b;
  const int bp = std::min(b, P.logN);
  C.Mp = 3 << bp;
  C.s = 3 * P.N / C.Mp;
  C.nprime = P.N / C.s;
  for (u64 c = 2; c < p; ++c)
    if (powmod(c, (p - 1) / 2, p) == p - 1) { C.gr_c = c; break; }
  if (!C.gr_c) throw std::runtime_error("no quadratic non-residue");
  // theta_0: the first element x0 + x1 u of F_{p^2} (index x0 + p x1) of order exactly M'
  const u64 Mp = (u64)C.Mp;
  GR2 th0{{0, 0}};
  for (u64 i = 1; i < p * p; ++i) {
    GR2 x{{i % p, i / p}};
    if (gr_is(gr_pow(x, Mp, C.gr_c, p), 1, 0) && !gr_is(gr_pow(x, Mp / 2, C.gr_c, p), 1, 0) &&
        !gr_is(gr_pow(x, Mp / 3, C.gr_c, p), 1, 0)) { th0 = x; break; }
  }
  if (gr_is(th0, 0, 0)) throw std::runtime_error("no primitive M'-th root in F_{p^2}");
  // Teichmueller lift: theta = theta_0^((p^2)^(r-1)) in GR(p^r, 2), the root of
  // unity of order M' that reduces to theta_0 mod p
  GR2 th = th0;
  for (int i = 1; i < P.r; ++i) th = gr_pow(th, p * p, C.gr_c, C.t);
  if (!gr_is(gr_pow(th, Mp, C.gr_c, C.t), 1, 0)) throw std::runtime_error("theta lift failed");
  C.theta[0] = th.x[0];
  C.theta[1] = th.x[1];
  // units of Z/M' and the subgroup generated by p
  auto unit = [&](int e) { return e % 2 != 0 && e % 3 != 0; };
  std::vector<char> H(C.Mp, 0);
  for (u64 x = 1 % Mp;;) {
    if (H[x]) break;
    H[x] = 1;
    x = x * (p % Mp) % Mp;
  }
  int o = 0;
  for (int e = 0; e < C.Mp; ++e) o += H[e];
  C.slots = C.nprime / o;
  // generators: repeatedly the smallest element of largest order modulo H,
  // then H <- H <g>
  C.gens.clear();
  auto order_mod_H = [&](int g) {
    int n = 1;
    for (long x = g; !H[x]; x = x * g % C.Mp) ++n;
    return n;
  };
  int covered = o;
  while (covered < C.nprime) {
    int best = -1, bn = 0;
    for (int g = 1; g < C.Mp; ++g)
      if (unit(g)) {
        int n = order_mod_H(g);
        if (n > bn) { bn = n; best = g; }
      }
    C.gens.push_back({best, bn});
    std::vector<char> H2(C.Mp, 0);
    for (int h = 0; h < C.Mp; ++h)
      if (H[h]) {
        long x = h;
        for (int j = 0; j < bn; ++j, x = x * best % C.Mp) H2[x] = 1;
      }
    H.swap(H2);
    covered = 0;
    for (int e = 0; e < C.Mp; ++e) covered += H[e];
  }
  // slot j = j_1 + n_1 (j_2 + n_2 (...)) holds the roots theta^(e p^i), e = prod g_i^j_i
  C.slot_exp.assign(C.slots, 1);
  for (int j = 0; j < C.slots; ++j) {
    long e = 1;
    int rest = j;
    for (auto& gn : C.gens) {
      for (int k = 0; k < rest % gn.second; ++k) e = e * gn.first % C.Mp;
      rest /= gn.second;
    }
    C.slot_exp[j] = (int)e;
  }
  // slot degree over X: ord_{3N}(p)
  int d = 1;
  for (u64 x = p % (3 * (u64)P.N); x != 1; x = x * p % (3 * (u64)P.N)) ++d;
  C.d = d;
  if (C.slots * d != P.N) throw std::runtime_error("slot count does not match ord_3N(p)");
}

// Smallest primitive (5N/2)-th root of unity mod q (q = 1 mod 5N/2): order
// exactly m = 5 * 2^k means x^m = 1, x^(m/2) != 1 and x^(m/5) != 1.
u64 find_root5(u64 q, int N) {
  const u64 m = 5 * (u64)N / 2;
  auto order_m = [&](u64 x) {
    return powmod(x, m, q) == 1 && powmod(x, m / 2, q) != 1 && powmod(x, m / 5, q) != 1;
  };
  u64 c = 0;
  for (u64 x = 2; !c; ++x) {
    u64 y = powmod(x, (q - 1) / m, q);
    if (order_m(y)) c = y;
  }
  u64 best = c, w = 1;
  for (u64 j = 1; j < m; ++j) {
    w = mulmod(w, c, q);
    if (j % 2 != 0 && j % 5 != 0 && w < best) best = w;
  }
  return best;
}

// ------------------------------------------------ Galois ring GR(p^k, 4)
// The tower GR(p^k, 2)[v] / (v^2 - w), w a non-square of F_{p^2}: an element
// is a + b v with a, b in GR(p^k, 2).
struct GR4 {
  GR2 a, b;
};
struct GR4Ring {
  u64 c, t;
  GR2 w;
  GR4 mul(const GR4& x, const GR4& y) const {
    GR2 ac = gr_mul(x.a, y.a, c, t), bd = gr_mul(x.b, y.b, c, t);
    GR2 ad = gr_mul(x.a, y.b, c, t), bc = gr_mul(x.b, y.a, c, t);
    return GR4{gr_add(ac, gr_mul(bd, w, c, t), t), gr_add(ad, bc, t)};
  }
  GR4 add(const GR4& x, const GR4& y) const { return GR4{gr_add(x.a, y.a, t), gr_add(x.b, y.b, t)}; }
  GR4 sub(const GR4& x, const GR4& y) const { return GR4{gr_sub(x.a, y.a, t), gr_sub(x.b, y.b, t)}; }
  GR4 one() const { return GR4{GR2{{1 % t, 0}}, GR2{{0, 0}}}; }
  GR4 pow(GR4 x, u64 e) const {
    GR4 r = one();
    while (e) {
      if (e & 1) r = mul(r, x);
      x = mul(x, x);
      e >>= 1;
    }
    return r;
  }
  // (a + b v)^-1 = (a - b v) / (a^2 - b^2 w)
  GR4 inv(const GR4& x) const {
    GR2 nrm = gr_sub(gr_mul(x.a, x.a, c, t), gr_mul(gr_mul(x.b, x.b, c, t), w, c, t), t);
    GR2 ni = gr_inv(nrm, c, t);
    return GR4{gr_mul(x.a, ni, c, t), gr_mul(gr_sub(GR2{{0, 0}}, x.b, t), ni, c, t)};
  }
  GR4 scale(const GR4& x, u64 k) const {
    return GR4{GR2{{mulmod(x.a.x[0], k, t), mulmod(x.a.x[1], k, t)}}, GR2{{mulmod(x.b.x[0], k, t), mulmod(x.b.x[1], k, t)}}};
  }
  static bool is(const GR4& x, u64 v) { return x.a.x[0] == v && x.a.x[1] == 0 && x.b.x[0] == 0 && x.b.x[1] == 0; }
  static u64 index(const GR4& x, u64 p) { return x.a.x[0] + p * (x.a.x[1] + p * (x.b.x[0] + p * x.b.x[1])); }
};

// Slot algebra of Phi_m, m = 5N/2 = 5 * 2^k (Section 2.1 with m = 5N/2):
// with 2^b the largest power of two dividing p^4 - 1, b' = min(b, k),
// M' = 5 * 2^b' and s = m / M', Phi_m(X) = Phi_M'(X^s) and Phi_M' splits
// over GR(p^r, 4) at theta^e, e in (Z/M')^*, because M' divides p^4 - 1.
// theta reduces to the element of smallest index of order exactly M' in
// F_{p^4} and is its Teichmueller lift. Slots, generators and slot order as
// for m = 3N.
static void make_slots_m5(Context& C) {
  const Params& P = C.P;
  const u64 p = (u64)P.p;
  int b = 0;
  const u64 p4 = p * p * p * p;
  for (u64 v = p4 - 1; v % 2 == 0; v /= 2) ++b;
  const int k = P.logN - 1;
  const int bp = std::min(b, k);
  C.Mp = 5 << bp;
  C.s = (5 << k) / C.Mp;
  C.nprime = P.N / C.s;
  for (u64 c = 2; c < p; ++c)
    if (powmod(c, (p - 1) / 2, p) == p - 1) { C.gr_c = c; break; }
  // w: first x0 + x1 u (index x0 + p x1) that is not a square in F_{p^2}
  GR2 w{{0, 0}};
  for (u64 i = 1; i < p * p; ++i) {
    GR2 x{{i % p, i / p}};
    if (!gr_is(gr_pow(x, (p * p - 1) / 2, C.gr_c, p), 1, 0)) { w = x; break; }
  }
  C.gr_w[0] = w.x[0];
  C.gr_w[1] = w.x[1];
  const GR4Ring F{C.gr_c, p, w};
  const u64 Mp = (u64)C.Mp;
  auto order_Mp = [&](const GR4& x) {
    return GR4Ring::is(F.pow(x, Mp), 1) && !GR4Ring::is(F.pow(x, Mp / 2), 1) && !GR4Ring::is(F.pow(x, Mp / 5), 1);
  };
  // one element of order M', then the smallest index among its powers prime to M'
  GR4 y{};
  bool found = false;
  for (u64 i = 1; !found; ++i) {
    u64 r = i;
    GR4 x{GR2{{r % p, (r / p) % p}}, GR2{{(r / (p * p)) % p, (r / (p * p * p)) % p}}};
    GR4 cand = F.pow(x, (p4 - 1) / Mp);
    if (order_Mp(cand)) { y = cand; found = true; }
  }
  GR4 th0 = y, cur = F.one();
  u64 best = ~0ULL;
  for (u64 j = 1; j < Mp; ++j) {
    cur = F.mul(cur, y);
    if (j % 2 != 0 && j % 5 != 0 && GR4Ring::index(cur, p) < best) { best = GR4Ring::index(cur, p); th0 = cur; }
  }
  // Teichmueller lift: theta = theta_0^((p^4)^(r-1)) in GR(p^r, 4)
  const GR4Ring R{C.gr_c, C.t, w};
  GR4 th = th0;
  for (int i = 1; i < P.r; ++i) th = R.pow(th, p4);
  if (!GR4Ring::is(R.pow(th, Mp), 1)) throw std::runtime_error("theta lift failed");
  C.theta4[0] = th.a.x[0];
  C.theta4[1] = th.a.x[1];
  C.theta4[2] = th.b.x[0];
  C.theta4[3] = th.b.x[1];
  auto unit = [&](int e) { return e % 2 != 0 && e % 5 != 0; };
  std::vector<char> H(C.Mp, 0);
  for (u64 x = 1 % Mp;;) {
    if (H[x]) break;
    H[x] = 1;
    x = x * (p % Mp) % Mp;
  }
  int o = 0;
  for (int e = 0; e < C.Mp; ++e) o += H[e];
  C.slots = C.nprime / o;
  C.gens.clear();
  auto order_mod_H = [&](int g) {
    int n = 1;
    for (long x = g; !H[x]; x = x * g % C.Mp) ++n;
    return n;
  };
  int covered = o;
  while (covered < C.nprime) {
    int bestg = -1, bn = 0;
    for (int g = 1; g < C.Mp; ++g)
      if (unit(g)) {
        int n = order_mod_H(g);
        if (n > bn) { bn = n; bestg = g; }
      }
    C.gens.push_back({bestg, bn});
    std::vector<char> H2(C.Mp, 0);
    for (int h = 0; h < C.Mp; ++h)
      if (H[h]) {
        long x = h;
        for (int j = 0; j < bn; ++j, x = x * bestg % C.Mp) H2[x] = 1;
      }
    H.swap(H2);
    covered = 0;
    for (int e = 0; e < C.Mp; ++e) covered += H[e];
  }
  C.slot_exp.assign(C.slots, 1);
  for (int j = 0; j < C.slots; ++j) {
    long e = 1;
    int rest = j;
    for (auto& gn : C.gens) {
      for (int kk = 0; kk < rest % gn.second; ++kk) e = e * gn.first % C.Mp;
      rest /= gn.second;
    }
    C.slot_exp[j] = (int)e;
  }
  const u64 m = 5 * (u64)P.N / 2;
  int d = 1;
  for (u64 x = p % m; x != 1; x = x * p % m) ++d;
  C.d = d;
  if (C.slots * d != P.N) throw std::runtime_error("slot count does not match ord_m(p)");
}

Context make_context(const Params& P0) {
  Context C;
  C.P = P0;
  Params& P = C.P;
  if (P.N != (1 << P.logN)) throw std::runtime_error("N must be 2^logN");
  if (P.m_odd == 0) P.m_odd = 1;
  if (P.m_odd != 1 && P.m_odd != 3 && P.m_odd != 5) throw std::runtime_error("m must be 2N, 3N or 5N/2");
  if (P.nmax == 0) P.nmax = P.N;
  if (P.nmax < P.N) throw std::runtime_error("nmax < N");
  C.t = ipow((u64)P.p, P.r);
  C.m = P.m_odd == 3 ? 3 * P.N : P.m_odd == 5 ? 5 * P.N / 2 : 2 * P.N;
  if (P.m_odd == 5) {
    if (P.p == 5 || P.p >= 32768 || P.logN < 3) throw std::runtime_error("m = 5N/2 needs p != 5, p < 2^15 and N >= 8");
    // primes q = 1 mod lcm(5*nmax/2, p^r) = 5*nmax*p^r/2
    C.primes = gen_primes(P.bits, 5 * (u64)P.nmax / 2 * C.t, P.L + P.alpha);
    for (u64 q : C.primes) C.psi.push_back(find_root5(q, P.N));
    make_slots_m5(C);
    return C;
  }
  if (P.m_odd == 3) {
    if (P.p % 3 == 0 || P.logN < 3) throw std::runtime_error("m = 3N needs p != 3 and N >= 8");
    // primes q = 1 mod lcm(3*nmax, p^r) = 3*nmax*p^r (q odd: nmax is even)
    C.primes = gen_primes(P.bits, 3 * (u64)P.nmax * C.t, P.L + P.alpha);
    for (u64 q : C.primes) C.psi.push_back(find_root3(q, P.N));
    make_slots_m3(C);
    return C;
  }
  // primes q = 1 mod lcm(2*nmax, p^r); p is odd, so the lcm is the product
  u64 M = 2 * (u64)P.nmax * C.t;
  C.primes = gen_primes(P.bits, M, P.L + P.alpha);
  for (u64 q : C.primes) C.psi.push_back(find_psi(q, P.N));
  // slots: X^N + 1 = prod_j (X^d - zeta_j) over Z_{p^r} when 2*slots | p - 1
  int d = 1;
  {
    u64 x = (u64)P.p % (2 * (u64)P.N);
    while (x != 1) { x = x * (u64)P.p % (2 * (u64)P.N); ++d; }
  }
  C.d = d;
  C.slots = P.N / d;
  if (((u64)P.p - 1) % (2 * (u64)C.slots) != 0)
    throw std::runtime_error("plaintext prime does not split X^N+1 into linear slot factors");
  // omega: smallest x mod p with x^slots = -1, Hensel-lifted to p^r
  u64 w0 = 0;
  for (u64 x = 2; x < (u64)P.p; ++x) {
    if (powmod(x, (u64)C.slots, (u64)P.p) == (u64)P.p - 1) { w0 = x; break; }
  }
  if (!w0) throw std::runtime_error("no slot root");
  u64 w = w0;
  for (int it = 0; it < P.r + 1; ++it) {
    u64 f = addmod(powmod(w, (u64)C.slots, C.t), 1, C.t);
    u64 fp = mulmod((u64)C.slots % C.t, powmod(w, (u64)C.slots - 1, C.t), C.t);
    w = submod(w, mulmod(f, invmod(fp, C.t), C.t), C.t);
  }
  if (powmod(w, (u64)C.slots, C.t) != C.t - 1) throw std::runtime_error("Hensel lift failed");
  C.omega = w;
  C.slot_exp.resize(C.slots);
  int two_l = 2 * C.slots;
  if (C.slots == 1) {
    C.slot_exp[0] = 1;
  } else {
    int half = C.slots / 2;
    int g = 1;
    for (int j = 0; j < half; ++j) {
      C.slot_exp[j] = g;
      C.slot_exp[j + half] = (two_l - g) % two_l;
      g = (g * 5) % two_l;
    }
  }
  return C;
}

// ================================================================= transform
// Negacyclic transform, written as the definition: twist by psi^i, then the
// textbook iterative radix-2 cyclic transform with omega = psi^2 (CLRS
// "iterative-FFT"), giving A[k] = a(psi^(2k+1)). The stored evaluation form is
// that vector in bit-reversed order: slot j holds a(psi^(2*bitrev(j)+1)).
static void cyclic_ntt(std::vector<u64>& A, u64 omega, u64 q, int logN) {
  int N = 1 << logN;
  std::vector<u64> B(N);
  for (int i = 0; i < N; ++i) B[bitrev(i, logN)] = A[i];
  for (int s = 1; s <= logN; ++s) {
    int m = 1 << s;
    u64 wm = powmod(omega, (u64)(N / m), q);
    for (int k = 0; k < N; k += m) {
      u64 w = 1;
      for (int j = 0; j < m / 2; ++j) {
        u64 t = mulmod(w, B[k + j + m / 2], q);
        u64 u = B[k + j];
        B[k + j] = addmod(u, t, q);
        B[k + j + m / 2] = submod(u, t, q);
        w = mulmod(w, wm, q);
      }
    }
  }
  A = B;
}

std::atomic<unsigned long long> g_ntt_count{0};

// m = 3N: Phi_3N(X) = X^N - X^(N/2) + 1 = (X^(N/2) - rho_0)(X^(N/2) - rho_1)
// with rho_h = omega^(e_h N/2), e_0 = 1, e_1 = 5, omega the primitive 3N-th
// root (rho_0 is a primitive 6th root of unity, rho_1 = rho_0^5). Half h of
// the evaluation form holds a mod (X^(N/2) - rho_h) at its roots
// omega^(e_h + 6k), k < N/2: twist by omega^(e_h i), then the cyclic transform
// of length N/2 with omega^6; word h N/2 + j = a(omega^(e_h + 6 bitrev(j))).
static void ntt_fwd_m3(const Context& C, int pi, Poly& a) {
  const int N = C.P.N, n = N / 2, logn = C.P.logN - 1;
  const u64 q = C.primes[pi], w = C.psi[pi];
  Poly out(N);
  for (int h = 0; h < 2; ++h) {
    const u64 eh = h == 0 ? 1 : 5;
    const u64 rho = powmod(w, eh * (u64)n, q), tw = powmod(w, eh, q);
    std::vector<u64> b(n);
    u64 pw = 1;
    for (int i = 0; i < n; ++i) {
      b[i] = mulmod(addmod(a[i], mulmod(rho, a[i + n], q), q), pw, q);
      pw = mulmod(pw, tw, q);
    }
    cyclic_ntt(b, powmod(w, 6, q), q, logn);
    for (int j = 0; j < n; ++j) out[(size_t)h * n + j] = b[bitrev(j, logn)];
  }
  a = out;
}

// Inverse of ntt_fwd_m3: per half the inverse cyclic transform and untwist
// give b_h = a mod (X^(N/2) - rho_h); then the Chinese remainder step
// a_hi = (b_0 - b_1) / (rho_0 - rho_1), a_lo = b_0 - rho_0 a_hi.
static void ntt_inv_m3(const Context& C, int pi, Poly& a) {
  const int N = C.P.N, n = N / 2, logn = C.P.logN - 1;
  const u64 q = C.primes[pi], w = C.psi[pi];
  const u64 n_inv = invmod((u64)n, q);
  std::vector<u64> b[2];
  u64 rho[2];
  for (int h = 0; h < 2; ++h) {
    const u64 eh = h == 0 ? 1 : 5;
    rho[h] = powmod(w, eh * (u64)n, q);
    const u64 tw_inv = invmod(powmod(w, eh, q), q);
    std::vector<u64> B(n);
    for (int k = 0; k < n; ++k) B[k] = a[(size_t)h * n + bitrev(k, logn)];
    cyclic_ntt(B, invmod(powmod(w, 6, q), q), q, logn);
    b[h].resize(n);
    u64 pw = 1;
    for (int i = 0; i < n; ++i) {
      b[h][i] = mulmod(mulmod(B[i], n_inv, q), pw, q);
      pw = mulmod(pw, tw_inv, q);
    }
  }
  const u64 dinv = invmod(submod(rho[0], rho[1], q), q);
  for (int i = 0; i < n; ++i) {
    u64 hi = mulmod(submod(b[0][i], b[1][i], q), dinv, q);
    a[i] = submod(b[0][i], mulmod(rho[0], hi, q), q);
    a[i + n] = hi;
  }
}

// m = 5N/2: Phi_m(X) = Phi_10(X^(N/4)) = prod_h (X^(N/4) - xi^(e_h)), xi =
// omega^(N/4) a primitive 10th root, e = (1, 3, 7, 9). Quarter h of the
// evaluation form holds a mod (X^(N/4) - xi^(e_h)) = sum_j xi^(e_h j) a_j
// (a_j the j-th quarter of the coefficients) at its roots omega^(e_h + 10k):
// twist by omega^(e_h i), cyclic transform of length N/4 with omega^10; word
// h N/4 + j = a(omega^(e_h + 10 bitrev(j))).
static const u64 kE5[4] = {1, 3, 7, 9};
static void ntt_fwd_m5(const Context& C, int pi, Poly& a) {
  const int N = C.P.N, n = N / 4, logn = C.P.logN - 2;
  const u64 q = C.primes[pi], w = C.psi[pi];
  const u64 xi = powmod(w, (u64)n, q);
  Poly out(N);
  for (int h = 0; h < 4; ++h) {
    const u64 eh = kE5[h], x = powmod(xi, eh, q), tw = powmod(w, eh, q);
    std::vector<u64> b(n);
    u64 pw = 1;
    for (int i = 0; i < n; ++i) {
      u64 v = 0, xj = 1;
      for (int j = 0; j < 4; ++j, xj = mulmod(xj, x, q)) v = addmod(v, mulmod(xj, a[i + (size_t)j * n], q), q);
      b[i] = mulmod(v, pw, q);
      pw = mulmod(pw, tw, q);
    }
    cyclic_ntt(b, powmod(w, 10, q), q, logn);
    for (int j = 0; j < n; ++j) out[(size_t)h * n + j] = b[bitrev(j, logn)];
  }
  a = out;
}

// Inverse of ntt_fwd_m5: b_h = a mod (X^(N/4) - x_h) per quarter, then the
// quarters a_j by Lagrange interpolation through the nodes x_h = xi^(e_h):
// sum_j a_j y^j = sum_h b_h prod_{h' != h} (y - x_h') / (x_h - x_h').
static void ntt_inv_m5(const Context& C, int pi, Poly& a) {
  const int N = C.P.N, n = N / 4, logn = C.P.logN - 2;
  const u64 q = C.primes[pi], w = C.psi[pi];
  const u64 xi = powmod(w, (u64)n, q), n_inv = invmod((u64)n, q);
  std::vector<u64> b[4];
  u64 x[4];
  for (int h = 0; h < 4; ++h) {
    const u64 eh = kE5[h];
    x[h] = powmod(xi, eh, q);
    const u64 tw_inv = invmod(powmod(w, eh, q), q);
    std::vector<u64> B(n);
    for (int k = 0; k < n; ++k) B[k] = a[(size_t)h * n + bitrev(k, logn)];
    cyclic_ntt(B, invmod(powmod(w, 10, q), q), q, logn);
    b[h].resize(n);
    u64 pw = 1;
    for (int i = 0; i < n; ++i) {
      b[h][i] = mulmod(mulmod(B[i], n_inv, q), pw, q);
      pw = mulmod(pw, tw_inv, q);
    }
  }
  // Lagrange basis coefficients L[h][j]
  u64 L[4][4];
  for (int h = 0; h < 4; ++h) {
    std::vector<u64> poly{1};  // prod_{h' != h} (y - x_h'), low degree first
    u64 den = 1;
    for (int h2 = 0; h2 < 4; ++h2) {
      if (h2 == h) continue;
      std::vector<u64> np(poly.size() + 1, 0);
      for (size_t i = 0; i < poly.size(); ++i) {
        np[i + 1] = addmod(np[i + 1], poly[i], q);
        np[i] = submod(np[i], mulmod(poly[i], x[h2], q), q);
      }
      poly = np;
      den = mulmod(den, submod(x[h], x[h2], q), q);
    }
    const u64 di = invmod(den, q);
    for (int j = 0; j < 4; ++j) L[h][j] = mulmod(poly[j], di, q);
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 4; ++j) {
      u64 v = 0;
      for (int h = 0; h < 4; ++h) v = addmod(v, mulmod(L[h][j], b[h][i], q), q);
      a[i + (size_t)j * n] = v;
    }
}

void ntt_fwd(const Context& C, int pi, Poly& a) {
  ++g_ntt_count;
  if (C.P.m_odd == 3) return ntt_fwd_m3(C, pi, a);
  if (C.P.m_odd == 5) return ntt_fwd_m5(C, pi, a);
  int N = C.P.N, logN = C.P.logN;
  u64 q = C.primes[pi], psi = C.psi[pi];
  std::vector<u64> b(N);
  u64 pw = 1;
  for (int i = 0; i < N; ++i) { b[i] = mulmod(a[i], pw, q); pw = mulmod(pw, psi, q); }
  cyclic_ntt(b, mulmod(psi, psi, q), q, logN);
  for (int j = 0; j < N; ++j) a[j] = b[bitrev(j, logN)];
}

void ntt_inv(const Context& C, int pi, Poly& a) {
  ++g_ntt_count;
  if (C.P.m_odd == 3) return ntt_inv_m3(C, pi, a);
  if (C.P.m_odd == 5) return ntt_inv_m5(C, pi, a);
  int N = C.P.N, logN = C.P.logN;
  u64 q = C.primes[pi], psi = C.psi[pi];
  std::vector<u64> A(N);
  for (int k = 0; k < N; ++k) A[k] = a[bitrev(k, logN)];
  u64 psi_inv = invmod(psi, q);
  cyclic_ntt(A, mulmod(psi_inv, psi_inv, q), q, logN);
  u64 n_inv = invmod((u64)N, q);
  u64 pw = 1;
  for (int i = 0; i < N; ++i) {
    a[i] = mulmod(mulmod(A[i], n_inv, q), pw, q);
    pw = mulmod(pw, psi_inv, q);
  }
}

Poly automorph_coeff(const Poly& a, int g, u64 q) {
  int N = (int)a.size();
  Poly out(N, 0);
  for (int i = 0; i < N; ++i) {
    long e = ((long)g * i) % (2L * N);
    if (e < N) out[e] = a[i];
    else out[e - N] = (q - a[i]) % q;
  }
  return out;
}

// a(X) -> a(X^g) mod Phi_m. For m = 3N: X^(3N/2) = -1 and X^N = X^(N/2) - 1
// modulo Phi_3N, so X^e (e mod 3N, folded to [0, 3N/2) with a sign) is X^e
// for e < N and X^(e - N/2) - X^(e - N) for N <= e < 3N/2.
Poly automorph_coeff(const Context& C, const Poly& a, int g, u64 q) {
  if (C.P.m_odd == 5) {
    // X^(5N/4) = -1 and X^N = X^(3N/4) - X^(N/2) + X^(N/4) - 1 modulo Phi_(5N/2)
    const long N = (long)a.size(), m = 5 * N / 2, half = m / 2;
    Poly out(N, 0);
    for (long i = 0; i < N; ++i) {
      long e = ((long)g * i) % m;
      u64 v = a[i] % q;
      if (e >= half) { e -= half; v = (q - v) % q; }
      if (e < N) {
        out[e] = addmod(out[e], v, q);
      } else {
        out[e - N / 4] = addmod(out[e - N / 4], v, q);
        out[e - N / 2] = submod(out[e - N / 2], v, q);
        out[e - 3 * N / 4] = addmod(out[e - 3 * N / 4], v, q);
        out[e - N] = submod(out[e - N], v, q);
      }
    }
    return out;
  }
  if (C.P.m_odd != 3) return automorph_coeff(a, g, q);
  const long N = (long)a.size(), m = 3 * N, half = m / 2;
  Poly out(N, 0);
  for (long i = 0; i < N; ++i) {
    long e = ((long)g * i) % m;
    u64 v = a[i] % q;
    if (e >= half) { e -= half; v = (q - v) % q; }
    if (e < N) {
      out[e] = addmod(out[e], v, q);
    } else {
      out[e - N / 2] = addmod(out[e - N / 2], v, q);
      out[e - N] = submod(out[e - N], v, q);
    }
  }
  return out;
}

// ===================================================================== slots
// m = 3N. Encoding constant slots v: the polynomial A of degree < n' = deg
// Phi_M' with A(theta^e) = v[slot of e] for every root theta^e of Phi_M',
// by Lagrange interpolation at the roots written with the node polynomial:
// A(y) = sum_e v_e Phi_M'(y) / ((y - theta^e) Phi_M''(theta^e)), where
// Phi_M'(y) = y^n' - y^(n'/2) + 1. The result has coefficients in Z_{p^t}
// (the values are Frobenius-invariant); m(X) = A(X^s).
static std::vector<u64> encode_m3(const Context& C, u64 t, const std::vector<u64>& v) {
  const int n = C.nprime, s = C.s, Mp = C.Mp;
  const u64 c = C.gr_c;
  const GR2 th{{C.theta[0] % t, C.theta[1] % t}};
  // slot of every exponent e in (Z/M')^*: the orbit representatives are slot_exp
  std::vector<int> slot_of(Mp, -1);
  for (int j = 0; j < C.slots; ++j) {
    long e = C.slot_exp[j];
    for (int k = 0; k < Mp && slot_of[e] < 0; ++k, e = e * (C.P.p % Mp) % Mp) slot_of[e] = j;
  }
  std::vector<GR2> A(n, GR2{{0, 0}});
  const u64 nn = (u64)n % t, nh = (u64)(n / 2) % t;
  for (int e = 1; e < Mp; ++e) {
    if (e % 2 == 0 || e % 3 == 0) continue;
    if (slot_of[e] < 0) throw std::runtime_error("encode: root outside every slot");
    const GR2 z = gr_pow(th, (u64)e, c, t);
    // Phi'(z) = n z^(n-1) - (n/2) z^(n/2-1)
    GR2 d1 = gr_pow(z, (u64)(n - 1), c, t), d2 = gr_pow(z, (u64)(n / 2 - 1), c, t);
    GR2 dphi = gr_sub(GR2{{mulmod(nn, d1.x[0], t), mulmod(nn, d1.x[1], t)}},
                      GR2{{mulmod(nh, d2.x[0], t), mulmod(nh, d2.x[1], t)}}, t);
    GR2 coef = gr_inv(dphi, c, t);
    const u64 val = v[slot_of[e]] % t;
    coef = GR2{{mulmod(coef.x[0], val, t), mulmod(coef.x[1], val, t)}};
    // synthetic division Phi(y) / (y - z): quotient digits from the top
    GR2 qk{{1 % t, 0}};  // coefficient of y^(n-1)
    for (int k = n - 1; k >= 0; --k) {
      A[k] = gr_add(A[k], gr_mul(coef, qk, c, t), t);
      if (k == 0) break;
      // q_{k-1} = phi_k + z q_k, phi_k = -1 at k = n/2, else 0 (0 < k < n)
      GR2 nq = gr_mul(z, qk, c, t);
      if (k == n / 2) nq = gr_sub(nq, GR2{{1 % t, 0}}, t);
      qk = nq;
    }
  }
  std::vector<u64> m(C.P.N, 0);
  for (int k = 0; k < n; ++k) {
    if (A[k].x[1] != 0) throw std::runtime_error("encode: interpolant leaves Z_{p^t}");
    m[(size_t)k * s] = A[k].x[0];
  }
  return m;
}

// m = 3N. Slot j's value: A_0(theta^e_j), A_0(y) = sum_k m[k s] y^k, read as
// its Z_{p^t} coordinate (exact for constant slots).
static std::vector<u64> decode_m3(const Context& C, u64 t, const std::vector<u64>& coeffs) {
  const GR2 th{{C.theta[0] % t, C.theta[1] % t}};
  std::vector<u64> v(C.slots, 0);
  for (int j = 0; j < C.slots; ++j) {
    const GR2 z = gr_pow(th, (u64)C.slot_exp[j], C.gr_c, t);
    GR2 acc{{0, 0}};
    for (int k = C.nprime - 1; k >= 0; --k)  // Horner
      acc = gr_add(gr_mul(acc, z, C.gr_c, t), GR2{{coeffs[(size_t)k * C.s] % t, 0}}, t);
    v[j] = acc.x[0];
  }
  return v;
}

// m = 5N/2. As encode_m3 over GR(p^t, 4), with the node polynomial
// Phi_M'(y) = y^(4h) - y^(3h) + y^(2h) - y^h + 1, h = n'/4.
static std::vector<u64> encode_m5(const Context& C, u64 t, const std::vector<u64>& v) {
  const int n = C.nprime, s = C.s, Mp = C.Mp, h = n / 4;
  const GR4Ring R{C.gr_c, t, GR2{{C.gr_w[0] % t, C.gr_w[1] % t}}};
  const GR4 th{GR2{{C.theta4[0] % t, C.theta4[1] % t}}, GR2{{C.theta4[2] % t, C.theta4[3] % t}}};
  std::vector<int> slot_of(Mp, -1);
  for (int j = 0; j < C.slots; ++j) {
    long e = C.slot_exp[j];
    for (int k = 0; k < Mp && slot_of[e] < 0; ++k, e = e * (C.P.p % Mp) % Mp) slot_of[e] = j;
  }
  std::vector<GR4> A(n, GR4{});
  auto phi_k = [&](int k) -> long { return k == 3 * h ? -1 : k == 2 * h ? 1 : k == h ? -1 : 0; };
  for (int e = 1; e < Mp; ++e) {
    if (e % 2 == 0 || e % 5 == 0) continue;
    if (slot_of[e] < 0) throw std::runtime_error("encode: root outside every slot");
    const GR4 z = R.pow(th, (u64)e);
    // Phi'(z) = 4h z^(4h-1) - 3h z^(3h-1) + 2h z^(2h-1) - h z^(h-1)
    GR4 dphi{};
    const long cs[4] = {4, -3, 2, -1};
    for (int i = 0; i < 4; ++i) {
      const int deg = (4 - i) * h;
      GR4 term = R.scale(R.pow(z, (u64)(deg - 1)), (u64)deg % t);
      dphi = cs[i] > 0 ? R.add(dphi, term) : R.sub(dphi, term);
    }
    GR4 coef = R.scale(R.inv(dphi), v[slot_of[e]] % t);
    GR4 qk = R.one();  // quotient coefficient of y^(n-1)
    for (int k = n - 1; k >= 0; --k) {
      A[k] = R.add(A[k], R.mul(coef, qk));
      if (k == 0) break;
      GR4 nq = R.mul(z, qk);
      const long ph = phi_k(k);
      if (ph > 0) nq = R.add(nq, R.one());
      if (ph < 0) nq = R.sub(nq, R.one());
      qk = nq;
    }
  }
  std::vector<u64> m(C.P.N, 0);
  for (int k = 0; k < n; ++k) {
    if (A[k].a.x[1] || A[k].b.x[0] || A[k].b.x[1]) throw std::runtime_error("encode: interpolant leaves Z_{p^t}");
    m[(size_t)k * s] = A[k].a.x[0];
  }
  return m;
}

static std::vector<u64> decode_m5(const Context& C, u64 t, const std::vector<u64>& coeffs) {
  const GR4Ring R{C.gr_c, t, GR2{{C.gr_w[0] % t, C.gr_w[1] % t}}};
  const GR4 th{GR2{{C.theta4[0] % t, C.theta4[1] % t}}, GR2{{C.theta4[2] % t, C.theta4[3] % t}}};
  std::vector<u64> v(C.slots, 0);
  for (int j = 0; j < C.slots; ++j) {
    const GR4 z = R.pow(th, (u64)C.slot_exp[j]);
    GR4 acc{};
    for (int k = C.nprime - 1; k >= 0; --k) {
      acc = R.mul(acc, z);
      acc.a.x[0] = addmod(acc.a.x[0], coeffs[(size_t)k * C.s] % t, t);
    }
    v[j] = acc.a.x[0];
  }
  return v;
}

std::vector<u64> encode(const Context& C, int t_exp, const std::vector<u64>& v) {
  u64 t = ipow((u64)C.P.p, t_exp);
  if ((int)v.size() != C.slots) throw std::runtime_error("encode: wrong slot count");
  if (C.P.m_odd == 3) return encode_m3(C, t, v);
  if (C.P.m_odd == 5) return encode_m5(C, t, v);
  u64 w = C.omega % t;
  u64 inv_l = invmod((u64)C.slots % t, t);
  std::vector<u64> m(C.P.N, 0);
  int two_l = 2 * C.slots;
  for (int k = 0; k < C.slots; ++k) {
    u64 acc = 0;
    for (int j = 0; j < C.slots; ++j) {
      // zeta_j^(-k) = omega^(-e_j k)
      long e = ((long)(two_l - C.slot_exp[j]) * k) % two_l;
      acc = addmod(acc, mulmod(v[j] % t, powmod(w, (u64)e, t), t), t);
    }
    m[(size_t)k * C.d] = mulmod(acc, inv_l, t);
  }
  return m;
}

std::vector<u64> decode(const Context& C, int t_exp, const std::vector<u64>& coeffs) {
  u64 t = ipow((u64)C.P.p, t_exp);
  if (C.P.m_odd == 3) return decode_m3(C, t, coeffs);
  if (C.P.m_odd == 5) return decode_m5(C, t, coeffs);
  u64 w = C.omega % t;
  int two_l = 2 * C.slots;
  std::vector<u64> v(C.slots, 0);
  for (int j = 0; j < C.slots; ++j) {
    u64 acc = 0;
    for (int k = 0; k < C.slots; ++k) {
      long e = ((long)C.slot_exp[j] * k) % two_l;
      acc = addmod(acc, mulmod(coeffs[(size_t)k * C.d] % t, powmod(w, (u64)e, t), t), t);
    }
    v[j] = acc;
  }
  return v;
}

// ====================================================================== keys
std::vector<i64> sample_secret(const Context& C) {
  int N = C.P.N;
  std::vector<int> idx(N);
  for (int i = 0; i < N; ++i) idx[i] = i;
  std::vector<i64> s(N, 0);
  for (int i = 0; i < C.P.h; ++i) {
    u32 x[4];
    draw(C, (u32)i, 0, 0, TAG_SK, x);
    u64 r64 = ((u64)x[1] << 32) | x[0];
    int j = i + (int)(r64 % (u64)(N - i));
    std::swap(idx[i], idx[j]);
    s[idx[i]] = (x[2] & 1) ? -1 : 1;
  }
  return s;
}

static Poly to_limb(const Context& C, const std::vector<i64>& v, int pi) {
  Poly a(C.P.N);
  for (int i = 0; i < C.P.N; ++i) a[i] = lift(v[i], C.primes[pi]);
  return a;
}

KSKey make_ksk(const Context& C, const std::vector<Poly>& sp_hat, u32 key_id) {
  const Params& P = C.P;
  int nl = P.L + P.alpha;
  int dnum = (P.L + P.alpha - 1) / P.alpha;
  // P = product of special primes, needed modulo each data prime
  KSKey K;
  K.b.resize(dnum);
  K.a.resize(dnum);
  for (int j = 0; j < dnum; ++j) {
    u32 id = key_id * 256u + (u32)j;
    std::vector<i64> e(P.N);
    for (int n = 0; n < P.N; ++n) e[n] = sample_cbd(C, (u32)n, id, TAG_KSK_E);
    K.b[j].resize(nl);
    K.a[j].resize(nl);
    limb_for(C, nl, [&](int i) {
      u64 q = C.primes[i];
      Poly a(P.N);
      for (int n = 0; n < P.N; ++n) a[n] = sample_uniform(C, (u32)n, (u32)i, id, TAG_KSK_A, q);
      Poly eh = to_limb(C, e, i);
      ntt_fwd(C, i, eh);
      u64 Pmod = 1;
      for (int k = 0; k < P.alpha; ++k) Pmod = mulmod(Pmod, C.primes[P.L + k] % q, q);
      bool in_digit = (i < P.L) && (i / P.alpha == j);
      Poly b(P.N);
      for (int n = 0; n < P.N; ++n) {
        u64 v = submod(mulmod(C.t % q, eh[n], q), mulmod(a[n], C.sk_hat[i][n], q), q);
        if (in_digit) v = addmod(v, mulmod(Pmod, sp_hat[i][n], q), q);
        b[n] = v;
      }
      K.b[j][i] = b;
      K.a[j][i] = a;
    });
  }
  return K;
}

void secret_keygen(Context& C) {
  int nl = C.P.L + C.P.alpha;
  C.sk = sample_secret(C);
  C.sk_hat.resize(nl);
  limb_for(C, nl, [&](int i) {
    C.sk_hat[i] = to_limb(C, C.sk, i);
    ntt_fwd(C, i, C.sk_hat[i]);
  });
  C.have_keys = true;
}

void keygen(Context& C, const std::vector<int>& galois) {
  const Params& P = C.P;
  int nl = P.L + P.alpha;
  secret_keygen(C);
  // relinearisation key: s' = s^2
  std::vector<Poly> s2(nl);
  limb_for(C, nl, [&](int i) {
    s2[i].resize(P.N);
    for (int n = 0; n < P.N; ++n) s2[i][n] = mulmod(C.sk_hat[i][n], C.sk_hat[i][n], C.primes[i]);
  });
  C.rlk = make_ksk(C, s2, 0);
  C.gk.clear();
  for (int g : galois) {
    std::vector<Poly> sg(nl);
    limb_for(C, nl, [&](int i) {
      sg[i] = automorph_coeff(C, to_limb(C, C.sk, i), g, C.primes[i]);
      ntt_fwd(C, i, sg[i]);
    });
    C.gk[g] = make_ksk(C, sg, (u32)g);
  }
  C.have_keys = true;
}

// ======================================================== encrypt / decrypt
Ct encrypt(const Context& C, const std::vector<u64>& m, u32 nonce, int t_exp) {
  const Params& P = C.P;
  if (!C.have_keys) throw std::runtime_error("encrypt: no keys");
  u64 t = ipow((u64)P.p, t_exp);
  Ct ct;
  ct.ncomp = 2;
  ct.level = P.L;
  ct.t_exp = t_exp;
  ct.c.assign(2, std::vector<Poly>(P.L));
  std::vector<i64> e(P.N);
  for (int n = 0; n < P.N; ++n) e[n] = sample_cbd(C, (u32)n, nonce, TAG_ENC_E);
  limb_for(C, P.L, [&](int i) {
    u64 q = C.primes[i];
    Poly a(P.N), me(P.N);
    for (int n = 0; n < P.N; ++n) a[n] = sample_uniform(C, (u32)n, (u32)i, nonce, TAG_ENC_A, q);
    for (int n = 0; n < P.N; ++n)
      me[n] = addmod(m[n] % t % q, mulmod(t % q, lift(e[n], q), q), q);
    ntt_fwd(C, i, me);
    Poly c0(P.N);
    for (int n = 0; n < P.N; ++n) c0[n] = submod(me[n], mulmod(a[n], C.sk_hat[i][n], q), q);
    ct.c[0][i] = c0;
    ct.c[1][i] = a;
  });
  return ct;
}

// v = c0 + c1 s (+ c2 s^2) as the centred integer representative modulo Q_level
static std::vector<std::pair<bool, Big>> decrypt_raw(const Context& C, const Ct& ct) {
  const Params& P = C.P;
  int l = ct.level;
  std::vector<Poly> v(l);
  limb_for(C, l, [&](int i) {
    u64 q = C.primes[i];
    Poly x(P.N);
    for (int n = 0; n < P.N; ++n) {
      u64 s = C.sk_hat[i][n];
      u64 acc = ct.c[0][i][n];
      acc = addmod(acc, mulmod(ct.c[1][i][n], s, q), q);
      if (ct.ncomp == 3) acc = addmod(acc, mulmod(ct.c[2][i][n], mulmod(s, s, q), q), q);
      x[n] = acc;
    }
    ntt_inv(C, i, x);
    v[i] = x;
  });
  // CRT: V = sum_i [v_i * (Q/q_i)^{-1}]_{q_i} * (Q/q_i) mod Q
  Big Q = Big::from(1);
  for (int i = 0; i < l; ++i) Q = big_mul_u64(Q, C.primes[i]);
  std::vector<Big> Qhat(l);
  std::vector<u64> Qhat_inv(l);
  for (int i = 0; i < l; ++i) {
    Big h = Big::from(1);
    for (int k = 0; k < l; ++k) if (k != i) h = big_mul_u64(h, C.primes[k]);
    Qhat[i] = h;
    Qhat_inv[i] = invmod(big_mod_u64(h, C.primes[i]), C.primes[i]);
  }
  Big half = big_shr1(Q);
  std::vector<std::pair<bool, Big>> out(P.N);
  // coefficients in blocks of 256 per worker task
  const int chunk = 256;
  limb_for(C, (P.N + chunk - 1) / chunk, [&](int blk) {
    for (int n = blk * chunk; n < std::min(P.N, (blk + 1) * chunk); ++n) {
      Big V;
      for (int i = 0; i < l; ++i) {
        u64 y = mulmod(v[i][n], Qhat_inv[i], C.primes[i]);
        V = big_add(V, big_mul_u64(Qhat[i], y));
      }
      while (big_cmp(V, Q) >= 0) V = big_sub(V, Q);
      if (big_cmp(V, half) > 0) out[n] = {true, big_sub(Q, V)};  // negative: -(Q - V)
      else out[n] = {false, V};
    }
  });
  return out;
}

std::vector<u64> decrypt(const Context& C, const Ct& ct) {
  u64 t = ipow((u64)C.P.p, ct.t_exp);
  auto raw = decrypt_raw(C, ct);
  std::vector<u64> m(C.P.N);
  for (int n = 0; n < C.P.N; ++n) {
    u64 r = big_mod_u64(raw[n].second, t);
    m[n] = raw[n].first ? (t - r) % t : r;
  }
  return m;
}

double noise_budget(const Context& C, const Ct& ct) {
  auto raw = decrypt_raw(C, ct);
  double mx = 0;
  for (auto& x : raw) mx = std::max(mx, big_log2(x.second));
  double logQ = 0;
  for (int i = 0; i < ct.level; ++i) logQ += std::log2((double)C.primes[i]);
  return logQ - 1.0 - mx;
}

// ==================================================================== BGV ops
static void need_same(const Ct& a, const Ct& b) {
  if (a.level != b.level) throw std::runtime_error("level mismatch");
  if (a.t_exp != b.t_exp) throw std::runtime_error("plaintext modulus mismatch");
}

static u64 cur_t(const Context& C, const Ct& a) { return ipow((u64)C.P.p, a.t_exp); }

Ct add(const Context& C, const Ct& a, const Ct& b) {
  need_same(a, b);
  Ct r = a.ncomp >= b.ncomp ? a : b;
  const Ct& o = a.ncomp >= b.ncomp ? b : a;
  for (int c = 0; c < o.ncomp; ++c)
    limb_for(C, a.level, [&](int i) {
      for (int n = 0; n < C.P.N; ++n)
        r.c[c][i][n] = addmod(r.c[c][i][n], o.c[c][i][n], C.primes[i]);
    });
  return r;
}

Ct sub(const Context& C, const Ct& a, const Ct& b) {
  return add(C, a, mul_scalar(C, b, -1));
}

Ct mul_scalar(const Context& C, const Ct& a, i64 s) {
  Ct r = a;
  for (int c = 0; c < a.ncomp; ++c)
    limb_for(C, a.level, [&](int i) {
      u64 q = C.primes[i], k = lift(s, q);
      for (int n = 0; n < C.P.N; ++n) r.c[c][i][n] = mulmod(a.c[c][i][n], k, q);
    });
  return r;
}

Ct add_scalar(const Context& C, const Ct& a, i64 s) {
  // the constant polynomial s evaluates to s at every point
  Ct r = a;
  limb_for(C, a.level, [&](int i) {
    u64 q = C.primes[i], k = lift(s, q);
    for (int n = 0; n < C.P.N; ++n) r.c[0][i][n] = addmod(r.c[0][i][n], k, q);
  });
  return r;
}

Ct tensor(const Context& C, const Ct& a, const Ct& b) {
  need_same(a, b);
  if (a.ncomp != 2 || b.ncomp != 2) throw std::runtime_error("tensor: needs 2-component inputs");
  Ct r;
  r.ncomp = 3; r.level = a.level; r.t_exp = a.t_exp;
  r.c.assign(3, std::vector<Poly>(a.level, Poly(C.P.N)));
  limb_for(C, a.level, [&](int i) {
    u64 q = C.primes[i];
    for (int n = 0; n < C.P.N; ++n) {
      u64 a0 = a.c[0][i][n], a1 = a.c[1][i][n], b0 = b.c[0][i][n], b1 = b.c[1][i][n];
      r.c[0][i][n] = mulmod(a0, b0, q);
      r.c[1][i][n] = addmod(mulmod(a0, b1, q), mulmod(a1, b0, q), q);
      r.c[2][i][n] = mulmod(a1, b1, q);
    }
  });
  return r;
}

// Drop the primes with global indices src[] from x (given in coefficient form on
// those primes): returns delta = t * conv(t^{-1} x mod Q_src) on each destination
// prime dst[m], in coefficient form. conv is the fast base conversion
//   conv(r) = sum_i [r_i * (Q_src/q_i)^{-1}]_{q_i} * (Q_src/q_i)   (mod q_dst).
static std::vector<Poly> scaled_base_conv(const Context& C, const std::vector<Poly>& x,
                                          const std::vector<int>& src, const std::vector<int>& dst,
                                          u64 t) {
  int N = C.P.N, k = (int)src.size();
  std::vector<Poly> y(k, Poly(N));
  limb_for(C, k, [&](int a) {
    u64 qa = C.primes[src[a]];
    u64 hat = 1;  // Q_src / q_a mod q_a
    for (int b = 0; b < k; ++b) if (b != a) hat = mulmod(hat, C.primes[src[b]] % qa, qa);
    u64 hat_inv = invmod(hat, qa);
    u64 t_inv = invmod(t % qa, qa);
    for (int n = 0; n < N; ++n) y[a][n] = mulmod(mulmod(x[a][n], t_inv, qa), hat_inv, qa);
  });
  std::vector<Poly> out(dst.size(), Poly(N));
  limb_for(C, (int)dst.size(), [&](int m) {
    u64 qm = C.primes[dst[m]];
    std::vector<u64> hat_m(k);
    for (int a = 0; a < k; ++a) {
      u64 h = 1;
      for (int b = 0; b < k; ++b) if (b != a) h = mulmod(h, C.primes[src[b]] % qm, qm);
      hat_m[a] = h;
    }
    for (int n = 0; n < N; ++n) {
      u64 acc = 0;
      for (int a = 0; a < k; ++a) acc = addmod(acc, mulmod(y[a][n] % qm, hat_m[a], qm), qm);
      out[m][n] = mulmod(acc, t % qm, qm);
    }
  });
  return out;
}

// ModUp of every digit of d and the inner product with the key: acc0, acc1 over
// the current data primes then the special primes (evaluation form).
static void keyswitch_acc(const Context& C, const std::vector<Poly>& d, int l, const KSKey& K,
                          std::vector<Poly>& acc0, std::vector<Poly>& acc1) {
  const Params& P = C.P;
  int N = P.N, alpha = P.alpha;
  std::vector<Poly> dc = d;
  limb_for(C, l, [&](int i) { ntt_inv(C, i, dc[i]); });
  // target primes: the current data primes, then the special primes
  std::vector<int> tgt;
  for (int i = 0; i < l; ++i) tgt.push_back(i);
  for (int k = 0; k < alpha; ++k) tgt.push_back(P.L + k);
  acc0.assign(tgt.size(), Poly(N, 0));
  acc1.assign(tgt.size(), Poly(N, 0));
  int dnum = (l + alpha - 1) / alpha;
  // one worker task per target prime m; it runs over the digits j in order
  limb_for(C, (int)tgt.size(), [&](int m) {
    for (int j = 0; j < dnum; ++j) {
      int lo = j * alpha, hi = std::min((j + 1) * alpha, l);
      int gm = tgt[m];
      u64 qm = C.primes[gm];
      Poly ext(N);
      if (gm >= lo && gm < hi) {
        ext = d[gm];
      } else {
        // fast base conversion of the digit's residues to prime gm:
        //   sum_i [d_i * (Q_j/q_i)^{-1}]_{q_i} * (Q_j/q_i)  (mod q_gm)
        std::vector<u64> hat_inv(hi - lo), hat_m(hi - lo);
        for (int i = lo; i < hi; ++i) {
          u64 qi = C.primes[i];
          u64 hat = 1, hm = 1;
          for (int b = lo; b < hi; ++b) if (b != i) {
            hat = mulmod(hat, C.primes[b] % qi, qi);
            hm = mulmod(hm, C.primes[b] % qm, qm);
          }
          hat_inv[i - lo] = invmod(hat, qi);
          hat_m[i - lo] = hm;
        }
        for (int n = 0; n < N; ++n) {
          u64 acc = 0;
          for (int i = lo; i < hi; ++i) {
            u64 y = mulmod(dc[i][n], hat_inv[i - lo], C.primes[i]);
            acc = addmod(acc, mulmod(y % qm, hat_m[i - lo], qm), qm);
          }
          ext[n] = acc;
        }
        ntt_fwd(C, gm, ext);
      }
      for (int n = 0; n < N; ++n) {
        acc0[m][n] = addmod(acc0[m][n], mulmod(ext[n], K.b[j][gm][n], qm), qm);
        acc1[m][n] = addmod(acc1[m][n], mulmod(ext[n], K.a[j][gm][n], qm), qm);
      }
    }
  });
}

void keyswitch(const Context& C, const std::vector<Poly>& d, int l, const KSKey& K, int t_exp,
               std::vector<Poly>& k0, std::vector<Poly>& k1) {
  const Params& P = C.P;
  int N = P.N, alpha = P.alpha;
  u64 t = ipow((u64)P.p, t_exp);
  std::vector<Poly> acc0, acc1;
  keyswitch_acc(C, d, l, K, acc0, acc1);
  // ModDown: (acc - t*conv(t^{-1} acc mod P)) * P^{-1} on the data primes
  std::vector<int> sp, dp;
  for (int k = 0; k < alpha; ++k) sp.push_back(P.L + k);
  for (int i = 0; i < l; ++i) dp.push_back(i);
  auto moddown = [&](std::vector<Poly>& acc, std::vector<Poly>& out) {
    std::vector<Poly> xs(alpha);
    limb_for(C, alpha, [&](int k) { xs[k] = acc[l + k]; ntt_inv(C, P.L + k, xs[k]); });
    std::vector<Poly> delta = scaled_base_conv(C, xs, sp, dp, t);
    out.assign(l, Poly(N));
    limb_for(C, l, [&](int i) {
      u64 q = C.primes[i];
      ntt_fwd(C, i, delta[i]);
      u64 Pm = 1;
      for (int k = 0; k < alpha; ++k) Pm = mulmod(Pm, C.primes[P.L + k] % q, q);
      u64 Pinv = invmod(Pm, q);
      for (int n = 0; n < N; ++n) out[i][n] = mulmod(submod(acc[i][n], delta[i][n], q), Pinv, q);
    });
  };
  moddown(acc0, k0);
  moddown(acc1, k1);
}

Ct relin(const Context& C, const Ct& a) {
  if (a.ncomp != 3) throw std::runtime_error("relin: needs 3 components");
  std::vector<Poly> k0, k1;
  keyswitch(C, a.c[2], a.level, C.rlk, a.t_exp, k0, k1);
  Ct r;
  r.ncomp = 2; r.level = a.level; r.t_exp = a.t_exp;
  r.c.assign(2, std::vector<Poly>(a.level, Poly(C.P.N)));
  limb_for(C, a.level, [&](int i) {
    u64 q = C.primes[i];
    for (int n = 0; n < C.P.N; ++n) {
      r.c[0][i][n] = addmod(a.c[0][i][n], k0[i][n], q);
      r.c[1][i][n] = addmod(a.c[1][i][n], k1[i][n], q);
    }
  });
  return r;
}

Ct modswitch(const Context& C, const Ct& a, int drop) {
  if (drop <= 0) return a;
  int l = a.level, nl = l - drop;
  if (nl < 1) throw std::runtime_error("modswitch: out of levels");
  u64 t = cur_t(C, a);
  std::vector<int> src, dst;
  for (int i = nl; i < l; ++i) src.push_back(i);
  for (int i = 0; i < nl; ++i) dst.push_back(i);
  Ct r;
  r.ncomp = a.ncomp; r.level = nl; r.t_exp = a.t_exp;
  r.c.assign(a.ncomp, std::vector<Poly>(nl, Poly(C.P.N)));
  for (int c = 0; c < a.ncomp; ++c) {
    std::vector<Poly> xs(drop);
    limb_for(C, drop, [&](int k) { xs[k] = a.c[c][nl + k]; ntt_inv(C, nl + k, xs[k]); });
    std::vector<Poly> delta = scaled_base_conv(C, xs, src, dst, t);
    limb_for(C, nl, [&](int i) {
      u64 q = C.primes[i];
      ntt_fwd(C, i, delta[i]);
      u64 Qd = 1;
      for (int k = nl; k < l; ++k) Qd = mulmod(Qd, C.primes[k] % q, q);
      u64 inv = invmod(Qd, q);
      for (int n = 0; n < C.P.N; ++n)
        r.c[c][i][n] = mulmod(submod(a.c[c][i][n], delta[i][n], q), inv, q);
    });
  }
  return r;
}

Ct modswitch_to(const Context& C, const Ct& a, int level) {
  if (level > a.level) throw std::runtime_error("modswitch_to: cannot raise level");
  return modswitch(C, a, a.level - level);
}

Ct rotate(const Context& C, const Ct& a, int g) {
  if (a.ncomp != 2) throw std::runtime_error("rotate: needs 2 components");
  auto it = C.gk.find(g);
  if (it == C.gk.end()) throw std::runtime_error("rotate: no Galois key");
  Ct s = a;
  limb_for(C, 2 * a.level, [&](int ci) {
    int c = ci / a.level, i = ci % a.level;
    Poly x = a.c[c][i];
    ntt_inv(C, i, x);
    x = automorph_coeff(C, x, g, C.primes[i]);
    ntt_fwd(C, i, x);
    s.c[c][i] = x;
  });
  std::vector<Poly> k0, k1;
  keyswitch(C, s.c[1], a.level, it->second, a.t_exp, k0, k1);
  Ct r = s;
  limb_for(C, a.level, [&](int i) {
    u64 q = C.primes[i];
    for (int n = 0; n < C.P.N; ++n) {
      r.c[0][i][n] = addmod(s.c[0][i][n], k0[i][n], q);
      r.c[1][i][n] = k1[i][n];
    }
  });
  return r;
}

Ct divide_by_p(const Context& C, const Ct& a) {
  if (a.t_exp < 2) throw std::runtime_error("divide_by_p: plaintext modulus already p");
  Ct r = a;
  for (int c = 0; c < a.ncomp; ++c)
    limb_for(C, a.level, [&](int i) {
      u64 q = C.primes[i], pinv = invmod((u64)C.P.p % q, q);
      for (int n = 0; n < C.P.N; ++n) r.c[c][i][n] = mulmod(a.c[c][i][n], pinv, q);
    });
  r.t_exp = a.t_exp - 1;
  return r;
}

// Relinearise a 3-component ciphertext and drop its last prime in one ModDown:
// over Q_l and P, c_j = P*d_j + acc_j (P*d_j vanishes on the special primes);
// with D = {q_{l-1}} and the special primes,
//   c'_j = (c_j - t*conv([t^{-1} c_j]_D)) * (q_{l-1} P)^{-1}   over Q_{l-1}.
Ct relin_drop(const Context& C, const Ct& a) {
  if (a.ncomp != 3) throw std::runtime_error("relin_drop: needs 3 components");
  const Params& P = C.P;
  int N = P.N, l = a.level, alpha = P.alpha;
  if (l < 2) throw std::runtime_error("relin_drop: out of levels");
  u64 t = ipow((u64)P.p, a.t_exp);
  std::vector<Poly> acc[2];
  keyswitch_acc(C, a.c[2], l, C.rlk, acc[0], acc[1]);
  std::vector<int> src, dst;
  src.push_back(l - 1);
  for (int k = 0; k < alpha; ++k) src.push_back(P.L + k);
  for (int i = 0; i < l - 1; ++i) dst.push_back(i);
  Ct r;
  r.ncomp = 2; r.level = l - 1; r.t_exp = a.t_exp;
  r.c.assign(2, std::vector<Poly>(l - 1, Poly(N)));
  for (int c = 0; c < 2; ++c) {
    // c_j on every data prime (index = prime) and special prime (index l + k)
    std::vector<Poly> ext(l + alpha);
    limb_for(C, l, [&](int i) {
      u64 q = C.primes[i], Pm = 1;
      for (int k = 0; k < alpha; ++k) Pm = mulmod(Pm, C.primes[P.L + k] % q, q);
      ext[i].resize(N);
      for (int n = 0; n < N; ++n) ext[i][n] = addmod(mulmod(Pm, a.c[c][i][n], q), acc[c][i][n], q);
    });
    for (int k = 0; k < alpha; ++k) ext[l + k] = acc[c][l + k];
    // D = {q_{l-1}} and the special primes, in that order, in coefficient form
    std::vector<Poly> xs(alpha + 1);
    limb_for(C, alpha + 1, [&](int k) {
      xs[k] = ext[l - 1 + k];
      ntt_inv(C, k == 0 ? l - 1 : P.L + k - 1, xs[k]);
    });
    std::vector<Poly> delta = scaled_base_conv(C, xs, src, dst, t);
    limb_for(C, l - 1, [&](int i) {
      u64 q = C.primes[i];
      ntt_fwd(C, i, delta[i]);
      u64 Dm = C.primes[l - 1] % q;
      for (int k = 0; k < alpha; ++k) Dm = mulmod(Dm, C.primes[P.L + k] % q, q);
      u64 inv = invmod(Dm, q);
      for (int n = 0; n < N; ++n) r.c[c][i][n] = mulmod(submod(ext[i][n], delta[i][n], q), inv, q);
    });
  }
  return r;
}

Ct mul(const Context& C, const Ct& a, const Ct& b) {
  int l = std::min(a.level, b.level);
  Ct x = modswitch_to(C, a, l), y = modswitch_to(C, b, l);
  return relin_drop(C, tensor(C, x, y));
}

}  // namespace orc
