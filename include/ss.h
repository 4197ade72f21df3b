/*
 * ss.h -- C ABI of the GB300 space-switching BGV library (libss.so).
 *
 * Method: "space switching" (arXiv 2604.19890): BGV arithmetic stays in the
 * number space Z_{p^r}; before a comparison each value is reduced
 * homomorphically to its r balanced base-p digits in Z_p (Algorithm 3), each
 * digit is compared with interpolation polynomials evaluated by
 * Paterson-Stockmeyer (Section 4.3, Algorithm 4), and the result is raised
 * back to Z_{p^r} with G_{p,r} (Section 4.4).
 *
 * Conventions shared by every call
 *  - Ring Z[X]/Phi_m(X), N a power of two: m = 2N, Phi_m = X^N+1 (the
 *    default), m = 3N, Phi_m = X^N - X^(N/2) + 1 (ss_params.m_odd = 3), or
 *    m = 5N/2, Phi_m = Phi_10(X^(N/4)) (m_odd = 5): the paper's general
 *    cyclotomic m, Section 2.1, with N / Ord(m, p) slots.
 *    RNS chain of L data primes q_0 > ... > q_{L-1} and alpha special primes,
 *    all = 1 mod (m/N)*nmax*p^r.
 *  - A ciphertext batch (ss_ct) lives in caller-owned DEVICE memory laid out
 *    uint64[count][ncomp][capacity][N]: limb i of component c of ciphertext b
 *    starts at data + ((b*ncomp + c)*capacity + i)*N. Limbs are stored in
 *    evaluation (NTT) form, psi_i the smallest primitive m-th root of unity
 *    mod q_i: for m = 2N word j of limb i is a(psi_i^(2*bitrev(j)+1)) mod q_i;
 *    for m = 3N word h*N/2 + j (h = 0, 1; j < N/2) is
 *    a(psi_i^(e_h + 6*bitrev(j))) with e_0 = 1, e_1 = 5 and bitrev over
 *    log2(N/2) bits; for m = 5N/2 word h*N/4 + j (h = 0..3; j < N/4) is
 *    a(psi_i^(e_h + 10*bitrev(j))), e = (1, 3, 7, 9), bitrev over log2(N/4).
 *    Only limbs 0..level-1 are meaningful. The library never frees caller
 *    memory; outputs must have capacity >= the level they receive.
 *  - Every device call is enqueued on the given stream (NULL = legacy default
 *    stream) and is asynchronous unless stated otherwise. The library keeps
 *    its own scratch in a stream-ordered pool (cudaMallocAsync).
 *  - Every call returns an ss_status; ss_last_error() gives a thread-local
 *    message for the last failure. Errors never cross the ABI as exceptions.
 *  - Calls that run an evaluation schedule (ss_mul_relin, ss_eval_g,
 *    ss_reduce_to_digits, ss_compare_lt, ss_compare, ss_raise_modulus,
 *    ss_rotate_sum, ss_query_*) first plan it on the host thread (levels and
 *    plaintext moduli only): a chain too short for the schedule returns
 *    SS_ERR_NOISE before anything is enqueued, copied or allocated. Planning
 *    state is per thread and never affects other threads' calls.
 *  - Keys and contexts are library-owned and released with *_destroy.
 */
#ifndef SS_H
#define SS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SS_OK = 0,
  SS_ERR_PARAM = 1,   /* invalid argument or parameter set */
  SS_ERR_LEVEL = 2,   /* not enough levels for the operation */
  SS_ERR_NOISE = 3,   /* the evaluation plan needs more depth than remains */
  SS_ERR_TMOD = 4,    /* mismatched plaintext modulus (t_exp) */
  SS_ERR_SHAPE = 5,   /* mismatched batch count, component count or capacity */
  SS_ERR_OOM = 6,     /* device allocation failed */
  SS_ERR_TIMEOUT = 7, /* a bounded wait gave up */
  SS_ERR_CUDA = 8     /* a CUDA call failed */
} ss_status;

typedef struct ss_ctx ss_ctx;   /* opaque: parameters, tables, keys */
typedef void* ss_stream;        /* a cudaStream_t */

typedef struct {
  int32_t logN;     /* ring dimension N = 2^logN (3..16) */
  int32_t L;        /* data primes */
  int32_t alpha;    /* special primes = key-switching digit width */
  int32_t bits;     /* primes lie in (2^(bits-1), 2^bits); 20 <= bits <= 58 */
  int32_t p;        /* plaintext prime >= 5; p = 1 mod 4 when m = 2N; p != 5, p < 2^15 when m = 5N/2 */
  int32_t r;        /* plaintext modulus p^r */
  int32_t h;        /* Hamming weight of the ternary secret (Section 5.1: 120) */
  int32_t nmax;     /* largest N the prime chain must support (0 = N) */
  uint64_t seed;    /* Philox4x32-10 key for every sampled value */
  int32_t m_odd;    /* odd part of the cyclotomic index m (Section 2.1, 5.1): 0 or 1 -> m = 2N,
                       ring Z[X]/(X^N + 1); 3 -> m = 3N, ring Z[X]/(X^N - X^(N/2) + 1);
                       5 -> m = 5N/2, ring Z[X]/(X^N - X^(3N/4) + X^(N/2) - X^(N/4) + 1), N >= 32 */
  int32_t reserved; /* 0 */
} ss_params;

typedef struct {
  uint64_t* data;   /* device pointer, see layout above */
  int32_t count;    /* ciphertexts in the batch */
  int32_t ncomp;    /* 2, or 3 after ss_mul */
  int32_t level;    /* data primes held */
  int32_t t_exp;    /* plaintext modulus p^t_exp */
  int32_t capacity; /* limbs allocated per component */
  int32_t reserved;
} ss_ct;

const char* ss_last_error(void);

/* Named parameter sets. id 0: N=2^13, 36-bit primes, p^r=17^2 (toy);
 * 1: N=2^15, 55-bit, 257^2; 2: N=2^16, 55-bit, 257^3; 3: as 2 on the ring
 * m = 3N (256 slots); 4: as 2 on the ring m = 5N/2 (512 slots). The chain
 * length L is the one the query needs (the depth of Algorithms 3/4, raise and
 * SUM). */
ss_status ss_params_preset(int id, ss_params* out);

/* Builds the prime chain, transform tables, base-conversion constants and
 * slot structure (Section 2.1: R_{p^r} splits into `slots` factors). */
ss_status ss_context_create(const ss_params* prm, ss_ctx** out);
void ss_context_destroy(ss_ctx* ctx);

/* Sizes: N, L, alpha, slots, d = N/slots, p, r, primes[L+alpha] (may be NULL). */
ss_status ss_context_info(const ss_ctx* ctx, int32_t* N, int32_t* L, int32_t* alpha, int32_t* slots,
                          int32_t* d, uint64_t* primes);

/* Secret key (ternary, Hamming weight h; Section 2.1 and 5.1), the
 * relinearisation key for s^2 and one Galois key per element of `galois`
 * (units mod m: residues prime to m). Keys are hybrid key-switching keys over the data and
 * special primes, device-resident and owned by ctx. Synchronous. */
ss_status ss_keygen(ss_ctx* ctx, const int32_t* galois, int32_t ngalois);

/* Galois elements ss_rotate_sum uses; returns the count, writes up to cap
 * elements. m = 2N: 5^(2^i) mod 2N for i < log2(slots/2), then 2N-1.
 * m = 3N, 5N/2: for each slot-group generator g of order n (below), g^(2^i)
 * mod m for i < log2 n, generators in their order. */
int32_t ss_rotate_sum_elements(const ss_ctx* ctx, int32_t* out, int32_t cap);

/* Slot encoding over Z_{p^t_exp} (host, synchronous): slots[slots] ->
 * coefficients[N]. m = 2N: slot j is the constant value modulo X^d - zeta_j.
 * m = 3N: with 2^b the largest power of two dividing p^2 - 1, b' = min(b,
 * log2 N), M' = 3*2^b' and s = 3N/M', Phi_3N(X) = Phi_M'(X^s) and Phi_M'
 * splits over the Galois ring GR(p^r, 2) = Z_{p^r}[u]/(u^2 - c) (c the
 * smallest quadratic non-residue mod p) at theta^e, e in (Z/M')^*, theta the
 * root of unity of order M' lifting the first element x0 + x1 u of F_{p^2}
 * (in the order x0 + p*x1) of that order. Slots are the orbits of (Z/M')^*
 * under multiplication by p; slot j = j_1 + n_1 (j_2 + n_2 (...)) is the
 * orbit of g_1^j_1 g_2^j_2 ..., where g_i is the smallest residue of largest
 * order n_i modulo the subgroup generated by p, g_1, ..., g_{i-1}. The
 * encoding is A(X^s) with A(theta^e) = the value of e's slot; decoding
 * returns the Z_{p^t} coordinate of A_0(theta^e_j), A_0 = sum_k c[k s] y^k.
 * m = 5N/2: the same with 2^b || p^4 - 1, b' = min(b, log2 N - 1), M' =
 * 5*2^b', s = m/M', units prime to 10, and GR(p^r, 4) = GR(p^r, 2)[v]/(v^2 -
 * w), w the first non-square x0 + x1 u of F_{p^2}; theta lifts the element of
 * smallest index x0 + p x1 + p^2 x2 + p^3 x3 (basis 1, u, v, uv) of order M'. */
ss_status ss_encode(const ss_ctx* ctx, int32_t t_exp, const uint64_t* slots, uint64_t* coeffs);
ss_status ss_decode(const ss_ctx* ctx, int32_t t_exp, const uint64_t* coeffs, uint64_t* slots);

/* Algorithm 1 (secret-key BGV encryption) for a batch: coeffs is a DEVICE
 * array uint64[count][N] of plaintext coefficients in [0, p^t_exp);
 * ciphertext b uses Philox nonce (nonce0 + b). out gets level L. */
ss_status ss_encrypt(ss_ctx* ctx, const uint64_t* coeffs, int32_t count, uint32_t nonce0, int32_t t_exp,
                     ss_ct* out, ss_stream stream);

/* Algorithm 2: m = c0 + c1 s (+ c2 s^2) mod Q, centred, reduced mod the
 * ciphertext's current p^t_exp (Lemma 4). Writes DEVICE uint64[count][N].
 * Only the coefficients at multiples of d are computed (the slot
 * coefficients); the others are written as zero. */
ss_status ss_decrypt(ss_ctx* ctx, const ss_ct* in, uint64_t* coeffs, ss_stream stream);
/* (For m = 3N and 5N/2 the computed coefficients are those at multiples of s.) */

/* ---- BGV operations (Section 2.1); operands must share level and t_exp ---- */
ss_status ss_add(ss_ctx* ctx, const ss_ct* a, const ss_ct* b, ss_ct* out, ss_stream stream);
ss_status ss_sub(ss_ctx* ctx, const ss_ct* a, const ss_ct* b, ss_ct* out, ss_stream stream);
ss_status ss_mul_scalar(ss_ctx* ctx, const ss_ct* a, int64_t c, ss_ct* out, ss_stream stream);
ss_status ss_add_scalar(ss_ctx* ctx, const ss_ct* a, int64_t c, ss_ct* out, ss_stream stream);
/* tensor product: out gets 3 components */
ss_status ss_mul(ss_ctx* ctx, const ss_ct* a, const ss_ct* b, ss_ct* out, ss_stream stream);
/* hybrid key switch of c2 with the relinearisation key: 3 -> 2 components */
ss_status ss_relin(ss_ctx* ctx, const ss_ct* a, ss_ct* out, ss_stream stream);
/* BGV multiplication as the evaluation schedules run it (Section 2.1: the
 * product of two ciphertexts, then relinearisation and modulus switching):
 * both operands are switched to the lower of their levels l, tensored, and the
 * result is relinearised and divided by q_{l-1} in one ModDown over
 * {q_{l-1}} and the special primes. 2-component inputs of equal count and
 * t_exp; out receives 2 components at level l - 1 (capacity >= l - 1). */
ss_status ss_mul_relin(ss_ctx* ctx, const ss_ct* a, const ss_ct* b, ss_ct* out, ss_stream stream);
/* Same result as ss_relin, for callers that cannot allocate device memory
 * while they run (a host framework that owns all device memory through its
 * own allocator, or a service that must not risk an allocation stalling or
 * failing mid-request). The paper has no counterpart: this is a deployment
 * variant. Scratch comes from one file-scope device array of 64 MiB that
 * every GPU loading the library holds until the process exits; the call
 * allocates nothing. A call needs count*(l + dnum*(l+alpha) + 2*(l+alpha) +
 * 2*l)*N words at level l (dnum = ceil(l/alpha)); larger calls fail with
 * SS_ERR_PARAM. All calls share the array, so calls that overlap on the GPU
 * race. The first call on a device looks up the array's address (with that
 * device current); make it before any stream capture. */
ss_status ss_relin_noalloc(ss_ctx* ctx, const ss_ct* a, ss_ct* out, ss_stream stream);
/* drops the last `drop` primes at once: c' = (c - t*conv(t^-1 c mod Q_drop)) / Q_drop */
ss_status ss_modswitch(ss_ctx* ctx, const ss_ct* a, int32_t drop, ss_ct* out, ss_stream stream);
/* sigma_g (X -> X^g) then key switch back to s with the Galois key of g */
ss_status ss_rotate(ss_ctx* ctx, const ss_ct* a, int32_t g, ss_ct* out, ss_stream stream);
/* total over all slots into every slot (SUM, Section 5.2) */
ss_status ss_rotate_sum(ss_ctx* ctx, const ss_ct* a, ss_ct* out, ss_stream stream);
/* out = sum_i coeffs[i] * terms[i] + cst (cst added to component 0): the
 * Paterson-Stockmeyer inner step (Theorem 2) in one pass. Every term must
 * share count, level and t_exp; |coeffs[i]|, |cst| < the smallest prime. */
ss_status ss_linear_combination(ss_ctx* ctx, const ss_ct* terms, const int64_t* coeffs, int32_t nterms, int64_t cst,
                                ss_ct* out, ss_stream stream);
/* Several combinations of the same terms in one pass, as Paterson-Stockmeyer
 * forms its leaves from one set of baby steps (Theorem 2): for k < nout,
 * outs[k] = sum_i coeffs[k*nterms + i] * terms[i]. 1 <= nterms, nout <= 16;
 * every term shares count, level and t_exp; |coeffs| < the smallest prime.
 * Each term is read once for all outputs; each output equals the
 * corresponding ss_linear_combination (with cst 0) word for word. */
ss_status ss_linear_combinations(ss_ctx* ctx, const ss_ct* terms, int32_t nterms, const int64_t* coeffs,
                                 int32_t nout, ss_ct* outs, ss_stream stream);
/* DivideByP (Section 4.2): times p^-1 mod Q, t_exp - 1 */
ss_status ss_divide_by_p(ss_ctx* ctx, const ss_ct* a, ss_ct* out, ss_stream stream);

/* ---- space switching ---- */
/* G_{p,e}(x) (Lemma 3) evaluated as x*H(x^2) by Paterson-Stockmeyer (Theorem 2) */
ss_status ss_eval_g(ss_ctx* ctx, const ss_ct* x, int32_t e, ss_ct* out, ss_stream stream);
/* Algorithm 3: digits[i] (i < r) receive the balanced base-p digits at t = p */
ss_status ss_reduce_to_digits(ss_ctx* ctx, const ss_ct* a, ss_ct* digits, ss_stream stream);
/* Algorithm 4: out = [centred(a - b) < 0] at t = p; b may have count 1 (broadcast) */
ss_status ss_compare_lt(ss_ctx* ctx, const ss_ct* a, const ss_ct* b, ss_ct* out, ss_stream stream);
/* Section 4.3 predicates of a against b, out at t = p (1 where it holds, else 0):
 *   LT  [centred(a - b) < 0]  (Algorithm 4)     LE  1 - GT
 *   GT  LT(b, a)                                GE  1 - LT
 *   EQ  prod_i F_EQ(d_i) over the digits d_i of a - b, F_EQ(x) = 1 - x^(p-1)
 *   NEQ 1 - EQ
 * centred() maps Z_{p^r} to [-(p^r-1)/2, (p^r-1)/2]. Either operand may have
 * count 1 (broadcast against the other). */
typedef enum { SS_PRED_LT = 0, SS_PRED_LE = 1, SS_PRED_GT = 2, SS_PRED_GE = 3, SS_PRED_EQ = 4, SS_PRED_NEQ = 5 } ss_predicate;
ss_status ss_compare(ss_ctx* ctx, int32_t pred, const ss_ct* a, const ss_ct* b, ss_ct* out, ss_stream stream);
/* Section 4.4: t <- p^r, out = G_{p,r}(in) */
ss_status ss_raise_modulus(ss_ctx* ctx, const ss_ct* in, ss_ct* out, ss_stream stream);
/* compare-then-SUM query (Section 1, Fig. 1; Section 5.2): one ciphertext whose
 * every slot holds sum over rows of A*B*[C1 < C2] mod p^r. A, B, C1 have the
 * same count; C2 has that count or 1 (an encrypted threshold). */
ss_status ss_query_sum_where_lt(ss_ctx* ctx, const ss_ct* A, const ss_ct* B, const ss_ct* C1, const ss_ct* C2,
                                ss_ct* out, ss_stream stream);
/* Conjunctive WHERE (Section 4.3 predicates joined by AND; the paper's
 * database workload filters on several columns): one ciphertext whose every
 * slot holds sum over rows of A*B*prod_k [x_k pred_k y_k] mod p^r. The
 * conditions' indicators are multiplied at t = p in order and raised once.
 * Every x_k has A's count; y_k has that count or 1. conds is a host array of
 * n_conds >= 1 entries; the ciphertexts it points to are device-resident. */
typedef struct {
  int32_t pred; /* ss_predicate */
  int32_t pad;
  const ss_ct* x;
  const ss_ct* y;
} ss_cond;
ss_status ss_query_sum_where(ss_ctx* ctx, const ss_ct* A, const ss_ct* B, const ss_cond* conds, int32_t n_conds,
                             ss_ct* out, ss_stream stream);
/* Same query with every input in HOST memory: copies the four columns to the
 * device, runs the query and copies the result ciphertext back to host_out
 * (uint64[2][out_level][N]); writes its level and t_exp. Synchronous. */
ss_status ss_query_sum_where_lt_host(ss_ctx* ctx, const uint64_t* A, const uint64_t* B, const uint64_t* C1,
                                     const uint64_t* C2, int32_t count, int32_t count2, int32_t level,
                                     uint64_t* host_out, int32_t* out_level, int32_t* out_t_exp,
                                     ss_stream stream);
/* ---- batched form ----
 * Many ciphertext pairs of mixed ring dimension (one context per parameter
 * set) and level: each pair is multiplied (tensor, relinearisation, one prime
 * dropped; the BGV multiplication of Section 2.1) into *prod and, when
 * `reduce` is set and the remaining levels allow it, reduced to its r digits
 * (Algorithm 3) into digits[0..r-1]. Items are grouped by (context, level);
 * each group is joined into one batch, split into chunks over several streams,
 * and the whole run can be captured once as a CUDA graph and replayed. The
 * results do not depend on the chunking, stream count or NTT tile. */
typedef struct {
  int32_t ctx;      /* index into the context array */
  int32_t reduce;   /* 1: also run Algorithm 3 on the product */
  ss_ct a, b;       /* count 1 each, same level, t = p^r */
  ss_ct* prod;      /* receives the product (count 1, capacity >= level - 1) */
  ss_ct* digits;    /* r outputs when reduce is set, else NULL */
} ss_batch_item;
typedef struct ss_batch ss_batch;
/* Groups the items (copies of the descriptors are kept; the caller keeps the
 * data and the output descriptors alive). Items whose reduction does not fit
 * in their remaining levels have it skipped and counted. */
ss_status ss_batch_create(ss_ctx* const* ctxs, int32_t nctx, const ss_batch_item* items, int32_t n, ss_batch** out);
/* chunk: ciphertexts per pass; nstreams: 1..8 streams, each issuing its own
 * launches, or 0: merged lanes (each chunk a host thread with its own stream;
 * the transforms of all lanes, of rings N >= 8192, run together as one
 * persistent launch per phase over all their tiles); ntt_tile_log: 11 or 12
 * (words per transform tile). Kernel timing does not cover merged lanes. */
ss_status ss_batch_config(ss_batch* b, int32_t chunk, int32_t nstreams, int32_t ntt_tile_log);
ss_status ss_batch_get_config(const ss_batch* b, int32_t* chunk, int32_t* nstreams, int32_t* ntt_tile_log,
                              int32_t* groups, int32_t* skipped);
/* Autotuner: times the run for chunk in {8, 32, 64} x streams in {1, 3, 0 (merged lanes)} x tile in
 * {2^11, 2^12} words on this work list and keeps the fastest setting. Synchronous. */
ss_status ss_batch_tune(ss_batch* b, ss_stream stream, int32_t* best_chunk, int32_t* best_streams,
                        int32_t* best_tile_log);
/* Captures the whole run (current setting) as one CUDA graph on `stream` (not the legacy stream). */
ss_status ss_batch_capture(ss_batch* b, ss_stream stream);
/* Runs the batch: replays the captured graph if there is one, else launches eagerly. */
ss_status ss_batch_run(ss_batch* b, ss_stream stream);
void ss_batch_destroy(ss_batch* b);

/* ---- served form: request loop with continuous batching ----
 * A server owns `workers` host threads, each with its own CUDA stream. A free
 * worker takes the oldest pending query plus every other pending query of the
 * same level and plaintext modulus that fits the HBM budget (at most
 * max_merge in all), runs them as one batch and splits the results, so
 * queries that arrive while others run are admitted as soon as a worker and
 * memory free up and their work overlaps on the device. Every result equals
 * the same query run alone (ss_query_sum_where_lt). hbm_budget = 0 takes 80 %
 * of the free device memory. Kernel timing and tracing must be off while a
 * server runs. */
typedef struct ss_server ss_server;
ss_status ss_server_create(ss_ctx* ctx, int32_t workers, int32_t max_merge, uint64_t hbm_budget, ss_server** out);
/* A server over several contexts (parameter sets of any ring dimension and
 * plaintext modulus, keys of all of them resident): queries name their
 * context at submission (ss_server_submit_to); only queries of the same
 * context, level and plaintext modulus are merged into one pass, and one HBM
 * budget admits the queries of all contexts. ss_server_create(ctx, ...) is
 * the one-context case. */
ss_status ss_server_create_multi(ss_ctx* const* ctxs, int32_t nctx, int32_t workers, int32_t max_merge,
                                 uint64_t hbm_budget, ss_server** out);
/* Queues one query on device-resident columns (as ss_query_sum_where_lt);
 * `out` (count 1, capacity >= the columns' level) receives the result. The
 * caller keeps the columns and *out alive until ss_server_wait returns. */
ss_status ss_server_submit(ss_server* s, const ss_ct* A, const ss_ct* B, const ss_ct* C1, const ss_ct* C2,
                           ss_ct* out, uint64_t* ticket);
/* The same for the server's context number ctx_index (0-based, in the order
 * given to ss_server_create_multi); ss_server_submit is ctx_index 0. A chain
 * too short for the query is rejected here with SS_ERR_NOISE. */
ss_status ss_server_submit_to(ss_server* s, int32_t ctx_index, const ss_ct* A, const ss_ct* B, const ss_ct* C1,
                              const ss_ct* C2, ss_ct* out, uint64_t* ticket);
/* Waits at most timeout_ms (negative: no bound) for a ticket: SS_ERR_TIMEOUT if
 * it is still running; otherwise releases it and returns its status with the
 * time it waited for admission and the time its batch ran (host clock). */
ss_status ss_server_wait(ss_server* s, uint64_t ticket, int32_t timeout_ms, double* queued_ms, double* run_ms);
ss_status ss_server_stats(ss_server* s, uint64_t* completed, uint64_t* batches, uint64_t* peak_inflight_bytes);
/* Finishes every queued query, then stops the workers. */
void ss_server_destroy(ss_server* s);

/* Number of levels a query consumes on inputs at `level` (the plan's depth);
 * SS_ERR_NOISE if the chain is too short. */
ss_status ss_query_depth(ss_ctx* ctx, int32_t level, int32_t* out_level);
/* Device bytes a query over n_ct ciphertexts per column at `level` holds at
 * its peak: the estimate the served form admits queries by. */
ss_status ss_query_bytes(const ss_ctx* ctx, int32_t n_ct, int32_t level, uint64_t* bytes);
/* Coefficients of G_{p,e} used by ss_eval_g, the reduction, the raising and
 * the queries: 0 = the canonical table (Newton interpolation, centred mod p^e,
 * the default); 1 = the lattice-reduced representative (Section 4.2, after
 * Geelen et al.): the odd polynomial equal to G_{p,e} on all of Z_{p^e} with
 * the least sum of |centred coefficients|, found exactly for e = 2, 3 (other e:
 * the canonical table). Smaller coefficients grow the noise less. */
ss_status ss_set_g_table(ss_ctx* ctx, int32_t mode);
/* Ciphertexts the query evaluates together per pass (memory/throughput knob). */
ss_status ss_set_batch(ss_ctx* ctx, int32_t batch);

/* ---- raw transform (for kernel-level measurement) ---- */
/* In-place NTT over the context's ring of `npoly` consecutive limbs of N words; limb k uses
 * data prime (first_prime + k % nprimes). Input words must be residues below
 * their prime (the forward transform keeps lazy sums below 40q, which needs
 * inputs below 4q); outputs are residues below the prime, forward in the
 * evaluation order given above. */
ss_status ss_ntt_forward(ss_ctx* ctx, uint64_t* data, int32_t npoly, int32_t first_prime, int32_t nprimes,
                         ss_stream stream);
ss_status ss_ntt_inverse(ss_ctx* ctx, uint64_t* data, int32_t npoly, int32_t first_prime, int32_t nprimes,
                         ss_stream stream);

/* ---- evaluation trace (schedule check) ---- */
ss_status ss_trace(ss_ctx* ctx, int32_t on);
int32_t ss_trace_get(ss_ctx* ctx, char* buf, int32_t len);

/* ---- kernel timing (measurement) ----
 * When on, every library kernel launch is bracketed by CUDA events recorded on
 * the stream it is launched on, and attributed to a class with the bytes the
 * operation must move (its algorithmic traffic, not the measured traffic):
 *   0 NTT (both phases of one transform; 16 N bytes per limb)
 *   1 base conversion   2 key-switch inner product   3 tensor product
 *   4 subtract-and-scale (ModDown / modulus-switch epilogue)
 *   5 automorphism   6 other elementwise   7 sampling.
 * ss_kernel_stats synchronises on the recorded events and returns, for one
 * class, the launches, total milliseconds and total algorithmic bytes since
 * timing was switched on. Switching it on resets the counters. */
ss_status ss_kernel_timing(ss_ctx* ctx, int32_t on);
ss_status ss_kernel_stats(ss_ctx* ctx, int32_t cls, uint64_t* launches, double* ms, double* bytes);

/* Shoup products (one 64-bit modular product by a precomputed constant each)
 * that the timed transform launches performed since kernel timing was switched
 * on: per polynomial N/2 log2 N forward, less N/2 when the base conversion
 * that wrote the input already applied the first stage's twiddle (ring
 * X^N + 1), and N/2 (log2 N + 1) inverse for N > 4096 (the last stage also
 * scales the sums by N^-1), N/2 (log2 N + 2) for N <= 4096 (N^-1 on every
 * word), N/2 (log2 N - 1) when the last stage's factors are left to the base
 * conversion that reads the output (ring X^N + 1, N > 4096). The
 * split stages of the m = 3N and 5N/2 rings count as the radix-2 stages they
 * replace. Written to *products; SS_ERR_PARAM on a null argument. The paper has
 * no counterpart of this call; it is measurement (the work term of the
 * transform's integer-multiply roofline). */
ss_status ss_ntt_products(ss_ctx* ctx, double* products);

/* Per-stage breakdown of the query while kernel timing is on, mirroring the
 * runtime breakdown of LT in Section 5 (reduction, comparison, aggregation,
 * modulus raising) plus the rest of the query:
 *   0 reduction (d = a - b and Algorithm 3)   1 comparison (F_LT, F_EQ per digit)
 *   2 aggregation (the fold of Algorithm 4)   3 modulus raising (Section 4.4)
 *   4 masked product ind * (a * b)            5 SUM (batch total and rotate-and-sum)
 * Returns how many times the stage ran and its total milliseconds (CUDA events
 * on the query's stream) since timing was switched on. The paper has no
 * counterpart of this call; it is measurement. */
ss_status ss_stage_stats(ss_ctx* ctx, int32_t stage, uint64_t* count, double* ms);

/* Integer-pipe ceilings on the current device, for the roofline of the
 * ALU-bound kernels (measurement; the paper has no counterpart). kind 0:
 * 32-bit multiply-adds per second; kind 1: forward butterflies per second
 * (Harvey's form: one conditional subtraction, one 64-bit Shoup product, the
 * lazy add and subtract; residues held in registers, no memory traffic);
 * kind 2: 32 x 32 -> 64-bit widening multiply-adds per second (the partial
 * products of a 64-bit modular product).
 * iters in [1, 2^20] sets the loop length (every thread of one full wave of
 * CTAs runs 8 operations per iteration). Allocates and frees a small buffer;
 * synchronises its own stream. */
ss_status ss_alu_probe(int32_t kind, int32_t iters, double* per_second);

/* Count of kernels this library has launched since context creation. */
uint64_t ss_launch_count(const ss_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SS_H */
