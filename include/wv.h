/*
 * wv.h -- C ABI of the GB300 Wolstenholme / Vandiver residue library.
 *
 * For primes p the library computes B_{p-3} mod p and E_{p-3} mod p
 * (Bernoulli numbers from z/(e^z-1), Euler numbers from sec z; Sec. 1) with
 * the computation-friendly congruences of Sec. 3 (eqns 3.1-3.7) and Sec. 5
 * (eqns 5.1-5.6), and flags the primes where a residue is 0: p is a
 * Wolstenholme prime iff p | B_{p-3} (Sec. 1, eqn 1.2 and the remark after
 * it) and a Vandiver prime iff p | E_{p-3} (Sec. 1).
 *
 * Conventions for every entry point:
 *  - Pointers named d_* are DEVICE pointers (global memory of the current
 *    CUDA device), owned and allocated by the caller.  Pointers named h_* or
 *    plain out-parameters (n_out, count, ...) are HOST pointers.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on `stream` unless stated otherwise;
 *    library-internal scratch is allocated stream-ordered on `stream`.
 *  - Every call returns a wv_status.  Nothing aborts, throws or traps; on
 *    failure wv_last_error() returns a message for the calling thread.
 *  - Residues are the canonical representatives in [0, p), as uint64.
 *  - Supported primes: 5 <= p < 2^37 (WV_P_MAX).  Primality is the caller's
 *    contract for d_primes; an odd p outside the range, or an even p, gives
 *    WV_RESIDUE_INVALID in its output slot (the call itself still succeeds).
 *    wv_options.check_primes makes the calls verify it (a composite's slot
 *    is then WV_RESIDUE_INVALID too); wv_is_prime is the same test on the host.
 *  - The Euler numbers use the sec convention (E_2 = +1), as the paper does.
 */
#ifndef WV_H
#define WV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int wv_status;
#define WV_OK 0
#define WV_EINVAL 1      /* bad argument */
#define WV_ENOMEM 2      /* device or host allocation failed */
#define WV_ERANGE 3      /* output capacity too small; the full count is still reported */
#define WV_ECUDA 4       /* a CUDA runtime call failed */
#define WV_ETIMEOUT 5    /* a bounded wait expired */
#define WV_ECANCELLED 6  /* the work was cancelled */
#define WV_EBUSY 7       /* the object is busy (e.g. a server queue is full) */

#define WV_P_MAX (1ull << 37)
#define WV_RESIDUE_INVALID UINT64_MAX

/* hit kinds (wv_hit.kind bit mask) */
#define WV_KIND_BERNOULLI 1u /* B_{p-3} = 0 mod p: Wolstenholme prime */
#define WV_KIND_EULER 2u     /* E_{p-3} = 0 mod p: Vandiver prime     */

typedef void *wv_stream; /* a cudaStream_t */

/* Library version string (static storage). */
const char *wv_version(void);

/* Message for the last failing call made on this host thread ("" if none). */
const char *wv_last_error(void);

/* 1 if n is a prime, else 0; host only, no device work.  Deterministic
 * Miller-Rabin with the bases 2..17, exact for n < 2^37 (Jaeschke 1993);
 * n >= 2^37 returns -1 (outside the supported range).  The same test that
 * wv_options.check_primes runs on the device. */
int wv_is_prime(uint64_t n);

/* ---------------------------------------------------------------------- */
/* a1: prime enumeration (the paper enumerates primes over intervals with */
/* a CPU sieve, Sec. 3 "Results" and Sec. 5; here a segmented GPU sieve)  */
/* ---------------------------------------------------------------------- */

/*
 * All primes in [lo, hi), ascending, written to d_out[0 .. min(count,cap)).
 *  lo, hi : 0 <= lo <= hi <= WV_P_MAX.
 *  d_out  : device array of `cap` uint64 (may be NULL if cap == 0).
 *  n_out  : host; receives the number of primes in [lo, hi).
 * SYNCHRONOUS: returns after the count is known (stream synchronised).
 * Returns WV_ERANGE if count > cap (the first cap primes are written and
 * *n_out holds the full count), WV_EINVAL on a bad range.
 */
wv_status wv_sieve(uint64_t lo, uint64_t hi, uint64_t *d_out, size_t cap,
                   size_t *n_out, wv_stream stream);

/* Number of primes in [lo, hi) without materialising them.  SYNCHRONOUS. */
wv_status wv_sieve_count(uint64_t lo, uint64_t hi, uint64_t *count, wv_stream stream);

/* ---------------------------------------------------------------------- */
/* a2-a6: residues                                                         */
/* ---------------------------------------------------------------------- */

/*
 * d_out[i] = B_{p_i - 3} mod p_i for the n primes d_primes[0..n).
 * Follows Sec. 3: B_{p-3} from eqn 3.7 (BB30) for p >= 11 by default, or
 * any congruence of the library (wv_options.cong_b), each sum
 * S_{p-4}(x,y) = sum_{xp<s<yp} s^-3 evaluated as c1/c0 of
 * prod (z + s^3) (the polynomial trick and eqn 3.12), partial products
 * combined with eqn 3.14, one modular inverse per prime; p = 5, 7 from the
 * definition.  d_primes and d_out: device arrays of n uint64 (may alias
 * only if d_out == d_primes).  Asynchronous.
 */
wv_status wv_bernoulli_pm3(const uint64_t *d_primes, size_t n, uint64_t *d_out,
                           wv_stream stream);

/*
 * d_out[i] = E_{p_i - 3} mod p_i (sec convention).  Follows Sec. 5: eqn 5.6
 * (EE33) for p >= 11 by default, or any congruence of the library, with
 * S_{p-3}(x,y) = sum s^-2 evaluated through
 * prod (z + s^2) (the remark after eqn 5.6).  Same layout and behaviour as
 * wv_bernoulli_pm3.  Asynchronous.
 */
wv_status wv_euler_pm3(const uint64_t *d_primes, size_t n, uint64_t *d_out,
                       wv_stream stream);

/*
 * Both residues in one launch sequence (one persistent accumulation launch
 * covers the sums of both congruences).  Either output may be NULL.
 * Asynchronous.
 */
wv_status wv_residues_pm3(const uint64_t *d_primes, size_t n, uint64_t *d_out_b,
                          uint64_t *d_out_e, wv_stream stream);

/*
 * wv_residues_pm3 for callers that cannot allocate device memory during a
 * call: hosts whose device memory is entirely owned by their own pool
 * allocator (so a cudaMalloc would fail or fragment it), and real-time loops
 * that cannot afford the device-wide synchronisation cudaMalloc/cudaFree
 * imply.  The paper has no counterpart to this call.
 *
 * It returns the same residues as wv_residues_pm3 but allocates nothing: all
 * scratch lives in one fixed device array inside the library, about 12 MB,
 * that every GPU which loads the library keeps until the process exits.  It
 * always sums BB30 (eqn 3.7) and EE33 (eqn 5.6), for which that array is
 * sized, with a fixed launch shape (at most 8 tiles per sum, hot-loop
 * formulation 9, grids sized by occupancy); options and the automatic
 * tile shape for short lists do not apply, so a short list may run slower
 * than through wv_residues_pm3.  Limits and behaviour:
 *  - n <= 1024 primes per call; larger n returns WV_ERANGE (split the list).
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current, uploads the two
 *    congruences into fixed device tables and waits for the device once;
 *    make that first call before any stream capture.
 *  - Every call uses the same array and leaves its contents behind; the call
 *    itself clears what must start at zero.  Calls that overlap on the GPU
 *    (different streams, or different host threads, without ordering between
 *    them) race on the array and must not be issued.
 *  - d_primes, d_out_b, d_out_e are device arrays of n uint64 owned by the
 *    caller; either output may be NULL.  Asynchronous on `stream`.
 */
wv_status wv_residues_pm3_noalloc(const uint64_t *d_primes, size_t n, uint64_t *d_out_b,
                                  uint64_t *d_out_e, wv_stream stream);

/*
 * General index near the top (Sec. 2 and Sec. 4 with t = 2k - 1, resp.
 * t = p - 1 - 2k, and p - 1 - t small): for every prime p of d_primes,
 *   d_out_b[i] = B_{p-e_b} mod p   (e_b odd, 3 <= e_b <= 15; 0 skips B),
 *   d_out_e[i] = E_{p-1-e_e} mod p (e_e even, 2 <= e_e <= 16; 0 skips E),
 * canonical in [0, p).  Every sum is then S_t = sum s^-e: B by Vandiver's
 * congruence (eqn 2.5, cost p/10) and E by the three-sum congruence of
 * eqn 4.2 (cost 3p/16), with their coefficients d^t and left-hand constants
 * evaluated per prime; the sums by eqn 3.12 with terms s^e from difference
 * tables of degree e.  e_b = 3, e_e = 2 reproduce wv_residues_pm3.
 * A slot is WV_RESIDUE_INVALID where p < 11, p < e + 3, p is not a valid
 * prime, or the left-hand constant vanishes mod p (C_k(2,5,6) for B).
 * Device arrays of n uint64, caller-owned; asynchronous on `stream`.
 * Errors: WV_EINVAL for an exponent outside the ranges above.
 */
wv_status wv_residues_general(const uint64_t *d_primes, size_t n, uint32_t e_b, uint32_t e_e,
                              uint64_t *d_out_b, uint64_t *d_out_e, wv_stream stream);

/* Options for the *_ex entry points.  Zero-initialise, then set fields;
 * a zero / negative field means "library default". */
typedef struct {
  int cong_b;       /* congruence id (wv_congruence_info) for B; <0: the default (BB30,
                       or by range in the range-aware calls: wv_congruence_for_range) */
  int cong_e;       /* congruence id for E; <0: as for B (EE33 / by range) */
  int block;        /* accumulation block size (threads): 32..256, multiple of 32;
                       default 256.  Smaller blocks release their registers warp by
                       warp at the end of a launch and round occupancy differently */
  int ilp;          /* independent accumulator chains per thread for p < 2^31: 1, 2 or 4
                       (4 only with arith 9, 12..18, 21 or 23; default 1).  The grouped 64-bit forms
                       (arith >= 9) run one chain per thread; the single-term 64-bit
                       form takes this value too */
  int tile_terms;   /* target terms per warp tile (default 2^20) */
  int max_tiles;    /* maximum tiles per (prime, sum) (default 8).  With neither set, a
                       call with few primes gets more and shorter tiles (up to 64 per
                       sum) so that one launch still holds ~1e5 tiles */
  int blocks_per_sm;/* persistent grid = SMs x this */
  int arith;        /* hot-loop formulation (default 50).  Every value gives the same
                       residues; the others exist for ablation.  32-bit path (p < 2^31;
                       signed words below 2^30, unsigned from 2^30 to 2^31):
                       1, 2, 4 single terms (1: shared t p^-1; 2: one wide product and
                       REDC; 4: 2 with the additions as ALU three-input adds); 9
                       grouped terms (2 cubes / 3 squares per eqn 3.14 step, REDC folded
                       into wide multiply-adds); 25..28 form 9 with none, 4, 6 or all of a
                       group's difference-table additions as ALU-only three-input adds
                       (9 itself: 4 of a Bernoulli group's 9 and 2 of an Euler group's
                       10); 29, 30, 31 groups of 3 cubes, of 4 squares, or both; 39
                       groups of 4 cubes / 5 squares; lane chains only (39 with warp
                       tiles): 40, 41, 44 groups of 5 cubes / 6 squares, 4 / 6, 4 / 7;
                       45, 46, 47 the u form (G0 = u^e from a table of u = prod (s+i),
                       K + e(K-1) table additions per group instead of 2eK - e) with
                       groups of 8 / 10, 6 / 8, 10 / 12; 51, 52 form 45 with 12 / 10 and
                       4 / 4 of its table additions ALU-only; 48, 49, 50 (default) per
                       warp 45 on pieces of at least uform_min31 terms and 41 on shorter
                       ones.  64-bit
                       path (2^31 <= p < 2^37): 1, 2, 4 the single-term 64-bit kernel;
                       12..18 and 21 other group sizes, shrink intervals and register
                       budgets; 32..36 the default with a quarter to all of its 64-bit
                       table additions as PTX carry chains (32: plain; 33..36: with a
                       three-input high word); 37 the default with the earlier, longer
                       shrink of its difference tables; 38 the default with its
                       per-chain set-up unrolled; 42, 43 (lane chains only) the default
                       with Euler groups of 10 or 11 squares; 49 (lane chains only) the u
                       form, groups of 12 cubes / 16 squares; 50 (default; lane chains only)
                       per warp 49 on pieces of at least uform_min64 terms and the grouped form
                       below; every other value the grouped form (8 cubes / 12 squares).  23: the paper's own arithmetic on both
                       paths (plain residues, eqn 3.15 split products, remainders from
                       a double-precision quotient, single terms).  Other values:
                       WV_EINVAL */
  int check_primes; /* nonzero: the planner also verifies that every input is a prime
                       (deterministic Miller-Rabin, bases 2..17, exact below 2^37); a
                       composite gets WV_RESIDUE_INVALID in its slot like an input
                       outside the supported range.  Default 0: primality stays the
                       caller's contract and a composite's slot is unspecified */
  int tiling;       /* work unit of the accumulation.  0 (default) or 2: lane chains --
                       every lane of a warp sums its own piece of one (prime, sum), the
                       pieces sorted by length so that a warp's lanes finish together;
                       used with the grouped formulations 50 (default), 31 and 39..49
                       and ILP 1 or 2, warp tiles otherwise.  1: warp tiles -- the 32
                       lanes of a warp split one piece and merge by shuffles (the earlier
                       work unit, kept for ablation).  Other values: WV_EINVAL */
  int uform_min31;  /* forms 48..50, lane chains: shortest piece (terms) that the 32-bit
                       kernel sums in the u form (default 3072) */
  int uform_min64;  /* form 50, lane chains: the same for the 64-bit kernel (default 32768) */
  int reserved[4];
} wv_options;

/* wv_residues_pm3 with explicit congruence choice and launch shape.
 * Any valid congruence gives the identical residue (the choice only changes
 * the cost, Sec. 3 and Sec. 5).  Asynchronous. */
wv_status wv_residues_ex(const uint64_t *d_primes, size_t n, uint64_t *d_out_b,
                         uint64_t *d_out_e, const wv_options *opt, wv_stream stream);

/* ---------------------------------------------------------------------- */
/* a7: search (sieve + both residues + flag/compact)                      */
/* ---------------------------------------------------------------------- */

typedef struct {
  uint64_t p;
  uint32_t kind; /* WV_KIND_BERNOULLI | WV_KIND_EULER */
  uint32_t pad;
} wv_hit;

/*
 * All primes p in [lo, hi) (5 <= p) with B_{p-3} = 0 or E_{p-3} = 0 mod p
 * (Sec. 3 and Sec. 5 searches), ascending by p, written to
 * d_hits[0 .. min(count, cap)).  n_hits (host) receives the count.
 * SYNCHRONOUS.  WV_ERANGE if count > cap.
 */
wv_status wv_search(uint64_t lo, uint64_t hi, wv_hit *d_hits, size_t cap,
                    size_t *n_hits, wv_stream stream);

/*
 * Search with residues: like wv_search, and also writes, for every prime of
 * [lo, hi) in ascending order, p to d_primes[i], B_{p-3} mod p to d_res_b[i]
 * and E_{p-3} mod p to d_res_e[i] (any of the three may be NULL).  Those
 * arrays hold `cap_primes` entries; *n_primes receives the prime count.
 * `near` > 0 also reports primes whose symmetric residue <r>_p in
 * (-p/2, p/2] satisfies |<r>_p| < near (the near-miss tables of Sec. 3 and
 * Sec. 5); near-miss entries carry kind bit 2 (B) / bit 3 (E).
 * SYNCHRONOUS.
 */
#define WV_KIND_NEAR_B 4u
#define WV_KIND_NEAR_E 8u
wv_status wv_search_ex(uint64_t lo, uint64_t hi, uint64_t near, wv_hit *d_hits,
                       size_t cap, size_t *n_hits, uint64_t *d_primes,
                       uint64_t *d_res_b, uint64_t *d_res_e, size_t cap_primes,
                       size_t *n_primes, const wv_options *opt, wv_stream stream);

/*
 * Histogram mode (Sec. 3 "Results": the histogram of <B_{p-3}>_p / p over
 * 2000 equal bins, where <r>_p is the representative of r mod p in
 * (-p/2, p/2]).  For every prime p of [lo, hi) (5 <= p), with
 * u = <r>_p / p + 1/2 in (0, 1), ADDS 1 to hist[floor(u * bins)]: bin b holds
 * u in [b / bins, (b + 1) / bins) (only r = 0 lies on an edge, u = 1/2).
 * d_hist_b receives the counts of r = B_{p-3} mod p, d_hist_e those of
 * r = E_{p-3} mod p (either may be NULL, not both); each is a caller-owned
 * device array of `bins` uint64 counters, 1 <= bins <= 2^20, which the call
 * adds to (zero it first; disjoint ranges may be accumulated over calls).
 * *n_primes (may be NULL) receives the number of primes counted.
 * SYNCHRONOUS: the counts are complete on return.
 */
wv_status wv_histogram(uint64_t lo, uint64_t hi, uint32_t bins, unsigned long long *d_hist_b,
                       unsigned long long *d_hist_e, size_t *n_primes, wv_stream stream);

/* ---------------------------------------------------------------------- */
/* host-side inspection of the congruence tables (no GPU needed)           */
/* ---------------------------------------------------------------------- */

/* Number of congruences in the library: ids 0..12 are the paper's (BB1..BB30,
 * EE3..EE33, Sec. 3 and Sec. 5); the ids after them were generated from
 * BB30 and EE33 by the greedy search over Prop. 2.1 (Sec. 2, "Heuristic
 * searches"), named by their number of sums (BB249 ... EE4122). */
int wv_congruence_count(void);

/* The id of the congruence the residue calls on a device prime list use by
 * default for kind 0 (B_{p-3}) or 1 (E_{p-3}): the paper's BB30 and EE33. */
int wv_congruence_default(int kind);

/* The congruences the range-aware calls (wv_search*, wv_histogram, the
 * serving loop, the batch's per-prime grouping) use for primes of [lo, hi)
 * when the caller chose none, each kind by hi on its own:
 *   B: BB30 up to 5e6, BB249 up to 2e7, BB476 up to 5e7, BB1115 up to
 *      1.5e8, BB2244 up to 1.2e9, then BB3802;
 *   E: EE33 up to 3e6, EE200 up to 2e7, EE404 up to 5e7, EE967 up to 1.5e8,
 *      EE2004 up to 1.2e9, then EE4122
 * (the measured fastest on GB300 with the default lane chains; all give the
 * identical residues). */
void wv_congruence_for_range(uint64_t lo, uint64_t hi, int *cong_b, int *cong_e);

/* Congruence `id`: kind 0 = B_{p-3}, 1 = E_{p-3}; n_rows sums; lhs = the
 * constant on the left; name (static string).  Any out-pointer may be NULL. */
wv_status wv_congruence_info(int id, int *kind, int *n_rows, int64_t *lhs,
                             const char **name);

/* Row `row` of congruence `id`: coef * S(xn/xd, yn/yd) for a row whose
 * coefficient is a plain integer (every row of ids 0..12).  A row with a
 * coefficient sum_k c_k d_k^t returns WV_ERANGE with *coef = 0 (the interval
 * is still written): read it with wv_congruence_terms. */
wv_status wv_congruence_row(int id, int row, int64_t *coef, uint32_t *xn,
                            uint32_t *xd, uint32_t *yn, uint32_t *yd);

/* The coefficient of row `row` of congruence `id` as terms c[k] d[k]^t
 * (t = p - 4 for B_{p-3}, p - 3 for E_{p-3}, so d^t = d^-3 resp. d^-2):
 * writes up to `cap` terms, *n = their number; WV_ERANGE if n > cap. */
wv_status wv_congruence_terms(int id, int row, int64_t *c, uint64_t *d, int cap, int *n);

/* The general-index forms used by wv_residues_general (host only):
 * kind 0 = B (Vandiver, eqn 2.5), kind 1 = E (eqn 4.2).  Row `row` is
 * (sum_i c[i] d[i]^t) * S_t(xn/xd, yn/yd) with t = p - 1 - e; lhs = (a, b, c)
 * of C_k(a, b, c) for kind 0 (unused for kind 1).  wv_general_rows(kind)
 * returns the number of rows (0 for an unknown kind). */
int wv_general_rows(int kind);
wv_status wv_general_row(int kind, int row, uint32_t *xn, uint32_t *xd, uint32_t *yn,
                         uint32_t *yd, int32_t c[3], uint32_t d[3], uint32_t lhs[3]);

/* ---------------------------------------------------------------------- */
/* profiling: per-kernel CUDA-event timing on the launching stream         */
/* ---------------------------------------------------------------------- */

/* Enable (1) / disable (0) event timing of every library kernel launch. */
void wv_profile_enable(int on);
/* Clear accumulated timings and launch counts. */
void wv_profile_reset(void);
/* Synchronise pending events and fold them into the totals. */
wv_status wv_profile_collect(void);
/* Number of distinct kernels seen; then per index its name, launch count
 * and total milliseconds (totals are those folded in by wv_profile_collect;
 * launch counts are kept even when timing is disabled). */
int wv_profile_kernels(void);
wv_status wv_profile_get(int idx, const char **name, uint64_t *launches, double *total_ms);
/* Total kernel launches issued by the library since the last reset. */
uint64_t wv_profile_launches(void);

/* Algorithmic work of one residue call: the number of terms s summed for the
 * given primes (host array h_primes) under congruences cong_b / cong_e
 * (<0: defaults; pass -2 to skip that kind).  Each term costs two modular
 * multiplications (eqn 3.12).  Host only.  */
wv_status wv_count_terms(const uint64_t *h_primes, size_t n, int cong_b, int cong_e,
                         uint64_t *terms_b, uint64_t *terms_e);

#ifdef __cplusplus
}
#endif
#endif /* WV_H */
