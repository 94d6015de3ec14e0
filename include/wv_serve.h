/*
 * wv_serve.h -- serving loop for range and single-prime queries (C ABI).
 *
 * The paper's search runs a fixed plan over ranges (Sec. 3 "Results",
 * Sec. 5).  A server here accepts queries as they arrive -- "all primes of
 * [lo, hi)" or "one prime p" -- and answers each with B_{p-3} mod p and
 * E_{p-3} mod p for its primes (Sec. 3, Sec. 5) plus its zero residues.
 *
 * Continuous batching: a worker thread keeps every admitted query's primes,
 * plan and per-tile partial products resident on the device, and runs the
 * accumulation in bounded "epochs", each one persistent launch over tiles
 * drawn from all active queries (smallest remaining work first).  Queries
 * that arrive while others run are admitted as slots and memory free up and
 * join the next epoch; a query is finalised and its memory released as soon
 * as its last tile is done.  Results are identical to computing each query
 * alone.
 */
#ifndef WV_SERVE_H
#define WV_SERVE_H

#include "wv.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wv_server_s *wv_server;

typedef struct {
  size_t mem_budget;     /* device bytes for admitted queries (0: 64 GiB)           */
  uint32_t max_active;   /* queries admitted at once (0: 256)                        */
  double epoch_terms;    /* summed terms per epoch, bounds its duration (0: 4e10)    */
  int device;            /* CUDA device (-1: current device at creation)              */
  int epoch_form;        /* epoch launch: 0 or 1 one persistent launch over both
                            arithmetic paths (default), 2 one warp per tile
                            (non-persistent, both paths), 3 one persistent launch
                            per arithmetic path                                       */
  int epoch_block;       /* threads per block of an epoch launch, 32..256 (0: 32)     */
  int piece_log2;        /* longest lane chain (piece of a sum) of a query's plan:
                            2^piece_log2 terms, 12..24 (0: 17).  Longer pieces pay
                            fewer per-piece set-ups; shorter ones bound how long one
                            lane can hold an epoch                                    */
  int reserved[4];
} wv_server_config;

typedef struct {
  uint64_t id;
  int kind;              /* 0 = range, 1 = single prime                              */
  int state;             /* 0 pending, 1 active, 2 done, 3 failed, 4 cancelled       */
  wv_status status;      /* final status once done/failed                            */
  uint64_t n_primes;     /* primes in the query (an upper bound until it is admitted) */
  uint64_t n_hits;       /* primes with a zero residue                                */
  double t_submit, t_admit, t_done; /* seconds since the server was created            */
} wv_query_info;

/* Create a server and start its worker thread.  `cfg` may be NULL (defaults). */
wv_status wv_server_create(const wv_server_config *cfg, wv_server *out);

/* Queue a query; returns its id.  Range: all primes of [lo, hi), hi <= 2^37.
 * Prime: one odd p, 5 <= p < 2^37 (primality is the caller's contract). */
wv_status wv_server_submit_range(wv_server s, uint64_t lo, uint64_t hi, uint64_t *id);
wv_status wv_server_submit_prime(wv_server s, uint64_t p, uint64_t *id);

/* Wait up to timeout_s seconds (< 0: forever) for query `id`; fills `info`.
 * Returns WV_ETIMEOUT if it is not finished in time. */
wv_status wv_server_wait(wv_server s, uint64_t id, double timeout_s, wv_query_info *info);

/* Non-blocking state of query `id`. */
wv_status wv_server_query(wv_server s, uint64_t id, wv_query_info *info);

/* Host copies of a finished query's primes and residues (ascending p); up to
 * `cap` entries each (any pointer may be NULL); *n receives the count. */
wv_status wv_server_result(wv_server s, uint64_t id, uint64_t *h_primes, uint64_t *h_res_b,
                           uint64_t *h_res_e, size_t cap, size_t *n);

/* Forget a finished query (frees its host copies). */
wv_status wv_server_release(wv_server s, uint64_t id);

/* Counters: epochs run, tiles done, device bytes in use now, peak active queries. */
wv_status wv_server_stats(wv_server s, uint64_t *epochs, uint64_t *tiles, size_t *bytes_in_use,
                          uint32_t *peak_active);

/* Stop the worker (pending and active queries are cancelled) and free everything. */
wv_status wv_server_destroy(wv_server s);

#ifdef __cplusplus
}
#endif
#endif /* WV_SERVE_H */
