/*
 * wv_batch.h -- many residue requests in one launch sequence (C ABI).
 *
 * The paper processes 81920 primes per GPU launch, one prime per thread, and
 * notes that the launch then waits for its slowest thread (Sec. 3, "Method
 * for primes p > 6*10^10", third improvement).  A batch here concatenates
 * the prime lists of many requests of very uneven per-prime cost, groups the
 * primes by the congruence pair that suits their size (as the paper switches
 * congruences with p, Sec. 3; the bands of wv_congruence_for_range), plans
 * each group with the primes ordered by size, and runs persistent
 * work-stealing accumulation launches, largest primes first, so no launch
 * waits on one long prime.  The groups run on forked streams, so the tail of
 * one group's launch overlaps the next.  The whole sequence is captured once
 * into a CUDA graph and replayed by wv_batch_run.
 *
 * Residues are the same as wv_residues_pm3 gives for each request alone (any
 * valid congruence gives the same residue).
 */
#ifndef WV_BATCH_H
#define WV_BATCH_H

#include "wv.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  const uint64_t *d_primes; /* device, n primes (5 <= p < 2^37), caller-owned  */
  size_t n;
  uint64_t *d_out_b;        /* device, n entries for B_{p-3} mod p, or NULL     */
  uint64_t *d_out_e;        /* device, n entries for E_{p-3} mod p, or NULL     */
} wv_request;

typedef struct wv_batch_s *wv_batch;

/*
 * Build a batch over k requests (host array `reqs`; the device buffers it
 * points to must stay valid for the life of the batch).  Waits for the
 * device, reads the requests' primes once to group them by size, allocates
 * the batch's device buffers, captures the launch sequence into a CUDA graph
 * and instantiates it.  SYNCHRONOUS.  `opt` (may be NULL) selects the launch
 * shape; a congruence it names is used for every prime of that kind (one
 * group), otherwise each prime gets the pair wv_congruence_for_range picks
 * for [p, p + 1).  Both residues are computed.  Later replays read the
 * buffers again: new values keep the grouping made here, which changes the
 * speed but never the residues.
 * Errors: WV_EINVAL for no requests, more than 65535, a NULL prime buffer or
 * a request of 2^48 or more primes.
 */
wv_status wv_batch_create(const wv_request *reqs, size_t k, const wv_options *opt, wv_batch *out);

/* Replay the captured launch sequence on `stream` (asynchronous).  Inputs are
 * read from the request buffers at replay time. */
wv_status wv_batch_run(wv_batch b, wv_stream stream);

/* Requests, total primes and graph node count of a batch (any pointer may be NULL). */
wv_status wv_batch_info(wv_batch b, size_t *n_requests, size_t *n_primes, size_t *graph_nodes);

/* Number of congruence groups (each one plan and one set of launches). */
wv_status wv_batch_groups(wv_batch b, size_t *n_groups);

/* Synchronise the device and free the batch. */
wv_status wv_batch_destroy(wv_batch b);

#ifdef __cplusplus
}
#endif
#endif /* WV_BATCH_H */
