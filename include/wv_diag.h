/*
 * wv_diag.h -- hardware diagnostics used to derive the integer-pipe roofline.
 *
 * The residue kernels are bound by 32-bit integer multiplies (the IMAD pipe);
 * the paper has no counterpart to these calls.  They run short loops of
 * independent instructions of one kind on every SM and report the measured
 * issue rate, so the peak used for the roofline is checked on the device
 * rather than assumed.
 */
#ifndef WV_DIAG_H
#define WV_DIAG_H

#include <stdint.h>

#include "wv.h"

#ifdef __cplusplus
extern "C" {
#endif

#define WV_DIAG_IMAD 0      /* mad.lo.u32                                   */
#define WV_DIAG_IMAD_HI 1   /* mul.hi.s32                                   */
#define WV_DIAG_IMAD_WIDE 2 /* mul.wide.u32                                 */
#define WV_DIAG_IADD 3      /* add.u32                                      */
#define WV_DIAG_IMNMX 4     /* min.u32                                      */
#define WV_DIAG_TERM_B 5    /* one term of the p < 2^30 Bernoulli hot loop  */
#define WV_DIAG_TERM_E 6    /* one term of the p < 2^30 Euler hot loop      */
#define WV_DIAG_TERM_B_WIDE 7 /* the same, wide-product formulation         */
#define WV_DIAG_TERM_E_WIDE 8 /* the same, wide-product formulation         */
#define WV_DIAG_IMAD_WIDE_S 9 /* mul.wide.s32                               */
#define WV_DIAG_IMAD_HI_U 10  /* mul.hi.u32                                 */
#define WV_DIAG_MONT_MUL 11   /* one signed Montgomery product (4 instr.)   */
#define WV_DIAG_SHOUP_MUL 12  /* one Shoup product (3 instr.)               */
#define WV_DIAG_TERM_E_SHOUP 13 /* Euler term with Shoup products           */

/*
 * Runs diagnostic `op` on the current device with one full wave of resident
 * blocks and returns, per SM per clock (SM cycles from clock64):
 *   *per_clk = warp-lane operations (instructions x 32 lanes, or terms for
 *              the TERM ops) completed per SM per clock.
 * `iters` is the loop count per thread (>= 1024 recommended).  Synchronous.
 */
wv_status wv_diag_throughput(int op, int iters, double *per_clk);

#ifdef __cplusplus
}
#endif
#endif /* WV_DIAG_H */
