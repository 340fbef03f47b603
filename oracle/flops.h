/*
 * flops.h -- the oracle's flop counter (TEST INFRASTRUCTURE, part of the
 * oracle).  Compiled in with -DORC_COUNT_FLOPS, a separate build used to
 * measure the method's arithmetic per stage and iteration; the default
 * build expands every macro to nothing.
 *
 * What is counted: the floating-point operations of the method's steps, one
 * per add, multiply, divide, square root, sine or cosine.  Products with
 * structurally zero Jacobian entries are not counted, and the symmetric
 * local model is counted on its lower triangle.  Work that only this plain
 * implementation repeats is not counted: the constant row scales, dense
 * zero fills, Jacobians evaluated for merit values, and the rows the step
 * re-evaluates at the point the measures have just taken.
 */
#ifndef COMET_ORACLE_FLOPS_H
#define COMET_ORACLE_FLOPS_H
#include <stdint.h>

#ifdef ORC_COUNT_FLOPS
extern __thread uint64_t orc_g_flops;
/* what a row evaluation counts: values and Jacobians */
extern __thread int orc_g_rows_on, orc_g_jac_on;
#define FLOPS(n) (orc_g_flops += (uint64_t)(n))
#define FLOPS_ROWS(n) (orc_g_flops += orc_g_rows_on ? (uint64_t)(n) : 0)
#define FLOPS_JAC(n) (orc_g_flops += orc_g_jac_on ? (uint64_t)(n) : 0)
#define COUNT_ROWS(r, j) (orc_g_rows_on = (r), orc_g_jac_on = (j))
#else
#define FLOPS(n) ((void)0)
#define FLOPS_ROWS(n) ((void)0)
#define FLOPS_JAC(n) ((void)0)
#define COUNT_ROWS(r, j) ((void)0)
#endif

#endif
