/*
 * lbm_oracle_cs.c -- complex-step twin of orc_step.  The step body of
 * step_body.inc is compiled with complex arithmetic; evaluating it at
 * A + i*h*v gives the directional derivative J v = Im(B)/h to rounding, with
 * no cancellation.  The tests use it to pin the oracle's adjoint by the
 * identity <J v, w> = <v, J^T w>.
 * TEST INFRASTRUCTURE ONLY (see lbm_oracle.h).
 */
#include <complex.h>
#include <string.h>
#include "lbm_oracle.h"
#include "lattice.inc"

#define ORC_REAL double _Complex
#define ORC_STEP_NAME orc_step_cs_impl
static void orc_step_cs_impl(const orc_params *p, const uint8_t *mask,
                             const ORC_REAL *force, const ORC_REAL *A, ORC_REAL *B);
#include "step_body.inc"

void orc_step_cs(const orc_params *p, const uint8_t *mask, const double *force,
                 const double *A, double *B)
{
    orc_step_cs_impl(p, mask, (const ORC_REAL *)force, (const ORC_REAL *)A,
                     (ORC_REAL *)B);
}
