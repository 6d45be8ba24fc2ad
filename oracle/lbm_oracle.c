/*
 * lbm_oracle.c -- plain, slow FP64 CPU oracle for the D2Q9 BGK
 * stream-and-collide update (Tomczak, arXiv 2108.13241).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * benchmark's CPU-baseline leg to check and time the CUDA library.  It is
 * independent of the CUDA path: no shared code, headers or tables.
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (see oracle.py).
 *
 * What each function follows:
 *   orc_link_mask        node-type field + bitmask of present neighbours
 *                        (Sec. 3, boundary-condition paragraph), half-way
 *                        bounce-back reading;
 *   orc_tile_map         16x16 tiles, only tiles holding a fluid node stored
 *                        ("pointer tile" layout, Sec. 4.2.2), with a table of
 *                        the 9 neighbour tiles;
 *   orc_init_equilibrium Algorithm 1, initialisation (f = f^eq(rho, v));
 *   orc_step / orc_run   Algorithm 1, one/many fused pull steps + swap
 *                        (body in step_body.inc);
 *   orc_macros           Eq. 2 on the gathered f', F/2 shift of the
 *                        Guo forcing;
 *   open sides           constant velocity / constant pressure (Sec. 3,
 *                        after Zou & He 1997), in the gather of the step
 *                        and the macros (orc_open_side, step_body.inc);
 *   orc_adjoint_step     discrete adjoint (transpose of the linearisation) of
 *                        orc_step, open sides included (their rules are
 *                        affine in f', orc_open_transpose);
 *   orc_macros_adjoint   transpose of orc_macros.
 * Pins: tests/test_oracle_*.py (closed forms, invariants, Poiseuille,
 * Taylor-Green decay, brute-force tables, dot-product and complex-step checks).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include "lbm_oracle.h"
#include "lattice.inc"

#define ORC_REAL double
#define ORC_STEP_NAME orc_step
#include "step_body.inc"
#undef ORC_REAL
#undef ORC_STEP_NAME

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the later parallel loops (timing of the oracle only). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

void orc_lattice(int cx[9], int cy[9], double w[9], int opp[9])
{
    for (int i = 0; i < 9; ++i) {
        cx[i] = CX[i];
        cy[i] = CY[i];
        w[i] = W[i];
        opp[i] = OPP[i];
    }
}

/*
 * Link mask: for a fluid node, bit (i-1) is set iff its link i pulls from a
 * solid node or from beyond a wall (so it bounces back).  Solid nodes get
 * ORC_SOLID.  A fluid node all 8 of whose links bounce has no link to any
 * other node; its mask is all ones, the same value, so it counts as solid.
 * Returns the number of fluid nodes, or -1 on invalid input.
 */
int orc_link_mask(const orc_params *p, const uint8_t *solid, uint8_t *mask)
{
    if (p->nx < 1 || p->ny < 1) return -1;
    int nfluid = 0;
    for (int y = 0; y < p->ny; ++y) {
        for (int x = 0; x < p->nx; ++x) {
            const long n = (long)y * p->nx + x;
            if (solid && solid[n]) { mask[n] = ORC_SOLID; continue; }
            unsigned bits = 0;
            for (int i = 1; i < 9; ++i) {
                long s = 0;
                int side = 0;
                int inside = orc_source(p, x, y, i, &s, &side);
                if (!inside || (solid && solid[s])) bits |= 1u << (i - 1);
            }
            mask[n] = (uint8_t)bits;
            if (bits != ORC_SOLID) ++nfluid;
        }
    }
    return nfluid;
}

/*
 * Tile map: tile (tx, ty) covers nodes [16tx, 16tx+16) x [16ty, 16ty+16).  It
 * is kept iff it holds a fluid node; kept tiles are numbered 0, 1, ... in
 * row-major tile order (ty outer, tx inner); tile_id[ty*ntx + tx] is that
 * number or -1.  nbr[9*t + i] is the number of the tile at (tx + c_ix,
 * ty + c_iy), wrapped on periodic axes, -1 beyond a wall or when absent.
 * A periodic axis must be a multiple of 16 long.  Returns 0, or -1.
 */
int orc_tile_map(const orc_params *p, const uint8_t *mask, int32_t *tile_id,
                 int32_t *nbr, int *ntiles)
{
    const int T = 16;
    if ((p->periodic_x && p->nx % T) || (p->periodic_y && p->ny % T)) return -1;
    const int ntx = (p->nx + T - 1) / T, nty = (p->ny + T - 1) / T;
    int count = 0;
    for (int ty = 0; ty < nty; ++ty) {
        for (int tx = 0; tx < ntx; ++tx) {
            int keep = 0;
            for (int y = ty * T; y < ty * T + T && y < p->ny; ++y)
                for (int x = tx * T; x < tx * T + T && x < p->nx; ++x)
                    if (mask[(long)y * p->nx + x] != ORC_SOLID) keep = 1;
            tile_id[ty * ntx + tx] = keep ? count++ : -1;
        }
    }
    for (int ty = 0; ty < nty; ++ty) {
        for (int tx = 0; tx < ntx; ++tx) {
            const int t = tile_id[ty * ntx + tx];
            if (t < 0) continue;
            for (int i = 0; i < 9; ++i) {
                int ux = tx + CX[i], uy = ty + CY[i];
                int id = -1;
                int ok = 1;
                if (ux < 0 || ux >= ntx) {
                    if (p->periodic_x) ux = (ux + ntx) % ntx; else ok = 0;
                }
                if (uy < 0 || uy >= nty) {
                    if (p->periodic_y) uy = (uy + nty) % nty; else ok = 0;
                }
                if (ok) id = tile_id[uy * ntx + ux];
                nbr[9 * t + i] = id;
            }
        }
    }
    *ntiles = count;
    return 0;
}

/* Algorithm 1, initialisation: A_i = f^eq_i(rho, u) (Eq. 6) at fluid
 * nodes; solid nodes hold w_i.  NULL fields mean rho = 1, u = 0. */
void orc_init_equilibrium(const orc_params *p, const uint8_t *mask,
                          const double *rho, const double *ux, const double *uy,
                          double *A)
{
    const long N = (long)p->nx * p->ny;
    for (long n = 0; n < N; ++n) {
        const double r = (rho && mask[n] != ORC_SOLID) ? rho[n] : 1.0;
        const double vx = (ux && mask[n] != ORC_SOLID) ? ux[n] : 0.0;
        const double vy = (uy && mask[n] != ORC_SOLID) ? uy[n] : 0.0;
        const double uu = vx * vx + vy * vy;
        for (int i = 0; i < 9; ++i) {
            const double cu = CX[i] * vx + CY[i] * vy;
            A[i * N + n] = W[i] * r * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
        }
    }
}

/* Algorithm 1, time loop: nsteps fused steps with the swap.  The final state
 * is left in A. */
void orc_run(const orc_params *p, const uint8_t *mask, const double *force,
             double *A, double *B, int nsteps)
{
    const long N = (long)p->nx * p->ny;
    double *a = A, *b = B;
    for (int t = 0; t < nsteps; ++t) {
        orc_step(p, mask, force, a, b);
        double *tmp = a; a = b; b = tmp;
    }
    if (a != A) memcpy(A, a, sizeof(double) * 9 * N);
}

static int orc_has_open(const orc_params *p)
{
    for (int s = 0; s < 4; ++s)
        if (p->open_kind[s] != ORC_OPEN_NONE) return 1;
    return 0;
}

/* Transpose of the open-side rules at node (x, y), applied to g: the rules
 * are affine in the gathered f' (orc_open_side), so their linear part is
 * M[:, j] = R(e_j) - R(0); g becomes M^T g.  Identity away from open sides. */
static void orc_open_transpose(const orc_params *p, int x, int y, double g[9])
{
    double r0[9] = {0}, M[9][9];
    for (int s = 0; s < 4; ++s)
        if (p->open_kind[s] != ORC_OPEN_NONE) orc_open_side(p, s, x, y, r0);
    for (int j = 0; j < 9; ++j) {
        double e[9] = {0};
        e[j] = 1.0;
        for (int s = 0; s < 4; ++s)
            if (p->open_kind[s] != ORC_OPEN_NONE) orc_open_side(p, s, x, y, e);
        for (int i = 0; i < 9; ++i) M[i][j] = e[i] - r0[i];
    }
    double out[9];
    for (int j = 0; j < 9; ++j) {
        out[j] = 0.0;
        for (int i = 0; i < 9; ++i) out[j] += M[i][j] * g[i];
    }
    for (int j = 0; j < 9; ++j) g[j] = out[j];
}

/* Shared by the macros and the adjoints: the gather of step 1 at node (x, y),
 * also reporting for each link whether it bounced and, if not, its source. */
static void orc_gather(const orc_params *p, const uint8_t *mask, const double *A,
                       int x, int y, double f[9], int bounced[9], long src[9])
{
    const long N = (long)p->nx * p->ny;
    const long n = (long)y * p->nx + x;
    f[0] = A[n];
    bounced[0] = 0;
    src[0] = n;
    for (int i = 1; i < 9; ++i) {
        long s = 0;
        int side = 0;
        int inside = orc_source(p, x, y, i, &s, &side);
        bounced[i] = (mask[n] >> (i - 1)) & 1;
        src[i] = s;
        if (!bounced[i])
            f[i] = A[i * N + s];
        else
            f[i] = A[OPP[i] * N + n] + orc_wall_term(p, i, !inside, side);
    }
}

/* Eq. 2 applied to the gathered f' of the next step, with the F/2
 * velocity shift of the Guo forcing.  Solid nodes report rho = 1, u = 0. */
void orc_macros(const orc_params *p, const uint8_t *mask, const double *force,
                const double *A, double *rho, double *ux, double *uy)
{
    const long N = (long)p->nx * p->ny;
    for (int y = 0; y < p->ny; ++y) {
        for (int x = 0; x < p->nx; ++x) {
            const long n = (long)y * p->nx + x;
            if (mask[n] == ORC_SOLID) { rho[n] = 1.0; ux[n] = 0.0; uy[n] = 0.0; continue; }
            double f[9];
            int bounced[9];
            long src[9];
            orc_gather(p, mask, A, x, y, f, bounced, src);
            for (int s = 0; s < 4; ++s)
                if (p->open_kind[s] != ORC_OPEN_NONE) orc_open_side(p, s, x, y, f);
            double r = 0, mx = 0, my = 0;
            for (int i = 0; i < 9; ++i) {
                r += f[i];
                mx += CX[i] * f[i];
                my += CY[i] * f[i];
            }
            const double Fx = force ? force[n] : p->fx;
            const double Fy = force ? force[N + n] : p->fy;
            rho[n] = r;
            ux[n] = (mx + 0.5 * Fx) / r;
            uy[n] = (my + 0.5 * Fy) / r;
        }
    }
}

/*
 * Discrete adjoint of orc_step.  Input lam_next = dL/dB (B = A_{t+1});
 * output lam = dL/dA_t (overwritten); grad_force += dL/dF (per-node field F,
 * or the uniform force when force == NULL).
 *
 * At a fluid node, with f' the gathered values, rho, u, f^eq as in the step:
 *   du/df'_j = (v_j - u)/rho,  drho/df'_j = 1,  du/dF = 1/(2 rho);
 *   df^eq_i/du = w_i rho (3 v_i + 9 (v_i.u) v_i - 3 u),
 *   df^eq_i/drho (u fixed) = f^eq_i / rho,
 *   dS_i/du = (1 - omega/2) w_i (-3 F + 9 (v_i.F) v_i),
 *   dS_i/dF (u fixed) = (1 - omega/2) w_i (3 (v_i - u) + 9 (v_i.u) v_i).
 * With V = sum_i lam_i (omega df^eq_i/du + dS_i/du) and
 *      a = omega sum_i lam_i f^eq_i / rho:
 *   dL/df'_j = (1 - omega) lam_j + a + (v_j - u).V / rho,
 *   dL/dF   += V / (2 rho) + sum_i lam_i dS_i/dF.
 * The gather is then transposed: a link j that pulled A_j(s) adds dL/df'_j to
 * lam_j(s); a bounced link adds it to lam_opp(j)(x) (the moving-wall term is
 * a constant and carries no gradient).
 */
void orc_adjoint_step(const orc_params *p, const uint8_t *mask,
                      const double *force, const double *A,
                      const double *lam_next, double *lam, double *grad_force)
{
    const long N = (long)p->nx * p->ny;
    const double omega = 1.0 / p->tau;
    const double k = 1.0 - 0.5 * omega;
    const int open = orc_has_open(p);
    memset(lam, 0, sizeof(double) * 9 * N);
    for (int y = 0; y < p->ny; ++y) {
        for (int x = 0; x < p->nx; ++x) {
            const long n = (long)y * p->nx + x;
            if (mask[n] == ORC_SOLID) continue;
            double f[9];
            int bounced[9];
            long src[9];
            orc_gather(p, mask, A, x, y, f, bounced, src);
            for (int s = 0; s < 4; ++s)
                if (p->open_kind[s] != ORC_OPEN_NONE) orc_open_side(p, s, x, y, f);
            double rho = 0, mx = 0, my = 0;
            for (int i = 0; i < 9; ++i) {
                rho += f[i];
                mx += CX[i] * f[i];
                my += CY[i] * f[i];
            }
            const double Fx = force ? force[n] : p->fx;
            const double Fy = force ? force[N + n] : p->fy;
            const double ux = (mx + 0.5 * Fx) / rho;
            const double uy = (my + 0.5 * Fy) / rho;
            const double uu = ux * ux + uy * uy;
            double Vx = 0, Vy = 0, a = 0, gFx = 0, gFy = 0;
            for (int i = 0; i < 9; ++i) {
                const double li = lam_next[i * N + n];
                const double cu = CX[i] * ux + CY[i] * uy;
                const double cF = CX[i] * Fx + CY[i] * Fy;
                const double feq = W[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
                const double dfeq_x = W[i] * rho * (3.0 * CX[i] + 9.0 * cu * CX[i] - 3.0 * ux);
                const double dfeq_y = W[i] * rho * (3.0 * CY[i] + 9.0 * cu * CY[i] - 3.0 * uy);
                const double dS_x = k * W[i] * (-3.0 * Fx + 9.0 * cF * CX[i]);
                const double dS_y = k * W[i] * (-3.0 * Fy + 9.0 * cF * CY[i]);
                Vx += li * (omega * dfeq_x + dS_x);
                Vy += li * (omega * dfeq_y + dS_y);
                a += omega * li * feq / rho;
                gFx += li * k * W[i] * (3.0 * (CX[i] - ux) + 9.0 * cu * CX[i]);
                gFy += li * k * W[i] * (3.0 * (CY[i] - uy) + 9.0 * cu * CY[i]);
            }
            double g[9];
            for (int j = 0; j < 9; ++j) {
                const double lj = lam_next[j * N + n];
                g[j] = (1.0 - omega) * lj + a + ((CX[j] - ux) * Vx + (CY[j] - uy) * Vy) / rho;
            }
            if (open) orc_open_transpose(p, x, y, g);
            for (int j = 0; j < 9; ++j) {
                if (!bounced[j])
                    lam[j * N + src[j]] += g[j];
                else
                    lam[OPP[j] * N + n] += g[j];
            }
            if (grad_force) {
                const long gn = force ? n : 0;
                const long gN = force ? N : 1;
                grad_force[gn] += Vx / (2.0 * rho) + gFx;
                grad_force[gN + gn] += Vy / (2.0 * rho) + gFy;
            }
        }
    }
}

/*
 * Transpose of orc_macros.  Given dL/drho, dL/du at every node (solid nodes
 * ignored), adds dL/dA to lam and dL/dF to grad_force:
 *   dL/df'_j = dL/drho + (v_j - u).(dL/du) / rho,  dL/dF += (dL/du)/(2 rho),
 * then the same transpose of the gather as in orc_adjoint_step.
 */
void orc_macros_adjoint(const orc_params *p, const uint8_t *mask,
                        const double *force, const double *A,
                        const double *g_rho, const double *g_ux,
                        const double *g_uy, double *lam, double *grad_force)
{
    const long N = (long)p->nx * p->ny;
    const int open = orc_has_open(p);
    for (int y = 0; y < p->ny; ++y) {
        for (int x = 0; x < p->nx; ++x) {
            const long n = (long)y * p->nx + x;
            if (mask[n] == ORC_SOLID) continue;
            double f[9];
            int bounced[9];
            long src[9];
            orc_gather(p, mask, A, x, y, f, bounced, src);
            for (int s = 0; s < 4; ++s)
                if (p->open_kind[s] != ORC_OPEN_NONE) orc_open_side(p, s, x, y, f);
            double rho = 0, mx = 0, my = 0;
            for (int i = 0; i < 9; ++i) {
                rho += f[i];
                mx += CX[i] * f[i];
                my += CY[i] * f[i];
            }
            const double Fx = force ? force[n] : p->fx;
            const double Fy = force ? force[N + n] : p->fy;
            const double ux = (mx + 0.5 * Fx) / rho;
            const double uy = (my + 0.5 * Fy) / rho;
            const double gr = g_rho ? g_rho[n] : 0.0;
            const double gx = g_ux ? g_ux[n] : 0.0;
            const double gy = g_uy ? g_uy[n] : 0.0;
            double g[9];
            for (int j = 0; j < 9; ++j) g[j] = gr + ((CX[j] - ux) * gx + (CY[j] - uy) * gy) / rho;
            if (open) orc_open_transpose(p, x, y, g);
            for (int j = 0; j < 9; ++j) {
                if (!bounced[j])
                    lam[j * N + src[j]] += g[j];
                else
                    lam[OPP[j] * N + n] += g[j];
            }
            if (grad_force) {
                const long gn = force ? n : 0;
                const long gN = force ? N : 1;
                grad_force[gn] += gx / (2.0 * rho);
                grad_force[gN + gn] += gy / (2.0 * rho);
            }
        }
    }
}
