/*
 * lbm3_oracle.c -- plain, slow FP64 CPU oracle for the D3Q19 BGK
 * stream-and-collide update (Algorithm 1 of arXiv 2108.13241 in three
 * dimensions; the paper names three-dimensional geometries as future work,
 * Sec. 5).
 *
 * TEST INFRASTRUCTURE ONLY (see lbm3_oracle.h).  Build: part of
 * liblbm_oracle.so (oracle.py).
 *
 * What each function follows:
 *   orc3_link_mask        the per-node field of present neighbours (Sec. 3),
 *                         half-way bounce-back on solid nodes and on the
 *                         faces of non-periodic axes;
 *   orc3_init_equilibrium Algorithm 1, initialisation (f = f^eq(rho, v));
 *   orc3_step / orc3_run  Algorithm 1: pull gather f'_i = f_i(x - c_i),
 *                         moments (Eq. 2 with the Guo F/2 shift), equilibrium
 *                         (Eq. 6 with the D3Q19 velocities and weights), BGK
 *                         relaxation (Eq. 3-5) plus the Guo source, store,
 *                         swap;
 *   orc3_macros           Eq. 2 on the gathered f' with the F/2 shift.
 * Pins: tests/test_oracle3_pins.py.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "lbm3_oracle.h"

/* D3Q19 velocities: rest, the six axis links, the twelve edge diagonals,
 * opposite links adjacent (2k-1, 2k). */
static const int C3[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

/* Weights of the D3Q19 equilibrium: 1/3 rest, 1/18 axis, 1/36 diagonal. */
static double w3(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }
static int opp3(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

void orc3_lattice(int c[19][3], double w[19], int opp[19])
{
    for (int i = 0; i < 19; ++i) {
        for (int a = 0; a < 3; ++a) c[i][a] = C3[i][a];
        w[i] = w3(i);
        opp[i] = opp3(i);
    }
}

/* Source of link i of node (x, y, z): x - c_i, periodic axes wrapped.
 * Returns 1 and the node index in *s, or 0 when it lies beyond a wall. */
static int src3(const orc3_params *p, int x, int y, int z, int i, long *s)
{
    int q[3] = {x - C3[i][0], y - C3[i][1], z - C3[i][2]};
    const int n[3] = {p->nx, p->ny, p->nz};
    const int per[3] = {p->periodic_x, p->periodic_y, p->periodic_z};
    for (int a = 0; a < 3; ++a) {
        if (q[a] < 0 || q[a] >= n[a]) {
            if (!per[a]) return 0;
            q[a] = (q[a] + n[a]) % n[a];
        }
    }
    *s = ((long)q[2] * p->ny + q[1]) * p->nx + q[0];
    return 1;
}

/*
 * Link mask: for a fluid node, bit (i-1) (i = 1..18) is set iff its link i
 * pulls from a solid node or from beyond a wall face, so that it bounces
 * back.  Solid nodes get ORC3_SOLID.  Returns the number of fluid nodes.
 */
long orc3_link_mask(const orc3_params *p, const uint8_t *solid, uint32_t *mask)
{
    long nf = 0;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                const long n = ((long)z * p->ny + y) * p->nx + x;
                if (solid && solid[n]) { mask[n] = ORC3_SOLID; continue; }
                uint32_t m = 0;
                for (int i = 1; i < 19; ++i) {
                    long s;
                    if (!src3(p, x, y, z, i, &s) || (solid && solid[s])) m |= 1u << (i - 1);
                }
                mask[n] = m;
                ++nf;
            }
    return nf;
}

/* f^eq_i(rho, u) of Eq. 6 with the D3Q19 velocities and weights. */
static double feq3(int i, double rho, const double u[3])
{
    const double cu = C3[i][0] * u[0] + C3[i][1] * u[1] + C3[i][2] * u[2];
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return w3(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

/* A = f^eq(rho, u) at fluid nodes (rho = 1, u = 0 where NULL); solid nodes
 * hold w_i. */
void orc3_init_equilibrium(const orc3_params *p, const uint32_t *mask, const double *rho,
                           const double *u, double *A)
{
    const long N = (long)p->nx * p->ny * p->nz;
    for (long n = 0; n < N; ++n) {
        const double r = rho ? rho[n] : 1.0;
        double v[3] = {0.0, 0.0, 0.0};
        if (u)
            for (int a = 0; a < 3; ++a) v[a] = u[a * N + n];
        for (int i = 0; i < 19; ++i) A[i * N + n] = mask[n] == ORC3_SOLID ? w3(i) : feq3(i, r, v);
    }
}

/* Algorithm 1's gather for node n at (x, y, z): f'_i = A_i(x - c_i), or, for
 * a bounced link, the node's own post-collision value of the opposite link
 * (half-way bounce-back, stationary walls and obstacles). */
static void gather3(const orc3_params *p, const uint32_t *mask, const double *A, int x, int y, int z, long n,
                    double f[19])
{
    const long N = (long)p->nx * p->ny * p->nz;
    f[0] = A[n];
    for (int i = 1; i < 19; ++i) {
        long s;
        if (mask[n] & (1u << (i - 1))) f[i] = A[opp3(i) * N + n];
        else {
            src3(p, x, y, z, i, &s);
            f[i] = A[i * N + s];
        }
    }
}

/* Moments of Eq. 2 with the Guo shift: rho = sum f', u = (sum c f' + F/2)/rho. */
static void moments3(const orc3_params *p, const double f[19], double *rho, double u[3])
{
    const double F[3] = {p->fx, p->fy, p->fz};
    double r = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 19; ++i) {
        r += f[i];
        for (int a = 0; a < 3; ++a) m[a] += C3[i][a] * f[i];
    }
    *rho = r;
    for (int a = 0; a < 3; ++a) u[a] = (m[a] + 0.5 * F[a]) / r;
}

/* One step A -> B: for every fluid node, gather, moments, BGK relaxation
 * toward f^eq (omega = 1/tau, Eq. 5) plus the Guo source
 * S_i = (1 - omega/2) w_i [3 (c_i - u) + 9 (c_i . u) c_i] . F.
 * Solid nodes are copied (they hold w_i and are never read). */
void orc3_step(const orc3_params *p, const uint32_t *mask, const double *A, double *B)
{
    const long N = (long)p->nx * p->ny * p->nz;
    const double om = 1.0 / p->tau;
    const double F[3] = {p->fx, p->fy, p->fz};
    /* the planes are independent: OpenMP splits them over threads, each
     * node's arithmetic is the same whatever the thread count */
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                const long n = ((long)z * p->ny + y) * p->nx + x;
                if (mask[n] == ORC3_SOLID) {
                    for (int i = 0; i < 19; ++i) B[i * N + n] = A[i * N + n];
                    continue;
                }
                double f[19], rho, u[3];
                gather3(p, mask, A, x, y, z, n, f);
                moments3(p, f, &rho, u);
                const double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
                for (int i = 0; i < 19; ++i) {
                    const double cu = C3[i][0] * u[0] + C3[i][1] * u[1] + C3[i][2] * u[2];
                    const double cF = C3[i][0] * F[0] + C3[i][1] * F[1] + C3[i][2] * F[2];
                    const double S = (1.0 - 0.5 * om) * w3(i) * (3.0 * (cF - uF) + 9.0 * cu * cF);
                    B[i * N + n] = f[i] - om * (f[i] - feq3(i, rho, u)) + S;
                }
            }
}

void orc3_run(const orc3_params *p, const uint32_t *mask, double *A, double *B, int nsteps)
{
    const long N = (long)p->nx * p->ny * p->nz;
    for (int t = 0; t < nsteps; ++t) {
        orc3_step(p, mask, A, B);
        memcpy(A, B, sizeof(double) * 19 * (size_t)N);
    }
}

/* rho and u at the current time: the gather of the next step without the
 * collision (Eq. 2, F/2 shift); 0 at solid nodes. */
void orc3_macros(const orc3_params *p, const uint32_t *mask, const double *A, double *rho, double *u)
{
    const long N = (long)p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                const long n = ((long)z * p->ny + y) * p->nx + x;
                if (mask[n] == ORC3_SOLID) {
                    rho[n] = 0.0;
                    for (int a = 0; a < 3; ++a) u[a * N + n] = 0.0;
                    continue;
                }
                double f[19], r, v[3];
                gather3(p, mask, A, x, y, z, n, f);
                moments3(p, f, &r, v);
                rho[n] = r;
                for (int a = 0; a < 3; ++a) u[a * N + n] = v[a];
            }
}
