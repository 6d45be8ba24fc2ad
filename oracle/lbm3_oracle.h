/*
 * lbm3_oracle.h -- plain, slow FP64 CPU oracle for a three-dimensional
 * (D3Q19) BGK stream-and-collide update: Algorithm 1 of Tomczak (arXiv
 * 2108.13241) carried to three dimensions, the extension the paper names as
 * future work (Sec. 5).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite and the CPU-baseline leg of
 * the benchmark may load this code.  It shares no code, header, table or
 * helper with the CUDA library; the CUDA library never loads it.
 *
 * Conventions (row-major, x fastest):
 *   node n = (z*ny + y)*nx + x;  distributions A[i*N + n], N = nx*ny*nz,
 *   i = 0..18;  vector fields V[c*N + n], c = 0 (x), 1 (y), 2 (z).
 * Lattice: 0 rest; 1 (+1,0,0) 2 (-1,0,0) 3 (0,+1,0) 4 (0,-1,0) 5 (0,0,+1)
 *   6 (0,0,-1); 7 (+1,+1,0) 8 (-1,-1,0) 9 (+1,-1,0) 10 (-1,+1,0)
 *   11 (+1,0,+1) 12 (-1,0,-1) 13 (+1,0,-1) 14 (-1,0,+1)
 *   15 (0,+1,+1) 16 (0,-1,-1) 17 (0,+1,-1) 18 (0,-1,+1):
 *   links 2k-1 and 2k are opposite (k = 1..9).
 */
#ifndef LBM3_ORACLE_H
#define LBM3_ORACLE_H
#include <stdint.h>

/* Geometry and physics of one three-dimensional run.  An axis that is not
 * periodic has a stationary half-way bounce-back wall on both faces. */
typedef struct {
    int nx, ny, nz;
    int periodic_x, periodic_y, periodic_z;
    double tau;          /* BGK relaxation time, omega = 1/tau */
    double fx, fy, fz;   /* uniform body-force density          */
} orc3_params;

/* Link-mask value of a node that takes no part in the update. */
#define ORC3_SOLID 0xFFFFFFFFu

void orc3_lattice(int c[19][3], double w[19], int opp[19]);
long orc3_link_mask(const orc3_params *p, const uint8_t *solid, uint32_t *mask);
void orc3_init_equilibrium(const orc3_params *p, const uint32_t *mask, const double *rho,
                           const double *u, double *A);
void orc3_step(const orc3_params *p, const uint32_t *mask, const double *A, double *B);
void orc3_run(const orc3_params *p, const uint32_t *mask, double *A, double *B, int nsteps);
void orc3_macros(const orc3_params *p, const uint32_t *mask, const double *A, double *rho, double *u);

#endif
