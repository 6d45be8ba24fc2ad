/*
 * lbm_oracle.h -- plain, slow FP64 CPU oracle for the D2Q9 BGK
 * stream-and-collide update of Tomczak, "Data-Oriented Language
 * Implementation of Lattice-Boltzmann Method for Dense and Sparse
 * Geometries" (arXiv 2108.13241).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this code.  It shares no code,
 * header, table or helper with the CUDA library; the CUDA library never
 * loads it.
 *
 * Conventions (all arrays row-major, x fastest):
 *   node n = y*nx + x;  distributions A[i*N + n], N = nx*ny, i = 0..8;
 *   per-node vector fields V[c*N + n], c = 0 (x) / 1 (y).
 * Lattice (Sec. 2.2, Fig. "D2Q9 lattice arrangement"):
 *   0 rest, 1 (+1,0), 2 (0,+1), 3 (-1,0), 4 (0,-1),
 *   5 (+1,+1), 6 (-1,+1), 7 (-1,-1), 8 (+1,-1).
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H
#include <stdint.h>

/* Geometry and physics of one run.  A side is a half-way bounce-back wall
 * moving at (wall_ux[s], wall_uy[s]) unless its axis is periodic or it is
 * open.  Sides: 0 west (x<0), 1 east (x>=nx), 2 south (y<0), 3 north (y>=ny).
 *
 * Open sides (the paper's constant-velocity and constant-pressure boundary
 * conditions after Zou & He, Sec. 3): the nodes of the outermost row or
 * column are boundary nodes; the links that would pull from beyond the side
 * get the values for which the node has the side's velocity (open_kind
 * ORC_OPEN_VELOCITY: open_ux, open_uy) or density (ORC_OPEN_PRESSURE:
 * open_rho, zero tangential velocity).  open_val[s], when not NULL, gives the
 * values node by node along the side instead: velocity [2][len] (all u_x,
 * then all u_y), pressure [len]; len = ny on west/east (index y), nx on
 * south/north (index x). */
#define ORC_OPEN_NONE 0
#define ORC_OPEN_VELOCITY 1
#define ORC_OPEN_PRESSURE 2
typedef struct {
    int nx, ny;
    int periodic_x, periodic_y;
    double wall_ux[4], wall_uy[4];
    double tau;          /* BGK relaxation time, omega = 1/tau        */
    double fx, fy;       /* uniform body-force density (no field given) */
    double rho_w;        /* wall density in the moving-wall term       */
    int open_kind[4];
    double open_ux[4], open_uy[4], open_rho[4];
    const double *open_val[4];
    /* Collision operator: 0 = BGK (Eq. 4); > 0 = the two-relaxation-time
     * (TRT) operator, whose odd parts relax at this rate while the even
     * parts relax at 1/tau (step_body.inc). */
    double omega_m;
} orc_params;

/* Per-node link mask value of a node that takes no part in the update. */
#define ORC_SOLID 0xFF

void orc_lattice(int cx[9], int cy[9], double w[9], int opp[9]);
int  orc_link_mask(const orc_params *p, const uint8_t *solid, uint8_t *mask);
int  orc_tile_map(const orc_params *p, const uint8_t *mask, int32_t *tile_id,
                  int32_t *nbr, int *ntiles);
void orc_init_equilibrium(const orc_params *p, const uint8_t *mask,
                          const double *rho, const double *ux, const double *uy,
                          double *A);
void orc_step(const orc_params *p, const uint8_t *mask, const double *force,
              const double *A, double *B);
void orc_run(const orc_params *p, const uint8_t *mask, const double *force,
             double *A, double *B, int nsteps);
void orc_macros(const orc_params *p, const uint8_t *mask, const double *force,
                const double *A, double *rho, double *ux, double *uy);
void orc_adjoint_step(const orc_params *p, const uint8_t *mask,
                      const double *force, const double *A,
                      const double *lam_next, double *lam, double *grad_force);
void orc_macros_adjoint(const orc_params *p, const uint8_t *mask,
                        const double *force, const double *A,
                        const double *g_rho, const double *g_ux,
                        const double *g_uy, double *lam, double *grad_force);
/* complex-step twin of orc_step (same body, complex arithmetic); arrays
 * hold interleaved (re, im) pairs. */
void orc_step_cs(const orc_params *p, const uint8_t *mask, const double *force,
                 const double *A, double *B);
int  orc_num_threads(void);
void orc_set_threads(int n);

#endif
