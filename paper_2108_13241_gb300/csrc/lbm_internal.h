// lbm_internal.h -- declarations shared by the C-ABI layer (lbm_api.cu) and
// the per-precision kernel translation units (kern_*.cu).  Not public.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "lbm.h"

namespace lbm {

constexpr int TILE = 16;        // sparse tile edge (nodes)
constexpr int TILE_N = 256;     // nodes per tile
constexpr int STEP_BLOCK = 256; // threads per block of the step kernels
constexpr int AUX_BLOCK = 256;  // threads per block of the per-node kernels
constexpr int RED_BLOCKS = 608; // blocks of the reduction pass (4 x 152 SMs)
constexpr int WALL_SIDES = 5;   // W, E, S, N, and "solid obstacle" (term 0)

// Halo chunk h of the staged tiled step's stage (E stored values = 16 bytes
// of one tile row): which slot it serves, the neighbour it comes from
// (3 x 3 index dir = 3 (oy + 1) + (ox + 1)), its source row and first
// column in that tile, and where it lands around the tile core (dlx: -E or
// 16 for a column chunk, else its first column; dly: -1 or 16 for a row
// chunk, else its row).  Chunks 0 .. 3 CPR - 1: the row below (slots 2, 5,
// 6 pulling from y - 1), then the row above (4, 7, 8), the left column (1,
// 5, 8; one chunk per row), the right column (3, 6, 7), and the four
// corners (5 SW, 6 SE, 7 NE, 8 NW).  Shared by the kernel, which copies the
// chunks, and the host, which marks the ones whose source holds fluid.
struct HaloSrc {
    int dir, slot, srow, scol, dlx, dly;
};
__host__ __device__ constexpr int halo_chunks(int E) { return 6 * (TILE / E) + 6 * TILE + 4; }
__host__ __device__ inline HaloSrc halo_source(int h, int E) {
    const int CPR = TILE / E;
    HaloSrc c;
    int ox, oy;
    if (h < 3 * CPR) { // row below the tile (ly = -1)
        const int s3 = h / CPR, k = h - s3 * CPR;
        c.slot = s3 == 0 ? 2 : (s3 == 1 ? 5 : 6);
        ox = 0; oy = -1; c.srow = TILE - 1; c.scol = k * E; c.dly = -1; c.dlx = k * E;
    } else if (h < 6 * CPR) { // row above (ly = 16)
        const int hh = h - 3 * CPR, s3 = hh / CPR, k = hh - s3 * CPR;
        c.slot = s3 == 0 ? 4 : (s3 == 1 ? 7 : 8);
        ox = 0; oy = 1; c.srow = 0; c.scol = k * E; c.dly = TILE; c.dlx = k * E;
    } else if (h < 6 * CPR + 3 * TILE) { // left column chunk
        const int hh = h - 6 * CPR, s3 = hh / TILE, r = hh - s3 * TILE;
        c.slot = s3 == 0 ? 1 : (s3 == 1 ? 5 : 8);
        ox = -1; oy = 0; c.srow = r; c.scol = TILE - E; c.dly = r; c.dlx = -E;
    } else if (h < 6 * CPR + 6 * TILE) { // right column chunk
        const int hh = h - 6 * CPR - 3 * TILE, s3 = hh / TILE, r = hh - s3 * TILE;
        c.slot = s3 == 0 ? 3 : (s3 == 1 ? 6 : 7);
        ox = 1; oy = 0; c.srow = r; c.scol = 0; c.dly = r; c.dlx = TILE;
    } else { // corners, one diagonal slot each
        const int k = h - 6 * CPR - 6 * TILE;
        c.slot = 5 + k;
        ox = (k == 0 || k == 3) ? -1 : 1;
        oy = (k <= 1) ? -1 : 1;
        c.srow = oy < 0 ? TILE - 1 : 0;
        c.scol = ox < 0 ? TILE - E : 0;
        c.dly = oy < 0 ? -1 : TILE;
        c.dlx = ox < 0 ? -E : TILE;
    }
    c.dir = 3 * (oy + 1) + (ox + 1);
    return c;
}

// Kernel kinds of one time step.
enum StepMode {
    MODE_TWO_LATTICE = 0, // gather from src, store aligned into dst
    MODE_AA_PULLPUSH = 1, // in place, from the swapped state: gather+scatter
    MODE_AA_LOCAL = 2     // in place, from the streamed state: local only
};

// How the lattice currently holds A_t (see lbm_api.cu).
enum Phase {
    PH_PLAIN = 0,   // slot i at x holds A_i(x)                 (two-lattice)
    PH_SWAPPED = 1, // slot opp(i) at x holds A_i(x)            (AA, even)
    PH_STREAMED = 2 // slot i at x holds f'_i(x) (pre-collision) (AA, odd)
};

enum ForceMode { FORCE_NONE = 0, FORCE_UNIFORM = 1, FORCE_FIELD = 2 };

// Geometry as the kernels see it (device pointers into the workspace).
struct Geo {
    int nx, ny;
    int periodic_x, periodic_y;
    int layout;            // lbm_layout
    int ntx, nty, ntiles;  // sparse tile grid / kept tiles
    long long nslot;       // elements per distribution slot (dense: nx*ny)
    long long nnode;       // nx*ny: component stride of canonical arrays
    const uint8_t *mask;   // dense [ny][nx]; sparse [ntiles][256]
    const int32_t *nbr;    // sparse [ntiles][9]
    const int32_t *tile_xy;// sparse [ntiles]: (ty << 16) | tx
    const int32_t *tile_id;// sparse [nty][ntx]
    int has_mask;          // 0: every node fluid, both axes periodic
    int frame_y;           // dense, > 2^21 nodes, bounced links only in rows 0 and ny-1
    // sparse: vectors of 2 / 4 nodes that hold a fluid node, as t * TPT +
    // position in the tile (TPT = 256 / vector size), in tile order
    int use_list;
    float active_frac;     // listed 2-node vectors / all vectors of kept tiles
    int nlist2, nlist4;
    const unsigned *vlist2, *vlist4;
    // sparse: per tile, bit 8 * row + v set iff 2-node vector v of that tile
    // row holds a fluid node (row r in 32-bit word r / 4)
    const uint4 *tile_vmask;
    // sparse: per tile 128 bytes, the 2-node vectors (8 * row + v) whose
    // 32-byte DRAM sector holds a fluid node, ascending, then 0xFF
    const uint8_t *tile_order;
    // sparse: per tile 128 bits, bit h (word h / 32) set iff halo chunk h of
    // the staged step (halo_source) exists and its source holds a fluid
    // node; the other chunks are never pulled unbounced, and are not read
    const uint4 *tile_hmask;
    // device error word: set when a kernel's bounded wait gave up
    unsigned *err;
};

// Physics as the kernels see it.
struct Phys {
    double omega;
    double fx, fy;
    const void *force;     // FORCE_FIELD: [2][ny][nx] compute type
    int force_mode;
    int has_wall;          // some wall term is nonzero
    double wt[WALL_SIDES][9];
    // the same constants rounded to FP32 on the host (FP32 / FP16s kernels)
    float omega_f, om1_f, kk_f, fx_f, fy_f;
    float wt_f[WALL_SIDES][9];
    // omega/3 and omega/12 (3 omega w for axis and diagonal links): FP64, and
    // for FP32 the float pair (hi + lo) of omega_f/3, omega_f/12
    double kq[2];
    float kq_hi[2], kq_lo[2];
    // tau - 1/2 = (1 - omega/2) / omega: the Guo source's weight relative to
    // the equilibrium's (FP64, and from omega_f for FP32 / FP16s)
    double tau_h;
    float tau_h_f;
    // two-relaxation-time collision (trt != 0): the odd rate omega_m and
    // f_i <- tp (f_i + f_opp) + tm (f_i - f_opp) + ..., tp = (1 - omega)/2,
    // tm = (1 - omega_m)/2; odd constants omega_m/3, omega_m/12 (FP64; FP32
    // float pair), 1/omega_m - 1/2, and 1 - omega_m/2 (FP32)
    int trt;
    double omega_m, tp, tm, kqm[2], thm;
    float tp_f, tm_f, kqm_hi[2], kqm_lo[2], thm_f, kkm_f;
    // when set, the step kernel's time-step index is *tbase + its step
    // argument (steps replayed from a CUDA graph, whose arguments are fixed)
    const unsigned long long *tbase;
    // open sides (lbm_side_kind per side; uniform values; optional per-node
    // values along the side, compute type)
    int has_open;
    int open_kind[4];
    double open_u[4][2], open_rho[4];
    float open_u_f[4][2], open_rho_f[4];
    const void *open_val[4];
};

// Launchers, defined in lbm_kernels.cuh and instantiated per precision P
// (an lbm_precision value) in kern_f64.cu, kern_f32.cu, kern_f16s.cu.
// t: index of the time step (random bits of FP16s stochastic rounding);
// TRT: the two-relaxation-time collision instead of BGK (launch_step picks
// it from ph.trt); its instances are built in kern_*_trt.cu.
template <int P, bool TRT> cudaError_t launch_step_op(const Geo &g, const Phys &ph, int mode,
                                                      const void *src, void *dst, unsigned long long t,
                                                      cudaStream_t s);
template <int P> inline cudaError_t launch_step(const Geo &g, const Phys &ph, int mode, const void *src,
                                                void *dst, unsigned long long t, cudaStream_t s) {
    return ph.trt ? launch_step_op<P, true>(g, ph, mode, src, dst, t, s)
                  : launch_step_op<P, false>(g, ph, mode, src, dst, t, s);
}
template <int P> cudaError_t launch_init(const Geo &g, int phase, const void *rho,
                                         const void *u, void *lat, cudaStream_t s);
template <int P> cudaError_t launch_set_f(const Geo &g, int phase, const void *f, void *lat,
                                          cudaStream_t s);
template <int P> cudaError_t launch_get_f(const Geo &g, int phase, const void *lat, void *f,
                                          cudaStream_t s);
template <int P> cudaError_t launch_macros(const Geo &g, const Phys &ph, int phase,
                                           const void *lat, void *rho, void *u,
                                           cudaStream_t s);
// FP64 partial sums -> partial[RED_BLOCKS][4], then a fixed-order final sum
// into out[4].  kind: 0 mass/momentum of A_t; 1 MSE vs target; 2 kinetic
// energy.
template <int P> cudaError_t launch_reduce(const Geo &g, const Phys &ph, int phase, int kind,
                                           const void *lat, const void *target,
                                           double *partial, double *out, cudaStream_t s);
template <int P> cudaError_t launch_adjoint(const Geo &g, const Phys &ph, const void *state,
                                            const void *lam_in, void *lam_out,
                                            void *grad_force, cudaStream_t s);
template <int P> cudaError_t launch_macros_adjoint(const Geo &g, const Phys &ph,
                                                   const void *state, const void *g_rho,
                                                   const void *g_u, void *lam,
                                                   void *grad_force, cudaStream_t s);

// Host geometry preparation (lbm_geometry.cpp).
// Link mask: bit (i-1) set iff link i pulls from a solid node or across a
// wall; 0xFF for solid nodes and for fluid nodes with no link to any node.
long long build_link_mask(const lbm_params &p, uint8_t *mask);
// Tile map (16x16): tile_id[nty][ntx] (-1 absent), nbr[ntiles][9],
// tile_xy[ntiles].  Returns the number of kept tiles.
int build_tile_map(const lbm_params &p, const uint8_t *mask, int32_t *tile_id,
                   int32_t *nbr, int32_t *tile_xy);
// Per-tile masks [ntiles][256] from the canonical mask (0xFF outside).
void build_tile_masks(const lbm_params &p, const uint8_t *mask, const int32_t *tile_xy,
                      int ntiles, uint8_t *tile_mask);

} // namespace lbm
