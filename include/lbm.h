/*
 * lbm.h -- C ABI of the GB300 (sm_103a) D2Q9 lattice-Boltzmann library.
 *
 * The library implements the fused pull stream-and-collide update of
 * Tomczak, "Data-Oriented Language Implementation of Lattice-Boltzmann Method
 * for Dense and Sparse Geometries" (arXiv 2108.13241), Algorithm 1, with the
 * BGK operator (Eq. 4, Eq. 5, Eq. 6), the moments of
 * Eq. 2, half-way bounce-back walls and obstacles (Sec. 3, boundary
 * paragraph), dense and 16x16-tiled sparse storage (Sec. 4.2.2, "tile" and
 * "pointer tile" layouts), the constant-velocity and constant-pressure
 * open sides of Sec. 3 (after Zou & He), plus a Guo body force, an in-place
 * AA pattern, FP64 / FP32 / FP16-shifted storage and a hand-written adjoint.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  Lattice (Sec. 2.2, Fig. D2Q9): i = 0 rest, 1 (+1,0), 2 (0,+1), 3 (-1,0),
 *  4 (0,-1), 5 (+1,+1), 6 (-1,+1), 7 (-1,-1), 8 (+1,-1).
 *  Node (x, y) has index n = y*nx + x (x fastest).  Canonical device arrays:
 *    distributions  f[i][ny][nx]  -- the post-collision state A_t, i.e. the
 *                                    array the next step gathers
 *                                    f'_i(x) = A_i(x - c_i) from;
 *    vector fields  v[2][ny][nx]  (x component first);
 *    scalar fields  s[ny][nx].
 *  "Compute type" = double for LBM_F64, float for LBM_F32 and LBM_F16S; every
 *  canonical device array passed to or from the library is in compute type.
 *  Device pointers must be 16-byte aligned (torch allocations are).  The
 *  field arguments of lbm_init_equilibrium and lbm_macros may also be
 *  pinned host memory that the device maps (cudaHostAlloc / torch
 *  pin_memory under unified addressing): the kernels then read or write
 *  host memory directly -- on GB300 over NVLink-C2C, overlapping the
 *  transfer with the kernel instead of staging it in a separate copy.
 *  Ownership: all device memory belongs to the caller.  lbm_create carves
 *  its lattices and tables out of the caller's workspace; the context owns
 *  host memory only.  Caller buffers must outlive the calls that use them
 *  (the force field: until it is replaced or the context destroyed).
 *  Streams: every call is asynchronous on params.stream unless it says it
 *  synchronises.  Errors: every call returns a status and never aborts; a
 *  CUDA launch or runtime error is also kept in the context ("sticky") and
 *  returned by every later call; lbm_last_error gives the message.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_ERR_INVALID = 1,      /* bad argument or geometry                    */
    LBM_ERR_CUDA = 2,         /* CUDA runtime error (sticky)                 */
    LBM_ERR_OOM = 3,          /* workspace smaller than lbm_workspace_bytes  */
    LBM_ERR_DIVERGED = 4,     /* a reduction met NaN/Inf                     */
    LBM_ERR_TIMEOUT = 5,      /* a kernel's bounded wait expired (sticky)    */
    LBM_ERR_UNSUPPORTED = 6   /* valid request this build does not serve     */
} lbm_status;

/* Storage of the distributions.  Every mode stores f_i - w_i ("shifted");
 * LBM_F64 stores and computes FP64, LBM_F32 FP32.  LBM_F16S computes in FP32
 * and stores (f_i - w_i) * 2^10 in binary16 (exact power-of-two scale;
 * |f_i - w_i| <= 64); the time step rounds it stochastically (13 random bits
 * added below the last kept bit, then truncation) with random bits that
 * depend only on the node pair (x even and x + 1), the link and the step
 * index, so runs are deterministic and identical across layouts and
 * patterns; every other encode (init, set_f) rounds to nearest. */
typedef enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16S = 2 } lbm_precision;

/* LBM_DENSE: f[i][ny][nx].  LBM_SPARSE_TILE16: only 16x16 tiles that hold a
 * fluid node are stored, f[tile][i][16][16], with a 9-entry neighbour-tile
 * table (the paper's "pointer tile" layout without pointers). */
typedef enum { LBM_DENSE = 0, LBM_SPARSE_TILE16 = 1 } lbm_layout;

/* LBM_TWO_LATTICE: read A, write B, swap (Algorithm 1).  LBM_AA: one lattice
 * updated in place, alternating a local step and a gather/scatter step (the
 * single-copy scheme the paper cites in Sec. 3). */
typedef enum { LBM_TWO_LATTICE = 0, LBM_AA = 1 } lbm_pattern;

/* Kind of a non-periodic side: a half-way bounce-back wall, or an open side
 * with constant velocity or constant pressure (the boundary conditions after
 * Zou & He that the paper lists in Sec. 3). */
typedef enum { LBM_SIDE_WALL = 0, LBM_SIDE_VELOCITY = 1, LBM_SIDE_PRESSURE = 2 } lbm_side_kind;

/* A domain side.  periodic != 0: the axis wraps (both sides of an axis must
 * agree; kind must be 0).  periodic == 0 and kind == LBM_SIDE_WALL:
 * half-way bounce-back wall half a spacing outside the outermost nodes,
 * moving at (ux, uy); a link that crosses it gets the term
 * 6 w_i rho_0 (c_i . u_w), rho_0 = 1.  A link that leaves the domain across
 * two sides is decided by the south/north side first.
 *
 * Open sides (periodic == 0, kind != 0): the outermost row or column of
 * nodes are boundary nodes.  Each link of a boundary node that would pull
 * from beyond the side takes the value for which the node has velocity
 * (ux, uy) (LBM_SIDE_VELOCITY; |u . n| < 1 for the outward normal n) or
 * density rho > 0 with zero tangential velocity (LBM_SIDE_PRESSURE):
 *   f_i = f_opp(i) + 6 w_i rho (c_i . u) - (c_i . t) N_t,
 *   N_t = 1/2 sum_{c.n=0} (c_j . t) f_j - rho (u . t)/3,
 *   rho (1 + u . n) = sum_{c.n=0} f_j + 2 sum_{c.n>0} f_j,
 * t the tangent along the side (Zou & He 1997 for every side).  Corner links
 * that also cross a wall follow the wall.  Two adjacent sides cannot both be
 * open.  Open sides work with every precision, layout and pattern, and in the
 * adjoint calls (whose rules are the transpose of these affine maps).
 * lbm_set_side_values gives per-node values. */
typedef struct {
    int periodic;
    double ux, uy;   /* wall velocity, or the velocity of a velocity side */
    int kind;        /* lbm_side_kind */
    double rho;      /* density of a pressure side */
} lbm_side;

/* Collision operator.  LBM_BGK: the single-relaxation-time operator of
 * Eq. 3-4, omega = 1/tau.  LBM_TRT: the two-relaxation-time operator
 * (Ginzburg), a collision model beyond BGK of the kind the paper leaves to
 * future work (Sec. 5): with g^+/- = (g_i +/- g_opp(i))/2,
 *   f_i <- f_i - omega (f^+ - f^eq+) - omega_m (f^- - f^eq-)
 *          + (1 - omega/2) G^+ + (1 - omega_m/2) G^-,
 * G_i the Guo term w_i [3 (c_i - u) + 9 (c_i . u) c_i] . F; the even rate
 * omega = 1/tau sets the viscosity, the odd rate omega_m follows from the
 * magic parameter Lambda = (1/omega - 1/2)(1/omega_m - 1/2).  Lambda = 3/16
 * puts half-way bounce-back walls exactly half-way for channel flow at any
 * tau; Lambda = (tau - 1/2)^2 gives BGK again. */
typedef enum { LBM_BGK = 0, LBM_TRT = 1 } lbm_collision;

typedef struct {
    int nx, ny;               /* nx % 16 == 0; LBM_SPARSE_TILE16 with a
                                 periodic y axis also needs ny % 16 == 0;
                                 9 * (stored nodes) < 2^32 (32-bit element
                                 indices: up to ~21800^2 nodes)             */
    const uint8_t *solid;     /* HOST [ny][nx], nonzero = solid; NULL = all
                                 fluid; read during lbm_workspace_bytes and
                                 lbm_create only                           */
    double tau;               /* BGK relaxation time > 0.5; omega = 1/tau,
                                 nu = (tau - 1/2)/3 (Eq. 5)            */
    double fx, fy;            /* uniform body-force density (Guo forcing)  */
    lbm_side west, east, south, north;
    lbm_precision precision;
    lbm_layout layout;
    lbm_pattern pattern;
    void *stream;             /* cudaStream_t, NULL = legacy default stream */
    lbm_collision collision;  /* LBM_BGK (0) or LBM_TRT                     */
    double magic;             /* LBM_TRT: Lambda > 0; 0 = 3/16             */
} lbm_params;

typedef struct lbm_ctx lbm_ctx;

/* Bytes of device workspace lbm_create needs for these parameters.  Host
 * only; builds the link mask and, for the sparse layout, the tile map. */
lbm_status lbm_workspace_bytes(const lbm_params *p, size_t *bytes);

/* Validates p, builds the per-node link mask (bit i-1 set iff link i pulls
 * from a solid node or across a wall; 0xFF marks a node that is solid or has
 * no link to any other node, Sec. 3 "bitmask containing information about
 * which neighbour nodes are present") and, for the sparse layout, the tile
 * map; copies them into d_workspace (>= lbm_workspace_bytes, 256-byte
 * aligned) and initialises the lattice to rest (rho = 1, u = 0) (Algorithm 1,
 * initialisation).  Synchronises the stream.  *out is NULL on error. */
lbm_status lbm_create(const lbm_params *p, void *d_workspace, size_t bytes, lbm_ctx **out);

/* Frees the host context and its recorded CUDA graphs (synchronising the
 * stream first when there are any).  The workspace stays the caller's. */
lbm_status lbm_destroy(lbm_ctx *ctx);

/* Per-node values of open side `side` (0 west, 1 east, 2 south, 3 north),
 * compute type, along the side (index y on west/east, x on south/north):
 * velocity side [2][len] (all u_x, then all u_y), pressure side [len]
 * densities; len = ny on west/east, nx on south/north.  NULL returns to the
 * uniform value of the parameters.  The pointer is kept, not copied, and
 * read by every later step and lbm_macros.  LBM_ERR_INVALID if the side is
 * not open or the pointer is not aligned to the compute type. */
lbm_status lbm_set_side_values(lbm_ctx *ctx, int side, const void *d_values);

/* Per-node body force F[2][ny][nx] (compute type), used by every later step,
 * macros and adjoint instead of (fx, fy); NULL returns to the uniform force.
 * The pointer is kept, not copied. */
lbm_status lbm_set_force(lbm_ctx *ctx, const void *d_force);

/* Algorithm 1, initialisation: A_i = f^eq_i(rho, u) (Eq. 6) at fluid
 * nodes.  d_rho [ny][nx] and d_u [2][ny][nx] in compute type; NULL means
 * rho = 1 / u = 0.  Resets the step counter and the AA phase. */
lbm_status lbm_init_equilibrium(lbm_ctx *ctx, const void *d_rho, const void *d_u);

/* n time steps of Algorithm 1 (n >= 0): per fluid node, pull gather with
 * bounce-back, moments (Eq. 2, u shifted by F/2), f^eq (Eq. 6), BGK
 * relaxation (Eq. 3, Eq. 4) plus the Guo source
 * (1 - omega/2) w_i [3 (c_i - u) + 9 (c_i . u) c_i] . F, aligned store.
 * With graphs enabled (the default, lbm_set_graphs), runs of 32 steps or
 * more are replayed from a CUDA graph recorded on the first such call (the
 * same kernels and arguments, so the results are bit-identical); the graph
 * is recorded again after lbm_set_force or lbm_set_side_values. */
lbm_status lbm_step(lbm_ctx *ctx, int n);

/* Whether lbm_step, lbm_forward_states and lbm_backward replay CUDA graphs
 * (enable != 0, the default) or issue every kernel launch from the host.
 * Launch-bound runs (small grids) gain from the graphs; a context whose
 * graph could not be recorded switches to direct launches by itself.
 * Replacing a recorded graph (new pointers, another run length, or after
 * lbm_set_force / lbm_set_side_values) synchronises the context's stream
 * first, since the old graph may still be running; so does lbm_destroy of a
 * context that recorded graphs. */
lbm_status lbm_set_graphs(lbm_ctx *ctx, int enable);

/* Density and velocity of the current state (Eq. 2 on the gathered f'
 * of the next step, u = (m + F/2)/rho).  d_rho [ny][nx], d_u [2][ny][nx]
 * (compute type); either may be NULL.  Solid nodes give rho = 1, u = 0. */
lbm_status lbm_macros(lbm_ctx *ctx, void *d_rho, void *d_u);

/* Canonical state A_t out / in: d_f [9][ny][nx] compute type.  Solid nodes
 * read as w_i and are ignored on input.  lbm_set_f resets the AA phase. */
lbm_status lbm_get_f(lbm_ctx *ctx, void *d_f);
lbm_status lbm_set_f(lbm_ctx *ctx, const void *d_f);

/* FP64 reductions over fluid nodes of the canonical state: mass
 * sum_i A_i and momentum sum_i c_i A_i.  Deterministic (fixed-order tree,
 * no atomics).  Synchronises; LBM_ERR_DIVERGED on NaN/Inf.  Either output
 * pointer may be NULL.  Like lbm_loss, it also reads the context's device
 * error word: LBM_ERR_TIMEOUT (sticky) if a step kernel's wait on its own
 * copy pipeline gave up (after about two seconds) since the context was
 * created. */
lbm_status lbm_reduce(lbm_ctx *ctx, double *h_mass, double h_mom[2]);

/* FP64 loss of the current state over fluid nodes, Nf = fluid-node count:
 * kind 0: (1/Nf) sum |u - u*|^2 with d_u_target [2][ny][nx] (compute type);
 * kind 1: 1/2 sum rho |u|^2 (d_u_target unused).  Synchronises. */
lbm_status lbm_loss(lbm_ctx *ctx, int kind, const void *d_u_target, double *h_loss);

/* Native checkpoints: the lattice the next step reads, in the storage
 * layout and type, plus nothing else (the AA phase is part of the context;
 * checkpoints need the two-lattice pattern).  *bytes = one state. */
lbm_status lbm_state_bytes(const lbm_ctx *ctx, size_t *bytes);
lbm_status lbm_save_state(lbm_ctx *ctx, void *d_dst);
lbm_status lbm_load_state(lbm_ctx *ctx, const void *d_src);

/* Forward recompute for the adjoint: runs n steps from native state
 * d_states[0] and writes A_{k+1} into d_states[k+1] (k = 0..n-1);
 * h_states is a HOST array of n+1 device pointers; t0 is the step index of
 * d_states[0] (FP16s stochastic rounding then reproduces the original run).
 * The context's own lattice and step counter are not touched.  Two-lattice
 * only.  Runs of 8 steps or more replay a CUDA graph, recorded again when
 * n or a pointer of h_states changes (see lbm_set_graphs). */
lbm_status lbm_forward_states(lbm_ctx *ctx, void *const *h_states, int n, long long t0);

/* Discrete adjoint of n steps (transpose of the linearised Algorithm 1
 * step, with the bounce-back gather transposed into a push).
 * h_states: HOST array of n device pointers to native states A_{t0+k}.
 * d_lambda [9][ny][nx] compute type: in dL/dA_{t0+n}, out dL/dA_{t0};
 * d_lambda_tmp: same size, scratch.  d_grad_force [2][ny][nx] compute type,
 * accumulated (+=): dL/dF(x) for the per-node force (the uniform force's
 * gradient is its node sum).  Entries of solid nodes come out 0.
 * LBM_ERR_UNSUPPORTED unless dense, two-lattice and BGK.  Runs of 8 steps or
 * more replay a CUDA graph, recorded again when n or a pointer changes. */
lbm_status lbm_backward(lbm_ctx *ctx, const void *const *h_states, int n,
                        void *d_lambda, void *d_lambda_tmp, void *d_grad_force);

/* Transpose of lbm_macros at the current state: from dL/drho [ny][nx] and
 * dL/du [2][ny][nx] (compute type, either NULL = 0) writes
 * d_lambda = dL/dA_t [9][ny][nx] and accumulates dL/dF into d_grad_force
 * (+=, may be NULL).  Dense two-lattice BGK only. */
lbm_status lbm_macros_backward(lbm_ctx *ctx, const void *d_grad_rho, const void *d_grad_u,
                               void *d_lambda, void *d_grad_force);

/* Host copies of the geometry tables: link mask [ny][nx] (see lbm_create),
 * and for the sparse layout tile_id [ceil(ny/16)][ceil(nx/16)] (compact
 * tile number in row-major tile order, -1 absent) and nbr [ntiles][9]
 * (tile at offset c_i, wrapped on periodic axes, -1 beyond a wall or
 * absent).  Any output may be NULL; lbm_tile_map returns
 * LBM_ERR_UNSUPPORTED for the dense layout. */
lbm_status lbm_link_mask(const lbm_ctx *ctx, uint8_t *h_mask);
lbm_status lbm_tile_map(const lbm_ctx *ctx, int32_t *h_tile_id, int32_t *h_nbr, int *h_ntiles);

/* Host-only: the same link mask and tile tables lbm_create would build for
 * p (no device work, no context).  h_mask [ny][nx]; h_tile_id and h_nbr as
 * for lbm_tile_map (sparse layout only; may be NULL); *h_nfluid = fluid
 * nodes.  Lets a caller (or a test without a GPU) inspect the geometry. */
lbm_status lbm_geometry(const lbm_params *p, uint8_t *h_mask, int32_t *h_tile_id, int32_t *h_nbr,
                        int *h_ntiles, long long *h_nfluid);

/* Largest ny lbm_reduce_f_noalloc accepts (its scratch is sized for it). */
#define LBM_NOALLOC_MAX_ROWS 16384

/* lbm_reduce_f_noalloc -- the paper has no counterpart; this is a service
 * for callers that must not allocate device memory at the moment they need a
 * reduction: code running while its stream is captured into a CUDA graph,
 * plugins whose host application owns every device buffer, real-time loops
 * that never enter an allocator.  It computes, in FP64, over the nodes of a
 * canonical array d_f [9][ny][nx] (compute type of `precision`: double for
 * LBM_F64, float otherwise) whose d_mask [ny][nx] byte is not 0xFF (NULL:
 * all nodes): d_out[0] = sum_i f_i, d_out[1..2] = sum_i c_i f_i (device
 * pointer, 3 doubles), asynchronously on `stream`.  It needs no context and
 * calls no allocator: its scratch is a static device array of
 * LBM_NOALLOC_MAX_ROWS * 32 + 256 bytes (512.25 KiB) that every GPU loading
 * the library keeps until the process exits.  ny > LBM_NOALLOC_MAX_ROWS (or
 * a NULL pointer, nx or ny < 1) returns LBM_ERR_INVALID before any device
 * work.  `stream` (NULL = the legacy default stream) and every pointer must
 * belong to the current device; a stream of another device returns
 * LBM_ERR_INVALID.  The first call on a device looks up the scratch array's
 * device address (cudaGetSymbolAddress) and caches it per device: make that
 * first call before any stream capture; the cached address does not survive
 * cudaDeviceReset.  A call clears a CUDA error that an earlier call left
 * unreported (cudaGetLastError) before it launches, and returns LBM_ERR_CUDA
 * if either of its two launches fails.  All calls share the scratch: calls
 * that overlap on the GPU (other streams, other host threads) race.  Every
 * call overwrites the scratch it reads, so nothing carries over between
 * calls. */
lbm_status lbm_reduce_f_noalloc(lbm_precision precision, const void *d_f, const uint8_t *d_mask, int nx, int ny,
                                double *d_out, void *stream);

/* Measurement aid, with no counterpart in the paper: the data movement of
 * one time step at DRAM-sector granularity without its arithmetic.  Copies,
 * n times, every 32-byte sector (8 FP32, 16 FP16s or 4 FP64 consecutive
 * nodes of one distribution slot) of the current lattice that holds a fluid
 * node, in all nine slots, into the other lattice of a two-lattice context,
 * asynchronously on the context's stream.  Any step must move at least
 * these bytes on the geometry; timing this call measures what HBM delivers
 * for the geometry's access pattern (scattered sectors on porous media), the
 * ceiling the step kernels are compared with.  The state A_t (the current
 * lattice) is not changed; the other lattice is the next step's output.
 * h_bytes (host, may be NULL) receives the bytes one copy reads and writes,
 * 2 * 9 * 32 * (sectors holding fluid).  LBM_ERR_UNSUPPORTED for the AA
 * pattern (one lattice); LBM_ERR_INVALID for n < 0. */
lbm_status lbm_sector_copy(lbm_ctx *ctx, int n, long long *h_bytes);

long long lbm_fluid_nodes(const lbm_ctx *ctx);
long long lbm_step_count(const lbm_ctx *ctx);

/* Kernel launches of one lbm_step time step (1 for most configurations; 2
 * when the dense grid runs its boundary rows with the masked kernel and the
 * rest without, more for grids of over 65535 rows).  -1 for a NULL ctx. */
int lbm_launches_per_step(const lbm_ctx *ctx);

/* Kernel launches (graph nodes included) that lbm_step(ctx, n) makes now:
 * n * lbm_launches_per_step, plus, when graphs replay, one to set the
 * device step counter and one per 32-step replay to advance it.  -1 for a
 * NULL ctx or n < 0. */
long long lbm_step_launches(const lbm_ctx *ctx, int n);
const char *lbm_status_string(lbm_status s);
const char *lbm_last_error(const lbm_ctx *ctx);

/* ------------------------------------------------------------------------
 * Three-dimensional D3Q19 step (lbm3_*): Algorithm 1 carried to three
 * dimensions, the extension the paper names as future work (Sec. 5).  The
 * moments (Eq. 2 with the Guo F/2 shift), the BGK relaxation (Eq. 3-5) and
 * the equilibrium (Eq. 6, with the D3Q19 weights 1/3 rest, 1/18 axis, 1/36
 * diagonal) are the two-dimensional step's; dense storage, two lattices or
 * the in-place AA pattern, stationary half-way bounce-back walls and
 * obstacles, uniform body force, FP64 / FP32 / FP16-shifted storage.
 *  Lattice: i = 0 rest; 1 (+1,0,0), 2 (-1,0,0), 3 (0,+1,0), 4 (0,-1,0),
 *  5 (0,0,+1), 6 (0,0,-1); 7 (+1,+1,0), 8 (-1,-1,0), 9 (+1,-1,0),
 *  10 (-1,+1,0); 11 (+1,0,+1), 12 (-1,0,-1), 13 (+1,0,-1), 14 (-1,0,+1);
 *  15 (0,+1,+1), 16 (0,-1,-1), 17 (0,+1,-1), 18 (0,-1,+1) -- links 2k-1 and
 *  2k are opposite.
 *  Node (x, y, z) has index n = (z*ny + y)*nx + x.  Canonical device arrays
 *  (compute type: double for LBM_F64, float for LBM_F32): distributions
 *  f[19][nz][ny][nx] (the post-collision state A_t, solid nodes read w_i),
 *  vector fields v[3][nz][ny][nx], scalar fields s[nz][ny][nx].  Device
 *  pointers 16-byte aligned; ownership, streams and errors as above (the
 *  workspace is the caller's, 256-byte aligned; calls are asynchronous on
 *  params.stream except lbm3_create, which synchronises; a CUDA error is
 *  sticky). */
typedef struct lbm3_ctx lbm3_ctx;
typedef struct {
    int nx, ny, nz;              /* ny, nz <= 65535; nx*ny*nz < 2^32 (1024^3 FP32 two-lattice: 163 GB) */
    const uint8_t *solid;        /* host [nz][ny][nx], 1 = solid; NULL = all fluid; read at create */
    double tau;                  /* > 0.5 (omega = 1/tau, Eq. 5) */
    double fx, fy, fz;           /* uniform body-force density (Guo) */
    int periodic_x, periodic_y, periodic_z; /* 0: stationary half-way bounce-back walls on both faces */
    lbm_precision precision;     /* LBM_F64, LBM_F32, or LBM_F16S (nx even; two-lattice only) */
    lbm_pattern pattern;         /* LBM_TWO_LATTICE, or LBM_AA (one lattice, in place) */
    void *stream;                /* cudaStream_t; NULL = legacy default stream */
    int node_list;               /* FP64 / FP32 with a link mask: 0 = a node list with the
                                    AA pattern when it holds at most 90% of the nodes (two
                                    lattices: the dense grid, measured faster), 1 = never
                                    (the dense grid), 2 = always; ignored for FP16s (below) */
} lbm3_params;

/* The node list (sparse geometries; the porous-media counterpart of the
 * two-dimensional tiles of Sec. 4.2.2): the step runs one thread per listed
 * node instead of one per grid node, so no lane idles on a solid node.  It
 * lists, ascending, every fluid node and, with two lattices, every solid
 * node sharing a 32-byte sector of the slot planes with a fluid node (it
 * stores zeros, so sectors are written whole); 8 bytes an entry in the
 * workspace (the node index and its link mask, read by one load).  Results are bit-identical to the dense grid's. */

/* Workspace bytes for p: two lattices (one for LBM_AA; 19 values a node),
 * when some link bounces a 32-bit link mask per node, and the node list.  Pure host;
 * LBM_ERR_INVALID for bad parameters (lbm3_create: LBM_ERR_UNSUPPORTED for
 * FP16s with the AA pattern). */
lbm_status lbm3_workspace_bytes(const lbm3_params *p, size_t *bytes);
/* Builds the link mask on the host (bit i-1: link i pulls from a solid node
 * or across a wall face), carves the lattices and the mask out of
 * d_workspace (256-byte aligned, at least lbm3_workspace_bytes), zeroes the
 * lattices (every node at rest, rho = 1) and synchronises.  LBM_ERR_OOM when
 * the workspace is too small. */
lbm_status lbm3_create(const lbm3_params *p, void *d_workspace, size_t bytes, lbm3_ctx **out);
/* Frees the context's host memory (the workspace stays the caller's). */
lbm_status lbm3_destroy(lbm3_ctx *ctx);
/* A_0 = f^eq(rho, u) (Algorithm 1, initialisation); NULL rho: 1, NULL u: 0. */
lbm_status lbm3_init_equilibrium(lbm3_ctx *ctx, const void *d_rho, const void *d_u);
/* n fused pull stream-and-collide steps (Algorithm 1), one launch each. */
lbm_status lbm3_step(lbm3_ctx *ctx, int n);
/* rho and u = (sum c f' + F/2)/rho at the current time (Eq. 2), 0 at solid
 * nodes; either pointer may be NULL. */
lbm_status lbm3_macros(lbm3_ctx *ctx, void *d_rho, void *d_u);
/* Canonical state out / in (checkpoints, tests). */
lbm_status lbm3_get_f(lbm3_ctx *ctx, void *d_f);
lbm_status lbm3_set_f(lbm3_ctx *ctx, const void *d_f);
long long lbm3_fluid_nodes(const lbm3_ctx *ctx);
/* Entries of the node list the step runs over; 0 when it runs over the
 * dense grid; -1 for a NULL ctx. */
long long lbm3_list_nodes(const lbm3_ctx *ctx);
long long lbm3_step_count(const lbm3_ctx *ctx);
const char *lbm3_last_error(const lbm3_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
