// lbm_api.cu -- the C ABI of include/lbm.h: argument checks, the host context,
// workspace carving, lattice-phase bookkeeping and kernel dispatch.
//
// Lattice phases (how the device lattice holds the state A_t):
//   two-lattice: lat[cur] holds A_t in slot order (PH_PLAIN); a step reads
//     lat[cur], writes lat[1-cur] and flips cur (Algorithm 1 with the swap
//     done by exchanging pointers, not by a copy kernel).
//   AA: one lattice.  PH_SWAPPED: slot opp(i) of x holds A_i(x).  A
//     gather/scatter step moves it to PH_STREAMED (slot i of x holds the
//     pulled f'_i(x) of the next step); a local step moves it back.
//
// Runs of steps replay recorded CUDA graphs, which removes the host's launch
// cost (the bound on small grids, where a step's kernel takes about as long
// as the host needs to issue it) and the gaps between launches: lbm_step in
// chunks of GRAPH_CHUNK steps, lbm_forward_states and lbm_backward as a whole
// once they are GRAPH_MIN steps or longer.  A graph is recorded once and replayed while
// the pointers and physics it was recorded with stay the same (the autograd
// segments reuse their state buffers, so every full segment replays); the
// FP16s steps of a graph read their time-step index from a device counter.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lbm_internal.h"

using namespace lbm;

struct lbm_ctx {
    lbm_params p;
    Geo geo;
    Phys phys;
    size_t esize;      // bytes per stored value
    size_t csize;      // bytes per compute value
    long long nfluid;
    std::vector<uint8_t> mask;    // canonical link mask [ny][nx]
    std::vector<int32_t> tile_id; // [nty][ntx]
    std::vector<int32_t> nbr;     // [ntiles][9], D2Q9 order
    void *lat[2];
    size_t lat_bytes;
    double *partial;
    double *red_out;
    int cur;
    int phase;
    long long steps;
    cudaStream_t stream;
    lbm_status sticky;
    std::string err;
    // CUDA graphs (see the top of this file)
    struct GraphCache {
        cudaGraphExec_t exec = nullptr;
        std::vector<unsigned long long> key;
    } gc[4];
    cudaStream_t cap = nullptr;       // stream the graphs are recorded on
    int graphs = 1;                   // replay graphs (lbm_set_graphs)
    unsigned long long *tb = nullptr; // device time-step counter of replayed steps
    unsigned long long version = 0;   // bumped when the physics' pointers change
    long long fluid_sectors = 0;      // 32-byte sectors of one slot that hold a fluid node
    const uint32_t *secs = nullptr;   // their list (NULL: every sector holds fluid)
};

namespace {

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t elem_size(int prec) { return prec == LBM_F64 ? 8 : (prec == LBM_F32 ? 4 : 2); }
size_t comp_size(int prec) { return prec == LBM_F64 ? 8 : 4; }

const char *check_params(const lbm_params *p) {
    if (!p) return "params is NULL";
    if (p->nx < 16 || p->nx % 16) return "nx must be a positive multiple of 16";
    if (p->ny < 1) return "ny must be >= 1";
    // element indices of the lattices and of canonical [9][ny][nx] arrays are
    // 32-bit in the kernels
    if (9ll * p->nx * p->ny >= (1ll << 32)) return "9*nx*ny must be < 2^32";
    if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return "tau must be > 0.5";
    if (!std::isfinite(p->fx) || !std::isfinite(p->fy)) return "force must be finite";
    if ((p->west.periodic != 0) != (p->east.periodic != 0))
        return "west and east must both be periodic or both be walls";
    if ((p->south.periodic != 0) != (p->north.periodic != 0))
        return "south and north must both be periodic or both be walls";
    if (p->precision < LBM_F64 || p->precision > LBM_F16S) return "unknown precision";
    if (p->layout != LBM_DENSE && p->layout != LBM_SPARSE_TILE16) return "unknown layout";
    if (p->pattern != LBM_TWO_LATTICE && p->pattern != LBM_AA) return "unknown pattern";
    if (p->collision != LBM_BGK && p->collision != LBM_TRT) return "unknown collision";
    if (p->collision == LBM_TRT && (!std::isfinite(p->magic) || p->magic < 0.0))
        return "TRT magic parameter must be finite and >= 0 (0 = 3/16)";
    if (p->layout == LBM_SPARSE_TILE16 && p->south.periodic && p->ny % 16)
        return "sparse layout with a periodic y axis needs ny % 16 == 0";
    const lbm_side *s[4] = {&p->west, &p->east, &p->south, &p->north};
    const int nrm[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
    for (int k = 0; k < 4; ++k) {
        if (!std::isfinite(s[k]->ux) || !std::isfinite(s[k]->uy)) return "side velocity must be finite";
        if (s[k]->kind < LBM_SIDE_WALL || s[k]->kind > LBM_SIDE_PRESSURE) return "unknown side kind";
        if (s[k]->periodic && s[k]->kind != LBM_SIDE_WALL) return "a periodic side cannot be open";
        if (s[k]->kind == LBM_SIDE_PRESSURE && !(s[k]->rho > 0.0 && std::isfinite(s[k]->rho)))
            return "pressure side needs a finite density > 0";
        if (s[k]->kind == LBM_SIDE_VELOCITY && !(std::fabs(s[k]->ux * nrm[k][0] + s[k]->uy * nrm[k][1]) < 1.0))
            return "velocity side needs |u.n| < 1";
    }
    const bool open_x = s[0]->kind != LBM_SIDE_WALL || s[1]->kind != LBM_SIDE_WALL;
    const bool open_y = s[2]->kind != LBM_SIDE_WALL || s[3]->kind != LBM_SIDE_WALL;
    if (open_x && open_y) return "two adjacent sides cannot both be open";
    return nullptr;
}

struct Plan {
    long long nfluid;
    int ntiles, ntx, nty;
    bool has_mask;
    long long nslot;
    size_t off_lat1, off_mask, off_nbr, off_txy, off_tid, off_part, off_out, off_tb, off_list2, off_list4, off_vmask,
        off_order, off_hmask, off_sec, total;
    size_t lat_bytes, mask_bytes;
    bool use_list;
};

// Sparse layout: tile masks [ntiles][256] and the lists of vectors of 2 and
// of 4 nodes (along a tile row) that hold a fluid node, entry t * TPT + k for
// the k-th vector of tile t (TPT = 128 or 64), in tile order.
struct SparseTables {
    std::vector<uint8_t> tmask;
    std::vector<uint32_t> list2, list4;
    size_t fluid2 = 0; // 2-node vectors of the kept tiles that hold fluid
    // per tile 4 words: bit 8 * (row % 4) + v of word row / 4 set iff 2-node
    // vector v of that row holds a fluid node
    std::vector<uint32_t> vmask;
    // per tile 128 bytes: the 2-node vectors (8 * row + v) of the DRAM
    // sectors (32 bytes of one slot) that hold a fluid node, then 0xFF
    std::vector<uint8_t> order;
    // two-lattice contexts with a mask: the 32-byte sectors of a slot that
    // hold a fluid node, ascending (lbm_sector_copy)
    std::vector<uint32_t> secs;
};

// The staged step's tables: per tile, which 2-node vectors hold fluid (it
// copies only those chunks) and which it computes and stores (every vector
// of a sector that holds fluid; esize: bytes per stored value).
void build_vector_masks(int ntiles, const std::vector<uint8_t> &tmask, size_t esize, SparseTables &st) {
    st.vmask.assign((size_t)ntiles * 4, 0u);
    st.order.assign((size_t)ntiles * (TILE_N / 2), 0xFF);
    const int vps = (int)(16 / esize); // 2-node vectors per 32-byte sector
    for (int t = 0; t < ntiles; ++t) {
        int n = 0;
        for (int row = 0; row < TILE; ++row) {
            unsigned bits = 0;
            for (int v = 0; v < TILE / 2; ++v) {
                const uint8_t *m = &tmask[(size_t)t * TILE_N + row * TILE + 2 * v];
                if (m[0] != 0xFF || m[1] != 0xFF) bits |= 1u << v;
            }
            st.vmask[(size_t)t * 4 + row / 4] |= bits << (8 * (row % 4));
            for (int v = 0; v < TILE / 2; ++v) {
                const unsigned sec = ((1u << vps) - 1u) << (v / vps * vps);
                if (bits & sec) st.order[(size_t)t * (TILE_N / 2) + n++] = (uint8_t)(row * 8 + v);
            }
        }
    }
}

// The lists the tiled step can run over: the 2- and 4-node vectors of the
// kept tiles (t * TPT + position, tile order) that hold a fluid node, or,
// with sec > 0, that lie in a DRAM sector holding one (sec nodes of a tile
// row: 32 bytes of one slot).  Sector granularity lists the solid vectors of
// such a sector too (solid nodes hold 0 and are written 0), so that the
// step writes every sector it touches whole: in the FP32 two-lattice step a
// partly written sector of the other lattice costs the L2 a fill from DRAM
// (measured +4-7% on porous media at phi 0.2-0.5).  The AA steps write
// sectors they have just read, and an FP16s sector is a whole tile row, so
// they keep the fluid vectors (sec = 0).
void build_vector_lists(int ntiles, const std::vector<uint8_t> &tmask, int sec, SparseTables &st) {
    st.fluid2 = 0;
    for (int vec = 2; vec <= 4; vec += 2) {
        std::vector<uint32_t> &out = vec == 2 ? st.list2 : st.list4;
        out.clear();
        const int tpt = TILE_N / vec;
        for (int t = 0; t < ntiles; ++t)
            for (int k = 0; k < tpt; ++k) {
                const uint8_t *m = &tmask[(size_t)t * TILE_N];
                const int n0 = k * vec, s0 = sec > 0 ? n0 / sec * sec : 0;
                bool own = false, sector = false;
                for (int j = 0; j < vec; ++j) own = own || m[n0 + j] != 0xFF;
                for (int j = 0; j < sec; ++j) sector = sector || m[s0 + j] != 0xFF;
                if (sec <= 0) sector = own;
                if (vec == 2 && own) ++st.fluid2;
                if (sector) out.push_back((uint32_t)t * (uint32_t)tpt + (uint32_t)k);
            }
    }
}

// The 32-byte sectors (e consecutive nodes of a slot: 8 FP32, 16 FP16s, 4
// FP64; never across a row or tile row, nx being a multiple of 16) that hold
// a fluid node, ascending.
void fluid_sectors(const std::vector<uint8_t> &mask, long long nslot, int e, std::vector<uint32_t> &out) {
    out.clear();
    for (long long k = 0; k + e <= nslot; k += e) {
        bool f = false;
        for (int j = 0; j < e; ++j) f = f || mask[(size_t)(k + j)] != 0xFF;
        if (f) out.push_back((uint32_t)(k / e));
    }
}

// The staged step's halo masks: per tile 4 words, bit h of word h / 32 set
// iff halo chunk h (halo_source, E values of esize bytes) comes from an
// existing neighbour (nbr3: [tile][3 x 3]) and its E source nodes include a
// fluid node.  Only unbounced pulls read a halo value, and they pull from
// fluid nodes, so the other chunks need not be read.
void build_halo_masks(int ntiles, const std::vector<uint8_t> &tmask, const std::vector<int32_t> &nbr3, size_t esize,
                      std::vector<uint32_t> &out) {
    const int E = (int)(16 / esize);
    const int nh = halo_chunks(E) < 128 ? halo_chunks(E) : 128;
    out.assign((size_t)ntiles * 4, 0u);
    for (int t = 0; t < ntiles; ++t)
        for (int h = 0; h < nh; ++h) {
            const HaloSrc hs = halo_source(h, E);
            const int n = nbr3[(size_t)t * 9 + hs.dir];
            if (n < 0) continue;
            bool f = false;
            for (int j = 0; j < E; ++j) f = f || tmask[(size_t)n * TILE_N + hs.srow * TILE + hs.scol + j] != 0xFF;
            if (f) out[(size_t)t * 4 + h / 32] |= 1u << (h % 32);
        }
}

// Geometry tables and the workspace layout for p.
void make_plan(const lbm_params &p, std::vector<uint8_t> &mask, std::vector<int32_t> &tile_id,
               std::vector<int32_t> &nbr, std::vector<int32_t> &txy, SparseTables &sp, Plan &pl) {
    const long long N = (long long)p.nx * p.ny;
    mask.assign((size_t)N, 0);
    pl.nfluid = build_link_mask(p, mask.data());
    bool any = false;
    for (long long n = 0; n < N && !any; ++n) any = mask[(size_t)n] != 0;
    pl.ntx = (p.nx + TILE - 1) / TILE;
    pl.nty = (p.ny + TILE - 1) / TILE;
    pl.ntiles = 0;
    if (p.layout == LBM_SPARSE_TILE16) {
        tile_id.assign((size_t)pl.ntx * pl.nty, -1);
        txy.assign((size_t)pl.ntx * pl.nty, 0);
        nbr.assign((size_t)pl.ntx * pl.nty * 9, -1);
        pl.ntiles = build_tile_map(p, mask.data(), tile_id.data(), nbr.data(), txy.data());
        txy.resize((size_t)pl.ntiles);
        nbr.resize((size_t)pl.ntiles * 9);
        // a tiled geometry without any bounced link (all fluid, both axes
        // periodic) runs the unmasked kernels, as the dense layout does
        pl.has_mask = any;
        pl.nslot = (long long)pl.ntiles * TILE_N;
        sp.tmask.assign((size_t)pl.ntiles * TILE_N, 0xFF);
        if (pl.ntiles > 0) build_tile_masks(p, mask.data(), txy.data(), pl.ntiles, sp.tmask.data());
        // sector granularity (8 nodes = 32 bytes of FP32) for the FP32
        // two-lattice step only
        const bool sectors = p.precision == LBM_F32 && p.pattern == LBM_TWO_LATTICE;
        build_vector_lists(pl.ntiles, sp.tmask, sectors ? 8 : 0, sp);
        build_vector_masks(pl.ntiles, sp.tmask, elem_size(p.precision), sp);
    } else {
        pl.has_mask = any;
        pl.nslot = N;
    }
    const size_t es = elem_size(p.precision);
    pl.lat_bytes = (size_t)9 * (size_t)pl.nslot * es;
    size_t off = align256(pl.lat_bytes);
    pl.off_lat1 = off;
    if (p.pattern == LBM_TWO_LATTICE) off += align256(pl.lat_bytes);
    pl.off_mask = off;
    pl.mask_bytes = p.layout == LBM_SPARSE_TILE16 ? (size_t)pl.ntiles * TILE_N : (pl.has_mask ? (size_t)N : 0);
    off += align256(pl.mask_bytes);
    pl.off_nbr = off;
    if (p.layout == LBM_SPARSE_TILE16) off += align256((size_t)pl.ntiles * 9 * 4);
    pl.off_txy = off;
    if (p.layout == LBM_SPARSE_TILE16) off += align256((size_t)pl.ntiles * 4);
    pl.off_tid = off;
    if (p.layout == LBM_SPARSE_TILE16) off += align256((size_t)pl.ntx * pl.nty * 4);
    pl.off_part = off;
    off += align256((size_t)RED_BLOCKS * 4 * sizeof(double));
    pl.off_out = off;
    off += align256(4 * sizeof(double));
    pl.off_tb = off;
    off += align256(sizeof(unsigned long long));
    // the list pays off when a good part of the kept tiles' vectors is solid
    // (measured on 4096^2 disc media: +10-33% at 42% active vectors, -3% at 87%)
    pl.use_list = p.layout == LBM_SPARSE_TILE16 && pl.ntiles > 0 &&
                  (double)sp.fluid2 < 0.85 * (double)pl.ntiles * (TILE_N / 2);
    pl.off_list2 = off;
    if (pl.use_list) off += align256(sp.list2.size() * 4);
    pl.off_list4 = off;
    if (pl.use_list) off += align256(sp.list4.size() * 4);
    pl.off_vmask = off;
    if (p.layout == LBM_SPARSE_TILE16) off += align256((size_t)pl.ntiles * 16);
    pl.off_order = off;
    if (p.layout == LBM_SPARSE_TILE16) off += align256((size_t)pl.ntiles * (TILE_N / 2));
    pl.off_hmask = off;
    if (p.layout == LBM_SPARSE_TILE16) off += align256((size_t)pl.ntiles * 16);
    // the sector copy's list (two-lattice with a mask; without one every
    // sector holds fluid)
    sp.secs.clear();
    if (p.pattern == LBM_TWO_LATTICE && (p.layout == LBM_SPARSE_TILE16 || pl.has_mask))
        fluid_sectors(p.layout == LBM_SPARSE_TILE16 ? sp.tmask : mask, pl.nslot, 32 / (int)es, sp.secs);
    pl.off_sec = off;
    off += align256(sp.secs.size() * 4);
    pl.total = off;
}

// Measurement aid: the listed 32-byte sectors (list NULL: every sector) of
// all nine slots, copied src -> dst in uint4 units.  Sector k of a slot is
// sector k % sb of block k / sb, a block being the whole slot in the dense
// layout (f[i][y][x], sb = the slot's sectors) and one tile in the tiled
// layout (f[tile][i][256], sb = a tile slot's sectors).  SLOT_MAJOR false:
// consecutive threads take the 18 halves (9 slots x 2) of one sector, so a
// warp's accesses stay within about two tiles' 9 KB (tiled layout);
// true: consecutive threads take 16 consecutive listed sectors of one slot
// (dense layout, whose slots lie nslot elements apart).
constexpr int SC_BLOCK = 256;
template <bool SLOT_MAJOR>
__global__ void __launch_bounds__(SC_BLOCK) k_sector_copy(const uint4 *src, uint4 *dst, const uint32_t *list,
                                                          long long nsec, long long sb) {
    // threads: 18 per sector (SLOT_MAJOR: 288 per group of 16 sectors, the
    // last group possibly partial)
    const long long tot = SLOT_MAJOR ? (nsec + 15) / 16 * 288 : nsec * 18;
    for (long long q = (long long)blockIdx.x * SC_BLOCK + threadIdx.x; q < tot; q += (long long)gridDim.x * SC_BLOCK) {
        long long e;
        int i, h;
        if constexpr (SLOT_MAJOR) {
            // groups of 16 sectors: 9 slots x 32 threads (16 sectors x 2 halves)
            const long long grp = q / 288;
            const int w = (int)(q - 288 * grp);
            i = w >> 5;
            e = grp * 16 + ((w & 31) >> 1);
            h = w & 1;
            if (e >= nsec) continue;
        } else {
            e = q / 18;
            const int r = (int)(q - 18 * e);
            i = r >> 1;
            h = r & 1;
        }
        const long long k = list ? (long long)__ldg(list + e) : e;
        const long long blk = k / sb;
        const long long off = (blk * 9 + i) * (2 * sb) + 2 * (k - blk * sb) + h;
        dst[off] = src[off];
    }
}

lbm_status fail(lbm_ctx *c, lbm_status s, const std::string &msg) {
    if (c) {
        if (s == LBM_ERR_CUDA) c->sticky = s;
        c->err = msg;
    }
    return s;
}

lbm_status cuda_check(lbm_ctx *c, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return LBM_OK;
    return fail(c, LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LBM_DISPATCH(prec, expr)                       \
    ([&]() -> cudaError_t {                            \
        switch (prec) {                                \
        case LBM_F64: { constexpr int P = LBM_F64; return expr; } \
        case LBM_F32: { constexpr int P = LBM_F32; return expr; } \
        default: { constexpr int P = LBM_F16S; return expr; }     \
        }                                              \
    }())

#define LBM_CTX_CHECK(ctx)                                   \
    do {                                                     \
        if (!(ctx)) return LBM_ERR_INVALID;                  \
        if ((ctx)->sticky != LBM_OK) return (ctx)->sticky;   \
    } while (0)

void set_force_mode(lbm_ctx *c) {
    if (c->phys.force) c->phys.force_mode = FORCE_FIELD;
    else if (c->phys.fx != 0.0 || c->phys.fy != 0.0) c->phys.force_mode = FORCE_UNIFORM;
    else c->phys.force_mode = FORCE_NONE;
}

void *current_lattice(lbm_ctx *c) { return c->p.pattern == LBM_AA ? c->lat[0] : c->lat[c->cur]; }
int current_phase(lbm_ctx *c) { return c->p.pattern == LBM_AA ? c->phase : PH_PLAIN; }

// One time step from lattice state (cur, phase), which it advances; t is the
// step's index (or its offset from *ph.tbase).
cudaError_t launch_one_step(lbm_ctx *c, const Phys &ph, int &cur, int &phase, unsigned long long t,
                            cudaStream_t s) {
    cudaError_t e;
    if (c->p.pattern == LBM_TWO_LATTICE) {
        e = LBM_DISPATCH(c->p.precision,
                         launch_step<P>(c->geo, ph, MODE_TWO_LATTICE, c->lat[cur], c->lat[1 - cur], t, s));
        cur = 1 - cur;
    } else {
        const int mode = phase == PH_SWAPPED ? MODE_AA_PULLPUSH : MODE_AA_LOCAL;
        e = LBM_DISPATCH(c->p.precision, launch_step<P>(c->geo, ph, mode, c->lat[0], c->lat[0], t, s));
        phase = phase == PH_SWAPPED ? PH_STREAMED : PH_SWAPPED;
    }
    return e;
}

// ---- CUDA graphs

// cache slots: lbm_step's chunk from either lattice parity (a run of odd
// length leaves the other one), the recompute, the adjoint sweep
enum { GC_STEP = 0, GC_FWD = 2, GC_BWD = 3 };
constexpr int GRAPH_CHUNK = 32; // steps per replay of lbm_step's graph (even)
constexpr int GRAPH_MIN = 8;    // shortest forward_states / backward run recorded

__global__ void k_counter(unsigned long long *c, unsigned long long v, int add) {
    if (add) *c += v;
    else *c = v;
}
cudaError_t set_counter(unsigned long long *c, unsigned long long v, cudaStream_t s) {
    k_counter<<<1, 1, 0, s>>>(c, v, 0);
    return cudaGetLastError();
}

// Destroys the recorded graphs (after the work they may have in flight).
void drop_graphs(lbm_ctx *c) {
    bool any = false;
    for (auto &g : c->gc) any = any || g.exec;
    if (!any) return;
    cudaStreamSynchronize(c->stream);
    for (auto &g : c->gc) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
        g.key.clear();
    }
}

// A graph could not be recorded or launched: clear the (non-sticky) error and
// issue this context's launches directly from now on.
void graphs_failed(lbm_ctx *c) {
    cudaGetLastError();
    c->graphs = 0;
}

// Launches cache slot `which`, recording it first with record(stream) when
// its key differs from the one it was recorded with.
template <class F>
cudaError_t replay(lbm_ctx *c, int which, const std::vector<unsigned long long> &key, F record) {
    lbm_ctx::GraphCache &gc = c->gc[which];
    if (!gc.exec || gc.key != key) {
        if (gc.exec) {
            cudaStreamSynchronize(c->stream); // the old graph may still run
            cudaGraphExecDestroy(gc.exec);
            gc.exec = nullptr;
            gc.key.clear();
        }
        cudaError_t e = cudaSuccess;
        if (!c->cap) e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        const cudaError_t er = record(c->cap);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(c->cap, &graph);
        if (er != cudaSuccess) e = er;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&gc.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            gc.exec = nullptr;
            return e;
        }
        gc.key = key;
    }
    return cudaGraphLaunch(gc.exec, c->stream);
}

// GRAPH_CHUNK steps from the context's (cur, phase), time-step indices read
// from the device counter, which the last node advances by GRAPH_CHUNK.
cudaError_t record_steps(lbm_ctx *c, cudaStream_t s) {
    Phys ph = c->phys;
    ph.tbase = c->tb;
    int cur = c->cur, phase = c->phase;
    for (int j = 0; j < GRAPH_CHUNK; ++j) {
        const cudaError_t e = launch_one_step(c, ph, cur, phase, (unsigned long long)j, s);
        if (e != cudaSuccess) return e;
    }
    k_counter<<<1, 1, 0, s>>>(c->tb, (unsigned long long)GRAPH_CHUNK, 1);
    return cudaGetLastError();
}

} // namespace

extern "C" {

const char *lbm_status_string(lbm_status s) {
    switch (s) {
    case LBM_OK: return "ok";
    case LBM_ERR_INVALID: return "invalid argument";
    case LBM_ERR_CUDA: return "CUDA error";
    case LBM_ERR_OOM: return "workspace too small";
    case LBM_ERR_DIVERGED: return "diverged (NaN/Inf)";
    case LBM_ERR_TIMEOUT: return "timeout";
    case LBM_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

lbm_status lbm_workspace_bytes(const lbm_params *p, size_t *bytes) {
    if (!bytes || check_params(p)) return LBM_ERR_INVALID;
    std::vector<uint8_t> mask;
    std::vector<int32_t> tid, nbr, txy;
    SparseTables sp;
    Plan pl;
    make_plan(*p, mask, tid, nbr, txy, sp, pl);
    if (9ll * pl.nslot >= (1ll << 32)) return LBM_ERR_INVALID;
    *bytes = pl.total;
    return LBM_OK;
}

lbm_status lbm_create(const lbm_params *p, void *d_workspace, size_t bytes, lbm_ctx **out) {
    if (!out) return LBM_ERR_INVALID;
    *out = nullptr;
    if (check_params(p)) return LBM_ERR_INVALID;
    if (!d_workspace || ((uintptr_t)d_workspace & 255)) return LBM_ERR_INVALID;
    lbm_ctx *c = new lbm_ctx();
    c->p = *p;
    c->p.solid = nullptr;
    c->stream = (cudaStream_t)p->stream;
    c->sticky = LBM_OK;
    std::vector<int32_t> txy;
    SparseTables sp;
    Plan pl;
    make_plan(*p, c->mask, c->tile_id, c->nbr, txy, sp, pl);
    if (9ll * pl.nslot >= (1ll << 32)) {
        delete c;
        return LBM_ERR_INVALID;
    }
    if (bytes < pl.total) {
        delete c;
        return LBM_ERR_OOM;
    }
    c->esize = elem_size(p->precision);
    c->csize = comp_size(p->precision);
    c->nfluid = pl.nfluid;
    const bool listed = p->pattern == LBM_TWO_LATTICE && (p->layout == LBM_SPARSE_TILE16 || pl.has_mask);
    c->fluid_sectors = listed ? (long long)sp.secs.size() : pl.nslot * (long long)elem_size(p->precision) / 32;
    c->secs = listed ? reinterpret_cast<const uint32_t *>(reinterpret_cast<char *>(d_workspace) + pl.off_sec)
                     : nullptr;
    c->lat_bytes = pl.lat_bytes;
    char *ws = reinterpret_cast<char *>(d_workspace);
    c->lat[0] = ws;
    c->lat[1] = p->pattern == LBM_TWO_LATTICE ? ws + pl.off_lat1 : ws;
    c->partial = reinterpret_cast<double *>(ws + pl.off_part);
    c->red_out = reinterpret_cast<double *>(ws + pl.off_out);
    c->tb = reinterpret_cast<unsigned long long *>(ws + pl.off_tb);
    // the error word shares the counter's 256-byte region
    unsigned *err_word = reinterpret_cast<unsigned *>(ws + pl.off_tb + 16);
    c->cur = 0;
    c->phase = p->pattern == LBM_AA ? PH_SWAPPED : PH_PLAIN;
    c->steps = 0;

    Geo &g = c->geo;
    std::memset(&g, 0, sizeof(g));
    g.nx = p->nx;
    g.ny = p->ny;
    g.periodic_x = p->west.periodic != 0;
    g.periodic_y = p->south.periodic != 0;
    g.layout = p->layout;
    g.ntx = pl.ntx;
    g.nty = pl.nty;
    g.ntiles = pl.ntiles;
    g.nslot = pl.nslot;
    g.nnode = (long long)p->nx * p->ny;
    g.has_mask = pl.has_mask;
    // the split costs a second launch (a few microseconds): worth it on large
    // grids only
    if (p->layout == LBM_DENSE && pl.has_mask && p->ny >= 3 && (long long)p->nx * p->ny > (1ll << 21)) {
        bool inner_free = true;
        for (size_t n = (size_t)p->nx; n < (size_t)p->nx * (size_t)(p->ny - 1) && inner_free; ++n)
            inner_free = c->mask[n] == 0;
        g.frame_y = inner_free;
    }
    g.mask = pl.mask_bytes ? reinterpret_cast<const uint8_t *>(ws + pl.off_mask) : nullptr;
    g.err = err_word;

    Phys &ph = c->phys;
    std::memset(&ph, 0, sizeof(ph));
    ph.omega = 1.0 / p->tau;
    ph.fx = p->fx;
    ph.fy = p->fy;
    const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1}, CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const double W[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    const lbm_side *sides[4] = {&p->west, &p->east, &p->south, &p->north};
    for (int s = 0; s < 4; ++s) {
        const bool wall = !sides[s]->periodic && sides[s]->kind == LBM_SIDE_WALL;
        for (int i = 0; i < 9; ++i) {
            // half-way bounce-back on a wall moving at u_w, rho_w = rho_0 = 1
            ph.wt[s][i] = wall ? 6.0 * W[i] * (CX[i] * sides[s]->ux + CY[i] * sides[s]->uy) : 0.0;
            if (ph.wt[s][i] != 0.0) ph.has_wall = 1;
        }
        ph.open_kind[s] = sides[s]->periodic ? LBM_SIDE_WALL : sides[s]->kind;
        if (ph.open_kind[s] != LBM_SIDE_WALL) ph.has_open = 1;
        ph.open_u[s][0] = sides[s]->ux;
        ph.open_u[s][1] = sides[s]->uy;
        ph.open_rho[s] = sides[s]->rho;
        ph.open_u_f[s][0] = (float)sides[s]->ux;
        ph.open_u_f[s][1] = (float)sides[s]->uy;
        ph.open_rho_f[s] = (float)sides[s]->rho;
    }
    // FP32 constants from the rounded omega in FP32 arithmetic, so that
    // om1_f + omega_f == 1 exactly (1 - omega is exact for omega in (0, 2)):
    // otherwise BGK would scale mass and momentum by (om1 + omega) each step.
    ph.omega_f = (float)ph.omega;
    ph.om1_f = 1.0f - ph.omega_f;
    ph.kk_f = 1.0f - 0.5f * ph.omega_f;
    ph.fx_f = (float)ph.fx;
    ph.fy_f = (float)ph.fy;
    for (int s = 0; s < WALL_SIDES; ++s)
        for (int i = 0; i < 9; ++i) ph.wt_f[s][i] = (float)ph.wt[s][i];
    ph.kq[0] = ph.omega / 3.0;
    ph.kq[1] = ph.omega / 12.0;
    for (int q = 0; q < 2; ++q) {
        const double k = (double)ph.omega_f / (q == 0 ? 3.0 : 12.0);
        ph.kq_hi[q] = (float)k;
        ph.kq_lo[q] = (float)(k - (double)ph.kq_hi[q]);
    }
    ph.tau_h = 1.0 / ph.omega - 0.5;
    ph.tau_h_f = (float)(1.0 / (double)ph.omega_f - 0.5);
    // two-relaxation-time: odd rate from Lambda = (1/omega - 1/2)(1/omega_m - 1/2)
    ph.trt = p->collision == LBM_TRT;
    {
        const double lam = p->magic > 0.0 ? p->magic : 3.0 / 16.0;
        ph.omega_m = ph.trt ? 1.0 / (0.5 + lam / (p->tau - 0.5)) : ph.omega;
        ph.tp = 0.5 * (1.0 - ph.omega);
        ph.tm = 0.5 * (1.0 - ph.omega_m);
        ph.kqm[0] = ph.omega_m / 3.0;
        ph.kqm[1] = ph.omega_m / 12.0;
        ph.thm = 1.0 / ph.omega_m - 0.5;
        const float omf = (float)ph.omega_m;
        ph.tp_f = 0.5f * ph.om1_f;   // exact: om1_f = 1 - omega_f exactly
        ph.tm_f = 0.5f * (1.0f - omf);
        for (int q = 0; q < 2; ++q) {
            const double k = (double)omf / (q == 0 ? 3.0 : 12.0);
            ph.kqm_hi[q] = (float)k;
            ph.kqm_lo[q] = (float)(k - (double)ph.kqm_hi[q]);
        }
        ph.thm_f = (float)(1.0 / (double)omf - 0.5);
        ph.kkm_f = 1.0f - 0.5f * omf;
    }
    set_force_mode(c);

    lbm_status st = LBM_OK;
    cudaStream_t s = c->stream;
    st = cuda_check(c, cudaMemsetAsync(c->lat[0], 0, pl.lat_bytes, s), "memset lattice");
    if (!st) st = cuda_check(c, cudaMemsetAsync(ws + pl.off_tb, 0, 256, s), "memset counter");
    if (!st && p->pattern == LBM_TWO_LATTICE)
        st = cuda_check(c, cudaMemsetAsync(c->lat[1], 0, pl.lat_bytes, s), "memset lattice");
    if (!st && !sp.secs.empty())
        st = cuda_check(c, cudaMemcpyAsync(ws + pl.off_sec, sp.secs.data(), sp.secs.size() * 4,
                                           cudaMemcpyHostToDevice, s), "copy sector list");
    if (!st && p->layout == LBM_DENSE && pl.mask_bytes)
        st = cuda_check(c, cudaMemcpyAsync(ws + pl.off_mask, c->mask.data(), pl.mask_bytes,
                                           cudaMemcpyHostToDevice, s), "copy mask");
    std::vector<int32_t> nbr3;
    const std::vector<uint8_t> &tmask = sp.tmask;
    if (!st && p->layout == LBM_SPARSE_TILE16 && pl.ntiles > 0) {
        // device neighbour table in 3x3 order: [t][3*(oy+1) + (ox+1)]
        nbr3.resize((size_t)pl.ntiles * 9);
        for (int t = 0; t < pl.ntiles; ++t)
            for (int i = 0; i < 9; ++i)
                nbr3[(size_t)t * 9 + 3 * (CY[i] + 1) + (CX[i] + 1)] = c->nbr[(size_t)t * 9 + i];
        st = cuda_check(c, cudaMemcpyAsync(ws + pl.off_mask, tmask.data(), tmask.size(),
                                           cudaMemcpyHostToDevice, s), "copy tile masks");
        if (!st)
            st = cuda_check(c, cudaMemcpyAsync(ws + pl.off_nbr, nbr3.data(), nbr3.size() * 4,
                                               cudaMemcpyHostToDevice, s), "copy neighbour table");
        if (!st)
            st = cuda_check(c, cudaMemcpyAsync(ws + pl.off_txy, txy.data(), txy.size() * 4,
                                               cudaMemcpyHostToDevice, s), "copy tile coordinates");
        if (!st)
            st = cuda_check(c, cudaMemcpyAsync(ws + pl.off_tid, c->tile_id.data(), c->tile_id.size() * 4,
                                               cudaMemcpyHostToDevice, s), "copy tile ids");
        if (!st && pl.use_list && !sp.list2.empty())
            st = cuda_check(c, cudaMemcpyAsync(ws + pl.off_list2, sp.list2.data(), sp.list2.size() * 4,
                                               cudaMemcpyHostToDevice, s), "copy vector list");
        if (!st && pl.use_list && !sp.list4.empty())
            st = cuda_check(c, cudaMemcpyAsync(ws + pl.off_list4, sp.list4.data(), sp.list4.size() * 4,
                                               cudaMemcpyHostToDevice, s), "copy vector list");
        if (!st)
            st = cuda_check(c, cudaMemcpyAsync(ws + pl.off_vmask, sp.vmask.data(), sp.vmask.size() * 4,
                                               cudaMemcpyHostToDevice, s), "copy vector masks");
        if (!st)
            st = cuda_check(c, cudaMemcpyAsync(ws + pl.off_order, sp.order.data(), sp.order.size(),
                                               cudaMemcpyHostToDevice, s), "copy vector order");
        std::vector<uint32_t> hmask;
        build_halo_masks(pl.ntiles, tmask, nbr3, elem_size(p->precision), hmask);
        if (!st)
            st = cuda_check(c, cudaMemcpyAsync(ws + pl.off_hmask, hmask.data(), hmask.size() * 4,
                                               cudaMemcpyHostToDevice, s), "copy halo masks");
        if (!st) st = cuda_check(c, cudaStreamSynchronize(s), "upload tables");
        g.tile_hmask = reinterpret_cast<const uint4 *>(ws + pl.off_hmask);
        g.tile_vmask = reinterpret_cast<const uint4 *>(ws + pl.off_vmask);
        g.tile_order = reinterpret_cast<const uint8_t *>(ws + pl.off_order);
        g.nbr = reinterpret_cast<const int32_t *>(ws + pl.off_nbr);
        g.tile_xy = reinterpret_cast<const int32_t *>(ws + pl.off_txy);
        g.tile_id = reinterpret_cast<const int32_t *>(ws + pl.off_tid);
        g.use_list = pl.use_list;
        g.active_frac = (float)((double)sp.fluid2 / ((double)pl.ntiles * (TILE_N / 2)));
        g.nlist2 = (int)sp.list2.size();
        g.nlist4 = (int)sp.list4.size();
        g.vlist2 = reinterpret_cast<const unsigned *>(ws + pl.off_list2);
        g.vlist4 = reinterpret_cast<const unsigned *>(ws + pl.off_list4);
    } else if (p->layout == LBM_SPARSE_TILE16) {
        g.tile_id = reinterpret_cast<const int32_t *>(ws + pl.off_tid);
        if (!st)
            st = cuda_check(c, cudaMemcpyAsync(ws + pl.off_tid, c->tile_id.data(), c->tile_id.size() * 4,
                                               cudaMemcpyHostToDevice, s), "copy tile ids");
    }
    if (!st)
        st = cuda_check(c, LBM_DISPATCH(p->precision, launch_init<P>(g, current_phase(c), nullptr, nullptr,
                                                                     current_lattice(c), s)),
                        "init kernel");
    if (!st) st = cuda_check(c, cudaStreamSynchronize(s), "create sync");
    if (st) {
        delete c;
        return st;
    }
    *out = c;
    return LBM_OK;
}

lbm_status lbm_destroy(lbm_ctx *ctx) {
    if (!ctx) return LBM_ERR_INVALID;
    drop_graphs(ctx);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    delete ctx;
    return LBM_OK;
}

lbm_status lbm_sector_copy(lbm_ctx *ctx, int n, long long *h_bytes) {
    LBM_CTX_CHECK(ctx);
    if (n < 0) return fail(ctx, LBM_ERR_INVALID, "n < 0");
    if (ctx->p.pattern != LBM_TWO_LATTICE)
        return fail(ctx, LBM_ERR_UNSUPPORTED, "the sector copy writes the other lattice of a two-lattice context");
    const bool tiled = ctx->geo.layout == LBM_SPARSE_TILE16;
    const long long sb = (tiled ? (long long)TILE_N : ctx->geo.nslot) * (long long)ctx->esize / 32;
    if (h_bytes) *h_bytes = 2ll * 9 * 32 * ctx->fluid_sectors;
    if (n == 0 || ctx->fluid_sectors == 0) return LBM_OK;
    // eight blocks per SM, grid-stride (measured best for this copy)
    static const int grid = [] {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        return (sms > 0 ? sms : 1) * 8;
    }();
    const uint4 *src = reinterpret_cast<const uint4 *>(ctx->lat[ctx->cur]);
    uint4 *dst = reinterpret_cast<uint4 *>(ctx->lat[1 - ctx->cur]);
#ifndef LBM_SC_DENSE_SLOT_MAJOR
#define LBM_SC_DENSE_SLOT_MAJOR 1
#endif
    for (int j = 0; j < n; ++j) {
        if (tiled || !LBM_SC_DENSE_SLOT_MAJOR)
            k_sector_copy<false><<<grid, SC_BLOCK, 0, ctx->stream>>>(src, dst, ctx->secs, ctx->fluid_sectors, sb);
        else
            k_sector_copy<true><<<grid, SC_BLOCK, 0, ctx->stream>>>(src, dst, ctx->secs, ctx->fluid_sectors, sb);
    }
    return cuda_check(ctx, cudaGetLastError(), "sector copy launch");
}

lbm_status lbm_set_graphs(lbm_ctx *ctx, int enable) {
    LBM_CTX_CHECK(ctx);
    ctx->graphs = enable != 0;
    return LBM_OK;
}

lbm_status lbm_set_side_values(lbm_ctx *ctx, int side, const void *d_values) {
    LBM_CTX_CHECK(ctx);
    if (side < 0 || side > 3 || ctx->phys.open_kind[side] == LBM_SIDE_WALL)
        return fail(ctx, LBM_ERR_INVALID, "side is not open");
    if (d_values && ((uintptr_t)d_values % ctx->csize)) return fail(ctx, LBM_ERR_INVALID, "values not aligned");
    ctx->phys.open_val[side] = d_values;
    ++ctx->version;
    return LBM_OK;
}

lbm_status lbm_set_force(lbm_ctx *ctx, const void *d_force) {
    LBM_CTX_CHECK(ctx);
    if (d_force && ((uintptr_t)d_force & 15)) return fail(ctx, LBM_ERR_INVALID, "force not 16-byte aligned");
    ctx->phys.force = d_force;
    set_force_mode(ctx);
    ++ctx->version;
    return LBM_OK;
}

lbm_status lbm_init_equilibrium(lbm_ctx *ctx, const void *d_rho, const void *d_u) {
    LBM_CTX_CHECK(ctx);
    if (ctx->p.pattern == LBM_AA) ctx->phase = PH_SWAPPED;
    ctx->steps = 0;
    const Geo &g = ctx->geo;
    return cuda_check(ctx, LBM_DISPATCH(ctx->p.precision, launch_init<P>(g, current_phase(ctx), d_rho, d_u,
                                                                         current_lattice(ctx), ctx->stream)),
                      "init kernel");
}

lbm_status lbm_step(lbm_ctx *ctx, int n) {
    LBM_CTX_CHECK(ctx);
    if (n < 0) return fail(ctx, LBM_ERR_INVALID, "negative step count");
    int k = 0;
    if (ctx->graphs && n >= GRAPH_CHUNK) {
        cudaError_t e = set_counter(ctx->tb, (unsigned long long)ctx->steps, ctx->stream);
        if (e != cudaSuccess) return cuda_check(ctx, e, "step counter");
        const std::vector<unsigned long long> key = {(unsigned long long)ctx->cur, (unsigned long long)ctx->phase,
                                                     ctx->version};
        const int slot = GC_STEP + (ctx->p.pattern == LBM_AA ? (ctx->phase == PH_SWAPPED ? 0 : 1) : ctx->cur);
        for (; k + GRAPH_CHUNK <= n; k += GRAPH_CHUNK) {
            e = replay(ctx, slot, key, [ctx](cudaStream_t s) { return record_steps(ctx, s); });
            if (e != cudaSuccess) {
                graphs_failed(ctx);
                break;
            }
            ctx->steps += GRAPH_CHUNK; // an even chunk: cur and phase are back
        }
    }
    for (; k < n; ++k) {
        const cudaError_t e =
            launch_one_step(ctx, ctx->phys, ctx->cur, ctx->phase, (unsigned long long)ctx->steps, ctx->stream);
        if (e != cudaSuccess) return cuda_check(ctx, e, "step kernel");
        ++ctx->steps;
    }
    return LBM_OK;
}

lbm_status lbm_macros(lbm_ctx *ctx, void *d_rho, void *d_u) {
    LBM_CTX_CHECK(ctx);
    if (!d_rho && !d_u) return LBM_OK;
    return cuda_check(ctx, LBM_DISPATCH(ctx->p.precision,
                                        launch_macros<P>(ctx->geo, ctx->phys, current_phase(ctx),
                                                         current_lattice(ctx), d_rho, d_u, ctx->stream)),
                      "macros kernel");
}

lbm_status lbm_get_f(lbm_ctx *ctx, void *d_f) {
    LBM_CTX_CHECK(ctx);
    if (!d_f) return fail(ctx, LBM_ERR_INVALID, "d_f is NULL");
    return cuda_check(ctx, LBM_DISPATCH(ctx->p.precision, launch_get_f<P>(ctx->geo, current_phase(ctx),
                                                                          current_lattice(ctx), d_f,
                                                                          ctx->stream)),
                      "get_f kernel");
}

lbm_status lbm_set_f(lbm_ctx *ctx, const void *d_f) {
    LBM_CTX_CHECK(ctx);
    if (!d_f) return fail(ctx, LBM_ERR_INVALID, "d_f is NULL");
    if (ctx->p.pattern == LBM_AA) ctx->phase = PH_SWAPPED;
    return cuda_check(ctx, LBM_DISPATCH(ctx->p.precision, launch_set_f<P>(ctx->geo, current_phase(ctx), d_f,
                                                                          current_lattice(ctx), ctx->stream)),
                      "set_f kernel");
}

static lbm_status run_reduce(lbm_ctx *ctx, int kind, const void *target, double out[4]) {
    lbm_status st = cuda_check(
        ctx, LBM_DISPATCH(ctx->p.precision, launch_reduce<P>(ctx->geo, ctx->phys, current_phase(ctx), kind,
                                                             current_lattice(ctx), target, ctx->partial,
                                                             ctx->red_out, ctx->stream)),
        "reduce kernel");
    if (st) return st;
    st = cuda_check(ctx, cudaMemcpyAsync(out, ctx->red_out, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                                         ctx->stream), "reduce copy");
    unsigned err = 0;
    if (!st)
        st = cuda_check(ctx, cudaMemcpyAsync(&err, ctx->geo.err, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                             ctx->stream), "error word copy");
    if (st) return st;
    st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "reduce sync");
    if (!st && err) {
        // a step kernel gave up waiting on its own pipeline: its results are
        // incomplete (sticky, like a CUDA error)
        ctx->sticky = LBM_ERR_TIMEOUT;
        return fail(ctx, LBM_ERR_TIMEOUT, "a step kernel's bounded wait expired");
    }
    return st;
}

lbm_status lbm_reduce(lbm_ctx *ctx, double *h_mass, double h_mom[2]) {
    LBM_CTX_CHECK(ctx);
    double out[4];
    lbm_status st = run_reduce(ctx, 0, nullptr, out);
    if (st) return st;
    // canonical values are w_i + shifted value; sum_i w_i = 1, sum_i c_i w_i = 0
    const double mass = (double)ctx->nfluid + out[0];
    if (h_mass) *h_mass = mass;
    if (h_mom) {
        h_mom[0] = out[1];
        h_mom[1] = out[2];
    }
    if (!std::isfinite(mass) || !std::isfinite(out[1]) || !std::isfinite(out[2]))
        return fail(ctx, LBM_ERR_DIVERGED, "non-finite mass or momentum");
    return LBM_OK;
}

lbm_status lbm_loss(lbm_ctx *ctx, int kind, const void *d_u_target, double *h_loss) {
    LBM_CTX_CHECK(ctx);
    if (!h_loss || (kind != 0 && kind != 1) || (kind == 0 && !d_u_target))
        return fail(ctx, LBM_ERR_INVALID, "bad loss arguments");
    double out[4];
    lbm_status st = run_reduce(ctx, kind == 0 ? 1 : 2, d_u_target, out);
    if (st) return st;
    *h_loss = kind == 0 ? (ctx->nfluid ? out[0] / (double)ctx->nfluid : 0.0) : out[0];
    if (!std::isfinite(*h_loss)) return fail(ctx, LBM_ERR_DIVERGED, "non-finite loss");
    return LBM_OK;
}

lbm_status lbm_state_bytes(const lbm_ctx *ctx, size_t *bytes) {
    if (!ctx || !bytes) return LBM_ERR_INVALID;
    *bytes = ctx->lat_bytes;
    return LBM_OK;
}

lbm_status lbm_save_state(lbm_ctx *ctx, void *d_dst) {
    LBM_CTX_CHECK(ctx);
    if (ctx->p.pattern != LBM_TWO_LATTICE) return fail(ctx, LBM_ERR_UNSUPPORTED, "checkpoints need two-lattice");
    if (!d_dst) return fail(ctx, LBM_ERR_INVALID, "d_dst is NULL");
    return cuda_check(ctx, cudaMemcpyAsync(d_dst, ctx->lat[ctx->cur], ctx->lat_bytes, cudaMemcpyDeviceToDevice,
                                           ctx->stream), "save state");
}

lbm_status lbm_load_state(lbm_ctx *ctx, const void *d_src) {
    LBM_CTX_CHECK(ctx);
    if (ctx->p.pattern != LBM_TWO_LATTICE) return fail(ctx, LBM_ERR_UNSUPPORTED, "checkpoints need two-lattice");
    if (!d_src) return fail(ctx, LBM_ERR_INVALID, "d_src is NULL");
    return cuda_check(ctx, cudaMemcpyAsync(ctx->lat[ctx->cur], d_src, ctx->lat_bytes, cudaMemcpyDeviceToDevice,
                                           ctx->stream), "load state");
}

lbm_status lbm_forward_states(lbm_ctx *ctx, void *const *h_states, int n, long long t0) {
    LBM_CTX_CHECK(ctx);
    if (ctx->p.pattern != LBM_TWO_LATTICE) return fail(ctx, LBM_ERR_UNSUPPORTED, "needs two-lattice");
    if (n < 0 || (n > 0 && !h_states)) return fail(ctx, LBM_ERR_INVALID, "bad state list");
    for (int k = 0; k < n; ++k) {
        if (!h_states[k] || !h_states[k + 1] || ((uintptr_t)h_states[k] & 15) || ((uintptr_t)h_states[k + 1] & 15))
            return fail(ctx, LBM_ERR_INVALID, "bad state pointer");
    }
    if (ctx->graphs && n >= GRAPH_MIN) {
        std::vector<unsigned long long> key = {(unsigned long long)n, ctx->version};
        for (int k = 0; k <= n; ++k) key.push_back((unsigned long long)(uintptr_t)h_states[k]);
        cudaError_t e = set_counter(ctx->tb, (unsigned long long)t0, ctx->stream);
        if (e != cudaSuccess) return cuda_check(ctx, e, "step counter");
        e = replay(ctx, GC_FWD, key, [ctx, h_states, n](cudaStream_t s) {
            Phys ph = ctx->phys;
            ph.tbase = ctx->tb;
            for (int k = 0; k < n; ++k) {
                const cudaError_t r = LBM_DISPATCH(ctx->p.precision,
                                                   launch_step<P>(ctx->geo, ph, MODE_TWO_LATTICE, h_states[k],
                                                                  h_states[k + 1], (unsigned long long)k, s));
                if (r != cudaSuccess) return r;
            }
            return cudaSuccess;
        });
        if (e == cudaSuccess) return LBM_OK;
        graphs_failed(ctx);
    }
    for (int k = 0; k < n; ++k) {
        cudaError_t e = LBM_DISPATCH(ctx->p.precision,
                                     launch_step<P>(ctx->geo, ctx->phys, MODE_TWO_LATTICE, h_states[k],
                                                    h_states[k + 1], (unsigned long long)(t0 + k), ctx->stream));
        if (e != cudaSuccess) return cuda_check(ctx, e, "forward_states kernel");
    }
    return LBM_OK;
}

lbm_status lbm_backward(lbm_ctx *ctx, const void *const *h_states, int n, void *d_lambda, void *d_lambda_tmp,
                        void *d_grad_force) {
    LBM_CTX_CHECK(ctx);
    if (ctx->p.layout != LBM_DENSE || ctx->p.pattern != LBM_TWO_LATTICE || ctx->phys.trt)
        return fail(ctx, LBM_ERR_UNSUPPORTED, "adjoint needs the dense two-lattice BGK configuration");
    if (n < 0 || (n > 0 && (!h_states || !d_lambda || !d_lambda_tmp || !d_grad_force)))
        return fail(ctx, LBM_ERR_INVALID, "bad backward arguments");
    if (((uintptr_t)d_lambda & 15) || ((uintptr_t)d_lambda_tmp & 15) || ((uintptr_t)d_grad_force & 15))
        return fail(ctx, LBM_ERR_INVALID, "buffers must be 16-byte aligned");
    for (int t = 0; t < n; ++t)
        if (!h_states[t]) return fail(ctx, LBM_ERR_INVALID, "NULL state");
    // the n adjoint steps, lambda ping-ponging between the two buffers and
    // ending in d_lambda
    auto sweep = [ctx, h_states, n, d_lambda, d_lambda_tmp, d_grad_force](cudaStream_t s) {
        void *in = d_lambda, *out = d_lambda_tmp;
        for (int t = n - 1; t >= 0; --t) {
            const cudaError_t e = LBM_DISPATCH(ctx->p.precision, launch_adjoint<P>(ctx->geo, ctx->phys, h_states[t],
                                                                                   in, out, d_grad_force, s));
            if (e != cudaSuccess) return e;
            void *tmp = in;
            in = out;
            out = tmp;
        }
        if (in != d_lambda)
            return cudaMemcpyAsync(d_lambda, in, (size_t)9 * ctx->geo.nnode * ctx->csize, cudaMemcpyDeviceToDevice,
                                   s);
        return cudaSuccess;
    };
    if (ctx->graphs && n >= GRAPH_MIN) {
        std::vector<unsigned long long> key = {(unsigned long long)n, ctx->version,
                                               (unsigned long long)(uintptr_t)d_lambda,
                                               (unsigned long long)(uintptr_t)d_lambda_tmp,
                                               (unsigned long long)(uintptr_t)d_grad_force};
        for (int t = 0; t < n; ++t) key.push_back((unsigned long long)(uintptr_t)h_states[t]);
        if (replay(ctx, GC_BWD, key, sweep) == cudaSuccess) return LBM_OK;
        graphs_failed(ctx);
    }
    return cuda_check(ctx, sweep(ctx->stream), "adjoint kernel");
}

lbm_status lbm_macros_backward(lbm_ctx *ctx, const void *d_grad_rho, const void *d_grad_u, void *d_lambda,
                               void *d_grad_force) {
    LBM_CTX_CHECK(ctx);
    if (ctx->p.layout != LBM_DENSE || ctx->p.pattern != LBM_TWO_LATTICE || ctx->phys.trt)
        return fail(ctx, LBM_ERR_UNSUPPORTED, "adjoint needs the dense two-lattice BGK configuration");
    if (!d_lambda) return fail(ctx, LBM_ERR_INVALID, "d_lambda is NULL");
    return cuda_check(ctx, LBM_DISPATCH(ctx->p.precision,
                                        launch_macros_adjoint<P>(ctx->geo, ctx->phys, ctx->lat[ctx->cur],
                                                                 d_grad_rho, d_grad_u, d_lambda, d_grad_force,
                                                                 ctx->stream)),
                      "macros adjoint kernel");
}

lbm_status lbm_link_mask(const lbm_ctx *ctx, uint8_t *h_mask) {
    if (!ctx || !h_mask) return LBM_ERR_INVALID;
    std::memcpy(h_mask, ctx->mask.data(), ctx->mask.size());
    return LBM_OK;
}

lbm_status lbm_tile_map(const lbm_ctx *ctx, int32_t *h_tile_id, int32_t *h_nbr, int *h_ntiles) {
    if (!ctx) return LBM_ERR_INVALID;
    if (ctx->p.layout != LBM_SPARSE_TILE16) return LBM_ERR_UNSUPPORTED;
    if (h_tile_id) std::memcpy(h_tile_id, ctx->tile_id.data(), ctx->tile_id.size() * 4);
    if (h_nbr) std::memcpy(h_nbr, ctx->nbr.data(), ctx->nbr.size() * 4);
    if (h_ntiles) *h_ntiles = ctx->geo.ntiles;
    return LBM_OK;
}

lbm_status lbm_geometry(const lbm_params *p, uint8_t *h_mask, int32_t *h_tile_id, int32_t *h_nbr,
                        int *h_ntiles, long long *h_nfluid) {
    if (check_params(p)) return LBM_ERR_INVALID;
    std::vector<uint8_t> mask;
    std::vector<int32_t> tid, nbr, txy;
    SparseTables sp;
    Plan pl;
    make_plan(*p, mask, tid, nbr, txy, sp, pl);
    if (h_mask) std::memcpy(h_mask, mask.data(), mask.size());
    if (p->layout == LBM_SPARSE_TILE16) {
        if (h_tile_id) std::memcpy(h_tile_id, tid.data(), tid.size() * 4);
        if (h_nbr) std::memcpy(h_nbr, nbr.data(), nbr.size() * 4);
        if (h_ntiles) *h_ntiles = pl.ntiles;
    } else if (h_ntiles) {
        *h_ntiles = 0;
    }
    if (h_nfluid) *h_nfluid = pl.nfluid;
    return LBM_OK;
}

long long lbm_fluid_nodes(const lbm_ctx *ctx) { return ctx ? ctx->nfluid : -1; }
long long lbm_step_count(const lbm_ctx *ctx) { return ctx ? ctx->steps : -1; }
int lbm_launches_per_step(const lbm_ctx *ctx) {
    if (!ctx) return -1;
    const Geo &g = ctx->geo;
    if (g.layout != LBM_DENSE) return 1;
    if (g.has_mask && g.frame_y) return 1 + (g.ny - 2 + 65534) / 65535;
    return (g.ny + 65534) / 65535;
}
long long lbm_step_launches(const lbm_ctx *ctx, int n) {
    if (!ctx || n < 0) return -1;
    const long long per = lbm_launches_per_step(ctx);
    if (!ctx->graphs || n < GRAPH_CHUNK) return per * n;
    return per * n + 1 + n / GRAPH_CHUNK; // + the counter's set and one add per replay
}
const char *lbm_last_error(const lbm_ctx *ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

} // extern "C"
