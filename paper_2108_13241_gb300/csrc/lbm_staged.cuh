// lbm_staged.cuh -- the tiled sparse two-lattice step with its tiles staged in
// shared memory (included by lbm_kernels.cuh inside its namespace, after the
// per-vector step kernel, whose node helpers it shares).
//
// Algorithm 1's pull step over the 16 x 16 tiles that hold fluid (the
// "pointer tile" layout of Sec. 4.2.2), built for GB300 as a warp-specialized
// pipeline:
//  * persistent blocks, tiles taken round-robin (block b: b, b + G, ...), so
//    the tiles in flight at any moment are neighbours and the halo reads of
//    one tile hit the L2 lines its neighbours' blocks are loading;
//  * one producer warp issues asynchronous 16-byte copies (cp.async) of the
//    next tiles into a ring of D shared-memory stages, up to D - 1 tiles
//    ahead; each stage's "full" mbarrier completes when the copies have landed
//    (cp.async.mbarrier.arrive), its "empty" mbarrier when the consumers are
//    done with it -- no block-wide barrier, so the copies stay in flight while
//    the consumer warps compute and a warp with little work in one tile moves
//    on to the next;
//  * chunks that hold no fluid node are zero-filled without a DRAM read (a
//    needed pull source is always a fluid node);
//  * each slot of a stage holds the tile's 16 x 16 values plus one halo row
//    and one 16-byte halo chunk of columns on exactly the edges that slot
//    pulls across, filled from the 3 x 3 neighbour tiles -- so the pull
//    f'_i(x) = A_i(x - c_i) is one shared-memory load at a fixed offset, with
//    no per-node test of tile edges; a halo chunk whose source nodes are all
//    solid (the tile's host-built halo mask) is zero-filled, not read, since
//    only unbounced pulls, from fluid nodes, use halo values;
//  * four consumer warps take the tile's 2-node vectors from a per-tile list
//    of the vectors whose DRAM sector holds fluid (host-built), so a consumer
//    warp whose share of a porous tile is solid skips the collision;
//  * the collision is the same `collide` as every other step kernel, on the
//    same operands, so results are bit-identical to the dense layout.
// Stores go straight to the other lattice: every 2-node vector of a DRAM
// sector that holds a fluid node (solid nodes there are written 0), nothing
// elsewhere.  Every wait on an mbarrier gives up after about two seconds: it
// then sets the device error word (reported as LBM_ERR_TIMEOUT) and the block
// returns, so a fault in the pipeline cannot hang the GPU.
#pragma once

// Compile-time tuning knob: stages in shared memory (FP32 and FP16s; FP64
// keeps 3, its stages being twice the size).
#ifndef LBM_STG_DEPTH
#define LBM_STG_DEPTH 3
#endif
constexpr int STG_CONSUMERS = 4;                      // consumer warps: 128 vectors of a tile
constexpr int STG_THREADS = 32 * (1 + STG_CONSUMERS); // + one producer warp
template <int P> struct StagedDepth {
    enum { value = P == LBM_F64 ? 3 : LBM_STG_DEPTH };
};
// Blocks per SM the registers are sized for (with 3 stages shared memory
// holds 6 FP32, 10 FP16s or 3 FP64 blocks).
#ifndef LBM_STG_BLOCKS32
#define LBM_STG_BLOCKS32 6
#endif
template <int P> struct StagedBlocks {
    enum { value = P == LBM_F32 ? LBM_STG_BLOCKS32 : (P == LBM_F16S ? 6 : 3) };
};
constexpr long long STG_WAIT_CYCLES = 4000000000ll; // about 2 s at 2 GHz

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// 16-byte asynchronous copy global -> shared; with pred false the 16 bytes
// are zero-filled and nothing is read (src must still be a valid address).
__device__ __forceinline__ void cp_async16(unsigned dst, const void *src, bool pred) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(pred ? 16 : 0)
                 : "memory");
}
// 4-byte asynchronous copy global -> shared
__device__ __forceinline__ void cp_async4(unsigned dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// the mbarrier gets one arrival when this thread's earlier cp.async copies
// have completed (the arrival is counted in its initial count)
__device__ __forceinline__ void cp_async_arrive(unsigned mbar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_init(unsigned mbar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned mbar, unsigned parity) {
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(mbar), "r"(parity)
                 : "memory");
    return ok != 0u;
}
// Waits for the phase of `parity` to complete; false after STG_WAIT_CYCLES.
__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned parity) {
    if (mbar_try_wait(mbar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(mbar, parity))
        if (clock64() - t0 > STG_WAIT_CYCLES) return false;
    return true;
}

// Layout of one stage for stored element type R.  Slot i keeps rows
// -HS .. 15 + HN and columns -HW .. 15 + HE, where HS / HN is 1 when the slot
// pulls from the row below / above (c_y = +1 / -1) and HW / HE is one 16-byte
// chunk (E elements) when it pulls from the column to the left / right
// (c_x = +1 / -1).
template <class R> struct StageLayout {
    static constexpr int E = 16 / (int)sizeof(R); // elements per 16-byte chunk
    static constexpr int CPR = TILE / E;          // chunks per tile row
    static __host__ __device__ constexpr int hw(int i) { return cx(i) == 1 ? E : 0; }
    static __host__ __device__ constexpr int he(int i) { return cx(i) == -1 ? E : 0; }
    static __host__ __device__ constexpr int hs(int i) { return cy(i) == 1 ? 1 : 0; }
    static __host__ __device__ constexpr int hn(int i) { return cy(i) == -1 ? 1 : 0; }
    static __host__ __device__ constexpr int rp(int i) { return TILE + hw(i) + he(i); }
    static __host__ __device__ constexpr int size(int i) { return (TILE + hs(i) + hn(i)) * rp(i); }
    // start of slot i: slots 0 (core only), 1 and 3 (one halo column chunk),
    // 2 and 4 (one halo row), 5 .. 8 (both); written out, not recursively, so
    // that it folds to a constant wherever i is one
    static __host__ __device__ constexpr int base(int i) {
        return i == 0 ? 0
                      : TILE_N + (i >= 2 ? size(1) : 0) + (i >= 3 ? size(2) : 0) + (i >= 4 ? size(3) : 0) +
                            (i >= 5 ? size(4) : 0) + (i > 5 ? (i - 5) * size(5) : 0);
    }
    // element (lx, ly) of slot i
    static __host__ __device__ constexpr int at(int i, int lx, int ly) {
        return base(i) + (ly + hs(i)) * rp(i) + lx + hw(i);
    }
    static constexpr int DATA = base(8) + size(8);         // elements of the 9 slots
    static constexpr int HALO = halo_chunks(E);            // halo chunks
    static_assert(HALO <= 128, "one bit per halo chunk in the tile's 128-bit halo mask");
    static constexpr int HALO_ROUNDS = (HALO + 31) / 32;   // per producer lane
    static constexpr int POS_ROUNDS = TILE * CPR / 32;     // (row, chunk) positions per lane
    static constexpr int MASK_OFF = DATA * (int)sizeof(R); // 256 node mask bytes
    static constexpr int ORDER_OFF = MASK_OFF + TILE_N;    // 128 vector order bytes
    static constexpr int XY_OFF = ORDER_OFF + TILE_N / 2;  // tile coordinates (one int)
    static constexpr int BYTES = XY_OFF + 16;              // one stage
    static_assert((TILE * CPR) % 32 == 0, "own-core chunk mapping");
    static_assert(MASK_OFF % 16 == 0 && BYTES % 16 == 0, "stage sections stay 16-byte aligned");
};

// One halo chunk: which neighbour (3 x 3 index 3 (oy+1) + (ox+1)), the source
// element in that tile (slot * 256 + row * 16 + column) and the destination
// element in the stage.
struct HaloChunk {
    int dir;
    unsigned src, dst;
};

template <class R> __device__ __forceinline__ HaloChunk halo_chunk(int h) {
    typedef StageLayout<R> L;
    const HaloSrc hs = halo_source(h, L::E);
    HaloChunk c;
    c.dir = hs.dir;
    c.src = (unsigned)(hs.slot * TILE_N + hs.srow * TILE + hs.scol);
    // the slot-specific layout, evaluated per slot (slot is not a constant here)
    unsigned d = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i)
        if (i == hs.slot) d = (unsigned)L::at(i, hs.dlx, hs.dly);
    c.dst = d;
    return c;
}

// What the producer needs of a tile to stage it.
template <int HR> struct TileRec {
    int t;      // tile id (< 0: nothing to stage)
    uint4 vm;   // 2-node vectors holding fluid: bit 8 * (row % 4) + v of word row / 4
    int nb[HR]; // neighbour tile of this lane's halo chunks (-1: absent, or no fluid at the source)
};

template <class R, int HR>
__device__ __forceinline__ void load_rec(const Geo &g, int t, const HaloChunk (&hc)[HR], int lane, TileRec<HR> &r) {
    typedef StageLayout<R> L;
    r.t = t;
    if (t < 0) return;
    r.vm = __ldg(g.tile_vmask + t);
#pragma unroll
    for (int k = 0; k < HR; ++k) r.nb[k] = (lane + 32 * k < L::HALO) ? __ldg(g.nbr + 9 * t + hc[k].dir) : -1;
    // halo chunks whose source holds no fluid are zero-filled, not read
    const uint4 hm = __ldg(g.tile_hmask + t);
#pragma unroll
    for (int k = 0; k < HR; ++k) {
        const unsigned w = k == 0 ? hm.x : (k == 1 ? hm.y : (k == 2 ? hm.z : hm.w));
        if (!((w >> lane) & 1u)) r.nb[k] = -1;
    }
}

// Fluid bits of tile row `row` (bit v: 2-node vector v of the row holds a
// fluid node) from the tile's 2-node-vector mask.
__device__ __forceinline__ unsigned row_bits(const uint4 &vm, int row) {
    const unsigned w = row < 4 ? vm.x : (row < 8 ? vm.y : (row < 12 ? vm.z : vm.w));
    return (w >> (8 * (row & 3))) & 0xFFu;
}

// Producer lane: issues its share of the copies of tile r.t into stage `st`.
// Own core: lane L copies (row, chunk) positions L, L + 32, ... of all nine
// slots; a position without a fluid node is zero-filled.
template <class R, int HR>
__device__ __forceinline__ void stage_tile(const Geo &g, const R *src, unsigned char *st, const TileRec<HR> &r,
                                           const HaloChunk (&hc)[HR], int lane) {
    typedef StageLayout<R> L;
    constexpr int E = L::E, CPR = L::CPR;
    if (r.t < 0) return;
    const R *tb = src + (size_t)r.t * (9 * TILE_N);
    R *sd = reinterpret_cast<R *>(st);
#pragma unroll
    for (int q = 0; q < L::POS_ROUNDS; ++q) {
        const int pos = lane + 32 * q, row = pos / CPR, c = pos - row * CPR;
        const bool f = ((row_bits(r.vm, row) >> (c * (E / 2))) & ((1u << (E / 2)) - 1u)) != 0u;
        const unsigned rc = (unsigned)(row * TILE + c * E);
#pragma unroll
        for (int slot = 0; slot < 9; ++slot)
            cp_async16(smem_addr(sd + L::at(slot, 0, 0) + row * L::rp(slot) + c * E),
                       f ? tb + slot * TILE_N + rc : tb, f);
    }
    // halo chunks from the neighbour tiles (absent neighbour: zeros; those
    // links bounce)
#pragma unroll
    for (int k = 0; k < HR; ++k) {
        if (lane + 32 * k < L::HALO) {
            const int n = r.nb[k];
            const R *p = n >= 0 ? src + (size_t)n * (9 * TILE_N) + hc[k].src : tb;
            cp_async16(smem_addr(sd + hc[k].dst), p, n >= 0);
        }
    }
    // the tile's 256 mask bytes and its 128-byte vector order
    if (lane < TILE_N / 16)
        cp_async16(smem_addr(st + L::MASK_OFF + 16 * lane), g.mask + (size_t)r.t * TILE_N + 16 * lane, true);
    else if (lane < TILE_N / 16 + TILE_N / 32)
        cp_async16(smem_addr(st + L::ORDER_OFF + 16 * (lane - 16)),
                   g.tile_order + (size_t)r.t * (TILE_N / 2) + 16 * (lane - 16), true);
    else if (lane == TILE_N / 16 + TILE_N / 32)
        cp_async4(smem_addr(st + L::XY_OFF), g.tile_xy + r.t);
}

// Node K (0 or 1) of the thread's 2-node vector at (lx0 + K, ly): gather from
// the stage, bounce-back, open sides, collision, encode into out[i].v[K].
template <class S, int FORCE, bool OPEN, int K, bool TRT>
__device__ __forceinline__ void staged_node(const Geo &g, const Phys &ph, const typename S::R *sd, int lx0, int ly,
                                            int gx0, int gy, unsigned m, const Coef<typename S::C> &co, SrState &sr,
                                            V16<typename S::R, 2> out[9]) {
    typedef typename S::R R;
    typedef typename S::C C;
    typedef StageLayout<R> L;
    const int lx = lx0 + K;
    if (m == 0xFFu) {
        if constexpr (S::STOCHASTIC) {
            const float z[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            put_sr<S, K>(z, sr, (long long)gy * g.nx + gx0, out);
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) out[i].v[K] = S::enc(C(0));
        }
        return;
    }
    C f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = S::dec_step(sd[L::at(i, lx - cx(i), ly - cy(i))]);
    if (m != 0u) {
        // half-way bounce-back: the node's own post-collision value of the
        // opposite link (plus the moving-wall term)
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            if (m & (1u << (i - 1))) {
                C v = S::dec_step(sd[L::at(opp(i), lx, ly)]);
                if (ph.has_wall) v = v + PC<C>::wt(ph, wall_side(g, gx0 + K, gy, i), i) * C(S::SCALE);
                f[i] = v;
            }
        }
    }
    if constexpr (OPEN) apply_open<C, S::SCALE>(g, ph, gx0 + K, gy, m, f);
    const C Fx = PC<C>::fx(ph), Fy = PC<C>::fy(ph);
    collide<C, FORCE != FORCE_NONE, (sizeof(C) == 4 && !S::STOCHASTIC), S::SCALE, TRT>(f, Fx, Fy, co);
    if constexpr (S::STOCHASTIC) {
        put_sr<S, K>(f, sr, (long long)gy * g.nx + gx0, out);
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) out[i].v[K] = S::enc(f[i]);
    }
}

// Range of the fraction of a geometry's kept-tile 2-node vectors holding
// fluid in which the staged step replaces the per-vector step.  Measured on
// 4096^2 disc media (phi 0.2 / 0.5 / 0.8, fractions 0.37 / 0.58 / 0.86) and
// the all-fluid box: FP32 staged 37.4 / 55.8 / 74.9 / 78.5 GLUPS against
// 37.0 / 48.3 / 72.1 / 94.4 per vector; FP16s staged 38.4 / 62.2 / 100.3 /
// 133.1 against 48.0 / 64.8 / 81.0 / 116.0 (its per-vector list kernel is
// persistent and prefetches, and wins on sparse tiles).
#ifndef LBM_STG_FP32_MAX
#define LBM_STG_FP32_MAX 0.95f
#endif
#ifndef LBM_STG_FP16S_MIN
#define LBM_STG_FP16S_MIN 0.70f
#endif
template <int P> __host__ __device__ inline bool staged_selected(float active_frac) {
    if (P == LBM_F32) return active_frac < LBM_STG_FP32_MAX;
    if (P == LBM_F16S) return active_frac >= LBM_STG_FP16S_MIN;
    return false;
}

// Shared memory of one staged block (the mbarriers are static).
template <int P> constexpr int staged_smem_bytes() {
    return StagedDepth<P>::value * StageLayout<typename St<P>::R>::BYTES;
}

template <int P, int FORCE, bool OPEN, bool TRT>
__global__ void __launch_bounds__(STG_THREADS, StagedBlocks<P>::value)
    k_step_staged(const Geo g, const Phys ph, const void *src_v, void *dst_v, unsigned step) {
    typedef StV<P, 2> S;
    typedef typename S::R R;
    typedef typename S::C C;
    typedef StageLayout<R> L;
    constexpr int D = StagedDepth<P>::value;
    constexpr int HR = L::HALO_ROUNDS;
    extern __shared__ __align__(16) unsigned char stg_smem[];
    __shared__ __align__(8) unsigned long long bar_full[D], bar_empty[D];
    const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
    const int G = (int)gridDim.x;
    const int nt = g.ntiles;
    const int b = (int)blockIdx.x;
    if (b >= nt) return; // block-uniform
    const int niter = (nt - 1 - b) / G + 1;
    if (threadIdx.x == 0) {
        for (int s = 0; s < D; ++s) {
            mbar_init(smem_addr(&bar_full[s]), 32);             // one cp.async arrival per producer lane
            mbar_init(smem_addr(&bar_empty[s]), STG_CONSUMERS); // one arrival per consumer warp
        }
    }
    __syncthreads();

    if (warp == 0) {
        // ---------------- producer
        const R *src = reinterpret_cast<const R *>(src_v);
        HaloChunk hc[HR];
#pragma unroll
        for (int k = 0; k < HR; ++k) hc[k] = halo_chunk<R>(lane + 32 * k < L::HALO ? lane + 32 * k : 0);
        // three records in turn, each loaded two tiles before its use (the
        // loop is unrolled by three so that no register copy waits on a load)
        TileRec<HR> ra, rb, rc;
        load_rec<R, HR>(g, b, hc, lane, ra);
        load_rec<R, HR>(g, 1 < niter ? b + G : -1, hc, lane, rb);
        bool ok = true;
        // stages tile k from `use` after loading tile k + 2 into `next`
        auto produce = [&](int k, const TileRec<HR> &use, TileRec<HR> &next) {
            const int s = k % D;
            load_rec<R, HR>(g, k + 2 < niter ? b + (k + 2) * G : -1, hc, lane, next);
            if (k >= D && !mbar_wait(smem_addr(&bar_empty[s]), (unsigned)((k / D - 1) & 1))) {
                atomicOr(g.err, 1u);
                ok = false;
                return;
            }
            stage_tile<R, HR>(g, src, stg_smem + s * L::BYTES, use, hc, lane);
            cp_async_arrive(smem_addr(&bar_full[s]));
        };
        for (int k = 0; k < niter && ok; k += 3) {
            produce(k, ra, rc);
            if (k + 1 < niter && ok) produce(k + 1, rb, ra);
            if (k + 2 < niter && ok) produce(k + 2, rc, rb);
        }
        cp_async_wait_all();
        return;
    }

    // -------------------- consumers: warp w takes the tile's vectors 32 (w - 1) ...
    R *dst = reinterpret_cast<R *>(dst_v);
    unsigned tbase = 0u;
    if constexpr (S::STOCHASTIC)
        if (ph.tbase) tbase = (unsigned)__ldg(ph.tbase);
    SrState sr;
    sr.tseed = S::STOCHASTIC ? fmix32((tbase + step) * 0x9E3779B9u + 0x632BE5ABu) : 0u;
    const Coef<C> co(ph);
    const int ent = 32 * (warp - 1) + lane;
    for (int k = 0; k < niter; ++k) {
        const int s = k % D;
        const int t = b + k * G;
        if (!mbar_wait(smem_addr(&bar_full[s]), (unsigned)((k / D) & 1))) {
            atomicOr(g.err, 1u);
            return;
        }
        const unsigned char *st = stg_smem + s * L::BYTES;
        // the lane's 2-node vector (8 row + v); 0xFF: none.  Any byte beyond
        // 127 is read as none, so every index stays inside the tile.
        const unsigned v = st[L::ORDER_OFF + ent];
        if (v < 128u) {
            const R *sd = reinterpret_cast<const R *>(st);
            const int ly = (int)(v >> 3), lx0 = 2 * (int)(v & 7u);
            const int xy = *reinterpret_cast<const int *>(st + L::XY_OFF);
            const int gx0 = (xy & 0xFFFF) * TILE + lx0, gy = (xy >> 16) * TILE + ly;
            const unsigned mv = *reinterpret_cast<const unsigned short *>(st + L::MASK_OFF + ly * TILE + lx0);
            V16<R, 2> out[9];
            staged_node<S, FORCE, OPEN, 0, TRT>(g, ph, sd, lx0, ly, gx0, gy, mv & 0xFFu, co, sr, out);
            staged_node<S, FORCE, OPEN, 1, TRT>(g, ph, sd, lx0, ly, gx0, gy, mv >> 8, co, sr, out);
            R *o = dst + (size_t)t * (9 * TILE_N) + ly * TILE + lx0;
#pragma unroll
            for (int i = 0; i < 9; ++i) st16<R, 2>(o + i * TILE_N, out[i]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&bar_empty[s]));
    }
}
