// lbm_kernels.cuh -- CUDA kernels of the D2Q9 BGK stream-and-collide update
// for sm_103a, templated on the storage precision.  Included only by the
// per-precision translation units kern_f64.cu, kern_f32.cu, kern_f16s.cu.
//
// The hot kernel (k_step) is Algorithm 1's fused pull kernel (Sec. 3):
// gather f'_i = A_i(x - c_i) with half-way bounce-back, moments (Eq. 2),
// equilibrium (Eq. 6), BGK relaxation (Eq. 3, Eq. 4) with a Guo
// body-force source, aligned store.  Design for GB300:
//  * SoA slots, one vector per thread and slot: 16 bytes = 2 FP64 or 4 FP32
//    nodes, 8 bytes = 4 FP16 nodes, consecutive along x;
//  * the x-shifted pulls (c_x != 0, the uncoalesced loads Sec. 4.2.2
//    reports) take the aligned vector and one value from the neighbouring
//    lane (__shfl_up/down_sync); only lanes at a warp or row edge load that
//    value from memory (an L1/L2 hit);
//  * a per-node link mask (one byte) selects a divergent slow path only at
//    nodes next to walls, open sides or obstacles; all-solid vectors move no
//    data; on porous tiled geometries threads run only over the vectors that
//    hold fluid (a host-built list);
//  * distributions are stored shifted, f_i - w_i, and the collision runs in
//    shifted variables (rho = 1 + sum, m = sum c_i (f_i - w_i)), so FP32 and
//    FP16 keep their mantissa for the small deviations from rest;
//  * every variant (dense / tiled / listed, two-lattice / AA) feeds the same
//    `collide` with the same operands, so results agree bit for bit.
#pragma once
#include <type_traits>

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lbm_internal.h"

namespace lbm {

#define LBM_FULL 0xffffffffu

// ------------------------------------------------------------- lattice

__host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
}
template <class C> __host__ __device__ constexpr C wgt(int i) {
    return i == 0 ? C(4.0 / 9.0) : (i <= 4 ? C(1.0 / 9.0) : C(1.0 / 36.0));
}

// ------------------------------------------------------------- storage

template <int P> struct St;
// dec/enc convert between the stored element and f_i - w_i in the compute
// type.  The step kernel works in units of SCALE (f_i - w_i times SCALE):
// dec_step decodes into them (FP16s encodes from them by a stochastically
// rounding conversion, put_sr); every other kernel uses dec/enc.
template <> struct St<LBM_F64> {
    typedef double R; // stored element
    typedef double C; // compute type
    enum { VEC = 2, STOCHASTIC = 0, SCALE = 1 };
    static __device__ __forceinline__ C dec(R r) { return r; }
    static __device__ __forceinline__ C dec_step(R r) { return r; }
    static __device__ __forceinline__ R enc(C c) { return c; }
};
template <> struct St<LBM_F32> {
    typedef float R;
    typedef float C;
    enum { VEC = 4, STOCHASTIC = 0, SCALE = 1 };
    static __device__ __forceinline__ C dec(R r) { return r; }
    static __device__ __forceinline__ C dec_step(R r) { return r; }
    static __device__ __forceinline__ R enc(C c) { return c; }
};
// FP16s: binary16 bits of (f_i - w_i) * 2^10.  The power-of-two scale is
// exact; it moves the small deviations of slow flows (|f_i - w_i| down to
// 6e-8) into binary16's normal range while keeping |f_i - w_i| up to 64
// finite.  The time step rounds stochastically, two values by one
// conversion (f16x2_rs below): 13 uniform random bits are added below
// binary16's last kept mantissa bit before truncation, so the rounding error
// has zero mean instead of repeating itself step after step in a slowly
// varying flow.
// log2 of the FP16s storage scale (compile-time)
#ifndef LBM_F16S_SHIFT
#define LBM_F16S_SHIFT 10
#endif
template <> struct St<LBM_F16S> {
    typedef unsigned short R;
    typedef float C;
    enum { VEC = 4, STOCHASTIC = 1, SCALE = 1 << LBM_F16S_SHIFT }; // 8-byte vectors: 4 nodes per thread
    static __device__ __forceinline__ C dec(R r) { return __half2float(__ushort_as_half(r)) * (1.0f / SCALE); }
    static __device__ __forceinline__ R enc(C c) { return __half_as_ushort(__float2half_rn(c * (float)SCALE)); }
    static __device__ __forceinline__ C dec_step(R r) { return __half2float(__ushort_as_half(r)); }
};

// Two values rounded stochastically to binary16 by one packed conversion
// (cvt.rs, sm_100 and later): lo goes to the low half of the word (the lower
// node index) and is rounded with random bits 12..0 of rbits, hi to the high
// half with bits 28..16 -- each adds its 13 bits below binary16's last kept
// mantissa bit and truncates.
__device__ __forceinline__ unsigned f16x2_rs(float lo, float hi, unsigned rbits) {
    unsigned r;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(r) : "f"(hi), "f"(lo), "r"(rbits));
    return r;
}

// Counter-based random bits for stochastic rounding: the 32-bit finaliser of
// Appleby's MurmurHash3 applied to (index of the even node of a node pair,
// time step), then one Numerical Recipes linear congruential step per link;
// the word h ^ (h >> 16) rounds the pair's two values of that link (the
// seed is well mixed, so both 13-bit fields are uniform and independent).
// Deterministic, and the same for a node pair, link and step in every layout
// and pattern.
__device__ __forceinline__ unsigned fmix32(unsigned h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}
__device__ __forceinline__ unsigned lcg_next(unsigned h) { return h * 1664525u + 1013904223u; }

// One aligned vector of VEC stored values: 16 bytes (FP64, FP32), 8 or 4
// bytes (FP16s), moved with one load or store instruction.
template <int BYTES> struct VecWord;
template <> struct VecWord<16> { typedef uint4 T; static __device__ __forceinline__ uint4 zero() { return make_uint4(0, 0, 0, 0); } };
template <> struct VecWord<4> { typedef unsigned T; static __device__ __forceinline__ unsigned zero() { return 0u; } };
template <> struct VecWord<8> { typedef uint2 T; static __device__ __forceinline__ uint2 zero() { return make_uint2(0, 0); } };

// The same storage with a different number of nodes per thread.
template <int P, int V> struct StV : St<P> {
    enum { VEC = V };
};
// Nodes per thread of the step kernel: one 16-byte (FP64, FP32) or 8-byte
// (FP16s) vector.  FP32 with a link mask moves 2 nodes (8-byte vectors), so
// that the preloaded bounce-back state fits 4 blocks per SM, in the AA steps,
// with a per-node force field and in the adjoint; its two-lattice step
// without a force field moves 4 (bounced values loaded on demand).  FP16s
// with a link mask moves 2 nodes (4-byte vectors) in the AA gather/scatter
// step, whose scattered stores otherwise spill at 3 blocks per SM (measured
// +14-24% on tiled and porous AA runs at 4 blocks per SM).
template <int P, bool HAS_MASK, int MODE, int FORCE> struct StepVec {
    enum {
        value = ((P == LBM_F32 && HAS_MASK && (MODE == MODE_AA_PULLPUSH || FORCE == FORCE_FIELD)) ||
                 (P == LBM_F16S && HAS_MASK && MODE == MODE_AA_PULLPUSH))
                    ? 2
                    : St<P>::VEC
    };
};
// Whether the step preloads the own-node vectors its bounced links read
// (issued with the gather, one vector per needed slot) or loads each bounced
// value when the node needs it: the FP32 two-lattice step with 16-byte
// vectors loads on demand, which keeps it at 4 blocks per SM.
template <class S, int MODE> struct OwnPreload {
    enum { value = !(sizeof(typename S::R) == 4 && S::VEC == 4 && MODE == MODE_TWO_LATTICE) };
};

template <class R, int VEC> union V16 {
    typename VecWord<(int)sizeof(R) * VEC>::T u;
    R v[VEC];
};

template <bool NC, class R, int VEC>
__device__ __forceinline__ V16<R, VEC> ld16(const R *p) {
    typedef typename VecWord<(int)sizeof(R) * VEC>::T W;
    V16<R, VEC> r;
    if (NC)
        r.u = __ldg(reinterpret_cast<const W *>(p));
    else
        r.u = *reinterpret_cast<const W *>(p);
    return r;
}
template <bool NC, class R> __device__ __forceinline__ R ld1(const R *p) {
    if (NC) return __ldg(p);
    return *p;
}
template <> __device__ __forceinline__ unsigned short ld1<true, unsigned short>(const unsigned short *p) {
    return __ldg(p);
}
template <class R, int VEC> __device__ __forceinline__ void st16(R *p, const V16<R, VEC> &v) {
    *reinterpret_cast<typename VecWord<(int)sizeof(R) * VEC>::T *>(p) = v.u;
}
template <class R, int VEC> __device__ __forceinline__ void zero16(V16<R, VEC> &v) {
    v.u = VecWord<(int)sizeof(R) * VEC>::zero();
}
// 32-bit word W of a 4-, 8- or 16-byte vector
template <int W> __device__ __forceinline__ void set_word(unsigned &u, unsigned v) { u = v; }
template <int W> __device__ __forceinline__ void set_word(uint2 &u, unsigned v) {
    if (W == 0) u.x = v;
    else u.y = v;
}
template <int W> __device__ __forceinline__ void set_word(uint4 &u, unsigned v) {
    if (W == 0) u.x = v;
    else if (W == 1) u.y = v;
    else if (W == 2) u.z = v;
    else u.w = v;
}

__device__ __forceinline__ double shfl_up1(double v) { return __shfl_up_sync(LBM_FULL, v, 1); }
__device__ __forceinline__ float shfl_up1(float v) { return __shfl_up_sync(LBM_FULL, v, 1); }
__device__ __forceinline__ unsigned short shfl_up1(unsigned short v) {
    return (unsigned short)__shfl_up_sync(LBM_FULL, (unsigned)v, 1);
}
__device__ __forceinline__ double shfl_down1(double v) { return __shfl_down_sync(LBM_FULL, v, 1); }
__device__ __forceinline__ float shfl_down1(float v) { return __shfl_down_sync(LBM_FULL, v, 1); }
__device__ __forceinline__ unsigned short shfl_down1(unsigned short v) {
    return (unsigned short)__shfl_down_sync(LBM_FULL, (unsigned)v, 1);
}
// the same among the lanes of mask m (a lane outside m gives an undefined
// value, which the caller does not use)
__device__ __forceinline__ double shfl_up1(unsigned m, double v) { return __shfl_up_sync(m, v, 1); }
__device__ __forceinline__ float shfl_up1(unsigned m, float v) { return __shfl_up_sync(m, v, 1); }
__device__ __forceinline__ unsigned short shfl_up1(unsigned m, unsigned short v) {
    return (unsigned short)__shfl_up_sync(m, (unsigned)v, 1);
}
__device__ __forceinline__ double shfl_down1(unsigned m, double v) { return __shfl_down_sync(m, v, 1); }
__device__ __forceinline__ float shfl_down1(unsigned m, float v) { return __shfl_down_sync(m, v, 1); }
__device__ __forceinline__ unsigned short shfl_down1(unsigned m, unsigned short v) {
    return (unsigned short)__shfl_down_sync(m, (unsigned)v, 1);
}

// VEC mask bytes of consecutive nodes, as one integer (node k in byte k).
template <int VEC> __device__ __forceinline__ unsigned long long ld_mask(const uint8_t *p);
template <> __device__ __forceinline__ unsigned long long ld_mask<2>(const uint8_t *p) {
    return __ldg(reinterpret_cast<const unsigned short *>(p));
}
template <> __device__ __forceinline__ unsigned long long ld_mask<4>(const uint8_t *p) {
    return __ldg(reinterpret_cast<const unsigned int *>(p));
}
template <> __device__ __forceinline__ unsigned long long ld_mask<8>(const uint8_t *p) {
    return __ldg(reinterpret_cast<const unsigned long long *>(p));
}
template <int VEC> __host__ __device__ constexpr unsigned long long mask_ones() {
    return VEC == 8 ? ~0ull : ((1ull << (8 * VEC)) - 1ull);
}
// bit b replicated into every node byte
template <int VEC> __host__ __device__ constexpr unsigned long long mask_rep(int b) {
    return VEC == 2 ? (0x0101ull << b) : (VEC == 4 ? (0x01010101ull << b) : (0x0101010101010101ull << b));
}

// ------------------------------------------------------------- addressing

__device__ __forceinline__ int pick3(int o, int a, int b, int c) { return o < 0 ? a : (o > 0 ? c : b); }

// Dense SoA f[slot][ny][nx]; thread = VEC nodes (x0..x0+VEC-1, y).
template <int VEC> struct DenseAddr {
    enum { VEC_ = VEC, LIST_ = 0 };
    int x0, y, xv, nvx, nx, ny;
    bool valid;
    unsigned nslot; // element indices fit 32 bits (checked at create)
    const uint8_t *mask;
    int roff[3];    // (row y-1, y, y+1) * nx: wrapped (periodic) or clamped (wall)
    int lcol, rcol; // columns x0 - 1 and x0 + VEC, wrapped or clamped

    // 2-D launch: (vector column, row) = (blockIdx.x * blockDim.x + tid, row).
    // Everything that depends on the wrap is resolved here, branch-free.
    __device__ __forceinline__ DenseAddr(const Geo &g, int col, int row_) {
        nx = g.nx;
        ny = g.ny;
        nslot = (unsigned)g.nslot;
        mask = g.mask;
        nvx = nx / VEC;
        valid = col < nvx;
        xv = valid ? col : nvx - 1;
        y = row_;
        x0 = xv * VEC;
        const bool px = g.periodic_x, py = g.periodic_y;
#pragma unroll
        for (int d = -1; d <= 1; ++d) {
            int r = y + d;
            r = r < 0 ? (py ? r + ny : 0) : r;
            r = r >= ny ? (py ? r - ny : ny - 1) : r;
            roff[d + 1] = r * nx;
        }
        const int l = x0 - 1, rr = x0 + VEC;
        lcol = l < 0 ? (px ? nx - 1 : 0) : l;
        rcol = rr >= nx ? (px ? 0 : nx - 1) : rr;
    }
    // aligned vector of slot at (x0, y + dy), dy in {-1, 0, 1}
    __device__ __forceinline__ unsigned vidx(int slot, int dy) const {
        return (unsigned)slot * nslot + (unsigned)(roff[dy + 1] + x0);
    }
    // element (x0 + k + dx, y + dy), k + dx in [-1, VEC], dy in {-1, 0, 1}
    __device__ __forceinline__ unsigned eidx(int slot, int k, int dx, int dy) const {
        const int c = (k + dx < 0) ? lcol : ((k + dx >= VEC) ? rcol : x0 + k + dx);
        return (unsigned)slot * nslot + (unsigned)(roff[dy + 1] + c);
    }
    __device__ __forceinline__ bool left_in_warp(int lane) const { return lane > 0 && xv > 0; }
    __device__ __forceinline__ bool right_in_warp(int lane) const { return lane < 31 && xv < nvx - 1; }
    __device__ __forceinline__ int gx(int k) const { return x0 + k; }
    __device__ __forceinline__ int gy() const { return y; }
    __device__ __forceinline__ bool in_domain() const { return true; }
    __device__ __forceinline__ long long node(int k) const { return (long long)y * nx + x0 + k; }
    __device__ __forceinline__ const uint8_t *mask_ptr() const { return mask + (long long)y * nx + x0; }
};

// Tiled sparse f[tile][slot][16][16]; thread = VEC nodes of one tile row.
// nbr3 is the device table [tile][3*(oy+1) + (ox+1)] (absent -> -1).
// LIST: thread k takes the k-th entry of the list of vectors that hold a
// fluid node (t * TPT + position in the tile), so that no warp idles on the
// solid part of a kept tile; without it, thread k takes position k % TPT of
// tile k / TPT.
template <int VEC, bool LIST = false> struct TileAddr {
    enum { VEC_ = VEC, LIST_ = LIST, TPR = TILE / VEC, TPT = TILE * (TILE / VEC) };
    int t, lx0, ly, xv, tx, ty, nx, ny;
    bool valid;
    bool lnb, rnb; // LIST: the lane below / above holds the vector just left / right
    const uint8_t *mask;
    // element index (slot 0) of this thread's first node in rows ly-1, ly,
    // ly+1 (rowb), and of the nodes just left (lb) and right (rb) of the
    // thread's vector in those rows, in whatever tile holds them (32-bit:
    // 9 * 256 * tiles < 2^32 is checked at create)
    unsigned rowb[3], lb[3], rb[3];

    // LIST: the list, its length, and entry k (clamped to the last one)
    static __device__ __forceinline__ const unsigned *list(const Geo &g) { return VEC == 4 ? g.vlist4 : g.vlist2; }
    static __device__ __forceinline__ int list_len(const Geo &g) { return VEC == 4 ? g.nlist4 : g.nlist2; }
    static __device__ __forceinline__ unsigned entry(const Geo &g, int k) {
        const int n = list_len(g);
        return __ldg(list(g) + (k < n ? k : n - 1));
    }

    // 1-D launch over tiles (TPT threads per tile) or over the list; the row
    // argument is unused
    __device__ __forceinline__ TileAddr(const Geo &g, int gtid, int) {
        if constexpr (LIST) {
            init(g, entry(g, gtid), gtid < list_len(g));
        } else {
            int tt = gtid / TPT;
            valid = tt < g.ntiles;
            if (!valid) tt = g.ntiles - 1;
            t = tt;
            init(g, 0u, valid, gtid - (gtid / TPT) * TPT);
        }
    }
    // LIST: list entry e (all lanes of the warp call this together)
    __device__ __forceinline__ TileAddr(const Geo &g, unsigned e, bool valid_) { init(g, e, valid_); }

    __device__ __forceinline__ void init(const Geo &g, unsigned e, bool valid_, int tl = 0) {
        nx = g.nx;
        ny = g.ny;
        mask = g.mask;
        if constexpr (LIST) {
            valid = valid_;
            t = (int)(e / TPT);
            tl = (int)(e - (unsigned)t * TPT);
            const unsigned ep = __shfl_up_sync(LBM_FULL, e, 1), en = __shfl_down_sync(LBM_FULL, e, 1);
            const int lane = threadIdx.x & 31;
            lnb = lane > 0 && ep + 1u == e && (tl % TPR) > 0;
            rnb = lane < 31 && en == e + 1u && (tl % TPR) < TPR - 1;
        }
        ly = tl / TPR;
        xv = tl - ly * TPR;
        lx0 = xv * VEC;
        const int txy = __ldg(g.tile_xy + t);
        tx = txy & 0xFFFF;
        ty = txy >> 16;
        int nb[9];
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const int n = __ldg(g.nbr + 9 * t + j);
            nb[j] = n < 0 ? t : n; // absent: any valid tile, the value is unused
        }
#pragma unroll
        for (int d = -1; d <= 1; ++d) {
            const int r = ly + d;
            const int oy = r < 0 ? -1 : (r >= TILE ? 1 : 0);
            const unsigned rr = (unsigned)((r & (TILE - 1)) * TILE);
            const unsigned base = (unsigned)pick3(oy, nb[1], nb[4], nb[7]) * (9u * TILE_N) + rr;
            rowb[d + 1] = base + lx0;
            lb[d + 1] = xv == 0 ? (unsigned)pick3(oy, nb[0], nb[3], nb[6]) * (9u * TILE_N) + rr + (TILE - 1)
                                : base + lx0 - 1;
            rb[d + 1] = xv == TPR - 1 ? (unsigned)pick3(oy, nb[2], nb[5], nb[8]) * (9u * TILE_N) + rr
                                      : base + lx0 + VEC;
        }
    }
    __device__ __forceinline__ unsigned vidx(int slot, int dy) const {
        return rowb[dy + 1] + (unsigned)(slot * TILE_N);
    }
    // element (x0 + k + dx, y + dy), k + dx in [-1, VEC], dy in {-1, 0, 1}
    __device__ __forceinline__ unsigned eidx(int slot, int k, int dx, int dy) const {
        if (k + dx < 0) return lb[dy + 1] + (unsigned)(slot * TILE_N);
        if (k + dx >= VEC) return rb[dy + 1] + (unsigned)(slot * TILE_N);
        return rowb[dy + 1] + (unsigned)(slot * TILE_N + k + dx);
    }
    __device__ __forceinline__ bool left_in_warp(int) const { return LIST ? lnb : xv > 0; }
    __device__ __forceinline__ bool right_in_warp(int) const { return LIST ? rnb : xv < TPR - 1; }
    __device__ __forceinline__ int gx(int k) const { return tx * TILE + lx0 + k; }
    __device__ __forceinline__ int gy() const { return ty * TILE + ly; }
    __device__ __forceinline__ bool in_domain() const { return gy() < ny; }
    __device__ __forceinline__ long long node(int k) const { return (long long)gy() * nx + gx(k); }
    __device__ __forceinline__ const uint8_t *mask_ptr() const {
        return mask + (long long)t * TILE_N + ly * TILE + lx0;
    }
};

// Which wall side link i of node (x, y) crosses (0 W, 1 E, 2 S, 3 N), or 4
// when its source is an obstacle node.  The y side is examined first.
__device__ __forceinline__ int wall_side(const Geo &g, int x, int y, int i) {
    const int sy = y - cy(i);
    if ((sy < 0 || sy >= g.ny) && !g.periodic_y) return sy < 0 ? 2 : 3;
    const int sx = x - cx(i);
    if ((sx < 0 || sx >= g.nx) && !g.periodic_x) return sx < 0 ? 0 : 1;
    return 4;
}

// ------------------------------------------------------------- physics

// Physics constants in the compute type (FP32 copies are rounded on the host,
// so no kernel converts FP64 to FP32).
template <class C> struct PC;
template <> struct PC<double> {
    static __device__ __forceinline__ double omega(const Phys &p) { return p.omega; }
    static __device__ __forceinline__ double om1(const Phys &p) { return 1.0 - p.omega; }
    static __device__ __forceinline__ double kk(const Phys &p) { return 1.0 - 0.5 * p.omega; }
    static __device__ __forceinline__ double tau_h(const Phys &p) { return p.tau_h; }
    static __device__ __forceinline__ double fx(const Phys &p) { return p.fx; }
    static __device__ __forceinline__ double fy(const Phys &p) { return p.fy; }
    static __device__ __forceinline__ double wt(const Phys &p, int s, int i) { return p.wt[s][i]; }
};
template <> struct PC<float> {
    static __device__ __forceinline__ float omega(const Phys &p) { return p.omega_f; }
    static __device__ __forceinline__ float om1(const Phys &p) { return p.om1_f; }
    static __device__ __forceinline__ float kk(const Phys &p) { return p.kk_f; }
    static __device__ __forceinline__ float tau_h(const Phys &p) { return p.tau_h_f; }
    static __device__ __forceinline__ float fx(const Phys &p) { return p.fx_f; }
    static __device__ __forceinline__ float fy(const Phys &p) { return p.fy_f; }
    static __device__ __forceinline__ float wt(const Phys &p, int s, int i) { return p.wt_f[s][i]; }
};

// Correctly rounded reciprocal (same value as 1/x in IEEE division).
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return __drcp_rn(x); }

// Rounded-to-nearest arithmetic the compiler may not contract or reorder,
// for the error-free transformations below.
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
// Knuth's TwoSum: s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = rn_add(a, b);
    const float bb = rn_sub(s, a);
    e = rn_add(rn_sub(a, rn_sub(s, bb)), rn_sub(b, bb));
}

// Moments of the gathered shifted f' (Eq. 2; u shifted by F/2), and the
// momentum j = m + F/2 = rho u.  COMP: j is returned as jx + jxl exactly
// (TwoSum), because F/2 is often below half an ulp of m and rounding it away
// would bias the momentum gain the same way every step.
// SC: f' in units of SC (f - w times SC); drho, jx, jy come out in those
// units, rho, inv and u in plain ones (inv = 1 / (SC rho), so u = j inv).
template <class C, bool HAS_F, bool COMP = false, int SC = 1>
__device__ __forceinline__ void moments_j(const C f[9], C Fx, C Fy, C &drho, C &rho, C &inv, C &ux, C &uy,
                                          C &jx, C &jy, C &jxl, C &jyl) {
    drho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    rho = C(1) + drho * C(1.0 / SC);
    const C a = f[5] - f[7], b = f[8] - f[6];
    const C mx = ((f[1] - f[3]) + a) + b;
    const C my = ((f[2] - f[4]) + a) - b;
    inv = recip(rho) * C(1.0 / SC);
    jxl = jyl = C(0);
    if (HAS_F) {
        if constexpr (COMP) {
            two_sum(mx, C(0.5) * Fx, jx, jxl);
            two_sum(my, C(0.5) * Fy, jy, jyl);
        } else {
            jx = mx + C(0.5 * SC) * Fx;
            jy = my + C(0.5 * SC) * Fy;
        }
    } else {
        jx = mx;
        jy = my;
    }
    ux = jx * inv;
    uy = jy * inv;
}
template <class C, bool HAS_F>
__device__ __forceinline__ void moments(const C f[9], C Fx, C Fy, C &drho, C &rho, C &inv, C &ux,
                                        C &uy) {
    C jx, jy, jxl, jyl;
    moments_j<C, HAS_F>(f, Fx, Fy, drho, rho, inv, ux, uy, jx, jy, jxl, jyl);
}

template <class C> struct Coef {
    C om, om1, kk, th;
    C kh[2], kl[2]; // omega/3, omega/12 (axis, diagonal); kl: low part (FP32)
    // two-relaxation-time: tp = (1 - omega)/2, tm = (1 - omega_m)/2, the odd
    // constants omega_m/3, omega_m/12 (float pair in FP32), 1/omega_m - 1/2,
    // 1 - omega_m/2
    int trt;
    C tp, tm, khm[2], klm[2], thm, kkm;
    __device__ __forceinline__ explicit Coef(const Phys &ph)
        : om(PC<C>::omega(ph)), om1(PC<C>::om1(ph)), kk(PC<C>::kk(ph)), th(PC<C>::tau_h(ph)), trt(ph.trt) {
        if constexpr (sizeof(C) == 8) {
            kh[0] = C(ph.kq[0]);
            kh[1] = C(ph.kq[1]);
            kl[0] = kl[1] = C(0);
            tp = C(ph.tp);
            tm = C(ph.tm);
            khm[0] = C(ph.kqm[0]);
            khm[1] = C(ph.kqm[1]);
            klm[0] = klm[1] = C(0);
            thm = C(ph.thm);
            kkm = C(1.0 - 0.5 * ph.omega_m);
        } else {
            kh[0] = C(ph.kq_hi[0]);
            kh[1] = C(ph.kq_hi[1]);
            kl[0] = C(ph.kq_lo[0]);
            kl[1] = C(ph.kq_lo[1]);
            tp = C(ph.tp_f);
            tm = C(ph.tm_f);
            khm[0] = C(ph.kqm_hi[0]);
            khm[1] = C(ph.kqm_hi[1]);
            klm[0] = C(ph.kqm_lo[0]);
            klm[1] = C(ph.kqm_lo[1]);
            thm = C(ph.thm_f);
            kkm = C(ph.kkm_f);
        }
    }
};

// Two-relaxation-time collision (Coef::trt) on the moments collide() has
// formed: the even part of every pair of opposite links relaxes exactly as
// in BGK at omega, the odd part at omega_m, and each part gets its share of
// the Guo source with its own factor (1 - rate/2):
//   f_i <- tp (f_i + f_opp) + tm (f_i - f_opp) + E_i + O_i,
//   f_opp <- tp (f_i + f_opp) - tm (f_i - f_opp) + E_i - O_i,
// E_i the even part of omega (f^eq_i - w_i) + (1 - omega/2) G_i (as in BGK),
// O_i = 3 w_i omega_m (c_i . (j + (1/omega_m - 1/2) F)) its odd part, j = rho u.
// COMP (FP32 storage): the odd constant as a float pair with an error-free
// product, tm from 1 - omega_m exactly, as in the BGK form.
template <class C, bool HAS_F, bool COMP, int SC>
__device__ __forceinline__ void collide_trt(C f[9], C Fx, C Fy, const Coef<C> &co, C drho, C rs, C ux, C uy,
                                            C jx, C jy, C jxl, C jyl, C usq, C uF) {
    const C om = co.om, om1 = co.om1, tp = co.tp, tm = co.tm;
    if constexpr (COMP) {
        C K0 = C(0), Ka = C(0), Kd = C(0), Kam = C(0), Kdm = C(0);
        if (HAS_F) {
            K0 = co.kk * C(4.0 / 9.0);
            Ka = co.kk * C(1.0 / 9.0);
            Kd = co.kk * C(1.0 / 36.0);
            Kam = co.kkm * C(1.0 / 9.0);
            Kdm = co.kkm * C(1.0 / 36.0);
        }
        const C R0 = (om * C(4.0 / 9.0)) * rs, Ra = (om * C(1.0 / 9.0)) * rs, Rd = (om * C(1.0 / 36.0)) * rs;
        const C E0 = (om * C(4.0 / 9.0)) * drho, Ea = (om * C(1.0 / 9.0)) * drho, Ed = (om * C(1.0 / 36.0)) * drho;
        {
            C G = E0 - R0 * usq;
            if (HAS_F) G = G + K0 * (C(-3) * uF);
            f[0] = om1 * f[0] + G;
        }
#define LBM_TRT_PAIR(I, J, T, SH, SL, CF, RQ, EQ, KQ, KQM, Q)                                 \
    {                                                                                       \
        const C t = (T);                                                                    \
        C P = EQ + RQ * (C(4.5) * (t * t) - usq);                                           \
        const C qh = rn_mul(co.khm[Q], (SH));                                               \
        C ql = rn_add(rn_fma(co.khm[Q], (SH), -qh), rn_fma(co.khm[Q], (SL), rn_mul(co.klm[Q], (SH)))); \
        if (HAS_F) {                                                                        \
            const C cf = (CF);                                                              \
            P = P + KQ * (C(9) * (t * cf) - C(3) * uF);                                     \
            ql = ql + (C(3) * KQM) * cf;                                                    \
        }                                                                                   \
        const C sp = f[I] + f[J], sm = f[I] - f[J];                                         \
        f[I] = tp * sp + tm * sm + rn_add(rn_add(P, qh), ql);                               \
        f[J] = tp * sp - tm * sm + rn_sub(rn_sub(P, qh), ql);                               \
    }
        C sd1h, sd1l, sd2h, sd2l;
        two_sum(jx, jy, sd1h, sd1l);
        two_sum(jy, -jx, sd2h, sd2l);
        if (HAS_F) {
            sd1l = sd1l + (jxl + jyl);
            sd2l = sd2l + (jyl - jxl);
        }
        LBM_TRT_PAIR(1, 3, ux, jx, jxl, Fx, Ra, Ea, Ka, Kam, 0)
        LBM_TRT_PAIR(2, 4, uy, jy, jyl, Fy, Ra, Ea, Ka, Kam, 0)
        LBM_TRT_PAIR(5, 7, ux + uy, sd1h, sd1l, Fx + Fy, Rd, Ed, Kd, Kdm, 1)
        LBM_TRT_PAIR(6, 8, uy - ux, sd2h, sd2l, Fy - Fx, Rd, Ed, Kd, Kdm, 1)
#undef LBM_TRT_PAIR
    } else {
        C Z = drho - rs * usq;
        const C r45 = C(4.5) * rs;
        const C w0 = om * C(4.0 / 9.0), wa = om * C(1.0 / 9.0), wd = om * C(1.0 / 36.0);
        C vx = jx, vy = jy, kx = jx, ky = jy;
        if (HAS_F) {
            const C h = co.th * C(SC), hm = co.thm * C(SC);
            Z = Z - (C(3) * h) * uF;
            kx = jx + hm * Fx;
            ky = jy + hm * Fy;
            vx = jx + (C(2) * h) * Fx;
            vy = jy + (C(2) * h) * Fy;
        }
        f[0] = om1 * f[0] + w0 * Z;
#define LBM_TRT_PAIR(I, J, T, TV, SK, WQ, Q)                                                \
    {                                                                                       \
        const C t = (T);                                                                    \
        C y;                                                                                \
        if (HAS_F) y = Z + (C(4.5) * t) * (TV);                                             \
        else y = Z + r45 * (t * t);                                                         \
        C q = co.khm[Q] * (SK);                                                             \
        if constexpr (sizeof(C) == 4) q = q + co.klm[Q] * (SK);                             \
        const C e = WQ * y, sp = f[I] + f[J], sm = f[I] - f[J];                             \
        f[I] = tp * sp + tm * sm + (e + q);                                                 \
        f[J] = tp * sp - tm * sm + (e - q);                                                 \
    }
        LBM_TRT_PAIR(1, 3, ux, vx, kx, wa, 0)
        LBM_TRT_PAIR(2, 4, uy, vy, ky, wa, 0)
        LBM_TRT_PAIR(5, 7, ux + uy, vx + vy, kx + ky, wd, 1)
        LBM_TRT_PAIR(6, 8, uy - ux, vy - vx, ky - kx, wd, 1)
#undef LBM_TRT_PAIR
    }
}

// BGK relaxation with Guo source, in shifted variables, in place on f:
//   f_i <- f_i + omega (f^eq_i - w_i - f_i) + S_i
// evaluated pairwise over opposite links (c_opp = -c): the even part of
// f^eq - w and S is shared, the odd part changes sign.  The odd part of
// omega f^eq is built from the momentum itself, 3 omega w_i (c_i . j) with
// j = rho u = m + F/2, so that its momentum is omega j by construction.
// COMP (FP32 storage): 3 omega w_i is carried as a float pair and the product
// is formed error-free, because a constant rounded to FP32 would scale the
// equilibrium momentum of every node by the same (1 + eps) each step -- a
// bias that grows linearly with the step count in slowly varying flows.
// FP16s (on its 2^10 scale) applies the float pair without the error-free
// product: that removes the bias of the rounded constant, the same for every
// node and step; what the product's rounding leaves varies from node to
// node and is far below binary16's storage rounding.
// SC: f in units of SC (the FP16s step works in f - w times 2^10, so its
// decode and encode need no scaling); the constants that multiply plain
// quantities (rho, u, F) carry the factor.
template <class C, bool HAS_F, bool COMP, int SC = 1, bool TRT = false>
__device__ __forceinline__ void collide(C f[9], C Fx, C Fy, const Coef<C> &co) {
    static_assert(SC == 1 || !COMP, "the compensated form works in plain units");
    C drho, rho, inv, ux, uy, jx, jy, jxl, jyl;
    moments_j<C, HAS_F, COMP, SC>(f, Fx, Fy, drho, rho, inv, ux, uy, jx, jy, jxl, jyl);
    const C usq = C(1.5) * (ux * ux + uy * uy);
    const C om = co.om, om1 = co.om1;
    const C rs = rho * C(SC);
    const C uF = HAS_F ? ux * Fx + uy * Fy : C(0);
    if constexpr (TRT) {
        collide_trt<C, HAS_F, COMP, SC>(f, Fx, Fy, co, drho, rs, ux, uy, jx, jy, jxl, jyl, usq, uF);
        return;
    }
    if constexpr (COMP) {
        // Guo source weights (1 - omega/2) w_q
        C K0 = C(0), Ka = C(0), Kd = C(0);
        if (HAS_F) {
            K0 = co.kk * C(4.0 / 9.0);
            Ka = co.kk * C(1.0 / 9.0);
            Kd = co.kk * C(1.0 / 36.0);
        }
        // omega * w_q * rho and omega * w_q * drho per weight class
        const C R0 = (om * C(4.0 / 9.0)) * rs, Ra = (om * C(1.0 / 9.0)) * rs, Rd = (om * C(1.0 / 36.0)) * rs;
        const C E0 = (om * C(4.0 / 9.0)) * drho, Ea = (om * C(1.0 / 9.0)) * drho, Ed = (om * C(1.0 / 36.0)) * drho;
        // rest
        {
            C G = E0 - R0 * usq;
            if (HAS_F) G = G + K0 * (C(-3) * uF);
            f[0] = om1 * f[0] + G;
        }
        // one pair of opposite links: T = c_i . u, S = c_i . j (SL: its low
        // part), CF = c_i . F, weight class Q (0 axis, 1 diagonal)
#define LBM_PAIR(I, J, T, SH, SL, CF, RQ, EQ, KQ, Q)                                        \
    {                                                                                       \
        const C t = (T);                                                                    \
        C P = EQ + RQ * (C(4.5) * (t * t) - usq);                                           \
        const C qh = rn_mul(co.kh[Q], (SH));                                                \
        C ql = rn_add(rn_fma(co.kh[Q], (SH), -qh), rn_fma(co.kh[Q], (SL), rn_mul(co.kl[Q], (SH)))); \
        if (HAS_F) {                                                                        \
            const C cf = (CF);                                                              \
            P = P + KQ * (C(9) * (t * cf) - C(3) * uF);                                     \
            ql = ql + (C(3) * KQ) * cf;                                                     \
        }                                                                                   \
        f[I] = om1 * f[I] + rn_add(rn_add(P, qh), ql);                                      \
        f[J] = om1 * f[J] + rn_sub(rn_sub(P, qh), ql);                                      \
    }
        C sd1h, sd1l, sd2h, sd2l;
        two_sum(jx, jy, sd1h, sd1l);
        two_sum(jy, -jx, sd2h, sd2l);
        if (HAS_F) {
            sd1l = sd1l + (jxl + jyl);
            sd2l = sd2l + (jyl - jxl);
        }
        LBM_PAIR(1, 3, ux, jx, jxl, Fx, Ra, Ea, Ka, 0)
        LBM_PAIR(2, 4, uy, jy, jyl, Fy, Ra, Ea, Ka, 0)
        LBM_PAIR(5, 7, ux + uy, sd1h, sd1l, Fx + Fy, Rd, Ed, Kd, 1)
        LBM_PAIR(6, 8, uy - ux, sd2h, sd2l, Fy - Fx, Rd, Ed, Kd, 1)
#undef LBM_PAIR
    } else {
        // FP64 and FP16s: the even part of omega (f^eq_i - w_i) is
        // omega w_q (Z + 4.5 rho t^2) with Z = drho - rho usq, one product
        // per link pair on top of t^2 (FP64 is bound by its FP64 pipe, FP16s
        // by instruction issue); the odd part, 3 omega w_q (c_i . j), is one
        // value q that the pair adds and subtracts (FP16s: the constant as a
        // float pair, kh S + kl S).  With a force, the Guo source joins both
        // parts per node instead of per link: with h = tau - 1/2,
        //   even: omega w_q (Z - 3 h (u . F) + 4.5 t (c_i . (j + 2 h F)))
        //   odd:  3 omega w_q (c_i . (j + h F)),
        // which is Eq. 6 and the source term, regrouped.
        C Z = drho - rs * usq;
        const C r45 = C(4.5) * rs;
        const C w0 = om * C(4.0 / 9.0), wa = om * C(1.0 / 9.0), wd = om * C(1.0 / 36.0);
        C vx = jx, vy = jy, kx = jx, ky = jy;
        if (HAS_F) {
            const C h = co.th * C(SC);
            Z = Z - (C(3) * h) * uF;
            kx = jx + h * Fx;
            ky = jy + h * Fy;
            vx = jx + (C(2) * h) * Fx;
            vy = jy + (C(2) * h) * Fy;
        }
        f[0] = om1 * f[0] + w0 * Z;
#define LBM_PAIR(I, J, T, TV, SK, WQ, Q)                                                    \
    {                                                                                       \
        const C t = (T);                                                                    \
        C y;                                                                                \
        if (HAS_F) y = Z + (C(4.5) * t) * (TV);                                             \
        else y = Z + r45 * (t * t);                                                         \
        C q = co.kh[Q] * (SK);                                                              \
        if constexpr (sizeof(C) == 4) q = q + co.kl[Q] * (SK);                              \
        f[I] = om1 * f[I] + (WQ * y + q);                                                   \
        f[J] = om1 * f[J] + (WQ * y - q);                                                   \
    }
        LBM_PAIR(1, 3, ux, vx, kx, wa, 0)
        LBM_PAIR(2, 4, uy, vy, ky, wa, 0)
        LBM_PAIR(5, 7, ux + uy, vx + vy, kx + ky, wd, 1)
        LBM_PAIR(6, 8, uy - ux, vy - vx, ky - kx, wd, 1)
#undef LBM_PAIR
    }
}

// ------------------------------------------------------------- open sides

// Open side `side` at boundary node (x, y) (Zou & He, for any side): the
// links of mask m that pull from beyond the side are unknown; the known
// shifted values f' fix rho (1 + u.n) = 1 + sum_{c.n=0} f'_j + 2 sum_{c.n>0} f'_j
// (the weights of those links sum to 1), with u given (velocity side) or rho
// given and u = (u.n) n (pressure side); then
//   f'_i = f'_opp(i) + 6 w_i rho (c_i . u) - (c_i . t) N_t,
//   N_t = 1/2 sum_{c.n=0} (c_j . t) f'_j - rho (u . t)/3.
// f in units of SC (f - w times SC, as in the step kernel).  Returns the set
// of links it wrote (bit i).
template <class C, int SC = 1>
__device__ unsigned open_side(const Geo &g, const Phys &ph, int x, int y, int side, unsigned m, C f[9]) {
    unsigned unk = 0;
#pragma unroll
    for (int i = 1; i < 9; ++i)
        if (((m >> (i - 1)) & 1u) && wall_side(g, x, y, i) == side) unk |= 1u << i;
    if (!unk) return 0u;
    const int nx_ = side == 0 ? -1 : (side == 1 ? 1 : 0), ny_ = side == 2 ? -1 : (side == 3 ? 1 : 0);
    const int tx = nx_ == 0, ty = ny_ == 0;
    C d = C(0), st = C(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int cn = cx(i) * nx_ + cy(i) * ny_;
        if (cn == 0) {
            d += f[i];
            st += C(cx(i) * tx + cy(i) * ty) * f[i];
        } else if (cn > 0) {
            d += C(2) * f[i];
        }
    }
    const int k = side < 2 ? y : x, len = side < 2 ? g.ny : g.nx;
    const C *val = reinterpret_cast<const C *>(ph.open_val[side]);
    C rho, ux, uy;
    if (ph.open_kind[side] == LBM_SIDE_VELOCITY) {
        if (val) {
            ux = val[k];
            uy = val[len + k];
        } else if constexpr (sizeof(C) == 8) {
            ux = ph.open_u[side][0];
            uy = ph.open_u[side][1];
        } else {
            ux = ph.open_u_f[side][0];
            uy = ph.open_u_f[side][1];
        }
        rho = (C(1) + d * C(1.0 / SC)) / (C(1) + (C(nx_) * ux + C(ny_) * uy));
    } else {
        if (val) rho = val[k];
        else if constexpr (sizeof(C) == 8) rho = ph.open_rho[side];
        else rho = ph.open_rho_f[side];
        const C un = (C(1) + d * C(1.0 / SC) - rho) / rho;
        ux = C(nx_) * un;
        uy = C(ny_) * un;
    }
    const C rs = rho * C(SC);
    const C Nt = C(0.5) * st - rs * (C(tx) * ux + C(ty) * uy) * C(1.0 / 3.0);
#pragma unroll
    for (int i = 1; i < 9; ++i)
        if ((unk >> i) & 1u)
            f[i] = f[opp(i)] + C(6) * wgt<C>(i) * rs * (C(cx(i)) * ux + C(cy(i)) * uy) -
                   C(cx(i) * tx + cy(i) * ty) * Nt;
    return unk;
}

// Every open side whose row or column holds (x, y).
template <class C, int SC = 1>
__device__ __forceinline__ void apply_open(const Geo &g, const Phys &ph, int x, int y, unsigned m, C f[9]) {
    if (!ph.has_open || m == 0u) return;
    const bool on[4] = {x == 0, x == g.nx - 1, y == 0, y == g.ny - 1};
#pragma unroll
    for (int s = 0; s < 4; ++s)
        if (ph.open_kind[s] != LBM_SIDE_WALL && on[s]) open_side<C, SC>(g, ph, x, y, s, m, f);
}



// ------------------------------------------------------------- step kernel

// Gather of the aligned vectors (and the one edge value per x-shifted slot)
// that hold f'_i of this thread's VEC nodes.  Slot pulled for link i: i
// (two-lattice) or opp(i) (AA gather/scatter step); AA local step reads the
// thread's own vectors.
template <class S, int MODE, class A>
__device__ __forceinline__ void gather_raw(const A &ad, const typename S::R *src, bool active, int lane,
                                           unsigned long long mv, V16<typename S::R, S::VEC> raw[9],
                                           typename S::R edge[9]) {
    typedef typename S::R R;
    constexpr int VEC = S::VEC;
    constexpr bool NC = (MODE == MODE_TWO_LATTICE);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int slot = (MODE == MODE_AA_PULLPUSH) ? opp(i) : i;
        const int dy = (MODE == MODE_AA_LOCAL) ? 0 : -cy(i);
        if (active) raw[i] = ld16<NC, R, VEC>(src + ad.vidx(slot, dy));
        else zero16(raw[i]);
        edge[i] = R(0);
    }
    if constexpr (MODE == MODE_AA_LOCAL) return;
    // Neighbour lanes whose VEC nodes are all solid (inactive) load nothing.
    // The values this lane pulls through them are then either solid (links
    // along x: bounced) or in the row above/below (diagonals), which this
    // lane loads itself unless its own mask bounces that link.  Over the
    // list the edge values are loaded whether bounced or not (the addresses
    // are in bounds, the bounce-back overwrites them), so that no load of
    // the gather waits for the mask.
    const bool lact = __shfl_up_sync(LBM_FULL, active ? 1 : 0, 1) != 0;
    const bool ract = __shfl_down_sync(LBM_FULL, active ? 1 : 0, 1) != 0;
    const bool lin = ad.left_in_warp(lane) && lact;
    const bool rin = ad.right_in_warp(lane) && ract;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const int slot = (MODE == MODE_AA_PULLPUSH) ? opp(i) : i;
        if (cx(i) == 1) {
            const bool bounced = !A::LIST_ && ((mv >> (i - 1)) & 1ull); // node 0
            if (active && !lin && !(ad.left_in_warp(lane) && cy(i) == 0) && !bounced)
                edge[i] = ld1<NC>(src + ad.eidx(slot, 0, -1, -cy(i)));
        }
        if (cx(i) == -1) {
            const bool bounced = !A::LIST_ && ((mv >> (8 * (VEC - 1) + i - 1)) & 1ull); // node VEC-1
            if (active && !rin && !(ad.right_in_warp(lane) && cy(i) == 0) && !bounced)
                edge[i] = ld1<NC>(src + ad.eidx(slot, VEC - 1, 1, -cy(i)));
        }
    }
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        if (cx(i) == 1) {
            const R l = shfl_up1(raw[i].v[VEC - 1]);
            if (lin) edge[i] = l;
        } else if (cx(i) == -1) {
            const R r = shfl_down1(raw[i].v[0]);
            if (rin) edge[i] = r;
        }
    }
}

// Stored value of link i for node k of the thread (before bounce-back).
template <class S, int I, int K>
__device__ __forceinline__ typename S::R pulled(const V16<typename S::R, S::VEC> raw[9],
                                                const typename S::R edge[9], int mode) {
    constexpr int VEC = S::VEC;
    if (mode == MODE_AA_LOCAL || cx(I) == 0) return raw[I].v[K];
    if (cx(I) == 1) return K == 0 ? edge[I] : raw[I].v[(K + VEC - 1) % VEC];
    return K == VEC - 1 ? edge[I] : raw[I].v[(K + 1) % VEC];
}

template <class S, int K, int MODE>
__device__ __forceinline__ void node_values(const V16<typename S::R, S::VEC> raw[9],
                                            const typename S::R edge[9], typename S::C f[9]) {
    f[0] = S::dec_step(pulled<S, 0, K>(raw, edge, MODE));
    f[1] = S::dec_step(pulled<S, 1, K>(raw, edge, MODE));
    f[2] = S::dec_step(pulled<S, 2, K>(raw, edge, MODE));
    f[3] = S::dec_step(pulled<S, 3, K>(raw, edge, MODE));
    f[4] = S::dec_step(pulled<S, 4, K>(raw, edge, MODE));
    f[5] = S::dec_step(pulled<S, 5, K>(raw, edge, MODE));
    f[6] = S::dec_step(pulled<S, 6, K>(raw, edge, MODE));
    f[7] = S::dec_step(pulled<S, 7, K>(raw, edge, MODE));
    f[8] = S::dec_step(pulled<S, 8, K>(raw, edge, MODE));
}

// Stored value of slot s at the thread's own node k.  Slots 0, 1, 3 are in
// the gathered vectors already (their pulls come from the node's own row,
// unshifted in memory); the others were preloaded into `own` when some node
// of the vector bounces a link that needs them.
template <class S, int MODE>
__device__ __forceinline__ typename S::R own_value(const V16<typename S::R, S::VEC> raw[9],
                                                   const V16<typename S::R, S::VEC> own[9], int s, int k) {
    if (s == 0 || s == 1 || s == 3) return MODE == MODE_TWO_LATTICE ? raw[s].v[k] : raw[opp(s)].v[k];
    return own[s].v[k];
}

// Own-node slot that half-way bounce-back of link i reads: the post-collision
// value of link opp(i) at x, held in slot opp(i) (two-lattice) or in slot i
// (AA gather/scatter step, where slot i of x holds link opp(i)'s value).
template <int MODE> __host__ __device__ constexpr int bounce_slot(int i) {
    return MODE == MODE_TWO_LATTICE ? opp(i) : i;
}

// Loads, right after the gather, the own-node vectors of the slots that the
// vector's bounced links need (union of the fluid nodes' mask bits).
template <class S, int MODE, class A>
__device__ __forceinline__ void preload_own(const A &ad, const typename S::R *src, unsigned long long mv,
                                            V16<typename S::R, S::VEC> own[9]) {
    constexpr int VEC = S::VEC;
    constexpr bool NC = (MODE == MODE_TWO_LATTICE);
    unsigned bits = 0;
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
        const unsigned m = (unsigned)((mv >> (8 * k)) & 0xFFu);
        bits |= (m == 0xFFu) ? 0u : m;
    }
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const int sl = bounce_slot<MODE>(i);
        if (sl == 0 || sl == 1 || sl == 3) continue;
        if (bits & (1u << (i - 1))) own[sl] = ld16<NC, typename S::R, VEC>(src + ad.vidx(sl, 0));
    }
}

// Half-way bounce-back for the links of node k whose mask bit is set:
// f'_i = (stored post-collision value of link opp(i) at x) + wall term.
template <class S, int MODE, class A>
__device__ __forceinline__ void bounce(const Geo &g, const Phys &ph, const A &ad, const typename S::R *src,
                                       const V16<typename S::R, S::VEC> raw[9],
                                       const V16<typename S::R, S::VEC> own[9], int k, unsigned m,
                                       typename S::C f[9]) {
    typedef typename S::C C;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        if (m & (1u << (i - 1))) {
            C v;
            constexpr bool NC = (MODE == MODE_TWO_LATTICE);
            const int sl = bounce_slot<MODE>(i);
            if (MODE == MODE_AA_LOCAL) v = f[i];
            else if (OwnPreload<S, MODE>::value || sl == 0 || sl == 1 || sl == 3)
                v = S::dec_step(own_value<S, MODE>(raw, own, sl, k));
            else
                v = S::dec_step(ld1<NC>(src + ad.eidx(sl, k, 0, 0)));
            if (ph.has_wall) v = v + PC<C>::wt(ph, wall_side(g, ad.gx(k), ad.gy(), i), i) * C(S::SCALE);
            f[i] = v;
        }
    }
}

template <class S, int FORCE, class A>
__device__ __forceinline__ void load_force(const Geo &g, const Phys &ph, const A &ad, bool active,
                                           typename S::C Fx[S::VEC], typename S::C Fy[S::VEC]) {
    typedef typename S::C C;
    constexpr int VEC = S::VEC;
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
        Fx[k] = PC<C>::fx(ph);
        Fy[k] = PC<C>::fy(ph);
    }
    if (FORCE == FORCE_FIELD && active && ad.in_domain()) {
        // VEC values of each component: one 8- or 16-byte vector
        static_assert(VEC * sizeof(C) == 8 || VEC * sizeof(C) == 16, "force vector width");
        const C *F = reinterpret_cast<const C *>(ph.force);
        const long long n = ad.node(0);
        const V16<C, VEC> a = ld16<true, C, VEC>(F + n);
        const V16<C, VEC> b = ld16<true, C, VEC>(F + g.nnode + n);
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            Fx[k] = a.v[k];
            Fy[k] = b.v[k];
        }
    }
}

// Stochastic rounding of the thread's nodes: the per-step seed, and the
// collided values of the even node of a pair until its odd partner is done.
struct SrState {
    unsigned tseed;
    float pend[9];
};

// Stores node K's nine collided FP16s values (units of the stored scale):
// nodes 2j and 2j+1 share a 32-bit word of each slot vector and are rounded
// together, with the pair's random stream (pair_node: index of node 2j).
template <class S, int K>
__device__ __forceinline__ void put_sr(const float d[9], SrState &sr, long long pair_node,
                                       V16<typename S::R, S::VEC> out[9]) {
    static_assert(S::VEC % 2 == 0, "FP16s vectors hold whole node pairs");
    if constexpr ((K & 1) == 0) {
#pragma unroll
        for (int i = 0; i < 9; ++i) sr.pend[i] = d[i];
    } else {
        unsigned h = fmix32((unsigned)pair_node ^ sr.tseed);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            h = lcg_next(h);
            set_word<K / 2>(out[i].u, f16x2_rs(sr.pend[i], d[i], h ^ (h >> 16)));
        }
    }
}

template <class S, class A, int MODE, bool HAS_MASK, int FORCE, bool OPEN, int K, bool TRT>
__device__ __forceinline__ void do_node(const Geo &g, const Phys &ph, const A &ad, const typename S::R *src,
                                        const V16<typename S::R, S::VEC> own[9],
                                        unsigned long long mv, const V16<typename S::R, S::VEC> raw[9],
                                        const typename S::R edge[9], const typename S::C Fx[],
                                        const typename S::C Fy[], const Coef<typename S::C> &co, SrState &sr,
                                        V16<typename S::R, S::VEC> out[9]) {
    typedef typename S::C C;
    C f[9];
    node_values<S, K, MODE>(raw, edge, f);
    const unsigned m = HAS_MASK ? (unsigned)((mv >> (8 * K)) & 0xFFu) : 0u;
    if (HAS_MASK && m == 0xFFu) {
        if constexpr (S::STOCHASTIC) {
            const float z[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            put_sr<S, K>(z, sr, ad.node(K & ~1), out);
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) out[i].v[K] = S::enc(C(0));
        }
        return;
    }
    if (HAS_MASK && m != 0u) bounce<S, MODE>(g, ph, ad, src, raw, own, K, m, f);
    if constexpr (OPEN) apply_open<C, S::SCALE>(g, ph, ad.gx(K), ad.gy(), m, f);
    collide<C, FORCE != FORCE_NONE, (sizeof(C) == 4 && !S::STOCHASTIC), S::SCALE, TRT>(f, Fx[K], Fy[K], co);
    if constexpr (S::STOCHASTIC) {
        put_sr<S, K>(f, sr, ad.node(K & ~1), out);
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) out[i].v[K] = S::enc(f[i]);
    }
}

// Nodes K0 .. K1-1 of the thread, in order (compile-time unrolled).
template <class S, class A, int MODE, bool HAS_MASK, int FORCE, bool OPEN, int K, int K1, bool TRT>
struct NodeRange {
    static __device__ __forceinline__ void run(const Geo &g, const Phys &ph, const A &ad, const typename S::R *src,
                                               const V16<typename S::R, S::VEC> own[9],
                                               unsigned long long mv,
                                               const V16<typename S::R, S::VEC> raw[9],
                                               const typename S::R edge[9], const typename S::C Fx[],
                                               const typename S::C Fy[], const Coef<typename S::C> &co,
                                               SrState &sr, V16<typename S::R, S::VEC> out[9]) {
        if constexpr (K < K1) {
            do_node<S, A, MODE, HAS_MASK, FORCE, OPEN, K, TRT>(g, ph, ad, src, own, mv, raw, edge, Fx, Fy, co, sr,
                                                                out);
            NodeRange<S, A, MODE, HAS_MASK, FORCE, OPEN, K + 1, K1, TRT>::run(g, ph, ad, src, own, mv, raw, edge, Fx, Fy,
                                                                         co, sr, out);
        }
    }
};

// Stores of the thread's VEC nodes for the three step kinds.  actm: the
// warp's lanes that store (all of them call this together); lane: this one.
template <class S, class A, int MODE, bool HAS_MASK>
__device__ __forceinline__ void store_all(const A &ad, typename S::R *dst, unsigned long long mv,
                                           const V16<typename S::R, S::VEC> out[9], unsigned actm, int lane) {
    typedef typename S::R R;
    constexpr int VEC = S::VEC;
    if constexpr (MODE == MODE_TWO_LATTICE) {
#pragma unroll
        for (int i = 0; i < 9; ++i) st16<R, VEC>(dst + ad.vidx(i, 0), out[i]);
    } else if constexpr (MODE == MODE_AA_LOCAL) {
        // post-collision value of link i goes to slot opp(i) of the same node
#pragma unroll
        for (int i = 0; i < 9; ++i) st16<R, VEC>(dst + ad.vidx(opp(i), 0), out[i]);
    } else {
        // AA gather/scatter step: f''_i(x) goes to slot i at x + c_i, or to
        // slot opp(i) at x when x + c_i is solid or beyond a wall (link
        // opp(i) of x bounces).  Each target slot has exactly one writer.
        st16<R, VEC>(dst + ad.vidx(0, 0), out[0]);
        // realigned stores without a mask, except FP16s on tiles, where one
        // lane in four starts a tile row and its element-wise 2-byte stores
        // cost more than they save (measured -2% on the tiled box)
        if constexpr (!HAS_MASK && (sizeof(R) >= 4 || std::is_same<A, DenseAddr<VEC>>::value)) {
            // no bounced link: the x-shifted targets of the thread's VEC
            // nodes are realigned by shuffles, so that each thread stores the
            // aligned vector x0 .. x0 + VEC - 1 of the target row (as the
            // gather realigns its loads); a value whose target vector
            // belongs to a lane outside the warp, the tile row or the
            // storing lanes is stored on its own, and that lane stores its
            // other elements one by one
            const bool lin = lane > 0 && ad.left_in_warp(lane) && ((actm >> (lane - 1)) & 1u);
            const bool rin = lane < 31 && ad.right_in_warp(lane) && ((actm >> (lane + 1)) & 1u);
            __syncwarp(actm);
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                if (cx(i) == 0) {
                    st16<R, VEC>(dst + ad.vidx(i, cy(i)), out[i]);
                } else if (cx(i) == 1) {
                    // target x + 1: element k of this vector is node k - 1's
                    const R l = shfl_up1(actm, out[i].v[VEC - 1]);
                    if (lin) {
                        V16<R, VEC> v;
                        v.v[0] = l;
#pragma unroll
                        for (int k = 1; k < VEC; ++k) v.v[k] = out[i].v[k - 1];
                        st16<R, VEC>(dst + ad.vidx(i, cy(i)), v);
                    } else {
#pragma unroll
                        for (int k = 0; k < VEC - 1; ++k) dst[ad.eidx(i, k, 1, cy(i))] = out[i].v[k];
                    }
                    if (!rin) dst[ad.eidx(i, VEC - 1, 1, cy(i))] = out[i].v[VEC - 1];
                } else {
                    // target x - 1: element k of this vector is node k + 1's
                    const R r = shfl_down1(actm, out[i].v[0]);
                    if (rin) {
                        V16<R, VEC> v;
#pragma unroll
                        for (int k = 0; k < VEC - 1; ++k) v.v[k] = out[i].v[k + 1];
                        v.v[VEC - 1] = r;
                        st16<R, VEC>(dst + ad.vidx(i, cy(i)), v);
                    } else {
#pragma unroll
                        for (int k = 1; k < VEC; ++k) dst[ad.eidx(i, k, -1, cy(i))] = out[i].v[k];
                    }
                    if (!lin) dst[ad.eidx(i, 0, -1, cy(i))] = out[i].v[0];
                }
            }
        } else {
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const unsigned long long rep = mask_rep<VEC>(opp(i) - 1);
                if (cx(i) == 0 && (!HAS_MASK || (mv & rep) == 0ull)) {
                    st16<R, VEC>(dst + ad.vidx(i, cy(i)), out[i]);
                } else {
#pragma unroll
                    for (int k = 0; k < VEC; ++k) {
                        const unsigned m = HAS_MASK ? (unsigned)((mv >> (8 * k)) & 0xFFu) : 0u;
                        if (m == 0xFFu) continue;
                        if (m & (1u << (opp(i) - 1)))
                            dst[ad.eidx(opp(i), k, 0, 0)] = out[i].v[k];
                        else
                            dst[ad.eidx(i, k, cx(i), cy(i))] = out[i].v[k];
                    }
                }
            }
        }
    }
}

// Blocks of 256 threads each SM must hold (the register cap that follows):
// the FP32 / FP16s step is memory-latency bound, so occupancy is fixed here
// rather than left to the register allocator -- 4 blocks (<= 64 registers)
// without a mask, for FP32 with a mask (2 nodes per thread) and for the
// FP16s AA gather/scatter step with a mask (2 nodes per thread), 3 blocks
// (<= 80) for the other FP16s steps with a mask.  FP64 is ALU-bound and
// left free.
template <int P, bool HAS_MASK, int MODE> struct MinBlocks {
    enum {
        value = P == LBM_F64 ? 1 : ((HAS_MASK && P == LBM_F16S && MODE != MODE_AA_PULLPUSH) ? 3 : 4)
    };
};

// One step of the thread's VEC nodes at address ad (every lane of the warp
// enters together; the gather's shuffles are the only collective operations).
template <int P, class A, int MODE, bool HAS_MASK, int FORCE, bool OPEN, bool TRT>
__device__ __forceinline__ void step_vector(const Geo &g, const Phys &ph, const void *src_v, void *dst_v,
                                            const A &ad, int lane, unsigned step) {
    typedef StV<P, A::VEC_> S;
    typedef typename S::R R;
    typedef typename S::C C;
    constexpr int VEC = S::VEC;
    const R *src = reinterpret_cast<const R *>(src_v);
    R *dst = reinterpret_cast<R *>(dst_v);
    // graph replays: the step index's base, loaded first so that its latency
    // hides behind the gather
    unsigned tbase = 0u;
    if constexpr (S::STOCHASTIC)
        if (ph.tbase) tbase = (unsigned)__ldg(ph.tbase);

    unsigned long long mv = 0;
    if (HAS_MASK) mv = ad.valid ? ld_mask<VEC>(ad.mask_ptr()) : mask_ones<VEC>();
    // every vector of the list lies in a DRAM sector that holds fluid and is
    // written whole (its solid nodes hold 0 and get 0): there the gather
    // need not wait for the mask
    const bool active = ad.valid && (A::LIST_ || !(HAS_MASK && mv == mask_ones<VEC>()));
    const unsigned actm = __ballot_sync(LBM_FULL, active);
    if (actm == 0u) return; // whole warp solid: no traffic

    V16<R, VEC> raw[9];
    R edge[9];
    gather_raw<S, MODE>(ad, src, active, lane, mv, raw, edge);
    // the inactive lanes leave; the store's shuffles run among actm
    if (!active) return;
    V16<R, VEC> own[9];
    if (HAS_MASK && MODE != MODE_AA_LOCAL && OwnPreload<S, MODE>::value && mv != 0ull)
        preload_own<S, MODE>(ad, src, mv, own);

    C Fx[VEC], Fy[VEC];
    load_force<S, FORCE>(g, ph, ad, active, Fx, Fy);
    const Coef<C> co(ph);

    V16<R, VEC> out[9];
    SrState sr;
    if constexpr (S::STOCHASTIC) {
        sr.tseed = fmix32((tbase + step) * 0x9E3779B9u + 0x632BE5ABu);
    } else {
        sr.tseed = 0u;
    }
    NodeRange<S, A, MODE, HAS_MASK, FORCE, OPEN, 0, VEC, TRT>::run(g, ph, ad, src, own, mv, raw, edge, Fx, Fy, co, sr,
                                                                   out);
    store_all<S, A, MODE, HAS_MASK>(ad, dst, mv, out, actm, lane);
}

// Whether the step over the list of fluid vectors runs as a persistent grid:
// FP16s (measured +4-9% on porous media); FP32 keeps one thread per list
// entry, because the loop's state pushes its 64-register step into spills
// (measured -5-18%).
template <int P, class A> struct ListPersist {
    enum { value = A::LIST_ && P == LBM_F16S };
};

// The step kernel.  Dense, tiled, and FP32 over the list: one thread per
// vector.  FP16s over the list: a persistent grid (as many blocks as the
// SMs hold), each warp taking chunks of 32 consecutive entries in turn and
// loading the entry of its next chunk before it works on the current one,
// so that the list read -- the first of the three dependent loads (entry,
// tile record, data) -- is off the critical path.
template <int P, class A, int MODE, bool HAS_MASK, int FORCE, bool OPEN, bool TRT>
__global__ void __launch_bounds__(STEP_BLOCK, MinBlocks<P, HAS_MASK, MODE>::value)
    k_step(const Geo g, const Phys ph, const void *src_v, void *dst_v, int y0, int ystride, unsigned step) {
    const int lane = threadIdx.x & 31;
    if constexpr (ListPersist<P, A>::value) {
        const int n = A::list_len(g);
        const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
        int c = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
        unsigned e = A::entry(g, c * 32 + lane);
        while (c * 32 < n) { // warp-uniform
            const int cn = c + nwarps;
            const unsigned en = A::entry(g, cn * 32 + lane);
            const A ad(g, e, c * 32 + lane < n);
            step_vector<P, A, MODE, HAS_MASK, FORCE, OPEN, TRT>(g, ph, src_v, dst_v, ad, lane, step);
            __syncwarp();
            e = en;
            c = cn;
        }
    } else {
        const A ad(g, (int)(blockIdx.x * blockDim.x + threadIdx.x), y0 + ystride * (int)blockIdx.y);
        step_vector<P, A, MODE, HAS_MASK, FORCE, OPEN, TRT>(g, ph, src_v, dst_v, ad, lane, step);
    }
}

#include "lbm_staged.cuh"

// ------------------------------------------------------------- adjoint kernel

// Discrete adjoint of one node's collision (see the oracle's derivation):
// from lam = dL/d(post-collision f) gives g = dL/df' and dL/dF.  With
// t_i = c_i . u, the chain rule through rho = sum f' and u = (m + F/2)/rho
// gives
//   g_j = (1 - omega) lam_j + omega a + (c_j - u) . V / rho
//   a   = sum_i lam_i w_i (1 + 3 t_i + 4.5 t_i^2 - 1.5 u^2)
//   V   = sum_i lam_i [omega rho w_i (3 c_i + 9 t_i c_i - 3 u)
//                      + (1 - omega/2) w_i (9 (c_i . F) c_i - 3 F)]
//   dL/dF = V / (2 rho) + (1 - omega/2) sum_i lam_i w_i (3 (c_i - u) + 9 t_i c_i),
// and every sum over i is a combination of the weighted moments of lam,
// Lw = sum w_i lam_i, P = sum w_i lam_i c_i, M = sum w_i lam_i c_i c_i^T
// (sum w t = P.u, sum w t^2 = u.M.u, sum w t c = M u, sum w (c.F) c = M F).
template <class C, bool HAS_F>
__device__ __forceinline__ void adjoint_node(const C f[9], const C lam[9], C Fx, C Fy, C omega,
                                             C g[9], C &dFx, C &dFy) {
    C drho, rho, inv, ux, uy;
    moments<C, HAS_F>(f, Fx, Fy, drho, rho, inv, ux, uy);
    const C usq = C(1.5) * (ux * ux + uy * uy);
    const C kk = C(1) - C(0.5) * omega;
    const C W0 = C(4.0 / 9.0), Wa = C(1.0 / 9.0), Wd = C(1.0 / 36.0);
    const C s13 = lam[1] + lam[3], s24 = lam[2] + lam[4], s57 = lam[5] + lam[7], s68 = lam[6] + lam[8];
    const C d13 = lam[1] - lam[3], d24 = lam[2] - lam[4], d57 = lam[5] - lam[7], d86 = lam[8] - lam[6];
    const C sd = s57 + s68;
    const C Lw = W0 * lam[0] + Wa * (s13 + s24) + Wd * sd;
    const C Px = Wa * d13 + Wd * (d57 + d86);
    const C Py = Wa * d24 + Wd * (d57 - d86);
    const C Mxx = Wa * s13 + Wd * sd, Myy = Wa * s24 + Wd * sd, Mxy = Wd * (s57 - s68);
    const C Mux = Mxx * ux + Mxy * uy, Muy = Mxy * ux + Myy * uy;
    const C a = omega * (Lw * (C(1) - usq) + C(3) * (Px * ux + Py * uy) + C(4.5) * (ux * Mux + uy * Muy));
    const C wr = omega * rho;
    C Vx = wr * (C(3) * (Px - ux * Lw) + C(9) * Mux);
    C Vy = wr * (C(3) * (Py - uy * Lw) + C(9) * Muy);
    if (HAS_F) {
        const C MFx = Mxx * Fx + Mxy * Fy, MFy = Mxy * Fx + Myy * Fy;
        Vx += kk * (C(9) * MFx - C(3) * Fx * Lw);
        Vy += kk * (C(9) * MFy - C(3) * Fy * Lw);
    }
    const C vx = Vx * inv, vy = Vy * inv;
    const C base = a - (ux * vx + uy * vy);
    const C om1 = C(1) - omega;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        C e = base;
        if (cx(j) == 1) e += vx;
        if (cx(j) == -1) e -= vx;
        if (cy(j) == 1) e += vy;
        if (cy(j) == -1) e -= vy;
        g[j] = om1 * lam[j] + e;
    }
    dFx = C(0.5) * vx + kk * (C(3) * (Px - ux * Lw) + C(9) * Mux);
    dFy = C(0.5) * vy + kk * (C(3) * (Py - uy * Lw) + C(9) * Muy);
}

// Transpose of the open-side rules at node (x, y) applied to g: the rules are
// affine in the gathered f', so their linear part is M[:, j] = R(e_j) - R(0)
// and g becomes M^T g (identity off the open sides' rows and columns).
template <class C>
__device__ void open_transpose(const Geo &g, const Phys &ph, int x, int y, unsigned m, C gv[9]) {
    if (!ph.has_open || m == 0u) return;
    if (!((x == 0 || x == g.nx - 1) && (ph.open_kind[0] || ph.open_kind[1])) &&
        !((y == 0 || y == g.ny - 1) && (ph.open_kind[2] || ph.open_kind[3])))
        return;
    C r0[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) r0[i] = C(0);
    apply_open<C>(g, ph, x, y, m, r0);
    C out[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        C e[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) e[i] = C(i == j ? 1 : 0);
        apply_open<C>(g, ph, x, y, m, e);
        C acc = C(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) acc += (e[i] - r0[i]) * gv[i];
        out[j] = acc;
    }
#pragma unroll
    for (int j = 0; j < 9; ++j) gv[j] = out[j];
}

// One adjoint step on the dense two-lattice layout: re-gathers f' from the
// stored state A_t, reads lam_in = dL/dA_{t+1} at the node, and pushes
// g_j = dL/df'_j back along each link (to slot j at x - c_j, or to slot
// opp(j) at x for a bounced link): the transpose of the pull gather.  Every
// target has one writer; solid nodes write 0 to their own slots.  OPEN: the
// gathered f' of nodes on an open side pass through the open-side rules, and
// their gradients through the rules' transpose.
template <int P, int FORCE, bool OPEN>
__global__ void __launch_bounds__(STEP_BLOCK) k_adjoint(const Geo g, const Phys ph, const void *state_v,
                                                        const void *lam_in_v, void *lam_out_v, void *gF_v,
                                                        int y0) {
    typedef StV<P, StepVec<P, true, MODE_TWO_LATTICE, FORCE_FIELD>::value> S; // FP32: 2 nodes per thread
    typedef typename S::R R;
    typedef typename S::C C;
    constexpr int VEC = S::VEC;
    constexpr int LC = VEC < 16 / (int)sizeof(C) ? VEC : 16 / (int)sizeof(C); // values per vector
    constexpr int CH = VEC / LC;                                               // vectors per slot
    const R *src = reinterpret_cast<const R *>(state_v);
    const C *lin = reinterpret_cast<const C *>(lam_in_v);
    C *lout = reinterpret_cast<C *>(lam_out_v);
    C *gF = reinterpret_cast<C *>(gF_v);
    DenseAddr<VEC> ad(g, (int)(blockIdx.x * blockDim.x + threadIdx.x), y0 + (int)blockIdx.y);
    const int lane = threadIdx.x & 31;
    unsigned long long mv = 0;
    if (g.has_mask) mv = ad.valid ? ld_mask<VEC>(ad.mask_ptr()) : mask_ones<VEC>();
    const bool active = ad.valid;
    if (!__any_sync(LBM_FULL, active)) return;

    V16<R, VEC> raw[9];
    R edge[9];
    gather_raw<S, MODE_TWO_LATTICE>(ad, src, active, lane, mv, raw, edge);
    V16<R, VEC> own[9];
    if (mv != 0ull) preload_own<S, MODE_TWO_LATTICE>(ad, src, mv, own);
    C Fx[VEC], Fy[VEC];
    load_force<S, FORCE>(g, ph, ad, active, Fx, Fy);
    const C omega = PC<C>::omega(ph);
    const long long n0 = ad.node(0);

    C gout[9][VEC];
    C dFx[VEC], dFy[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
        dFx[k] = C(0);
        dFy[k] = C(0);
#pragma unroll
        for (int j = 0; j < 9; ++j) gout[j][k] = C(0);
    }
    C lam[9][VEC];
#pragma unroll
    for (int j = 0; j < 9; ++j) {
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            V16<C, LC> v;
            if (active) v = ld16<true, C, LC>(lin + j * g.nnode + n0 + c * LC);
            else zero16(v);
#pragma unroll
            for (int q = 0; q < LC; ++q) lam[j][c * LC + q] = v.v[q];
        }
    }
#define LBM_ADJ_NODE(K)                                                                   \
    if constexpr ((K) < VEC) {                                                            \
        const unsigned m = (unsigned)((mv >> (8 * (K))) & 0xFFu);                         \
        if (m != 0xFFu) {                                                                 \
            C f[9];                                                                       \
            node_values<S, ((K) < VEC ? (K) : 0), MODE_TWO_LATTICE>(raw, edge, f);        \
            if (m != 0u) bounce<S, MODE_TWO_LATTICE>(g, ph, ad, src, raw, own, (K), m, f);\
            if constexpr (OPEN) apply_open<C>(g, ph, ad.gx(K), ad.gy(), m, f);           \
            C l[9], gg[9];                                                                \
            for (int j = 0; j < 9; ++j) l[j] = lam[j][(K)];                               \
            adjoint_node<C, FORCE != FORCE_NONE>(f, l, Fx[(K)], Fy[(K)], omega, gg,       \
                                                 dFx[(K)], dFy[(K)]);                     \
            if constexpr (OPEN) open_transpose<C>(g, ph, ad.gx(K), ad.gy(), m, gg);      \
            for (int j = 0; j < 9; ++j) gout[j][(K)] = gg[j];                             \
        }                                                                                 \
    }
    LBM_ADJ_NODE(0)
    LBM_ADJ_NODE(1)
    LBM_ADJ_NODE(2)
    LBM_ADJ_NODE(3)
    LBM_ADJ_NODE(4)
    LBM_ADJ_NODE(5)
    LBM_ADJ_NODE(6)
    LBM_ADJ_NODE(7)
#undef LBM_ADJ_NODE
    if (!active) return;

    // push
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const unsigned long long rep = j == 0 ? 0ull : mask_rep<VEC>(j - 1);
        if (cx(j) == 0 && (j == 0 || (mv & rep) == 0ull)) {
            // all VEC targets are the aligned vector at (x0, y - c_y)
            const long long base = j * g.nnode + ad.roff[1 - cy(j)] + ad.x0;
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                V16<C, LC> v;
#pragma unroll
                for (int q = 0; q < LC; ++q) v.v[q] = gout[j][c * LC + q];
                st16<C, LC>(lout + base + c * LC, v);
            }
        } else {
#pragma unroll
            for (int k = 0; k < VEC; ++k) {
                const unsigned m = (unsigned)((mv >> (8 * k)) & 0xFFu);
                long long dst;
                if (m == 0xFFu) dst = j * g.nnode + n0 + k;                  // solid: own slot, 0
                else if (j > 0 && (m & (1u << (j - 1)))) dst = opp(j) * g.nnode + n0 + k; // bounced
                else dst = ad.eidx(j, k, -cx(j), -cy(j));
                lout[dst] = gout[j][k];
            }
        }
    }
    // dL/dF accumulation (fluid nodes contribute, solid nodes add 0)
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        V16<C, LC> a = ld16<false, C, LC>(gF + n0 + c * LC);
        V16<C, LC> b = ld16<false, C, LC>(gF + g.nnode + n0 + c * LC);
#pragma unroll
        for (int q = 0; q < LC; ++q) {
            a.v[q] += dFx[c * LC + q];
            b.v[q] += dFy[c * LC + q];
        }
        st16<C, LC>(gF + n0 + c * LC, a);
        st16<C, LC>(gF + g.nnode + n0 + c * LC, b);
    }
}

// ------------------------------------------------------------- per-node helpers

// Index of slot j at in-domain node (x, y), both layouts.
__device__ __forceinline__ long long cidx(const Geo &g, int x, int y, int j) {
    if (g.layout == LBM_DENSE) return j * g.nslot + (long long)y * g.nx + x;
    const int t = __ldg(g.tile_id + (y >> 4) * g.ntx + (x >> 4));
    return ((long long)t * 9 + j) * TILE_N + (y & 15) * TILE + (x & 15);
}
__device__ __forceinline__ unsigned node_mask(const Geo &g, int x, int y) {
    if (g.layout == LBM_DENSE) return g.has_mask ? __ldg(g.mask + (long long)y * g.nx + x) : 0u;
    const int t = __ldg(g.tile_id + (y >> 4) * g.ntx + (x >> 4));
    return t < 0 ? 0xFFu : __ldg(g.mask + (long long)t * TILE_N + (y & 15) * TILE + (x & 15));
}
__device__ __forceinline__ void wrap_xy(const Geo &g, int &x, int &y) {
    if (x < 0) x += g.nx; else if (x >= g.nx) x -= g.nx;
    if (y < 0) y += g.ny; else if (y >= g.ny) y -= g.ny;
}

// Canonical A_i(x, y) (shifted) in each phase of the lattice.
template <class S>
__device__ __forceinline__ typename S::C canon_read(const Geo &g, int phase, const typename S::R *M, int x,
                                                    int y, int i, unsigned m) {
    if (phase == PH_PLAIN) return S::dec(M[cidx(g, x, y, i)]);
    if (phase == PH_SWAPPED) return S::dec(M[cidx(g, x, y, opp(i))]);
    if (i == 0) return S::dec(M[cidx(g, x, y, 0)]);
    if (m & (1u << (opp(i) - 1))) return S::dec(M[cidx(g, x, y, opp(i))]);
    int x2 = x + cx(i), y2 = y + cy(i);
    wrap_xy(g, x2, y2);
    return S::dec(M[cidx(g, x2, y2, i)]);
}
template <class S>
__device__ __forceinline__ void canon_write(const Geo &g, int phase, typename S::R *M, int x, int y, int i,
                                            typename S::C v) {
    M[cidx(g, x, y, phase == PH_SWAPPED ? opp(i) : i)] = S::enc(v);
}

// Gathered f'_i(x, y) of the next step (shifted), in each phase.
template <class S>
__device__ __forceinline__ void gather_node(const Geo &g, const Phys &ph, int phase, const typename S::R *M,
                                            int x, int y, unsigned m, typename S::C f[9]) {
    typedef typename S::C C;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const bool b = i > 0 && (m & (1u << (i - 1)));
        C v;
        if (phase == PH_STREAMED) {
            v = S::dec(M[cidx(g, x, y, i)]);
        } else if (b) {
            v = S::dec(M[cidx(g, x, y, phase == PH_PLAIN ? opp(i) : i)]);
        } else {
            int sx = x - cx(i), sy = y - cy(i);
            wrap_xy(g, sx, sy);
            v = S::dec(M[cidx(g, sx, sy, phase == PH_PLAIN ? i : opp(i))]);
        }
        if (b && ph.has_wall) v = v + PC<C>::wt(ph, wall_side(g, x, y, i), i);
        f[i] = v;
    }
}

template <class C>
__device__ __forceinline__ void node_force(const Geo &g, const Phys &ph, long long n, C &Fx, C &Fy) {
    if (ph.force_mode == FORCE_FIELD) {
        const C *F = reinterpret_cast<const C *>(ph.force);
        Fx = F[n];
        Fy = F[g.nnode + n];
    } else {
        Fx = PC<C>::fx(ph);
        Fy = PC<C>::fy(ph);
    }
}

// One thread per node on a 2-D grid: x along blockIdx.x, rows on blockIdx.y
// (blockIdx.z counts chunks of gridDim.y rows).  No integer division.
#define LBM_NODE_LOOP(g)                                                                   \
    const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x);                            \
    const int y = (int)(blockIdx.z * gridDim.y + blockIdx.y);                              \
    if (x >= (g).nx || y >= (g).ny) return;                                                \
    const long long n = (long long)y * (g).nx + x;

template <int P>
__global__ void k_init(const Geo g, int phase, const void *rho_v, const void *u_v, void *lat_v) {
    typedef St<P> S;
    typedef typename S::C C;
    LBM_NODE_LOOP(g)
    const unsigned m = node_mask(g, x, y);
    if (m == 0xFFu && g.layout != LBM_DENSE) {
        // node in an absent tile has no storage
        const int t = __ldg(g.tile_id + (y >> 4) * g.ntx + (x >> 4));
        if (t < 0) return;
    }
    typename S::R *M = reinterpret_cast<typename S::R *>(lat_v);
    const C *rho = reinterpret_cast<const C *>(rho_v);
    const C *u = reinterpret_cast<const C *>(u_v);
    C drho = C(0), ux = C(0), uy = C(0);
    if (m != 0xFFu) {
        if (rho) drho = rho[n] - C(1);
        if (u) {
            ux = u[n];
            uy = u[g.nnode + n];
        }
    }
    const C r = C(1) + drho;
    const C usq = C(1.5) * (ux * ux + uy * uy);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const C t = C(cx(i)) * ux + C(cy(i)) * uy;
        const C v = (m == 0xFFu) ? C(0) : wgt<C>(i) * (drho + r * (C(3) * t + C(4.5) * t * t - usq));
        canon_write<S>(g, phase, M, x, y, i, v);
    }
}

template <int P>
__global__ void k_set_f(const Geo g, int phase, const void *f_v, void *lat_v) {
    typedef St<P> S;
    typedef typename S::C C;
    LBM_NODE_LOOP(g)
    const unsigned m = node_mask(g, x, y);
    if (g.layout != LBM_DENSE && __ldg(g.tile_id + (y >> 4) * g.ntx + (x >> 4)) < 0) return;
    const C *f = reinterpret_cast<const C *>(f_v);
    typename S::R *M = reinterpret_cast<typename S::R *>(lat_v);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const C v = (m == 0xFFu) ? C(0) : f[i * g.nnode + n] - wgt<C>(i);
        canon_write<S>(g, phase, M, x, y, i, v);
    }
}

template <int P>
__global__ void k_get_f(const Geo g, int phase, const void *lat_v, void *f_v) {
    typedef St<P> S;
    typedef typename S::C C;
    LBM_NODE_LOOP(g)
    const unsigned m = node_mask(g, x, y);
    const typename S::R *M = reinterpret_cast<const typename S::R *>(lat_v);
    C *f = reinterpret_cast<C *>(f_v);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const C v = (m == 0xFFu) ? C(0) : canon_read<S>(g, phase, M, x, y, i, m);
        f[i * g.nnode + n] = wgt<C>(i) + v;
    }
}

template <int P>
__global__ void k_macros(const Geo g, const Phys ph, int phase, const void *lat_v, void *rho_v, void *u_v) {
    typedef St<P> S;
    typedef typename S::C C;
    LBM_NODE_LOOP(g)
    const unsigned m = node_mask(g, x, y);
    C r = C(1), ux = C(0), uy = C(0);
    if (m != 0xFFu) {
        C f[9];
        gather_node<S>(g, ph, phase, reinterpret_cast<const typename S::R *>(lat_v), x, y, m, f);
        apply_open<C>(g, ph, x, y, m, f);
        C Fx, Fy, drho, inv;
        node_force<C>(g, ph, n, Fx, Fy);
        moments<C, true>(f, Fx, Fy, drho, r, inv, ux, uy);
    }
    if (rho_v) reinterpret_cast<C *>(rho_v)[n] = r;
    if (u_v) {
        reinterpret_cast<C *>(u_v)[n] = ux;
        reinterpret_cast<C *>(u_v)[g.nnode + n] = uy;
    }
}

// FP64 block reduction of 4 values; thread 0 returns the sums.
__device__ __forceinline__ void block_sum4(double v[4], double *out) {
    __shared__ double sm[4][AUX_BLOCK / 32];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_xor_sync(LBM_FULL, v[c], o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < 4; ++c) sm[c][w] = v[c];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int c = 0; c < 4; ++c) {
            double s = 0.0;
            for (int k = 0; k < AUX_BLOCK / 32; ++k) s += sm[c][k];
            out[c] = s;
        }
    }
}

template <int P>
__global__ void __launch_bounds__(AUX_BLOCK) k_reduce(const Geo g, const Phys ph, int phase, int kind,
                                                      const void *lat_v, const void *target_v, double *partial) {
    typedef St<P> S;
    typedef typename S::C C;
    const typename S::R *M = reinterpret_cast<const typename S::R *>(lat_v);
    const C *tgt = reinterpret_cast<const C *>(target_v);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int y = blockIdx.x; y < g.ny; y += gridDim.x)
    for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
        const long long n = (long long)y * g.nx + x;
        const unsigned m = node_mask(g, x, y);
        if (m == 0xFFu) continue;
        if (kind == 0) {
            // the node's own 9 values summed in the storage's compute type
            // (error ~1e-7 of the node's deviation from w), accumulated over
            // nodes in FP64
            C v[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) v[i] = canon_read<S>(g, phase, M, x, y, i, m);
            acc[0] += (double)((((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]))) + v[8]);
            acc[1] += (double)(((v[1] - v[3]) + (v[5] - v[7])) + (v[8] - v[6]));
            acc[2] += (double)(((v[2] - v[4]) + (v[5] - v[7])) + (v[6] - v[8]));
        } else {
            C f[9];
            gather_node<S>(g, ph, phase, M, x, y, m, f);
            apply_open<C>(g, ph, x, y, m, f);
            C Fx, Fy, drho, r, inv, ux, uy;
            node_force<C>(g, ph, n, Fx, Fy);
            moments<C, true>(f, Fx, Fy, drho, r, inv, ux, uy);
            if (kind == 1) {
                const double dx = (double)ux - (double)tgt[n], dy = (double)uy - (double)tgt[g.nnode + n];
                acc[0] += dx * dx + dy * dy;
            } else {
                acc[0] += 0.5 * (double)r * ((double)ux * (double)ux + (double)uy * (double)uy);
            }
        }
    }
    block_sum4(acc, partial + 4 * blockIdx.x);
}

template <int P>
__global__ void __launch_bounds__(AUX_BLOCK) k_reduce_final(const double *partial, int nparts, double *out) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int p = threadIdx.x; p < nparts; p += blockDim.x)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] += partial[4 * p + c];
    block_sum4(acc, out);
}

// One adjoint step with one node per thread (dense two-lattice): the same
// transpose as k_adjoint -- re-gather of f' from A_t in plain units
// (gather_node), lambda_{t+1} at the node, adjoint_node, push of
// g_j = dL/df'_j to slot j at x - c_j (slot opp(j) at x for a bounced link),
// dL/dF accumulated -- with every access a scalar whose lanes touch
// consecutive nodes of a row (coalesced; the x-shifted ones one sector
// wider), no shuffles, and a small register footprint.
template <int P, int FORCE, bool OPEN>
__global__ void __launch_bounds__(STEP_BLOCK) k_adjoint1(const Geo g, const Phys ph, const void *state_v,
                                                         const void *lam_in_v, void *lam_out_v, void *gF_v,
                                                         int y0) {
    typedef St<P> S;
    typedef typename S::R R;
    typedef typename S::C C;
    const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int y = y0 + (int)blockIdx.y;
    if (x >= g.nx) return;
    const long long n = (long long)y * g.nx + x;
    const unsigned m = g.has_mask ? __ldg(g.mask + n) : 0u;
    C *lout = reinterpret_cast<C *>(lam_out_v);
    if (m == 0xFFu) {
#pragma unroll
        for (int j = 0; j < 9; ++j) lout[j * g.nnode + n] = C(0);
        return;
    }
    const C *lin = reinterpret_cast<const C *>(lam_in_v);
    C l[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) l[j] = __ldg(lin + j * g.nnode + n);
    C f[9];
    gather_node<S>(g, ph, PH_PLAIN, reinterpret_cast<const R *>(state_v), x, y, m, f);
    if constexpr (OPEN) apply_open<C>(g, ph, x, y, m, f);
    C Fx = PC<C>::fx(ph), Fy = PC<C>::fy(ph);
    if constexpr (FORCE == FORCE_FIELD) {
        const C *F = reinterpret_cast<const C *>(ph.force);
        Fx = __ldg(F + n);
        Fy = __ldg(F + g.nnode + n);
    }
    C gg[9], dFx, dFy;
    adjoint_node<C, FORCE != FORCE_NONE>(f, l, Fx, Fy, PC<C>::omega(ph), gg, dFx, dFy);
    if constexpr (OPEN) open_transpose<C>(g, ph, x, y, m, gg);
    lout[n] = gg[0];
#pragma unroll
    for (int j = 1; j < 9; ++j) {
        if (m & (1u << (j - 1))) {
            lout[opp(j) * g.nnode + n] = gg[j]; // bounced: the own node's opposite slot
        } else {
            int sx = x - cx(j), sy = y - cy(j);
            wrap_xy(g, sx, sy);
            lout[j * g.nnode + (long long)sy * g.nx + sx] = gg[j];
        }
    }
    C *gF = reinterpret_cast<C *>(gF_v);
    gF[n] += dFx;
    gF[g.nnode + n] += dFy;
}

// Transpose of the macros at the current (two-lattice, dense) state.
template <int P>
__global__ void k_macros_adjoint(const Geo g, const Phys ph, const void *state_v, const void *grho_v,
                                 const void *gu_v, void *lam_v, void *gF_v) {
    typedef St<P> S;
    typedef typename S::C C;
    LBM_NODE_LOOP(g)
    const unsigned m = node_mask(g, x, y);
    C *lam = reinterpret_cast<C *>(lam_v);
    if (m == 0xFFu) {
#pragma unroll
        for (int j = 0; j < 9; ++j) lam[j * g.nnode + n] = C(0);
        return;
    }
    C f[9];
    gather_node<S>(g, ph, PH_PLAIN, reinterpret_cast<const typename S::R *>(state_v), x, y, m, f);
    apply_open<C>(g, ph, x, y, m, f);
    C Fx, Fy, drho, r, inv, ux, uy;
    node_force<C>(g, ph, n, Fx, Fy);
    moments<C, true>(f, Fx, Fy, drho, r, inv, ux, uy);
    const C gr = grho_v ? reinterpret_cast<const C *>(grho_v)[n] : C(0);
    const C gx = gu_v ? reinterpret_cast<const C *>(gu_v)[n] : C(0);
    const C gy = gu_v ? reinterpret_cast<const C *>(gu_v)[g.nnode + n] : C(0);
    C gv[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) gv[j] = gr + ((C(cx(j)) - ux) * gx + (C(cy(j)) - uy) * gy) * inv;
    open_transpose<C>(g, ph, x, y, m, gv);
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const C v = gv[j];
        if (j > 0 && (m & (1u << (j - 1)))) {
            lam[opp(j) * g.nnode + n] = v;
        } else {
            int sx = x - cx(j), sy = y - cy(j);
            wrap_xy(g, sx, sy);
            lam[j * g.nnode + (long long)sy * g.nx + sx] = v;
        }
    }
    if (gF_v) {
        C *gF = reinterpret_cast<C *>(gF_v);
        gF[n] += C(0.5) * gx * inv;
        gF[g.nnode + n] += C(0.5) * gy * inv;
    }
}

// ------------------------------------------------------------- launchers

// Launch shape.  Dense: blockIdx.y = row (in chunks of at most 65535 rows),
// blockIdx.x * blockDim.x + tid = vector column, blockDim.x = the row's vector
// count rounded up to a warp, at most STEP_BLOCK.  Tiled: 1-D over tiles.
struct Shape {
    unsigned bx, gx, rows;
    bool dense;
};
template <int VEC, bool LIST = false> static Shape step_shape(const Geo &g) {
    Shape sh;
    sh.dense = g.layout == LBM_DENSE;
    if (sh.dense) {
        const int nvx = g.nx / VEC;
        sh.bx = (unsigned)(((nvx + 31) / 32) * 32);
        if (sh.bx > (unsigned)STEP_BLOCK) sh.bx = STEP_BLOCK;
        sh.gx = (unsigned)((nvx + sh.bx - 1) / sh.bx);
        sh.rows = (unsigned)g.ny;
    } else {
        const long long n = LIST ? (VEC == 4 ? g.nlist4 : g.nlist2) : (long long)g.ntiles * TileAddr<VEC>::TPT;
        sh.bx = STEP_BLOCK;
        sh.gx = (unsigned)((n + STEP_BLOCK - 1) / STEP_BLOCK);
        sh.rows = 1;
    }
    return sh;
}

// Rows row0, row0 + stride, ... (nrows of them) of the dense layout; all
// kept tiles of the tiled layout.
struct Rows {
    int row0, nrows, stride;
};
template <int P, class A, int MODE, bool HM, int F, bool OPEN, bool TRT>
static cudaError_t step_launch(const Geo &g, const Phys &ph, const void *src, void *dst, unsigned t, Rows r,
                               cudaStream_t s) {
    Shape sh = step_shape<A::VEC_, A::LIST_>(g);
    if (sh.gx == 0) return cudaSuccess;
    if constexpr (ListPersist<P, A>::value) {
        // persistent over the list: the blocks that are resident at once
        static const unsigned cap = [] {
            int dev = 0, sms = 0, per_sm = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step<P, A, MODE, HM, F, OPEN, TRT>, STEP_BLOCK, 0);
            return (unsigned)(sms > 0 && per_sm > 0 ? sms * per_sm : 1);
        }();
        if (sh.gx > cap) sh.gx = cap;
    }
    const unsigned rows = sh.dense ? (unsigned)r.nrows : 1u;
    for (unsigned k = 0; k < rows; k += 65535u) {
        const unsigned gy = rows - k < 65535u ? rows - k : 65535u;
        k_step<P, A, MODE, HM, F, OPEN, TRT><<<dim3(sh.gx, gy), sh.bx, 0, s>>>(g, ph, src, dst,
                                                                         r.row0 + (int)k * r.stride, r.stride, t);
    }
    return cudaGetLastError();
}
// Dense (TILED false) or tiled addressing with the vector width of the step
// kind, the force mode and the mask flag.
template <int P, class A, int MODE, bool HM, int F, bool TRT>
static cudaError_t step_open(const Geo &g, const Phys &ph, const void *src, void *dst, unsigned t, Rows r,
                             cudaStream_t s) {
    // open sides are only on masked kernels (their links are marked)
    if constexpr (HM)
        if (ph.has_open) return step_launch<P, A, MODE, HM, F, true, TRT>(g, ph, src, dst, t, r, s);
    return step_launch<P, A, MODE, HM, F, false, TRT>(g, ph, src, dst, t, r, s);
}
// The staged tiled two-lattice step: persistent, as many blocks as the SMs
// hold (shared memory bounds them), never more than there are tiles.
template <int P, int F, bool OPEN, bool TRT>
static cudaError_t staged_launch(const Geo &g, const Phys &ph, const void *src, void *dst, unsigned t,
                                 cudaStream_t s) {
    if (g.ntiles <= 0) return cudaSuccess;
    constexpr int smem = staged_smem_bytes<P>();
    static const unsigned cap = [] {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_step_staged<P, F, OPEN, TRT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(k_step_staged<P, F, OPEN, TRT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_staged<P, F, OPEN, TRT>, STG_THREADS, smem);
        return (unsigned)(sms > 0 && per_sm > 0 ? sms * per_sm : 1);
    }();
    const unsigned grid = (unsigned)g.ntiles < cap ? (unsigned)g.ntiles : cap;
    k_step_staged<P, F, OPEN, TRT><<<grid, STG_THREADS, smem, s>>>(g, ph, src, dst, t);
    return cudaGetLastError();
}

template <int P, bool TILED, int MODE, bool HM, int F, bool TRT>
static cudaError_t step_vec(const Geo &g, const Phys &ph, const void *src, void *dst, unsigned t, Rows r,
                            cudaStream_t s) {
    constexpr int V = StepVec<P, HM, MODE, F>::value;
    if constexpr (TILED && HM && MODE == MODE_TWO_LATTICE && F != FORCE_FIELD && P != LBM_F64) {
        // porous geometries: tiles staged in shared memory (uniform or no
        // force; FP64 is bound by its FP64 pipe and keeps the per-vector step)
        if (staged_selected<P>(g.active_frac)) {
            if (ph.has_open) return staged_launch<P, F, true, TRT>(g, ph, src, dst, t, s);
            return staged_launch<P, F, false, TRT>(g, ph, src, dst, t, s);
        }
    }
    if constexpr (TILED) {
        // over the list, FP32 keeps 8-byte vectors with the bounce-back
        // preload in every step kind (finer vectors skip more solid nodes);
        // the FP32 two-lattice step without it moves 16-byte vectors, which
        // wins until about a third of the vectors are solid
        constexpr int VL = P == LBM_F32 ? 2 : V;
        constexpr bool WIDE = P == LBM_F32 && MODE == MODE_TWO_LATTICE && F != FORCE_FIELD;
        if (g.use_list && g.active_frac < (WIDE ? 0.67f : 0.85f))
            return step_open<P, TileAddr<VL, true>, MODE, HM, F, TRT>(g, ph, src, dst, t, r, s);
        return step_open<P, TileAddr<V, false>, MODE, HM, F, TRT>(g, ph, src, dst, t, r, s);
    } else {
        return step_open<P, DenseAddr<V>, MODE, HM, F, TRT>(g, ph, src, dst, t, r, s);
    }
}
template <int P, bool TILED, int MODE, bool HM, bool TRT>
static cudaError_t step_force(const Geo &g, const Phys &ph, const void *src, void *dst, unsigned t, Rows r,
                              cudaStream_t s) {
    switch (ph.force_mode) {
    case FORCE_NONE: return step_vec<P, TILED, MODE, HM, FORCE_NONE, TRT>(g, ph, src, dst, t, r, s);
    case FORCE_UNIFORM: return step_vec<P, TILED, MODE, HM, FORCE_UNIFORM, TRT>(g, ph, src, dst, t, r, s);
    default: return step_vec<P, TILED, MODE, HM, FORCE_FIELD, TRT>(g, ph, src, dst, t, r, s);
    }
}
template <int P, bool TILED, bool HM, bool TRT>
static cudaError_t step_mode(const Geo &g, const Phys &ph, int mode, const void *src, void *dst, unsigned t, Rows r,
                             cudaStream_t s) {
    switch (mode) {
    case MODE_TWO_LATTICE: return step_force<P, TILED, MODE_TWO_LATTICE, HM, TRT>(g, ph, src, dst, t, r, s);
    case MODE_AA_PULLPUSH: return step_force<P, TILED, MODE_AA_PULLPUSH, HM, TRT>(g, ph, src, dst, t, r, s);
    default: return step_force<P, TILED, MODE_AA_LOCAL, HM, TRT>(g, ph, src, dst, t, r, s);
    }
}

// Dense grids whose only bounced links are in the first and last row (walls
// or open sides in y, periodic x, no obstacle): those two rows run the
// masked kernel, every other row the kernel without a mask.  Both read the
// state before the step and write disjoint nodes (two-lattice), or touch
// disjoint slot sets (AA), so the split is exact.  TRT: the
// two-relaxation-time collision (its kernels are separate instances, built
// in their own translation units).
template <int P, bool TRT>
cudaError_t launch_step_op(const Geo &g, const Phys &ph, int mode, const void *src, void *dst, unsigned long long t,
                           cudaStream_t s) {
    const unsigned tt = (unsigned)t;
    const Rows all = {0, g.ny, 1};
    if (g.layout == LBM_DENSE) {
        if (g.has_mask && g.frame_y) {
            cudaError_t e = step_mode<P, false, true, TRT>(g, ph, mode, src, dst, tt, Rows{0, 2, g.ny - 1}, s);
            if (e != cudaSuccess) return e;
            return step_mode<P, false, false, TRT>(g, ph, mode, src, dst, tt, Rows{1, g.ny - 2, 1}, s);
        }
        if (g.has_mask) return step_mode<P, false, true, TRT>(g, ph, mode, src, dst, tt, all, s);
        return step_mode<P, false, false, TRT>(g, ph, mode, src, dst, tt, all, s);
    }
    if (g.has_mask) return step_mode<P, true, true, TRT>(g, ph, mode, src, dst, tt, all, s);
    return step_mode<P, true, false, TRT>(g, ph, mode, src, dst, tt, all, s);
}

static inline dim3 node_blocks(const Geo &g) {
    const unsigned rows = (unsigned)(g.ny < 65535 ? g.ny : 65535);
    return dim3((unsigned)((g.nx + AUX_BLOCK - 1) / AUX_BLOCK), rows, (unsigned)((g.ny + rows - 1) / rows));
}

template <int P>
cudaError_t launch_init(const Geo &g, int phase, const void *rho, const void *u, void *lat, cudaStream_t s) {
    k_init<P><<<node_blocks(g), AUX_BLOCK, 0, s>>>(g, phase, rho, u, lat);
    return cudaGetLastError();
}
template <int P>
cudaError_t launch_set_f(const Geo &g, int phase, const void *f, void *lat, cudaStream_t s) {
    k_set_f<P><<<node_blocks(g), AUX_BLOCK, 0, s>>>(g, phase, f, lat);
    return cudaGetLastError();
}
template <int P>
cudaError_t launch_get_f(const Geo &g, int phase, const void *lat, void *f, cudaStream_t s) {
    k_get_f<P><<<node_blocks(g), AUX_BLOCK, 0, s>>>(g, phase, lat, f);
    return cudaGetLastError();
}
template <int P>
cudaError_t launch_macros(const Geo &g, const Phys &ph, int phase, const void *lat, void *rho, void *u,
                          cudaStream_t s) {
    k_macros<P><<<node_blocks(g), AUX_BLOCK, 0, s>>>(g, ph, phase, lat, rho, u);
    return cudaGetLastError();
}
template <int P>
cudaError_t launch_reduce(const Geo &g, const Phys &ph, int phase, int kind, const void *lat, const void *target,
                          double *partial, double *out, cudaStream_t s) {
    k_reduce<P><<<RED_BLOCKS, AUX_BLOCK, 0, s>>>(g, ph, phase, kind, lat, target, partial);
    k_reduce_final<P><<<1, AUX_BLOCK, 0, s>>>(partial, RED_BLOCKS, out);
    return cudaGetLastError();
}
// The adjoint kernel: FP64 and FP32 take the vector kernel k_adjoint
// (measured 4.99 against 3.99 TB/s for the one-node-per-thread kernel on a
// 2048^2 channel); FP16s takes k_adjoint1, whose gather decodes the stored
// values to plain units, as adjoint_node expects (the vector gather
// decodes in the step's stored scale).  LBM_ADJ_SCALAR=1 sends every
// precision to k_adjoint1.
#ifndef LBM_ADJ_SCALAR
#define LBM_ADJ_SCALAR 0
#endif
template <int P, int F, bool OPEN>
static void adjoint_rows(const Geo &g, const Phys &ph, const void *state, const void *lam_in, void *lam_out,
                         void *grad_force, const Shape &sh, cudaStream_t s) {
    if constexpr (LBM_ADJ_SCALAR != 0 || P == LBM_F16S) {
        const unsigned gx = (unsigned)((g.nx + STEP_BLOCK - 1) / STEP_BLOCK);
        for (unsigned y0 = 0; y0 < (unsigned)g.ny; y0 += 65535u) {
            const dim3 grid(gx, (unsigned)g.ny - y0 < 65535u ? (unsigned)g.ny - y0 : 65535u);
            k_adjoint1<P, F, OPEN><<<grid, STEP_BLOCK, 0, s>>>(g, ph, state, lam_in, lam_out, grad_force, (int)y0);
        }
    } else {
        for (unsigned y0 = 0; y0 < sh.rows; y0 += 65535u) {
            const dim3 grid(sh.gx, sh.rows - y0 < 65535u ? sh.rows - y0 : 65535u);
            k_adjoint<P, F, OPEN><<<grid, sh.bx, 0, s>>>(g, ph, state, lam_in, lam_out, grad_force, (int)y0);
        }
    }
}
template <int P, int F>
static void adjoint_open(const Geo &g, const Phys &ph, const void *state, const void *lam_in, void *lam_out,
                         void *grad_force, const Shape &sh, cudaStream_t s) {
    if (ph.has_open) adjoint_rows<P, F, true>(g, ph, state, lam_in, lam_out, grad_force, sh, s);
    else adjoint_rows<P, F, false>(g, ph, state, lam_in, lam_out, grad_force, sh, s);
}
template <int P>
cudaError_t launch_adjoint(const Geo &g, const Phys &ph, const void *state, const void *lam_in, void *lam_out,
                           void *grad_force, cudaStream_t s) {
    const Shape sh = step_shape<StepVec<P, true, MODE_TWO_LATTICE, FORCE_FIELD>::value>(g); // dense, as k_adjoint
    if (sh.gx == 0) return cudaSuccess;
    switch (ph.force_mode) {
    case FORCE_NONE: adjoint_open<P, FORCE_NONE>(g, ph, state, lam_in, lam_out, grad_force, sh, s); break;
    case FORCE_UNIFORM: adjoint_open<P, FORCE_UNIFORM>(g, ph, state, lam_in, lam_out, grad_force, sh, s); break;
    default: adjoint_open<P, FORCE_FIELD>(g, ph, state, lam_in, lam_out, grad_force, sh, s);
    }
    return cudaGetLastError();
}
template <int P>
cudaError_t launch_macros_adjoint(const Geo &g, const Phys &ph, const void *state, const void *g_rho,
                                  const void *g_u, void *lam, void *grad_force, cudaStream_t s) {
    k_macros_adjoint<P><<<node_blocks(g), AUX_BLOCK, 0, s>>>(g, ph, state, g_rho, g_u, lam, grad_force);
    return cudaGetLastError();
}

#define LBM_INSTANTIATE_STEP(P, TRT)                                                                        \
    template cudaError_t launch_step_op<P, TRT>(const Geo &, const Phys &, int, const void *, void *,          \
                                                unsigned long long, cudaStream_t);
#define LBM_INSTANTIATE(P)                                                                                  \
    LBM_INSTANTIATE_STEP(P, false)                                                                          \
    template cudaError_t launch_init<P>(const Geo &, int, const void *, const void *, void *, cudaStream_t); \
    template cudaError_t launch_set_f<P>(const Geo &, int, const void *, void *, cudaStream_t);             \
    template cudaError_t launch_get_f<P>(const Geo &, int, const void *, void *, cudaStream_t);             \
    template cudaError_t launch_macros<P>(const Geo &, const Phys &, int, const void *, void *, void *,    \
                                          cudaStream_t);                                                    \
    template cudaError_t launch_reduce<P>(const Geo &, const Phys &, int, int, const void *, const void *, \
                                          double *, double *, cudaStream_t);                                \
    template cudaError_t launch_adjoint<P>(const Geo &, const Phys &, const void *, const void *, void *,  \
                                           void *, cudaStream_t);                                           \
    template cudaError_t launch_macros_adjoint<P>(const Geo &, const Phys &, const void *, const void *,   \
                                                  const void *, void *, void *, cudaStream_t);

} // namespace lbm
