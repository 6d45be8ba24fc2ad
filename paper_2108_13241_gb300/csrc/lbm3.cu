// lbm3.cu -- the D3Q19 stream-and-collide step (Algorithm 1 of the paper in
// three dimensions, the extension named as future work in Sec. 5) and its
// C-ABI entry points (lbm3_* in include/lbm.h).
//
// Dense SoA storage f[i][z][y][x] of the shifted values f_i - w_i (FP64 or
// FP32), two lattices swapped by pointer.  One node per thread: the 19 pulls
// f'_i(x) = A_i(x - c_i) are 19 loads whose lanes read consecutive nodes of
// one (slot, row) -- coalesced, the x-shifted ones one 32-byte sector wider
// -- and the 19 stores are aligned.  Bounced links (a solid source or a wall
// face, one bit each in a per-node 32-bit link mask) read the node's own
// value of the opposite link (half-way bounce-back).  The collision is BGK
// (Eq. 3-5) toward Eq. 6 with the D3Q19 weights plus the Guo source,
// regrouped per pair of opposite links into an even part and an odd part
// (exact algebra, fewer operations).  The register footprint stays small
// (19 values a thread), the concern the paper raises for three dimensions.
// On sparse geometries a node list (index and link mask per entry) lets the
// step run one thread per fluid node instead of one per grid node.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "lbm.h"

namespace {

constexpr int Q3 = 19;
constexpr uint32_t SOLID3 = 0xFFFFFFFFu;
constexpr int BLOCK3 = 128;

// Velocities (the order of lbm.h): rest; +-x, +-y, +-z; the xy, xz and yz
// edge diagonals, opposite links adjacent (2k - 1, 2k).
__host__ __device__ constexpr int c3(int i, int a) {
    constexpr int t[Q3][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
                              {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
                              {-1, 0, 1}, {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    return t[i][a];
}
__host__ __device__ constexpr int opp3(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
template <class T> __host__ __device__ constexpr T w3(int i) {
    return i == 0 ? T(1.0 / 3.0) : (i <= 6 ? T(1.0 / 18.0) : T(1.0 / 36.0));
}

struct Geo3 {
    int nx, ny, nz;
    int px, py, pz;        // periodic axes
    unsigned long long N;  // nodes (node indices are 32-bit: N < 2^32, checked at create;
                           // slot offsets i N + n are 64-bit, so 19 N may exceed 2^32)
    const uint32_t *mask;  // [nz][ny][nx]; NULL: every node fluid, all axes periodic
    const uint2 *list;     // node list of the listed step (node index, link mask; ascending
                           // index); NULL: the dense grid runs
    unsigned nlist;        // entries of list
    unsigned mx, my;       // floor((2^32 - 1) / nx), floor((2^32 - 1) / ny): node index -> x, y, z
};

// q = n / d and r = n mod d for a divisor fixed for the run: the high word
// of n * floor((2^32 - 1) / d) lies between n / d - 2 and n / d (n < 2^32),
// so at most two corrections follow.
__device__ __forceinline__ unsigned divq3(unsigned n, unsigned d, unsigned magic, unsigned &r) {
    unsigned q = __umulhi(n, magic);
    r = n - q * d;
#pragma unroll
    for (int k = 0; k < 2; ++k)
        if (r >= d) {
            ++q;
            r -= d;
        }
    return q;
}
struct Phys3 {
    double om, kk, fx, fy, fz; // omega = 1/tau, 1 - omega/2, force
    float om_f, kk_f, fx_f, fy_f, fz_f;
};
template <class T> struct P3;
template <> struct P3<double> {
    static __device__ __forceinline__ double om(const Phys3 &p) { return p.om; }
    static __device__ __forceinline__ double kk(const Phys3 &p) { return p.kk; }
    static __device__ __forceinline__ void F(const Phys3 &p, double &x, double &y, double &z) {
        x = p.fx; y = p.fy; z = p.fz;
    }
};
template <> struct P3<float> {
    static __device__ __forceinline__ float om(const Phys3 &p) { return p.om_f; }
    static __device__ __forceinline__ float kk(const Phys3 &p) { return p.kk_f; }
    static __device__ __forceinline__ void F(const Phys3 &p, float &x, float &y, float &z) {
        x = p.fx_f; y = p.fy_f; z = p.fz_f;
    }
};

// Stored element R <-> compute type (C): FP64 and FP32 store f - w as is;
// FP16s stores binary16 bits of (f - w) * 2^10 (exact power-of-two scale, as
// in two dimensions) and computes in FP32.
template <class R> struct Cod3;
template <> struct Cod3<double> {
    typedef double C;
    static __device__ __forceinline__ double dec(double r) { return r; }
    static __device__ __forceinline__ double enc(double c) { return c; }
};
template <> struct Cod3<float> {
    typedef float C;
    static __device__ __forceinline__ float dec(float r) { return r; }
    static __device__ __forceinline__ float enc(float c) { return c; }
};
constexpr float H3_SCALE = 1024.0f;
template <> struct Cod3<unsigned short> {
    typedef float C;
    static __device__ __forceinline__ float dec(unsigned short r) {
        return __half2float(__ushort_as_half(r)) * (1.0f / H3_SCALE);
    }
    static __device__ __forceinline__ unsigned short enc(float c) {
        return __half_as_ushort(__float2half_rn(c * H3_SCALE));
    }
};

// The node a thread updates, and its neighbours' coordinates along each
// axis (periodic: wrapped; wall: clamped -- those links bounce and their
// address is never used).
struct Node3 {
    int x, y, z;
    unsigned n;
    int xs[3], ys[3], zs[3]; // coordinate - 1, itself, + 1
    __device__ __forceinline__ Node3(const Geo3 &g, int x_, int y_, int z_)
        : Node3(g, x_, y_, z_, ((unsigned)z_ * (unsigned)g.ny + (unsigned)y_) * (unsigned)g.nx + (unsigned)x_) {}
    __device__ __forceinline__ Node3(const Geo3 &g, int x_, int y_, int z_, unsigned n_) : x(x_), y(y_), z(z_), n(n_) {
        nb(x, g.nx, g.px, xs);
        nb(y, g.ny, g.py, ys);
        nb(z, g.nz, g.pz, zs);
    }
    // the node of index n_ (an entry of the node list)
    static __device__ __forceinline__ Node3 at(const Geo3 &g, unsigned n_) {
        unsigned x_, y_;
        const unsigned row = divq3(n_, (unsigned)g.nx, g.mx, x_);
        const unsigned z_ = divq3(row, (unsigned)g.ny, g.my, y_);
        return Node3(g, (int)x_, (int)y_, (int)z_, n_);
    }
    static __device__ __forceinline__ void nb(int c, int n, int per, int o[3]) {
        o[0] = c > 0 ? c - 1 : (per ? n - 1 : 0);
        o[1] = c;
        o[2] = c < n - 1 ? c + 1 : (per ? 0 : n - 1);
    }
    // node index of the pull source x - c_i
    __device__ __forceinline__ unsigned src(const Geo3 &g, int i) const {
        const int sx = xs[1 - c3(i, 0)], sy = ys[1 - c3(i, 1)], sz = zs[1 - c3(i, 2)];
        return ((unsigned)sz * (unsigned)g.ny + (unsigned)sy) * (unsigned)g.nx + (unsigned)sx;
    }
};

// The gather of Algorithm 1 for one node: f'_i = A_i(x - c_i), or the
// node's own value of the opposite link where link i bounces (bit i - 1).
template <class R, bool HM>
__device__ __forceinline__ void gather3(const Geo3 &g, const Node3 &nd, const R *A, uint32_t m,
                                        typename Cod3<R>::C f[Q3]) {
    f[0] = Cod3<R>::dec(A[nd.n]);
#pragma unroll
    for (int i = 1; i < Q3; ++i) {
        if (HM && (m & (1u << (i - 1)))) f[i] = Cod3<R>::dec(A[(unsigned)opp3(i) * g.N + nd.n]);
        else f[i] = Cod3<R>::dec(A[(unsigned)i * g.N + nd.src(g, i)]);
    }
}

// How the lattice holds the state A_t: two-lattice (slot i at x holds
// A_i(x)); AA after its gather/scatter step's partner, the local step
// (swapped: slot opp(i) at x holds A_i(x)); AA after a gather/scatter step
// (streamed: slot i at x holds the next step's pulled f'_i(x)).
enum Phase3 { P3_PLAIN = 0, P3_SWAPPED = 1, P3_STREAMED = 2 };

// The next step's f'_i at node nd in any phase (bounced links: the own
// node's value of the opposite link).
template <class R, bool HM>
__device__ __forceinline__ void gather3p(const Geo3 &g, const Node3 &nd, const R *A, uint32_t m, int phase,
                                         typename Cod3<R>::C f[Q3]) {
    if (phase == P3_PLAIN) {
        gather3<R, HM>(g, nd, A, m, f);
        return;
    }
    f[0] = Cod3<R>::dec(A[nd.n]);
#pragma unroll
    for (int i = 1; i < Q3; ++i) {
        unsigned long long k;
        if (phase == P3_STREAMED) k = (unsigned long long)i * g.N + nd.n;
        else if (HM && (m & (1u << (i - 1)))) k = (unsigned long long)i * g.N + nd.n;
        else k = (unsigned long long)opp3(i) * g.N + nd.src(g, i);
        f[i] = Cod3<R>::dec(A[k]);
    }
}

// Canonical A_i(x) read from any phase (streamed: the value the last
// gather/scatter step pushed to x + c_i, or kept in the own opposite slot
// where that link bounces).
template <class R>
__device__ __forceinline__ typename Cod3<R>::C canon3(const Geo3 &g, const Node3 &nd, const R *A, uint32_t m,
                                                      int phase, int i) {
    if (phase == P3_PLAIN || i == 0) return Cod3<R>::dec(A[(unsigned long long)i * g.N + nd.n]);
    if (phase == P3_SWAPPED) return Cod3<R>::dec(A[(unsigned long long)opp3(i) * g.N + nd.n]);
    if (m & (1u << (opp3(i) - 1))) return Cod3<R>::dec(A[(unsigned long long)opp3(i) * g.N + nd.n]);
    return Cod3<R>::dec(A[(unsigned long long)i * g.N + nd.src(g, opp3(i))]); // x - c_opp(i) = x + c_i
}

// Moments of the shifted f' (Eq. 2 with the Guo shift): drho = rho - 1,
// j = rho u = sum c f' + F/2.
template <class T>
__device__ __forceinline__ void moments3(const T f[Q3], T Fx, T Fy, T Fz, T &drho, T &jx, T &jy, T &jz) {
    drho = T(0);
    jx = jy = jz = T(0);
#pragma unroll
    for (int i = 0; i < Q3; ++i) {
        drho += f[i];
        if (c3(i, 0)) jx += c3(i, 0) > 0 ? f[i] : -f[i];
        if (c3(i, 1)) jy += c3(i, 1) > 0 ? f[i] : -f[i];
        if (c3(i, 2)) jz += c3(i, 2) > 0 ? f[i] : -f[i];
    }
    jx += T(0.5) * Fx;
    jy += T(0.5) * Fy;
    jz += T(0.5) * Fz;
}

// BGK relaxation toward Eq. 6 plus the Guo source, on shifted values:
//   f_i <- (1 - omega) f_i + omega (f^eq_i - w_i) + S_i,
//   f^eq_i - w_i = w_i [drho + rho (3 t + 4.5 t^2 - 1.5 u.u)], t = c_i . u,
//   S_i = (1 - omega/2) w_i [3 (c_i . F) - 3 u.F + 9 t (c_i . F)],
// taken per pair (i, opp(i)) as the even part E (the same for both) and the
// odd part O = 3 w_i [omega (c_i . j) + (1 - omega/2) (c_i . F)] (+ for i,
// - for opp(i)).  SC: f in units of 1/SC (FP16s computes on its stored
// scale, SC = 2^10, so that neither its decode nor its encode multiplies);
// the moments come back to plain units, the updates go out in f's units.
template <class T, bool HAS_F, int SC = 1>
__device__ __forceinline__ void collide3(T f[Q3], T om, T kk, T Fx, T Fy, T Fz) {
    T drho, jx, jy, jz;
    if constexpr (SC == 1) {
        moments3<T>(f, Fx, Fy, Fz, drho, jx, jy, jz);
    } else {
        moments3<T>(f, T(0), T(0), T(0), drho, jx, jy, jz);
        drho *= T(1.0 / SC);
        jx = jx * T(1.0 / SC) + T(0.5) * Fx;
        jy = jy * T(1.0 / SC) + T(0.5) * Fy;
        jz = jz * T(1.0 / SC) + T(0.5) * Fz;
    }
    const T rho = T(1) + drho;
    const T inv = T(1) / rho;
    const T ux = jx * inv, uy = jy * inv, uz = jz * inv;
    const T usq = T(1.5) * (ux * ux + uy * uy + uz * uz);
    const T uF = HAS_F ? ux * Fx + uy * Fy + uz * Fz : T(0);
    const T om1 = T(1) - om;
    const T base = drho - rho * usq;
    {
        T e = om * base;
        if (HAS_F) e -= kk * T(3) * uF;
        f[0] = om1 * f[0] + (w3<T>(0) * T(SC)) * e;
    }
    if constexpr (sizeof(T) == 8) {
        static_assert(SC == 1, "FP64 works in plain units");
        // FP64 (bound by its FP64 pipe): omega w and (1 - omega/2) w folded
        // per weight class (axis, diagonal), 4.5 rho hoisted -- fewer FP64
        // operations for the same algebra
        const T r45 = T(4.5) * rho;
        const T owa = om * w3<T>(1), owd = om * w3<T>(7);
        const T kwa = kk * w3<T>(1), kwd = kk * w3<T>(7);
#pragma unroll
        for (int i = 1; i < Q3; i += 2) {
            const T ow = i <= 6 ? owa : owd, kw = i <= 6 ? kwa : kwd;
            const T cx = T(c3(i, 0)), cy = T(c3(i, 1)), cz = T(c3(i, 2));
            const T t = cx * ux + cy * uy + cz * uz;
            const T cj = cx * jx + cy * jy + cz * jz;
            T e = ow * (base + r45 * (t * t));
            T o = (T(3) * ow) * cj;
            if (HAS_F) {
                const T cF = cx * Fx + cy * Fy + cz * Fz;
                e += kw * (T(9) * t * cF - T(3) * uF);
                o += (T(3) * kw) * cF;
            }
            f[i] = om1 * f[i] + (e + o);
            f[i + 1] = om1 * f[i + 1] + (e - o);
        }
    } else {
        // FP32 arithmetic (DRAM- or issue-bound): each factor rounded in
        // the order of the formula, which keeps the FP32 velocity closer to
        // FP64 on decaying flows (1.19e-5 against below 1e-5 with the FP64
        // folding on the periodic random-field box)
#pragma unroll
        for (int i = 1; i < Q3; i += 2) {
            const T cx = T(c3(i, 0)), cy = T(c3(i, 1)), cz = T(c3(i, 2));
            const T t = cx * ux + cy * uy + cz * uz;
            const T cj = cx * jx + cy * jy + cz * jz;
            T e = om * (base + T(4.5) * rho * t * t);
            T o = om * cj;
            if (HAS_F) {
                const T cF = cx * Fx + cy * Fy + cz * Fz;
                e += kk * (T(9) * t * cF - T(3) * uF);
                o += kk * cF;
            }
            e *= w3<T>(i) * T(SC);
            o *= T(3) * w3<T>(i) * T(SC);
            f[i] = om1 * f[i] + (e + o);
            f[i + 1] = om1 * f[i + 1] + (e - o);
        }
    }
}

// Whether a solid node shares its 32-byte DRAM sector with a fluid node of
// its warp (lanes in aligned groups of 32 / bytes-per-lane, which match the
// sectors when n_x is a multiple of the group; otherwise some writes stay
// partial, which costs time, not correctness): such a node
// writes zeros -- what every solid node holds, and never read -- so that the
// sector is stored whole and the memory does not first read the old sector
// to merge a partial write (the two-lattice step writes a lattice it has not
// read).  `fluid` is the warp's ballot of lanes holding fluid.
template <int LANE_BYTES> __device__ __forceinline__ bool sector_has_fluid(unsigned fluid) {
    constexpr int G = 32 / LANE_BYTES;
    const int lane = (int)(threadIdx.x & 31u);
    return ((fluid >> (lane & ~(G - 1))) & ((1u << G) - 1u)) != 0u;
}

// One node's two-lattice update (Algorithm 1): the gather, the collision and
// the aligned stores of its 19 values to B.
template <class T, bool HM, bool HAS_F>
__device__ __forceinline__ void step_node3(const Geo3 &g, const Phys3 &ph, const T *__restrict__ A,
                                           T *__restrict__ B, const Node3 &nd, uint32_t m) {
    T f[Q3];
    gather3<T, HM>(g, nd, A, m, f);
    T Fx, Fy, Fz;
    P3<T>::F(ph, Fx, Fy, Fz);
    collide3<T, HAS_F>(f, P3<T>::om(ph), P3<T>::kk(ph), Fx, Fy, Fz);
#pragma unroll
    for (int i = 0; i < Q3; ++i) B[(unsigned)i * g.N + nd.n] = f[i];
}

template <class T, bool HM, bool HAS_F>
__global__ void __launch_bounds__(BLOCK3) k3_step(const Geo3 g, const Phys3 ph, const T *__restrict__ A,
                                                  T *__restrict__ B) {
    const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (!HM && x >= g.nx) return;
    const Node3 nd(g, x, (int)blockIdx.y, (int)blockIdx.z);
    uint32_t m = 0u;
    if (HM) {
        // every lane of the warp takes part in the ballot (blocks are whole
        // warps); lanes beyond the row count as solid and touch no memory
        const bool in = x < g.nx;
        m = in ? g.mask[nd.n] : SOLID3;
        const unsigned fluid = __ballot_sync(0xFFFFFFFFu, m != SOLID3);
        if (!in) return;
        if (m == SOLID3) {
            if (sector_has_fluid<(int)sizeof(T)>(fluid)) {
#pragma unroll
                for (int i = 0; i < Q3; ++i) B[(unsigned)i * g.N + nd.n] = T(0);
            }
            return; // never read
        }
    }
    step_node3<T, HM, HAS_F>(g, ph, A, B, nd, m);
}

// The listed two-lattice step: one thread per entry of the node list -- the
// fluid nodes, and the solid nodes that share a DRAM sector with one (they
// store zeros, as above) -- so no lane of a porous box idles on a solid
// node; the entries' coordinates come from their index.
template <class T, bool HAS_F>
__global__ void __launch_bounds__(BLOCK3) k3_step_list(const Geo3 g, const Phys3 ph, const T *__restrict__ A,
                                                       T *__restrict__ B) {
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.nlist) return;
    const uint2 e = g.list[t]; // the node and its mask in one load: no dependent mask read
    const unsigned n = e.x;
    const uint32_t m = e.y;
    if (m == SOLID3) {
#pragma unroll
        for (int i = 0; i < Q3; ++i) B[(unsigned long long)i * g.N + n] = T(0);
        return;
    }
    step_node3<T, true, HAS_F>(g, ph, A, B, Node3::at(g, n), m);
}

// The in-place AA pattern, one lattice.  PULLPUSH (from the swapped
// phase): f'_i = slot opp(i) at x - c_i (bounced: own slot i), collision,
// f''_i to slot i at x + c_i (or, where that node is solid or beyond a
// wall, to the own slot opp(i)) -- the streamed phase.  Local (from the
// streamed phase): f'_i = own slot i, collision, f''_i to own slot opp(i)
// -- the swapped phase.  Every (slot, node) is read and written by one
// thread only, reads before writes, so the update in place is race-free.
template <class T, bool HM, bool HAS_F, bool PULLPUSH>
__device__ __forceinline__ void step_node3_aa(const Geo3 &g, const Phys3 &ph, T *A, const Node3 &nd, uint32_t m) {
    T f[Q3];
    gather3p<T, HM>(g, nd, A, m, PULLPUSH ? P3_SWAPPED : P3_STREAMED, f);
    T Fx, Fy, Fz;
    P3<T>::F(ph, Fx, Fy, Fz);
    collide3<T, HAS_F>(f, P3<T>::om(ph), P3<T>::kk(ph), Fx, Fy, Fz);
    A[nd.n] = f[0];
#pragma unroll
    for (int i = 1; i < Q3; ++i) {
        unsigned long long k;
        if (!PULLPUSH) k = (unsigned long long)opp3(i) * g.N + nd.n;
        else if (HM && (m & (1u << (opp3(i) - 1)))) k = (unsigned long long)opp3(i) * g.N + nd.n;
        else k = (unsigned long long)i * g.N + nd.src(g, opp3(i));
        A[k] = f[i];
    }
}

template <class T, bool HM, bool HAS_F, bool PULLPUSH>
__global__ void __launch_bounds__(BLOCK3, sizeof(T) == 4 ? 6 : 1) k3_step_aa(const Geo3 g, const Phys3 ph, T *A) {
    const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (x >= g.nx) return;
    const Node3 nd(g, x, (int)blockIdx.y, (int)blockIdx.z);
    uint32_t m = 0u;
    if (HM) {
        m = g.mask[nd.n];
        if (m == SOLID3) return;
    }
    step_node3_aa<T, HM, HAS_F, PULLPUSH>(g, ph, A, nd, m);
}

// The listed AA step: one thread per fluid node of the node list (the AA
// pattern's list holds fluid nodes only; its in-place stores touch sectors
// the same warp has just read).
template <class T, bool HAS_F, bool PULLPUSH>
__global__ void __launch_bounds__(BLOCK3, sizeof(T) == 4 ? 6 : 1) k3_step_aa_list(const Geo3 g, const Phys3 ph,
                                                                                 T *A) {
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.nlist) return;
    const uint2 e = g.list[t];
    const unsigned n = e.x;
    const uint32_t m = e.y;
    if (m == SOLID3) return;
    step_node3_aa<T, true, HAS_F, PULLPUSH>(g, ph, A, Node3::at(g, n), m);
}

// ---- FP16s storage: two nodes (x0 even, x0 + 1) per thread, rounded
// together stochastically by one packed conversion per link, as in two
// dimensions.
__device__ __forceinline__ unsigned f16x2_rs3(float lo, float hi, unsigned rbits) {
    unsigned r;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(r) : "f"(hi), "f"(lo), "r"(rbits));
    return r;
}
// counter-based random bits: the MurmurHash3 32-bit finaliser of (even
// node's index, step seed), then one linear congruential step per link
__device__ __forceinline__ unsigned fmix32_3(unsigned h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

template <bool HM, bool HAS_F>
__global__ void __launch_bounds__(BLOCK3) k3_step_h(const Geo3 g, const Phys3 ph, const unsigned short *__restrict__ A,
                                                    unsigned short *__restrict__ B, unsigned step) {
    const int x0 = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (!HM && x0 >= g.nx) return; // nx is even
    const int y = (int)blockIdx.y, z = (int)blockIdx.z;
    const Node3 a(g, x0, y, z), b(g, x0 + 1, y, z);
    uint32_t m0 = 0u, m1 = 0u;
    if (HM) {
        // the whole warp votes (as in k3_step); lanes beyond the row count
        // as solid and touch no memory
        const bool in = x0 < g.nx;
        if (in) {
            const uint2 mm = *reinterpret_cast<const uint2 *>(g.mask + a.n);
            m0 = mm.x;
            m1 = mm.y;
        } else {
            m0 = m1 = SOLID3;
        }
        const unsigned fluid = __ballot_sync(0xFFFFFFFFu, m0 != SOLID3 || m1 != SOLID3);
        if (!in) return;
        if (m0 == SOLID3 && m1 == SOLID3) {
            // never read; zeros where the sector holds fluid (whole-sector
            // stores)
            if (sector_has_fluid<4>(fluid)) {
#pragma unroll
                for (int i = 0; i < Q3; ++i)
                    *reinterpret_cast<unsigned *>(B + (unsigned long long)i * g.N + a.n) = 0u;
            }
            return;
        }
    }
    // gather in units of the stored scale: links along y and z (c_x = 0)
    // pull both nodes' values with one aligned 4-byte load
    float f[2][Q3];
#pragma unroll
    for (int i = 0; i < Q3; ++i) {
        const unsigned long long so = (unsigned long long)i * g.N;
        if (c3(i, 0) == 0) {
            const unsigned w = *reinterpret_cast<const unsigned *>(A + so + a.src(g, i));
            f[0][i] = __half2float(__ushort_as_half((unsigned short)(w & 0xFFFFu)));
            f[1][i] = __half2float(__ushort_as_half((unsigned short)(w >> 16)));
        } else {
            f[0][i] = __half2float(__ushort_as_half(A[so + a.src(g, i)]));
            f[1][i] = __half2float(__ushort_as_half(A[so + b.src(g, i)]));
        }
    }
    if (HM && (m0 | m1)) {
        // half-way bounce-back: the own node's value of the opposite link
#pragma unroll
        for (int i = 1; i < Q3; ++i) {
            const uint32_t bit = 1u << (i - 1);
            if ((m0 | m1) & bit) {
                const unsigned w = *reinterpret_cast<const unsigned *>(A + (unsigned long long)opp3(i) * g.N + a.n);
                if (m0 & bit) f[0][i] = __half2float(__ushort_as_half((unsigned short)(w & 0xFFFFu)));
                if (m1 & bit) f[1][i] = __half2float(__ushort_as_half((unsigned short)(w >> 16)));
            }
        }
    }
    float Fx = ph.fx_f, Fy = ph.fy_f, Fz = ph.fz_f;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        // the collision on the stored scale (values are (f - w) 2^10)
        collide3<float, HAS_F, (int)H3_SCALE>(f[k], ph.om_f, ph.kk_f, Fx, Fy, Fz);
        const bool solid = HM && (k == 0 ? m0 : m1) == SOLID3;
#pragma unroll
        for (int i = 0; i < Q3; ++i) f[k][i] = solid ? 0.0f : f[k][i];
    }
    unsigned h = fmix32_3(a.n ^ fmix32_3(step * 0x9E3779B9u + 0x632BE5ABu));
#pragma unroll
    for (int i = 0; i < Q3; ++i) {
        h = h * 1664525u + 1013904223u;
        *reinterpret_cast<unsigned *>(B + (unsigned long long)i * g.N + a.n) = f16x2_rs3(f[0][i], f[1][i], h ^ (h >> 16));
    }
}

// rho and u at the current time (the gather without the collision); 0 at
// solid nodes.
template <class R>
__global__ void __launch_bounds__(BLOCK3) k3_macros(const Geo3 g, const Phys3 ph, int phase, const R *A,
                                                    typename Cod3<R>::C *rho, typename Cod3<R>::C *u) {
    typedef typename Cod3<R>::C T;
    const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (x >= g.nx) return;
    const Node3 nd(g, x, (int)blockIdx.y, (int)blockIdx.z);
    const uint32_t m = g.mask ? g.mask[nd.n] : 0u;
    if (m == SOLID3) {
        if (rho) rho[nd.n] = T(0);
        if (u)
            for (int a = 0; a < 3; ++a) u[(unsigned)a * g.N + nd.n] = T(0);
        return;
    }
    T f[Q3];
    if (g.mask) gather3p<R, true>(g, nd, A, m, phase, f);
    else gather3p<R, false>(g, nd, A, m, phase, f);
    T Fx, Fy, Fz, drho, jx, jy, jz;
    P3<T>::F(ph, Fx, Fy, Fz);
    moments3<T>(f, Fx, Fy, Fz, drho, jx, jy, jz);
    const T r = T(1) + drho;
    if (rho) rho[nd.n] = r;
    if (u) {
        u[nd.n] = jx / r;
        u[g.N + nd.n] = jy / r;
        u[2u * g.N + nd.n] = jz / r;
    }
}

// A = f^eq(rho, u) - w at fluid nodes (rho = 1, u = 0 where NULL), 0 (that
// is, w) at solid nodes.
template <class R>
__global__ void __launch_bounds__(BLOCK3) k3_init(const Geo3 g, int phase, const typename Cod3<R>::C *rho,
                                                  const typename Cod3<R>::C *u, R *A) {
    typedef typename Cod3<R>::C T;
    const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (x >= g.nx) return;
    const unsigned n = (((unsigned)blockIdx.z * (unsigned)g.ny + blockIdx.y) * (unsigned)g.nx) + (unsigned)x;
    const bool solid = g.mask && g.mask[n] == SOLID3;
    const T r = rho ? rho[n] : T(1);
    const T ux = u ? u[n] : T(0), uy = u ? u[g.N + n] : T(0), uz = u ? u[2u * g.N + n] : T(0);
    const T usq = T(1.5) * (ux * ux + uy * uy + uz * uz);
#pragma unroll
    for (int i = 0; i < Q3; ++i) {
        const T t = T(c3(i, 0)) * ux + T(c3(i, 1)) * uy + T(c3(i, 2)) * uz;
        const T d = w3<T>(i) * ((r - T(1)) + r * (T(3) * t + T(4.5) * t * t - usq));
        A[(unsigned long long)(phase == P3_SWAPPED ? opp3(i) : i) * g.N + n] = Cod3<R>::enc(solid ? T(0) : d);
    }
}

// canonical f = stored + w (get, any phase), stored = f - w (set, plain or
// swapped phase); solid nodes read w_i
template <class R>
__global__ void __launch_bounds__(BLOCK3) k3_get(const Geo3 g, int phase, const R *in, typename Cod3<R>::C *out) {
    typedef typename Cod3<R>::C T;
    const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (x >= g.nx) return;
    const Node3 nd(g, x, (int)blockIdx.y, (int)blockIdx.z);
    const uint32_t m = g.mask ? g.mask[nd.n] : 0u;
#pragma unroll
    for (int i = 0; i < Q3; ++i) {
        const T v = m == SOLID3 ? T(0) : canon3<R>(g, nd, in, m, phase, i);
        out[(unsigned long long)i * g.N + nd.n] = v + w3<T>(i);
    }
}
template <class R>
__global__ void __launch_bounds__(BLOCK3) k3_set(const Geo3 g, int phase, const typename Cod3<R>::C *in, R *out) {
    typedef typename Cod3<R>::C T;
    const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (x >= g.nx) return;
    const unsigned n = (((unsigned)blockIdx.z * (unsigned)g.ny + blockIdx.y) * (unsigned)g.nx) + (unsigned)x;
#pragma unroll
    for (int i = 0; i < Q3; ++i) {
        const int slot = phase == P3_SWAPPED ? opp3(i) : i;
        out[(unsigned long long)slot * g.N + n] = Cod3<R>::enc(in[(unsigned long long)i * g.N + n] - w3<T>(i));
    }
}

} // namespace

// ------------------------------------------------------------- C ABI

struct lbm3_ctx {
    lbm3_params p;
    Geo3 g;
    Phys3 ph;
    size_t es = 0;   // bytes per stored value
    void *lat[2] = {nullptr, nullptr};
    int cur = 0;     // lattice holding A_t
    int phase = 0;   // Phase3 of the lattice
    long long steps = 0, nfluid = 0;
    cudaStream_t stream = nullptr;
    lbm_status sticky = LBM_OK;
    std::string err;
};

namespace {

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

const char *check3(const lbm3_params *p) {
    if (!p) return "params is NULL";
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return "nx, ny, nz must be >= 1";
    if (p->ny > 65535 || p->nz > 65535) return "ny and nz must be <= 65535";
    if ((double)p->nx * p->ny * p->nz >= 4294967296.0) return "nx*ny*nz must be < 2^32";
    if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return "tau must be > 0.5";
    if (!std::isfinite(p->fx) || !std::isfinite(p->fy) || !std::isfinite(p->fz)) return "force must be finite";
    if (p->precision != LBM_F64 && p->precision != LBM_F32 && p->precision != LBM_F16S) return "unknown precision";
    if (p->precision == LBM_F16S && (p->nx % 2)) return "FP16s storage needs an even nx (node pairs)";
    if (p->pattern != LBM_TWO_LATTICE && p->pattern != LBM_AA) return "unknown pattern";
    if (p->node_list < 0 || p->node_list > 2) return "node_list must be 0, 1 or 2";
    return nullptr;
}

// Link mask (host): bit i - 1 set iff link i of a fluid node pulls from a
// solid node or from beyond a wall face; SOLID3 for solid nodes.  Returns
// the fluid node count; `any` tells whether some link bounces.
long long build_mask3(const lbm3_params &p, std::vector<uint32_t> &m, bool &any) {
    const long long N = (long long)p.nx * p.ny * p.nz;
    m.assign((size_t)N, 0u);
    any = false;
    long long nf = 0;
    const int n[3] = {p.nx, p.ny, p.nz};
    const int per[3] = {p.periodic_x != 0, p.periodic_y != 0, p.periodic_z != 0};
    for (int z = 0; z < p.nz; ++z)
        for (int y = 0; y < p.ny; ++y)
            for (int x = 0; x < p.nx; ++x) {
                const long long k = ((long long)z * p.ny + y) * p.nx + x;
                if (p.solid && p.solid[k]) {
                    m[(size_t)k] = SOLID3;
                    any = true;
                    continue;
                }
                ++nf;
                uint32_t bits = 0;
                for (int i = 1; i < Q3; ++i) {
                    int q[3] = {x - c3(i, 0), y - c3(i, 1), z - c3(i, 2)};
                    bool out = false;
                    for (int a = 0; a < 3; ++a)
                        if (q[a] < 0 || q[a] >= n[a]) {
                            if (per[a]) q[a] = (q[a] + n[a]) % n[a];
                            else out = true;
                        }
                    if (out || (p.solid && p.solid[((long long)q[2] * p.ny + q[1]) * p.nx + q[0]]))
                        bits |= 1u << (i - 1);
                }
                m[(size_t)k] = bits;
                any = any || bits != 0u;
            }
    return nf;
}

// The node list of the listed step, ascending: every fluid node and, with
// two lattices, every solid node that shares a 32-byte sector of the stored
// slot planes with a fluid node (it stores zeros there, so the sector is
// written whole).  Built for FP64 / FP32 storage when some link bounces,
// and used when node_list is 2, or 0 with the AA pattern and at most 90% of
// the nodes listed (with two lattices the dense grid measured faster: its
// zero-storing solid lanes ride in warps that hold fluid anyway, while in
// the list they take lanes of their own); otherwise empty and the dense
// grid runs.  Returns the entries; with
// `mask` (the link mask) and `out`, writes them as (node index, its mask).
size_t node_list3(const lbm3_params &p, bool has_mask, const std::vector<uint32_t> *mask, std::vector<uint2> *out) {
    if (out) out->clear();
    if (!has_mask || p.precision == LBM_F16S || p.node_list == 1) return 0;
    const size_t N = (size_t)p.nx * p.ny * p.nz;
    const size_t G = p.precision == LBM_F64 ? 4 : 8; // nodes per 32-byte sector
    const bool two = p.pattern == LBM_TWO_LATTICE;
    auto fluid = [&](size_t k) { return !(p.solid && p.solid[k]); };
    // calls fn on the listed nodes in ascending order
    auto visit = [&](auto fn) {
        for (size_t s0 = 0; s0 < N; s0 += G) {
            const size_t s1 = s0 + G < N ? s0 + G : N;
            bool any = false;
            if (two)
                for (size_t k = s0; k < s1; ++k) any = any || fluid(k);
            for (size_t k = s0; k < s1; ++k)
                if (any || fluid(k)) fn(k);
        }
    };
    size_t len = 0;
    visit([&](size_t) { ++len; });
    if (len == 0 || (p.node_list == 0 && (two || 10 * len > 9 * N))) return 0;
    if (out && mask) {
        out->reserve(len);
        visit([&](size_t k) { out->push_back(make_uint2((unsigned)k, (*mask)[k])); });
    }
    return len;
}

struct Plan3 {
    size_t lat, off1, offm, offl, total;
    bool has_mask;
};
Plan3 plan3(const lbm3_params &p, bool has_mask, size_t nlist) {
    Plan3 pl;
    const size_t N = (size_t)p.nx * p.ny * p.nz;
    const size_t es = p.precision == LBM_F64 ? 8 : (p.precision == LBM_F32 ? 4 : 2);
    pl.lat = Q3 * N * es;
    pl.off1 = p.pattern == LBM_AA ? 0 : al256(pl.lat); // AA: one lattice
    pl.offm = pl.off1 + al256(pl.lat);
    pl.has_mask = has_mask;
    pl.offl = pl.offm + (has_mask ? al256(N * 4) : 0);
    pl.total = pl.offl + al256(nlist * sizeof(uint2));
    return pl;
}
bool any_bounce(const lbm3_params &p) {
    if (!p.periodic_x || !p.periodic_y || !p.periodic_z) return true;
    if (p.solid) {
        const size_t N = (size_t)p.nx * p.ny * p.nz;
        for (size_t k = 0; k < N; ++k)
            if (p.solid[k]) return true;
    }
    return false;
}

lbm_status fail3(lbm3_ctx *c, lbm_status s, const std::string &msg) {
    if (c) {
        if (s == LBM_ERR_CUDA) c->sticky = s;
        c->err = msg;
    }
    return s;
}
lbm_status cuda3(lbm3_ctx *c, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return LBM_OK;
    return fail3(c, LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
dim3 grid3(const Geo3 &g) {
    return dim3((unsigned)((g.nx + BLOCK3 - 1) / BLOCK3), (unsigned)g.ny, (unsigned)g.nz);
}
bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

cudaError_t step3h(lbm3_ctx *c) {
    const unsigned short *A = static_cast<const unsigned short *>(c->lat[c->cur]);
    unsigned short *B = static_cast<unsigned short *>(c->lat[1 - c->cur]);
    const bool F = c->p.fx != 0.0 || c->p.fy != 0.0 || c->p.fz != 0.0;
    const int pairs = c->g.nx / 2;
    const dim3 gr((unsigned)((pairs + BLOCK3 - 1) / BLOCK3), (unsigned)c->g.ny, (unsigned)c->g.nz);
    const unsigned t = (unsigned)c->steps;
    if (c->g.mask) {
        if (F) k3_step_h<true, true><<<gr, BLOCK3, 0, c->stream>>>(c->g, c->ph, A, B, t);
        else k3_step_h<true, false><<<gr, BLOCK3, 0, c->stream>>>(c->g, c->ph, A, B, t);
    } else {
        if (F) k3_step_h<false, true><<<gr, BLOCK3, 0, c->stream>>>(c->g, c->ph, A, B, t);
        else k3_step_h<false, false><<<gr, BLOCK3, 0, c->stream>>>(c->g, c->ph, A, B, t);
    }
    return cudaGetLastError();
}
template <class T> cudaError_t step3aa(lbm3_ctx *c) {
    T *A = static_cast<T *>(c->lat[0]);
    const bool F = c->p.fx != 0.0 || c->p.fy != 0.0 || c->p.fz != 0.0;
    const bool pp = c->phase == P3_SWAPPED;
    const dim3 gr = grid3(c->g);
#define LBM3_AA(HM, HF)                                                                    \
    (pp ? (k3_step_aa<T, HM, HF, true><<<gr, BLOCK3, 0, c->stream>>>(c->g, c->ph, A), 0)    \
        : (k3_step_aa<T, HM, HF, false><<<gr, BLOCK3, 0, c->stream>>>(c->g, c->ph, A), 0))
#define LBM3_AA_LIST(HF)                                                                    \
    (pp ? (k3_step_aa_list<T, HF, true><<<gl, BLOCK3, 0, c->stream>>>(c->g, c->ph, A), 0)   \
        : (k3_step_aa_list<T, HF, false><<<gl, BLOCK3, 0, c->stream>>>(c->g, c->ph, A), 0))
    if (c->g.list) {
        const dim3 gl((c->g.nlist + BLOCK3 - 1) / BLOCK3);
        if (F) LBM3_AA_LIST(true);
        else LBM3_AA_LIST(false);
    } else if (c->g.mask) {
        if (F) LBM3_AA(true, true);
        else LBM3_AA(true, false);
    } else {
        if (F) LBM3_AA(false, true);
        else LBM3_AA(false, false);
    }
#undef LBM3_AA
#undef LBM3_AA_LIST
    return cudaGetLastError();
}
template <class T> cudaError_t step3(lbm3_ctx *c) {
    const T *A = static_cast<const T *>(c->lat[c->cur]);
    T *B = static_cast<T *>(c->lat[1 - c->cur]);
    const bool F = c->p.fx != 0.0 || c->p.fy != 0.0 || c->p.fz != 0.0;
    const dim3 gr = grid3(c->g);
    if (c->g.list) {
        const dim3 gl((c->g.nlist + BLOCK3 - 1) / BLOCK3);
        if (F) k3_step_list<T, true><<<gl, BLOCK3, 0, c->stream>>>(c->g, c->ph, A, B);
        else k3_step_list<T, false><<<gl, BLOCK3, 0, c->stream>>>(c->g, c->ph, A, B);
    } else if (c->g.mask) {
        if (F) k3_step<T, true, true><<<gr, BLOCK3, 0, c->stream>>>(c->g, c->ph, A, B);
        else k3_step<T, true, false><<<gr, BLOCK3, 0, c->stream>>>(c->g, c->ph, A, B);
    } else {
        if (F) k3_step<T, false, true><<<gr, BLOCK3, 0, c->stream>>>(c->g, c->ph, A, B);
        else k3_step<T, false, false><<<gr, BLOCK3, 0, c->stream>>>(c->g, c->ph, A, B);
    }
    return cudaGetLastError();
}

// Calls f with a null pointer of the context's stored element type.
template <class F> cudaError_t by_storage3(const lbm3_ctx *c, F f) {
    if (c->es == 8) return f(static_cast<double *>(nullptr));
    if (c->es == 4) return f(static_cast<float *>(nullptr));
    return f(static_cast<unsigned short *>(nullptr));
}

} // namespace

extern "C" {

lbm_status lbm3_workspace_bytes(const lbm3_params *p, size_t *bytes) {
    if (check3(p) || !bytes) return LBM_ERR_INVALID;
    const bool any = any_bounce(*p);
    *bytes = plan3(*p, any, node_list3(*p, any, nullptr, nullptr)).total;
    return LBM_OK;
}

lbm_status lbm3_create(const lbm3_params *p, void *d_workspace, size_t bytes, lbm3_ctx **out) {
    if (!out) return LBM_ERR_INVALID;
    *out = nullptr;
    if (check3(p) || !d_workspace || ((uintptr_t)d_workspace & 255u)) return LBM_ERR_INVALID;
    if (p->pattern == LBM_AA && p->precision == LBM_F16S) return LBM_ERR_UNSUPPORTED;
    std::vector<uint32_t> mask;
    bool any = false;
    const long long nf = build_mask3(*p, mask, any);
    std::vector<uint2> list;
    const size_t nlist = node_list3(*p, any, &mask, &list);
    const Plan3 pl = plan3(*p, any, nlist);
    if (bytes < pl.total) return LBM_ERR_OOM;
    lbm3_ctx *c = new lbm3_ctx();
    c->p = *p;
    c->p.solid = nullptr; // read here only
    c->es = p->precision == LBM_F64 ? 8 : (p->precision == LBM_F32 ? 4 : 2);
    c->stream = static_cast<cudaStream_t>(p->stream);
    c->nfluid = nf;
    char *ws = static_cast<char *>(d_workspace);
    c->lat[0] = ws;
    c->lat[1] = ws + pl.off1;
    c->phase = p->pattern == LBM_AA ? P3_SWAPPED : P3_PLAIN;
    Geo3 &g = c->g;
    g.nx = p->nx;
    g.ny = p->ny;
    g.nz = p->nz;
    g.px = p->periodic_x != 0;
    g.py = p->periodic_y != 0;
    g.pz = p->periodic_z != 0;
    g.N = (unsigned long long)p->nx * p->ny * p->nz;
    g.mask = any ? reinterpret_cast<const uint32_t *>(ws + pl.offm) : nullptr;
    g.list = nlist ? reinterpret_cast<const uint2 *>(ws + pl.offl) : nullptr;
    g.nlist = (unsigned)nlist;
    g.mx = 0xFFFFFFFFu / (unsigned)p->nx;
    g.my = 0xFFFFFFFFu / (unsigned)p->ny;
    Phys3 &ph = c->ph;
    ph.om = 1.0 / p->tau;
    ph.kk = 1.0 - 0.5 * ph.om;
    ph.fx = p->fx;
    ph.fy = p->fy;
    ph.fz = p->fz;
    ph.om_f = (float)ph.om;
    ph.kk_f = 1.0f - 0.5f * ph.om_f;
    ph.fx_f = (float)p->fx;
    ph.fy_f = (float)p->fy;
    ph.fz_f = (float)p->fz;
    lbm_status st = cuda3(c, cudaMemsetAsync(ws, 0, pl.offm, c->stream), "memset lattices");
    if (!st && any)
        st = cuda3(c, cudaMemcpyAsync(ws + pl.offm, mask.data(), mask.size() * 4, cudaMemcpyHostToDevice, c->stream),
                   "copy link mask");
    if (!st && nlist)
        st = cuda3(c, cudaMemcpyAsync(ws + pl.offl, list.data(), nlist * sizeof(uint2), cudaMemcpyHostToDevice,
                                      c->stream),
                   "copy node list");
    if (!st) st = cuda3(c, cudaStreamSynchronize(c->stream), "create sync");
    if (st) {
        delete c;
        return st;
    }
    *out = c;
    return LBM_OK;
}

lbm_status lbm3_destroy(lbm3_ctx *ctx) {
    if (!ctx) return LBM_ERR_INVALID;
    delete ctx;
    return LBM_OK;
}

#define LBM3_CHECK(ctx)                                   \
    do {                                                  \
        if (!(ctx)) return LBM_ERR_INVALID;               \
        if ((ctx)->sticky != LBM_OK) return (ctx)->sticky; \
    } while (0)

lbm_status lbm3_init_equilibrium(lbm3_ctx *ctx, const void *d_rho, const void *d_u) {
    LBM3_CHECK(ctx);
    if ((d_rho && !aligned16(d_rho)) || (d_u && !aligned16(d_u)))
        return fail3(ctx, LBM_ERR_INVALID, "fields must be 16-byte aligned");
    const dim3 gr = grid3(ctx->g);
    ctx->phase = ctx->p.pattern == LBM_AA ? P3_SWAPPED : P3_PLAIN;
    const cudaError_t e = by_storage3(ctx, [&](auto tag) {
        typedef std::remove_pointer_t<decltype(tag)> R;
        typedef typename Cod3<R>::C C;
        k3_init<R><<<gr, BLOCK3, 0, ctx->stream>>>(ctx->g, ctx->phase, static_cast<const C *>(d_rho),
                                                   static_cast<const C *>(d_u), static_cast<R *>(ctx->lat[0]));
        return cudaGetLastError();
    });
    ctx->cur = 0;
    ctx->steps = 0;
    return cuda3(ctx, e, "init launch");
}

lbm_status lbm3_step(lbm3_ctx *ctx, int n) {
    LBM3_CHECK(ctx);
    if (n < 0) return fail3(ctx, LBM_ERR_INVALID, "n < 0");
    for (int k = 0; k < n; ++k) {
        cudaError_t e;
        if (ctx->p.pattern == LBM_AA) {
            e = ctx->es == 8 ? step3aa<double>(ctx) : step3aa<float>(ctx);
            ctx->phase = ctx->phase == P3_SWAPPED ? P3_STREAMED : P3_SWAPPED;
        } else {
            e = ctx->es == 8 ? step3<double>(ctx) : (ctx->es == 4 ? step3<float>(ctx) : step3h(ctx));
            ctx->cur = 1 - ctx->cur;
        }
        if (e != cudaSuccess) return cuda3(ctx, e, "step launch");
        ++ctx->steps;
    }
    return LBM_OK;
}

lbm_status lbm3_macros(lbm3_ctx *ctx, void *d_rho, void *d_u) {
    LBM3_CHECK(ctx);
    if ((d_rho && !aligned16(d_rho)) || (d_u && !aligned16(d_u)))
        return fail3(ctx, LBM_ERR_INVALID, "fields must be 16-byte aligned");
    const dim3 gr = grid3(ctx->g);
    return cuda3(ctx, by_storage3(ctx, [&](auto tag) {
                     typedef std::remove_pointer_t<decltype(tag)> R;
                     typedef typename Cod3<R>::C C;
                     k3_macros<R><<<gr, BLOCK3, 0, ctx->stream>>>(ctx->g, ctx->ph, ctx->phase,
                                                                  static_cast<const R *>(ctx->lat[ctx->cur]),
                                                                  static_cast<C *>(d_rho), static_cast<C *>(d_u));
                     return cudaGetLastError();
                 }),
                 "macros launch");
}

lbm_status lbm3_get_f(lbm3_ctx *ctx, void *d_f) {
    LBM3_CHECK(ctx);
    if (!d_f || !aligned16(d_f)) return fail3(ctx, LBM_ERR_INVALID, "f must be a 16-byte aligned pointer");
    const dim3 gr = grid3(ctx->g);
    return cuda3(ctx, by_storage3(ctx, [&](auto tag) {
                     typedef std::remove_pointer_t<decltype(tag)> R;
                     typedef typename Cod3<R>::C C;
                     k3_get<R><<<gr, BLOCK3, 0, ctx->stream>>>(ctx->g, ctx->phase,
                                                               static_cast<const R *>(ctx->lat[ctx->cur]),
                                                               static_cast<C *>(d_f));
                     return cudaGetLastError();
                 }),
                 "get launch");
}

lbm_status lbm3_set_f(lbm3_ctx *ctx, const void *d_f) {
    LBM3_CHECK(ctx);
    if (!d_f || !aligned16(d_f)) return fail3(ctx, LBM_ERR_INVALID, "f must be a 16-byte aligned pointer");
    const dim3 gr = grid3(ctx->g);
    ctx->phase = ctx->p.pattern == LBM_AA ? P3_SWAPPED : P3_PLAIN;
    return cuda3(ctx, by_storage3(ctx, [&](auto tag) {
                     typedef std::remove_pointer_t<decltype(tag)> R;
                     typedef typename Cod3<R>::C C;
                     k3_set<R><<<gr, BLOCK3, 0, ctx->stream>>>(ctx->g, ctx->phase, static_cast<const C *>(d_f),
                                                               static_cast<R *>(ctx->lat[ctx->cur]));
                     return cudaGetLastError();
                 }),
                 "set launch");
}

long long lbm3_fluid_nodes(const lbm3_ctx *ctx) { return ctx ? ctx->nfluid : -1; }

long long lbm3_list_nodes(const lbm3_ctx *ctx) { return ctx ? (long long)ctx->g.nlist : -1; }
long long lbm3_step_count(const lbm3_ctx *ctx) { return ctx ? ctx->steps : -1; }
const char *lbm3_last_error(const lbm3_ctx *ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

} // extern "C"
