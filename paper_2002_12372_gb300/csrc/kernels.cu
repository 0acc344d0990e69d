// QQMC device kernels for sm_103a.
//
//  * gf_table_kernel   -- g^<(tau), g^>(tau) of the wide-band dot by the
//                         contour-deformed Fourier integral of App. E.
//  * lead_*_kernel     -- the same for semicircular leads of finite width
//                         and bias, plus the dot-lead tables of the current.
//  * detsum_kernel     -- the hot path: Sobol' point generation with a digital
//                         shift, exponential product-model warp, pair
//                         interpolation of the Green-function tables and the
//                         Keldysh sum of det M_up * det M_down (App. E
//                         Eq. (integral_gf)), weighted and reduced per chunk.
//  * reduce_kernel     -- per shifted sequence, compensated sum of the chunk
//                         partials (Eq. (warped_int2)).
//  * sobol/warp/integrand kernels -- the same device code exposed for checks.
//
// Keldysh sum: the vertices are ordered t = u_0 > u_1 > ... > u_n > 0.  For a
// pair j < k the Keldysh matrix entry above the diagonal depends only on a_k
// (a_k = 0: g^>(u_j-u_k), a_k = 1: g^<(u_j-u_k)) and the one below only on a_k
// too (a_k = 0: g^<(u_k-u_j), a_k = 1: g^>(u_k-u_j)); the diagonal is g^<(0).
// Row 0 / column 0 of M_up are the measurement points (t, a=0) / (i, t, a=1):
// site i = 0 for the charge, lead site 1 for the current, whose column then
// holds the dot-lead functions gamma g^<_01, gamma g^>_01 (App. E).
// Hence, once the leading vertices are eliminated, every entry of the Schur
// complement depends only on the Keldysh indices of its own row and column
// vertices.  The kernel walks the binary tree of Keldysh indices depth first
// and keeps, per tree level, the Schur complement for BOTH choices of every
// remaining vertex: a (2R+2) x (2R+2) matrix (rows/columns = (vertex, choice)
// plus two copies of the measurement row/column, one per choice of a_1).
// Fixing a_k is one rank-1 update of that matrix with the pivot (k, a_k).
// det M_down is the product of the pivots, det M_up / det M_down is the final
// measurement entry, and sum_{a_1} (-1)^{a_1} det M_up det M_down =
// det M_down^2 (S_00(a_1=0) - S_00(a_1=1)).  The last F vertices are resolved
// per lane (one lane per choice path, 2^F paths).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <atomic>

#include "qqmc_internal.h"

namespace qqmc {

__constant__ uint32_t c_dirs[kMaxOrder][32];
__constant__ double c_gl_x[16];
__constant__ double c_gl_w[16];

constexpr unsigned FULL = 0xffffffffu;
constexpr size_t kSmemMax = 227 * 1024;  // dynamic shared memory one block can address

// ----------------------------------------------------------------------------
// complex helpers
// ----------------------------------------------------------------------------
template <class R>
struct __align__(2 * sizeof(R)) cx {
    R re, im;
};

__device__ __forceinline__ double fmaR(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaR(float a, float b, float c) { return fmaf(a, b, c); }

template <class R>
__device__ __forceinline__ cx<R> mk(R a, R b) {
    cx<R> z;
    z.re = a;
    z.im = b;
    return z;
}
template <class R>
__device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
    return mk<R>(fmaR(a.re, b.re, -a.im * b.im), fmaR(a.re, b.im, a.im * b.re));
}
// c - a * b
template <class R>
__device__ __forceinline__ cx<R> cfms(cx<R> c, cx<R> a, cx<R> b) {
    return mk<R>(fmaR(-a.re, b.re, fmaR(a.im, b.im, c.re)), fmaR(-a.re, b.im, fmaR(-a.im, b.re, c.im)));
}
// 1/x.  FP64: IEEE division.  FP32: the hardware approximation (PTX
// rcp.approx.ftz.f32) refined by one Newton-Raphson step r' = r + r (1 - x r),
// which leaves ~1 ulp, well inside the FP32 path's error budget and without
// the division's special-case branch.
// FP64 reciprocal: the hardware approximation refined by two Newton-Raphson
// steps r <- r + r (1 - x r) (each squares the relative error), fewer FP64
// instructions than an IEEE division; within an ulp or two of 1/x.
__device__ __forceinline__ double recip(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    r = fma(r, fma(-x, r, 1.0), r);
    return fma(r, fma(-x, r, 1.0), r);
}
__device__ __forceinline__ float recip(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return fmaf(r, fmaf(-x, r, 1.0f), r);
}
template <class R>
__device__ __forceinline__ cx<R> crcp(cx<R> a) {
    R s = recip(fmaR(a.re, a.re, a.im * a.im));
    return mk<R>(a.re * s, -a.im * s);
}
template <class R>
__device__ __forceinline__ cx<R> nconj(cx<R> a) {  // -conj(a)
    return mk<R>(-a.re, a.im);
}

// Lane accumulator of the Keldysh leaf terms, value = s + c.  FP32 leaves:
// Knuth two-sum (float-float), since the alternating-sign sum cancels by up to
// 1e5.  FP64 leaves: plain sum; a lane adds at most 2^(n-1)/32 terms, so its
// rounding stays below 1e-14 of the Keldysh-sum scale, and the lanes are
// combined with two-sum in warp_total.
template <class R>
struct Acc {
    R s, c;
    __device__ __forceinline__ void init() { s = R(0); c = R(0); }
    __device__ __forceinline__ void add(R x) {
        R t = s + x;
        R z = t - s;
        c += (s - (t - z)) + (x - z);
        s = t;
    }
};
template <>
__device__ __forceinline__ void Acc<double>::add(double x) { s += x; }

__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
    s = a + b;
    double z = s - a;
    e = (a - (s - z)) + (b - z);
}

// Deterministic butterfly reduction of (s, c) pairs over the warp.
__device__ __forceinline__ void warp_reduce_pair(double &s, double &c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double s2 = __shfl_xor_sync(FULL, s, o);
        double c2 = __shfl_xor_sync(FULL, c, o);
        double t, e;
        // combine in a lane-independent order (lower lane's value first)
        int lo = ((threadIdx.x & 31) & o) == 0;
        if (lo) two_sum(s, s2, t, e); else two_sum(s2, s, t, e);
        s = t;
        c = lo ? (c + c2) + e : (c2 + c) + e;
    }
}

// ----------------------------------------------------------------------------
// Sobol' point, shift and warp (shared by the integration and check kernels)
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t sobol_word(int d, uint64_t i) {
    uint64_t g = i ^ (i >> 1);
    uint32_t x = 0;
    while (g) {
        int j = __ffsll((long long)g) - 1;
        x ^= c_dirs[d][j];
        g &= g - 1;
    }
    return x;
}

// Shifted point word of dimension d for index i: Sobol' with a digital shift
// (XOR), or a rank-1 lattice of 2^m points, x = frac(i z / N + Delta) in 32-bit
// fixed point: ((i z_d mod 2^m) << (32 - m)) + S_d mod 2^32, optionally
// followed by the baker's transform x -> 1 - |2x - 1| (the word 2^31, which
// would map to exactly 1, stays at 1 - 2^-32).  lat_m: m, or 64 + m with the
// transform.
__device__ __forceinline__ uint32_t point_word(const uint32_t *lat_z, int lat_m, int d, uint64_t i, uint32_t s) {
    if (lat_z) {
        const int m = lat_m & 63;
        const uint64_t r = (i * (uint64_t)lat_z[d]) & ((1ull << m) - 1ull);
        const uint32_t w = (uint32_t)(r << (32 - m)) + s;
        if (lat_m < 64) return w;
        if (w < 0x80000000u) return w << 1;
        const uint64_t v = (1ull << 33) - 2ull * (uint64_t)w;
        return v > 0xffffffffull ? 0xffffffffu : (uint32_t)v;
    }
    return sobol_word(d, i) ^ s;
}

// ----------------------------------------------------------------------------
// Table interpolation: half table starting at node L/2 - 1 (tau = -h/2).
// ----------------------------------------------------------------------------
template <class R>
struct TabT;
template <>
struct TabT<double> {
    using V = dbl4;
};
template <>
struct TabT<float> {
    using V = float4;
};

// pair values for tau > 0: gl = g^<(tau), gg = g^>(tau).  Position on the
// mesh s = (tau + T) / h, formed as tau / h + T / h (one FP64 FMA); the blend
// runs in R.
template <class R>
__device__ __forceinline__ void interp_pair(const typename TabT<R>::V *tab, double inv_h, double s0, int L, double tau,
                                            cx<R> &gl, cx<R> &gg) {
    double s = fma(tau, inv_h, s0);
    int k = __double2int_rd(s);
    int kmin = L / 2 - 1, kmax = L - 2;
    k = k < kmin ? kmin : (k > kmax ? kmax : k);
    R fr = (R)(s - (double)k);
    R g = R(1) - fr;
    typename TabT<R>::V a = tab[k - kmin];
    typename TabT<R>::V b = tab[k - kmin + 1];
    gl = mk<R>(fmaR(fr, b.x, g * a.x), fmaR(fr, b.y, g * a.y));
    gg = mk<R>(fmaR(fr, b.z, g * a.z), fmaR(fr, b.w, g * a.w));
}

// Measurement-column values of the current at tau = u_k - t < 0 (a_k = 0:
// gamma g^<_01, a_k = 1: gamma g^>_01).  The column table holds the nodes
// k = 0 .. L/2 (tau from -T to +h/2).
template <class R>
__device__ __forceinline__ void interp_col(const typename TabT<R>::V *col, double inv_h, double s0, int L, double tau,
                                           cx<R> &cl, cx<R> &cg) {
    double s = fma(tau, inv_h, s0);
    int k = __double2int_rd(s);
    const int kmax = L / 2 - 1;
    k = k < 0 ? 0 : (k > kmax ? kmax : k);
    R fr = (R)(s - (double)k);
    R g = R(1) - fr;
    typename TabT<R>::V a = col[k];
    typename TabT<R>::V b = col[k + 1];
    cl = mk<R>(fmaR(fr, b.x, g * a.x), fmaR(fr, b.y, g * a.y));
    cg = mk<R>(fmaR(fr, b.z, g * a.z), fmaR(fr, b.w, g * a.w));
}

// ----------------------------------------------------------------------------
// Per-warp shared-memory layout for the Keldysh sum.
//
// The depth-first tree stops when kTreeLeaf vertices remain (or earlier for
// small n).  From there, B = Rleaf - RF levels are expanded breadth first
// (2, 4, ... 2^B sibling matrices, all lanes cooperating), and each lane
// resolves the last RF vertices of one node along one choice path in
// registers: 2^B nodes x 2^RF paths = 2^Rleaf <= 32 lanes.
// ----------------------------------------------------------------------------
constexpr int kTreeLeaf = 5;

template <class R>
struct WarpSmem {
    cx<R> *stack;   // tree levels, level l has (2 R_l + 2)^2 entries, R_l = n-1-l (shared memory)
    cx<R> *gstack;  // split stack: the levels wider than gs_level in device memory, or null
    cx<R> *wrow;    // scaled pivot row(s): <= max(2 n_max, 64) entries
    cx<R> *P;       // vertex k's block at o_k = (k-1)(k+2)/2: P[o_k + j] = g^>(u_j - u_k), 0 <= j < k,
                    // and P[o_k + k] = measurement-column entry (k, a_k = 1)
    cx<R> *Rr;      // Rr[o_k + j] = g^<(u_j - u_k); Rr[o_k + k] = column entry (k, a_k = 0)
    cx<R> *detD;    // per tree level, and (after the last) the sibling leaf's
    cx<R> *sib;     // the second leaf of a sibling pair (2 kTreeLeaf + 2)^2 entries
    cx<R> *lr;      // level 0: left and right factors of vertex 1 per block index (4 n_max)
    cx<R> *bfs;     // breadth-first levels (all nodes of one level contiguous)
    cx<R> *bdet;    // det M_down prefix per breadth-first node, two levels (2 x 32)
    cx<R> *bip;     // pivot reciprocal per child of the level being built (32)
    double *upt;    // [32][n_max+1] point times of the chunk (u_0 = t); device memory with the split stack
    int gs_level;   // split stack: levels with S > gs_level in device memory
};


// wrow, bdet and bip serve the general cooperative expansion: breadth-first
// levels (flat depth below the tree leaf) and depth-first steps wider than a
// warp (children of more than 32 rows, orders >= 18).
__host__ __device__ inline bool needs_wide_buffers(int n_max, int RF) {
    const int rl = n_max - 1 < kTreeLeaf ? n_max - 1 : kTreeLeaf;
    return RF < rl || 2 * (n_max - 1) > 32;
}

__host__ __device__ inline size_t stack_entries(int n_max) {
    size_t tot = 0;
    int R0 = n_max - 1;
    int levels = R0 > kTreeLeaf ? R0 - kTreeLeaf : 0;
    for (int l = 0; l <= levels; ++l) {
        size_t S = 2 * (size_t)(R0 - l) + 2;
        tot += S * S;
    }
    return tot;
}

// With the split stack the tree levels wider than gs_level (the top levels,
// built 1, 2, 4 ... times per point) live in device memory and the narrow, hot
// bottom levels stay in shared memory.
__host__ __device__ inline size_t stack_entries_split(int n_max, bool global_part, int gs_level) {
    size_t tot = 0;
    int R0 = n_max - 1;
    int levels = R0 > kTreeLeaf ? R0 - kTreeLeaf : 0;
    for (int l = 0; l <= levels; ++l) {
        size_t S = 2 * (size_t)(R0 - l) + 2;
        if (((int)S > gs_level) == global_part) tot += S * S;
    }
    return tot;
}

// entries of the breadth-first levels below a tree leaf of Rleaf vertices
__host__ __device__ inline size_t bfs_entries(int Rleaf, int RF) {
    size_t tot = 0;
    int B = Rleaf > RF ? Rleaf - RF : 0;
    for (int b = 1; b <= B; ++b) {
        size_t S = 2 * (size_t)(Rleaf - b) + 2;
        tot += ((size_t)1 << b) * S * S;
    }
    return tot;
}

__host__ __device__ inline size_t bfs_max_entries(int n_max, int RF) {
    size_t m = 0;
    for (int Rl = 0; Rl <= kTreeLeaf && Rl <= n_max - 1; ++Rl) {
        size_t e = bfs_entries(Rl, RF);
        m = e > m ? e : m;
    }
    return m;
}

// The mixed-precision path builds sibling leaves in pairs (one depth-first step
// for two leaves: its steps are latency-bound); the FP64 path, bound by its
// FP64 pipe, gains nothing from it and keeps the shared memory for warps.
template <class R>
__host__ __device__ constexpr bool twin_leaves() { return sizeof(R) == 4; }

// the sibling leaf buffer, used when the tree has depth-first levels
template <class R>
__host__ __device__ inline size_t sib_entries(int n_max) {
    return twin_leaves<R>() && n_max - 1 > kTreeLeaf ? (size_t)(2 * kTreeLeaf + 2) * (2 * kTreeLeaf + 2) : 0;
}

// entries of the packed pair values with the measurement column (P and Rr:
// blocks of k + 1 entries for the vertices k = 1 .. n_max)
__host__ __device__ inline size_t pair_entries(int n_max) { return (size_t)n_max * (n_max + 3); }

// Shared memory of one warp.  gs_level = 0: the whole tree stack and the point
// times in shared memory.  gs_level > 0 (split stack): the levels wider than
// gs_level and the point times in a per-warp slice of device memory.
template <class R>
__host__ __device__ inline size_t warp_smem_bytes_at(int n_max, int RF, int gs_level) {
    size_t wide = needs_wide_buffers(n_max, RF) ? (2 * (size_t)n_max > 64 ? 2 * (size_t)n_max : 64) + 64 + 32 : 0;
    size_t c = (gs_level ? stack_entries_split(n_max, false, gs_level) : stack_entries(n_max)) + pair_entries(n_max) +
               n_max + 1 + sib_entries<R>(n_max) + 4 * (size_t)n_max + bfs_max_entries(n_max, RF) + wide;
    size_t bytes = (c * sizeof(cx<R>) + 15) & ~(size_t)15;
    if (!gs_level) bytes += 32 * (size_t)(n_max + 1) * sizeof(double);
    return (bytes + 127) & ~(size_t)127;
}

// Split-stack boundary: the widest levels go to device memory, two rows at a
// time, until a warp's shared memory lets the SM hold the warps its bound pipe
// needs (FP64: 6 warps keep GB300's two FP64 lanes per SM busy; mixed: 12).
// Never the tree leaf (S = 12) or its parent (S = 14): the last depth-first
// step and the breadth-first and flat phases work in shared memory only.
template <class R>
__host__ __device__ inline int gs_level_of(int n_max, int RF) {
    const size_t budget = sizeof(R) == 8 ? 36 * 1024 : 18 * 1024;
    int lev = 20;
    while (lev > 2 * kTreeLeaf + 4 && warp_smem_bytes_at<R>(n_max, RF, lev) > budget) lev -= 2;
    return lev;
}

// Shared memory of one warp; with the split stack (gs) the wide top levels of
// the Schur tree live in a per-warp slice of device memory (FP64 orders >= 21,
// whose whole stack exceeds the 227 KB a block can address, and the orders the
// stack policy names).
template <class R>
__host__ __device__ inline size_t warp_smem_bytes(int n_max, int RF, bool gs = false) {
    return warp_smem_bytes_at<R>(n_max, RF, gs ? gs_level_of<R>(n_max, RF) : 0);
}

// Device-memory slice of one warp with the split stack: the wide levels, one
// spare entry, and the point times of the chunk.
template <class R>
__host__ __device__ inline size_t gstack_entries(int n_max, int RF) {
    return stack_entries_split(n_max, true, gs_level_of<R>(n_max, RF)) + 1 +
           (32 * (size_t)(n_max + 1) * sizeof(double) + sizeof(cx<R>) - 1) / sizeof(cx<R>);
}

template <class R>
__device__ __forceinline__ WarpSmem<R> carve(unsigned char *base, int n_max, int RF, cx<R> *gstack = nullptr) {
    WarpSmem<R> w;
    cx<R> *p = reinterpret_cast<cx<R> *>(base);
    w.gstack = gstack;
    w.gs_level = gstack ? gs_level_of<R>(n_max, RF) : 0;
    w.stack = p;
    p += gstack ? stack_entries_split(n_max, false, w.gs_level) : stack_entries(n_max);
    const int npair = n_max * (n_max + 3) / 2;
    w.P = p;
    p += npair;
    w.Rr = p;
    p += npair;
    w.detD = p;
    p += n_max + 1;
    w.sib = p;
    p += sib_entries<R>(n_max);
    w.lr = p;
    p += 4 * n_max;
    w.bfs = p;
    p += bfs_max_entries(n_max, RF);
    w.wrow = w.bdet = w.bip = nullptr;
    if (needs_wide_buffers(n_max, RF)) {
        w.wrow = p;
        p += 2 * n_max > 64 ? 2 * n_max : 64;
        w.bdet = p;
        p += 64;
        w.bip = p;
        p += 32;
    }
    size_t off = (reinterpret_cast<unsigned char *>(p) - base + 15) & ~(size_t)15;
    w.upt = gstack ? reinterpret_cast<double *>(gstack + stack_entries_split(n_max, true, w.gs_level) + 1)
                   : reinterpret_cast<double *>(base + off);
    return w;
}

// Leaf term after the last vertex p: with pivot pv and the copies' entries,
//   det' = det pv,   S_aa = m_aa - m_ap m_pa / pv   (a = copy 0, 1),
//   det'^2 (S_00 - S_11) = det^2 pv (pv (m_00 - m_11) - (m_0p m_p0 - m_1p m_p1)):
// the last elimination needs no reciprocal.
template <class R>
__device__ __forceinline__ cx<R> leaf_term(cx<R> m00, cx<R> m11, cx<R> m0p, cx<R> mp0, cx<R> m1p, cx<R> mp1, cx<R> pv,
                                           cx<R> det) {
    const cx<R> q = cfms(cmul(m0p, mp0), m1p, mp1);                        // m0p mp0 - m1p mp1
    const cx<R> r = cfms(q, pv, mk<R>(m00.re - m11.re, m00.im - m11.im));  // q - pv (m00 - m11)
    return cmul(cmul(det, det), cmul(pv, mk<R>(-r.re, -r.im)));
}

// Flat phase: one lane resolves the F remaining vertices of node matrix E
// (size S = 2F + 2) along the choice path `path` (bit q = Keldysh index of the
// q-th remaining vertex).  The first elimination is fused with the gather;
// the rest runs on an (F+1) x (F+1) register matrix whose rows and columns
// are {copy a_1 = 0, copy a_1 = 1, remaining vertices}.
template <class R, int F, int STRIDE = 1>
__device__ __forceinline__ void flat_phase(const cx<R> *E, cx<R> detD, int parity, int path, Acc<R> &acc_re,
                                           Acc<R> &acc_im) {
    constexpr int S = 2 * F + 2;
    if (F == 0) {
        cx<R> dd = cmul(detD, detD);
        cx<R> diff = mk<R>(E[0].re - E[(S + 1) * STRIDE].re, E[0].im - E[(S + 1) * STRIDE].im);
        cx<R> term = cmul(dd, diff);
        if (parity) term = mk<R>(-term.re, -term.im);
        acc_re.add(term.re);
        acc_im.add(term.im);
        return;
    }
    constexpr int M = F + 1;  // after the first elimination: 2 copies + F-1 vertices
    int idx[M];
    idx[0] = 0;
    idx[1] = 1;
#pragma unroll
    for (int q = 1; q < F; ++q) idx[q + 1] = 2 + 2 * q + ((path >> q) & 1);
    const int p0 = 2 + (path & 1);
    cx<R> piv = E[(p0 * S + p0) * STRIDE];
    detD = cmul(detD, piv);
    cx<R> ip = crcp(piv);
    cx<R> m[M][M];
    cx<R> prow[M];
#pragma unroll
    for (int y = 0; y < M; ++y) prow[y] = cmul(E[(p0 * S + idx[y]) * STRIDE], ip);
#pragma unroll
    for (int x = 0; x < M; ++x) {
        cx<R> cf = E[(idx[x] * S + p0) * STRIDE];
#pragma unroll
        for (int y = 0; y < M; ++y) {
            if (x < 2 && y < 2 && x != y) continue;  // copy cross terms are never used
            m[x][y] = cfms(E[(idx[x] * S + idx[y]) * STRIDE], cf, prow[y]);
        }
    }
#pragma unroll
    for (int q = 1; q < F - 1; ++q) {
        const int p = q + 1;
        cx<R> pv = m[p][p];
        detD = cmul(detD, pv);
        cx<R> iq = crcp(pv);
#pragma unroll
        for (int y = 0; y < M; ++y)
            if (y < 2 || y > p) m[p][y] = cmul(m[p][y], iq);
#pragma unroll
        for (int x = 0; x < M; ++x) {
            if (!(x < 2 || x > p)) continue;
#pragma unroll
            for (int y = 0; y < M; ++y) {
                if (!(y < 2 || y > p)) continue;
                if (x < 2 && y < 2 && x != y) continue;
                m[x][y] = cfms(m[x][y], m[x][p], m[p][y]);
            }
        }
    }
    cx<R> term;
    if constexpr (F >= 2) {  // the last vertex is eliminated inside the leaf term
        term = leaf_term(m[0][0], m[1][1], m[0][M - 1], m[M - 1][0], m[1][M - 1], m[M - 1][1], m[M - 1][M - 1], detD);
    } else {  // F = 1: the gather step eliminated the only vertex
        term = cmul(cmul(detD, detD), mk<R>(m[0][0].re - m[1][1].re, m[0][0].im - m[1][1].im));
    }
    parity ^= __popc(path) & 1;
    if (parity) term = mk<R>(-term.re, -term.im);
    acc_re.add(term.re);
    acc_im.add(term.im);
}

template <class R, int RF>
__device__ __forceinline__ void flat_dispatch(int Rf, const cx<R> *E, cx<R> detD, int parity, int path, Acc<R> &ar,
                                              Acc<R> &ai) {
    switch (Rf) {  // Rf <= RF
        case 0: flat_phase<R, 0>(E, detD, parity, path, ar, ai); break;
        case 1: flat_phase<R, 1>(E, detD, parity, path, ar, ai); break;
        case 2: flat_phase<R, 2>(E, detD, parity, path, ar, ai); break;
        case 3: if (RF >= 3) flat_phase<R, (RF >= 3 ? 3 : 0)>(E, detD, parity, path, ar, ai); break;
        case 4: if (RF >= 4) flat_phase<R, (RF >= 4 ? 4 : 0)>(E, detD, parity, path, ar, ai); break;
        default: if (RF >= 5) flat_phase<R, (RF >= 5 ? 5 : 0)>(E, detD, parity, path, ar, ai); break;
    }
}

// One cooperative elimination: child(ren) of S x S parent matrices.  Child j
// of the new level comes from parent j >> 1 with Keldysh index a = j & 1 on the
// parent's first remaining vertex (pivot row/column 2 + a).  The new matrices
// are (S-2) x (S-2), all children contiguous in `out`.
template <class R>
__device__ __forceinline__ void expand_level(const cx<R> *__restrict__ in, int S, int nchild, int first_a,
                                             cx<R> *__restrict__ out, const cx<R> *detD_in, cx<R> *detD_out,
                                             cx<R> *__restrict__ wrow, cx<R> *ip_buf, int lane) {
    const int S2 = S - 2;
    // child pivots: reciprocal and running det M_down
    for (int j = lane; j < nchild; j += 32) {
        const int a = nchild == 1 ? first_a : (j & 1);
        const int pj = nchild == 1 ? 0 : (j >> 1);
        const int pr = 2 + a;
        cx<R> piv = in[(size_t)pj * S * S + pr * S + pr];
        ip_buf[j] = crcp(piv);
        detD_out[j] = cmul(detD_in[pj], piv);
    }
    __syncwarp();
    // scaled pivot rows
    for (int q = lane; q < nchild * S2; q += 32) {
        const int j = q / S2, c2 = q - j * S2;
        const int a = nchild == 1 ? first_a : (j & 1);
        const int pj = nchild == 1 ? 0 : (j >> 1);
        const int pr = 2 + a;
        const int c = c2 < 2 ? c2 : c2 + 2;
        wrow[q] = cmul(in[(size_t)pj * S * S + pr * S + c], ip_buf[j]);
    }
    __syncwarp();
    // Only entries that are ever read are built: a choice path takes one copy of every vertex
    // (and one measurement copy per determinant), so the entry joining row r2 to its row's
    // other copy, column r2 ^ 1, is never used (1 / S2 of the updates).  lane -> (child j,
    // row r2, used column cc of W = S2 - 1) stepped by 32 entries without divisions.
    const int W = S2 - 1;
    const int dr = 32 / W, dc = 32 - dr * W;
    int r2 = lane / W, cc = lane - r2 * W, j = 0;
    while (r2 >= S2) { r2 -= S2; ++j; }
    const int total = nchild * S2 * W;
    for (int e = lane; e < total; e += 32) {
        const int c2 = cc < (r2 ^ 1) ? cc : cc + 1;
        const int a = nchild == 1 ? first_a : (j & 1);
        const int pj = nchild == 1 ? 0 : (j >> 1);
        const int pr = 2 + a;
        const int r = r2 < 2 ? r2 : r2 + 2;
        const int c = c2 < 2 ? c2 : c2 + 2;
        const cx<R> *P = in + (size_t)pj * S * S;
        out[((size_t)j * S2 + r2) * S2 + c2] = cfms(P[r * S + c], P[r * S + pr], wrow[j * S2 + c2]);
        cc += dc;
        r2 += dr;
        if (cc >= W) { cc -= W; ++r2; }
        while (r2 >= S2) { r2 -= S2; ++j; }
    }
    __syncwarp();
}

// Single child (a depth-first step, S - 2 <= 32): each lane owns one column of
// the child and a fixed row offset, so the scaled pivot-row entry of its
// column stays in a register and the pivot-column entry of a row is a
// broadcast load.  A step is latency-bound (a few hundred flops per warp), so
// every load of the step is issued before the pivot's reciprocal is formed,
// and the lane mapping needs no division.
//
// Children of 2T = 12, 14 or 16 rows (the deep, frequent steps): lanes 0-15
// take the even rows, lanes 16-31 the odd rows, column c2 = lane & 15.
template <class R, int T>
__device__ __forceinline__ void expand_one_t(const cx<R> *__restrict__ in, int a, cx<R> *__restrict__ out,
                                             const cx<R> *detD_in, cx<R> *detD_out, int lane) {
    constexpr int S2 = 2 * T, S = S2 + 2;
    const int pr = 2 + a;
    const int c2 = lane & 15, rsub = lane >> 4;
    const bool act = c2 < S2;
    const int c = c2 < 2 ? c2 : c2 + 2;
    const cx<R> piv = in[pr * S + pr];
    cx<R> prc = mk<R>(0, 0), ev[T], cv[T];
#pragma unroll
    for (int t = 0; t < T; ++t) ev[t] = cv[t] = mk<R>(0, 0);
    if (act) {
        prc = in[pr * S + c];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int r2 = rsub + 2 * t;
            const int r = r2 < 2 ? r2 : r2 + 2;
            ev[t] = in[r * S + c];
            cv[t] = in[r * S + pr];
        }
    }
    const cx<R> ip = crcp(piv);
    if (lane == 0) *detD_out = cmul(*detD_in, piv);
    if (act) {
        const cx<R> w = cmul(prc, ip);
#pragma unroll
        for (int t = 0; t < T; ++t) out[(rsub + 2 * t) * S2 + c2] = cfms(ev[t], cv[t], w);
    }
    __syncwarp();
}

// Both children (a = 0 into out0, a = 1 into out1) of a parent of 2T + 2 rows:
// the last depth-first step, whose two children are consecutive leaves.  The
// parent entries are loaded once for both, and both pivots' latencies overlap.
template <class R, int T>
__device__ __forceinline__ void expand_both_t(const cx<R> *__restrict__ in, cx<R> *__restrict__ out0,
                                              cx<R> *__restrict__ out1, const cx<R> *detD_in, cx<R> *detD_out0,
                                              cx<R> *detD_out1, int lane) {
    constexpr int S2 = 2 * T, S = S2 + 2;
    const int c2 = lane & 15, rsub = lane >> 4;
    const bool act = c2 < S2;
    const int c = c2 < 2 ? c2 : c2 + 2;
    const cx<R> piv0 = in[2 * S + 2], piv1 = in[3 * S + 3];
    cx<R> prc0 = mk<R>(0, 0), prc1 = mk<R>(0, 0), ev[T], cv0[T], cv1[T];
#pragma unroll
    for (int t = 0; t < T; ++t) ev[t] = cv0[t] = cv1[t] = mk<R>(0, 0);
    if (act) {
        prc0 = in[2 * S + c];
        prc1 = in[3 * S + c];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int r2 = rsub + 2 * t;
            const int r = r2 < 2 ? r2 : r2 + 2;
            ev[t] = in[r * S + c];
            cv0[t] = in[r * S + 2];
            cv1[t] = in[r * S + 3];
        }
    }
    const cx<R> ip0 = crcp(piv0), ip1 = crcp(piv1);
    if (lane == 0) *detD_out0 = cmul(*detD_in, piv0);
    if (lane == 1) *detD_out1 = cmul(*detD_in, piv1);
    if (act) {
        const cx<R> w0 = cmul(prc0, ip0), w1 = cmul(prc1, ip1);
#pragma unroll
        for (int t = 0; t < T; ++t) {
            out0[(rsub + 2 * t) * S2 + c2] = cfms(ev[t], cv0[t], w0);
            out1[(rsub + 2 * t) * S2 + c2] = cfms(ev[t], cv1[t], w1);
        }
    }
    __syncwarp();
}

// Wider children (S - 2 = 18 .. 32 rows, the rare top steps): lane = column,
// rows in batches (eight in FP32, four in FP64) with the batch's loads issued first.
template <class R>
__device__ __forceinline__ void expand_one_wide(const cx<R> *__restrict__ in, int S, int a, cx<R> *__restrict__ out,
                                                const cx<R> *detD_in, cx<R> *detD_out, int lane) {
    constexpr int NB = sizeof(R) == 4 ? 8 : 4;  // rows per batch (FP64: register budget)
    const int S2 = S - 2;
    const int pr = 2 + a;
    const cx<R> piv = in[pr * S + pr];
    const cx<R> ip = crcp(piv);
    if (lane == 0) *detD_out = cmul(*detD_in, piv);
    if (lane < S2) {
        const int c = lane < 2 ? lane : lane + 2;
        const cx<R> w = cmul(in[pr * S + c], ip);
        for (int r0 = 0; r0 < S2; r0 += NB) {
            cx<R> ev[NB], cv[NB];
#pragma unroll
            for (int t = 0; t < NB; ++t) {
                const int r2 = r0 + t < S2 ? r0 + t : S2 - 1;  // a clamped duplicate of the last row
                const int r = r2 < 2 ? r2 : r2 + 2;
                ev[t] = in[r * S + c];
                cv[t] = in[r * S + pr];
            }
#pragma unroll
            for (int t = 0; t < NB; ++t)
                if (r0 + t < S2) out[(r0 + t) * S2 + lane] = cfms(ev[t], cv[t], w);
        }
    }
    __syncwarp();
}

template <class R>
__device__ __forceinline__ void expand_one(const cx<R> *__restrict__ in, int S, int a, cx<R> *__restrict__ out,
                                           const cx<R> *detD_in, cx<R> *detD_out, int lane) {
    switch (S - 2) {
        case 12: expand_one_t<R, 6>(in, a, out, detD_in, detD_out, lane); break;
        case 14: expand_one_t<R, 7>(in, a, out, detD_in, detD_out, lane); break;
        case 16: expand_one_t<R, 8>(in, a, out, detD_in, detD_out, lane); break;
        default: expand_one_wide<R>(in, S, a, out, detD_in, detD_out, lane); break;
    }
}

// Float-float or double-double style butterfly of the lane accumulators:
// combines (s, c) pairs with two-sum in R, then returns s + c in double.
template <class R>
__device__ __forceinline__ void two_sum_r(R a, R b, R &s, R &e) {
    s = a + b;
    R z = s - a;
    e = (a - (s - z)) + (b - z);
}

template <class R>
__device__ __forceinline__ double warp_total(Acc<R> acc) {
    R s = acc.s, c = acc.c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        R s2 = __shfl_xor_sync(FULL, s, o);
        R c2 = __shfl_xor_sync(FULL, c, o);
        R t, e;
        int lo = ((threadIdx.x & 31) & o) == 0;
        if (lo) two_sum_r<R>(s, s2, t, e); else two_sum_r<R>(s2, s, t, e);
        s = t;
        c = lo ? (c + c2) + e : (c2 + c) + e;
    }
    return (double)s + (double)c;
}

// Keldysh sum for one point whose times are in u[0..n] (u_0 = t).
// Returns sum_{a_2..a_n} (-1)^{a_2+..+a_n} det M_down^2 (S00(0) - S00(1)),
// i.e. sum_a (-1)^{|a|} det M_up det M_down (without the i^n factor).
// The depth-first walk covers the subtree `sub` of 2^split: the first `split`
// tree levels follow the bits of sub (split <= levels); split = 0: whole tree.
template <class R, int RFMAX, bool GS>
__device__ cx<double> keldysh_sum(const WarpSmem<R> &ws, const double *u, int n, int n_max, cx<R> d, cx<R> dv,
                                  const typename TabT<R>::V *tab, const typename TabT<R>::V *col, double inv_h,
                                  double s0, int L, int RF, int lane, int sub = 0, int split = 0) {
    // 1. pair interpolation, 0 <= j < k <= n
    const int npairs = n * (n + 1) / 2;
    for (int p = lane; p < npairs; p += 32) {
        int k = (int)((1.0f + sqrtf(8.0f * p + 1.0f)) * 0.5f);
        while (k * (k - 1) / 2 > p) --k;
        while ((k + 1) * k / 2 <= p) ++k;
        int j = p - k * (k - 1) / 2;
        cx<R> gl, gg;
        interp_pair<R>(tab, inv_h, s0, L, u[j] - u[k], gl, gg);
        const int ok = p - j + k - 1;  // vertex k's block: (k-1)(k+2)/2
        ws.P[ok + j] = gg;
        ws.Rr[ok + j] = gl;
        if (j == 0) {  // measurement column of vertex k: g^<(u_k - t), g^>(u_k - t) for the charge
            cx<R> c0 = nconj(gl), c1 = nconj(gg);
            if (col) interp_col<R>(col, inv_h, s0, L, u[k] - u[0], c0, c1);
            ws.Rr[ok + k] = c0;
            ws.P[ok + k] = c1;
        }
    }
    __syncwarp();
    // 2. level 0: vertex 1 eliminated (both a_1 kept in the two measurement copies).
    // Built by 2x2 blocks: block row/column 0 = the measurement copies, block
    // q >= 1 = vertex q+1 with its two Keldysh indices.  Within a block the
    // entry is base(ai, aj) - left(ai) right(aj), with left = M(., vertex 1),
    // right = M(vertex 1, .) / d.
    const int R0 = n - 1;
    const int S0 = 2 * R0 + 2;
    // tree levels: offsets in shared memory, or (split stack) in device memory for the wide ones.
    // Level l holds S_l^2 = 4 (R0 + 1 - l)^2 entries, so the offset of level l within its part is
    // 4 (Q(R0 + 1 - l0) - Q(R0 + 1 - l)), Q(x) = x(x+1)(2x+1)/6, l0 = the part's first level.
    const int levels = R0 > kTreeLeaf ? R0 - kTreeLeaf : 0;
    int lg = 0;  // levels [0, lg) in device memory: S_l > gs_level
    if (GS) {
        lg = R0 + 1 - ws.gs_level / 2;
        lg = lg < 0 ? 0 : (lg > levels + 1 ? levels + 1 : lg);
    }
    auto sq_sum = [](int x) { return x * (x + 1) * (2 * x + 1) / 6; };
    const int qtop = sq_sum(R0 + 1), qsplit = sq_sum(R0 + 1 - lg);
    auto level = [&](int l) -> cx<R> * {
        const int ql = sq_sum(R0 + 1 - l);
        return (GS && l < lg) ? ws.gstack + 4 * (qtop - ql) : ws.stack + 4 * (qsplit - ql);
    };
    // the leaf and its parent are always in shared memory (gs_level >= 14)
    auto level_smem = [&](int l) -> cx<R> * { return ws.stack + 4 * (qsplit - sq_sum(R0 + 1 - l)); };
    const cx<R> id = crcp(dv);  // pivot of vertex 1
    {
        // Block row b's left factors M(., vertex 1) and block column b's right factors
        // M(vertex 1, .) / d, once per block index: b = 0 the measurement copies (row entries
        // r_1(a), column entries c_1(a) / d), b >= 1 vertex b + 1 (pair (1, b + 1)).
        if (lane < n) {
            cx<R> l0, l1, r0, r1;
            if (lane == 0) {
                l0 = ws.P[0];  // pair (0, 1)
                l1 = ws.Rr[0];
                r0 = cmul(ws.Rr[1], id);  // column entries of vertex 1
                r1 = cmul(ws.P[1], id);
            } else {
                const int t = (lane * (lane + 3)) >> 1;  // vertex lane + 1's block
                l0 = nconj(ws.Rr[t + 1]);
                l1 = nconj(ws.P[t + 1]);
                r0 = cmul(ws.P[t + 1], id);
                r1 = cmul(ws.Rr[t + 1], id);
            }
            ws.lr[4 * lane] = l0;
            ws.lr[4 * lane + 1] = l1;
            ws.lr[4 * lane + 2] = r0;
            ws.lr[4 * lane + 3] = r1;
        }
        __syncwarp();
        // lane -> block (bx, by), stepped by 32 blocks without divisions; i = bx + 1 and
        // j = by + 1 are the vertices, ti and tj the offsets of their packed blocks.  Within a
        // block the entry is base(ai, aj) - left(ai) right(aj); base is the pair value of the
        // later vertex's index: above the diagonal (row 0: the measurement row) it follows aj,
        // below it (column 0: the measurement column, stored as is) it follows ai.
        const int sq = 32 / n, sr = 32 - sq * n;
        int bx = lane / n, by = lane - bx * n;
        for (int bid = lane; bid < n * n; bid += 32) {
            const int i = bx + 1, j = by + 1;
            const int ti = (int)((unsigned)((i - 1) * (i + 2)) >> 1), tj = (int)((unsigned)((j - 1) * (j + 2)) >> 1);
            const bool up = bx < by, diag = bx == by;
            const int idx = up ? tj + (bx ? i : 0) : ti + (by ? j : i);
            const cx<R> vP = ws.P[idx], vR = ws.Rr[idx];
            const cx<R> left0 = ws.lr[4 * bx], left1 = ws.lr[4 * bx + 1];
            const cx<R> right0 = ws.lr[4 * by + 2], right1 = ws.lr[4 * by + 3];
            const R sg = (!up && by) ? R(-1) : R(1);  // lower entries of vertex pairs: -conj
            const cx<R> lo0 = mk<R>(sg * vR.re, vR.im), lo1 = mk<R>(sg * vP.re, vP.im);
            const cx<R> dd = bx == 0 ? d : dv;
            const cx<R> b00 = diag ? dd : (up ? vP : lo0), b01 = diag ? dd : (up ? vR : lo0);
            const cx<R> b10 = diag ? dd : (up ? vP : lo1), b11 = diag ? dd : (up ? vR : lo1);
            cx<R> *o = level(0) + (2 * bx) * S0 + 2 * by;
            o[0] = cfms(b00, left0, right0);
            o[1] = cfms(b01, left0, right1);
            o[S0] = cfms(b10, left1, right0);
            o[S0 + 1] = cfms(b11, left1, right1);
            by += sr;
            bx += sq;
            if (by >= n) {
                by -= n;
                ++bx;
            }
        }
    }
    if (lane == 0) ws.detD[0] = dv;
    __syncwarp();
    // 3. depth-first tree over a_2 .. a_{levels+1}
    const int Rleaf = R0 - levels;
    const int B = Rleaf > RF ? Rleaf - RF : 0;
    const int Rf = Rleaf - B;
    Acc<R> ar, ai;
    ar.init();
    ai.init();
    const int nleaf = 1 << (levels - split);
    const int node = lane >> Rf;
    const int path = lane & ((1 << Rf) - 1);
    const bool active = lane < (1 << Rleaf);
    // With two or more leaves in the walk, leaves come in sibling pairs: the last depth-first step
    // builds both (the second into ws.sib) and the pair is resolved one after the other.
    const int twin = twin_leaves<R>() && levels - split >= 1 ? 1 : 0;
    for (int bl = 0; bl < nleaf; bl += 1 + twin) {
        const int b = (sub << (levels - split)) | bl;  // tree path: the subtree's fixed prefix, then bl
        int from = (bl == 0) ? 0 : levels - (__ffs(b) - 1) - 1;
        for (int l = from; l < levels - twin; ++l) {
            const int a = (b >> (levels - 1 - l)) & 1;
            const int S = 2 * (R0 - l) + 2;
            if (S - 2 <= 32)
                expand_one<R>(level(l), S, a, level(l + 1), ws.detD + l, ws.detD + l + 1, lane);
            else
                expand_level<R>(level(l), S, 1, a, level(l + 1), ws.detD + l, ws.detD + l + 1, ws.wrow, ws.bip,
                                lane);
        }
        if (twin)  // the leaves' parent has 2 kTreeLeaf + 4 rows
            expand_both_t<R, kTreeLeaf + 1>(level_smem(levels - 1), level_smem(levels), ws.sib,
                                            ws.detD + levels - 1, ws.detD + levels, ws.detD + levels + 1, lane);
#pragma unroll 1
        for (int h = 0; h <= twin; ++h) {
            const int tparity = __popc(b + h) & 1;
            // 4. breadth-first expansion of B levels below the tree leaf
            const cx<R> *E = h ? ws.sib : level_smem(levels);
            int S = 2 * Rleaf + 2;
            const cx<R> *ndet = ws.detD + levels + h;
            cx<R> *dbuf = ws.bdet;
            size_t bo = 0;
            for (int lb = 0; lb < B; ++lb) {
                const int nparent = 1 << lb;
                cx<R> *out = ws.bfs + bo;
                expand_level<R>(E, S, 2 * nparent, 0, out, ndet, dbuf, ws.wrow, ws.bip, lane);
                bo += (size_t)(2 * nparent) * (S - 2) * (S - 2);
                E = out;
                S -= 2;
                ndet = dbuf;
                dbuf = (dbuf == ws.bdet) ? ws.bdet + 32 : ws.bdet;
            }
            // 5. per-lane flat phase on the last Rf vertices
            if (active) {
                const cx<R> *En = E + (size_t)node * S * S;
                const int parity = tparity ^ (__popc(node) & 1);
                flat_dispatch<R, RFMAX>(Rf, En, ndet[B > 0 ? node : 0], parity, path, ar, ai);
            }
            __syncwarp();
        }
    }
    return mk<double>(warp_total<R>(ar), warp_total<R>(ai));
}

// One point per lane (small orders), registers only: the lane interpolates
// its own pairs, and for every choice path of vertices 2..N builds the path's
// (N+1) x (N+1) matrix -- rows/columns {copy a_1 = 0, copy a_1 = 1, vertices
// 2..N with their chosen Keldysh index}, vertex 1 already eliminated -- from
// the pair values, then eliminates vertices 2..N.  All loops are unrolled, so
// every array index is static.
template <class R>
__device__ __forceinline__ cx<R> sel(int bit, cx<R> one, cx<R> zero) {
    return mk<R>(bit ? one.re : zero.re, bit ? one.im : zero.im);
}

template <class R, int N>
__device__ __forceinline__ cx<double> lane_keldysh_sum(const double *u, cx<R> d, cx<R> dv,
                                                       const typename TabT<R>::V *tab,
                                                       const typename TabT<R>::V *col, double inv_h, double s0,
                                                       int L) {
    constexpr int M = N + 1;
    cx<R> P[N + 1][N + 1], Rr[N + 1][N + 1];
    double uu[N + 1];
#pragma unroll
    for (int m = 0; m <= N; ++m) uu[m] = u[m];
#pragma unroll
    for (int k = 1; k <= N; ++k)
#pragma unroll
        for (int j = 0; j < k; ++j) interp_pair<R>(tab, inv_h, s0, L, uu[j] - uu[k], Rr[j][k], P[j][k]);
    // measurement column (a_k = 0, 1): g^<, g^> at u_k - t for the charge, dot-lead tables for the current
    cx<R> C0[N + 1], C1[N + 1];
#pragma unroll
    for (int k = 1; k <= N; ++k) {
        C0[k] = nconj(Rr[0][k]);
        C1[k] = nconj(P[0][k]);
        if (col) interp_col<R>(col, inv_h, s0, L, uu[k] - uu[0], C0[k], C1[k]);
    }
    const cx<R> id = crcp(dv);
    // row/column factors of vertex 1 (eliminated first, pivot dv)
    const cx<R> r1[2] = {P[0][1], Rr[0][1]};
    const cx<R> c1d[2] = {cmul(C0[1], id), cmul(C1[1], id)};
    Acc<R> ar, ai;
    ar.init();
    ai.init();
#pragma unroll
    for (int path = 0; path < (1 << (N - 1)); ++path) {
        // position x: 0, 1 = copies; x >= 2 = vertex v = x with Keldysh index a_v = bit (x-2) of path
        cx<R> left[M], right[M], m[M][M];
#pragma unroll
        for (int x = 0; x < M; ++x) {
            if (x < 2) {
                left[x] = r1[x];
                right[x] = c1d[x];
            } else {
                const int a = (path >> (x - 2)) & 1;
                left[x] = nconj(sel<R>(a, P[1][x], Rr[1][x]));
                right[x] = cmul(sel<R>(a, Rr[1][x], P[1][x]), id);
            }
        }
#pragma unroll
        for (int x = 0; x < M; ++x)
#pragma unroll
            for (int y = 0; y < M; ++y) {
                if (x < 2 && y < 2 && x != y) continue;  // copy cross terms are never used
                cx<R> base;
                if (x == y) {
                    base = x < 2 ? d : dv;
                } else if (x < 2) {  // measurement row, vertex y
                    base = sel<R>((path >> (y - 2)) & 1, Rr[0][y], P[0][y]);
                } else if (y < 2) {  // vertex x, measurement column
                    base = sel<R>((path >> (x - 2)) & 1, C1[x], C0[x]);
                } else if (x < y) {  // upper: index of the column vertex
                    base = sel<R>((path >> (y - 2)) & 1, Rr[x][y], P[x][y]);
                } else {  // lower: index of the row vertex
                    base = nconj(sel<R>((path >> (x - 2)) & 1, P[y][x], Rr[y][x]));
                }
                m[x][y] = cfms(base, left[x], right[y]);
            }
        cx<R> detD = dv;
#pragma unroll
        for (int p = 2; p < M - 1; ++p) {
            cx<R> pv = m[p][p];
            detD = cmul(detD, pv);
            cx<R> iq = crcp(pv);
#pragma unroll
            for (int y = 0; y < M; ++y)
                if (y < 2 || y > p) m[p][y] = cmul(m[p][y], iq);
#pragma unroll
            for (int x = 0; x < M; ++x) {
                if (!(x < 2 || x > p)) continue;
#pragma unroll
                for (int y = 0; y < M; ++y) {
                    if (!(y < 2 || y > p)) continue;
                    if (x < 2 && y < 2 && x != y) continue;
                    m[x][y] = cfms(m[x][y], m[x][p], m[p][y]);
                }
            }
        }
        cx<R> term;
        if constexpr (M > 2) {
            term = leaf_term(m[0][0], m[1][1], m[0][M - 1], m[M - 1][0], m[1][M - 1], m[M - 1][1], m[M - 1][M - 1],
                             detD);
        } else {  // order 1: vertex 1 was eliminated when the matrix was built
            term = cmul(cmul(detD, detD), mk<R>(m[0][0].re - m[1][1].re, m[0][0].im - m[1][1].im));
        }
        if (__popc(path) & 1) term = mk<R>(-term.re, -term.im);
        ar.add(term.re);
        ai.add(term.im);
    }
    return mk<double>((double)ar.s + (double)ar.c, (double)ai.s + (double)ai.c);
}

// i^n * z
__device__ __forceinline__ cx<double> times_i_pow(cx<double> z, int n) {
    switch (n & 3) {
        case 0: return z;
        case 1: return mk<double>(-z.im, z.re);
        case 2: return mk<double>(-z.re, -z.im);
        default: return mk<double>(z.im, -z.re);
    }
}

template <class R>
__device__ __forceinline__ const typename TabT<R>::V *item_table(const ItemDev &it);
template <>
__device__ __forceinline__ const dbl4 *item_table<double>(const ItemDev &it) { return it.table; }
template <>
__device__ __forceinline__ const float4 *item_table<float>(const ItemDev &it) { return it.table32; }

// dot-lead column table of the current observable, or null (charge)
template <class R>
__device__ __forceinline__ const typename TabT<R>::V *item_col(const ItemDev &it);
template <>
__device__ __forceinline__ const dbl4 *item_col<double>(const ItemDev &it) { return it.col; }
template <>
__device__ __forceinline__ const float4 *item_col<float>(const ItemDev &it) { return it.col32; }

// Gap v = -tau log(1 - x) of the exponential warp, x = y 2^-32.  FP64 for the
// FP64 path; FP32 for the mixed path (log1p for x < 1/2, log of the exactly
// formed 1 - x above), with the times accumulated in FP64 either way.
__device__ __forceinline__ void warp_gap(double, uint32_t y, double tau, double &v, double &omx) {
    double x = (double)y * 0x1p-32;
    v = -tau * log1p(-x);
    omx = 1.0 - x;
}
__device__ __forceinline__ void warp_gap(float, uint32_t y, double tau, double &v, double &omx) {
    float l;
    if (y < 0x80000000u) {
        l = log1pf(-(float)y * 0x1p-32f);
    } else {
        l = logf((float)(0x100000000ull - (unsigned long long)y) * 0x1p-32f);
    }
    v = (double)(-(float)tau * l);
    omx = (double)((float)(0x100000000ull - (unsigned long long)y) * 0x1p-32f);
}

// Learned (projection) warp, paper App. F "learning h from the integrand": the
// density of w_m in [0, 1) is piecewise constant on `cells` equal cells with
// CDF values cdf[0] = 0 .. cdf[cells] = 1; x -> w inverts the CDF (bisection
// for the cell, linear inside it) and dw/dx = 1 / (cells (cdf[k+1] - cdf[k])).
__device__ __forceinline__ double proj_map(const double *cdf, int cells, double x, double &jac) {
    int lo = 0, hi = cells;  // cdf[lo] <= x < cdf[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(cdf + mid) <= x) lo = mid; else hi = mid;
    }
    const double c0 = __ldg(cdf + lo), dc = __ldg(cdf + lo + 1) - c0;
    jac = 1.0 / ((double)cells * dc);
    return ((double)lo + (x - c0) / dc) / (double)cells;
}

// Gap and weight factors of dimension m for the plain or the learned warp.
template <class R>
__device__ __forceinline__ void point_gap(const ItemDev &I, int m, uint32_t y, double &v, double &omx,
                                          double &jac) {
    if (I.proj) {
        const double x = (double)y * 0x1p-32;
        const double w = proj_map(I.proj + (size_t)m * (I.proj_cells + 1), I.proj_cells, x, jac);
        v = -I.tau * log1p(-w);
        omx = 1.0 - w;
    } else {
        jac = 1.0;
        warp_gap(R(0), y, I.tau, v, omx);
    }
}

// ----------------------------------------------------------------------------
// Hot-path kernel: persistent warps pull chunks of 32 Sobol' indices.
// ----------------------------------------------------------------------------
template <class R, int RFMAX, bool GS>
__global__ void detsum_kernel(const ItemDev *__restrict__ items, int n_items, long long total_chunks,
                              unsigned long long *counter, int n_max, int rf_min, cx<R> *gstack) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    cx<R> *gst = nullptr;
    if (GS) gst = gstack + ((size_t)blockIdx.x * (blockDim.x >> 5) + warp) * gstack_entries<R>(n_max, rf_min);
    WarpSmem<R> ws = carve<R>(smem_raw + (size_t)warp * warp_smem_bytes<R>(n_max, rf_min, GS), n_max, rf_min, gst);
    const int NU = n_max + 1;
    while (true) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(counter, 1ull);
        c = __shfl_sync(FULL, c, 0);
        if ((long long)c >= total_chunks) break;
        int it = 0;
        while (it + 1 < n_items && items[it + 1].chunk_begin <= (long long)c) ++it;
        const ItemDev &I = items[it];
        const int n = I.order;
        const long long local = (long long)c - I.chunk_begin;
        const int k = (int)(local / I.chunks_per_shift);
        const long long unit = local - (long long)k * I.chunks_per_shift;
        const long long blk = unit >> (I.pbits + I.split);      // chunk of 32 points
        const int sub = (int)(unit & ((1ll << I.split) - 1));   // subtree of each point's Keldysh tree
        const int grp = (int)(unit >> I.split) & ((1 << I.pbits) - 1);  // the chunk's lanes [grp * g, grp * g + g)
        const long long idx = blk * kChunk + lane;
        const bool valid = idx < I.n_points && (lane >> (5 - I.pbits)) == grp;
        // point generation and warp (Sobol' integers are exact)
        bool inside = false;
        double w = 0.0;
        if (valid) {
            const uint64_t i = (uint64_t)(I.first_index + idx);
            double uprev = I.t, prod = 1.0;
            ws.upt[lane * NU] = I.t;
            double jt = 1.0;
            for (int m = 0; m < n; ++m) {
                uint32_t y = point_word(I.lat_z, I.lat_m, m, i, I.shifts[k * n + m]);
                double v, omx, jac;
                point_gap<R>(I, m, y, v, omx, jac);
                uprev = uprev - v;
                ws.upt[lane * NU + 1 + m] = uprev;
                prod *= omx;
                jt *= jac;
            }
            inside = uprev > 0.0;
            double tn = 1.0;
            for (int m = 0; m < n; ++m) tn *= I.tau;
            w = tn / prod * jt;
        }
        unsigned mask = __ballot_sync(FULL, inside);
        __syncwarp();
        cx<double> myval = mk<double>(0.0, 0.0);
        const cx<R> d = mk<R>((R)I.g0_re, (R)I.g0_im);
        const cx<R> dv = mk<R>((R)I.g0_re, (R)(I.g0_im - I.alpha));
        const typename TabT<R>::V *tab = item_table<R>(I);
        const double inv_h = 1.0 / I.h;
        const double s0 = I.T * inv_h;
        unsigned mm = mask;
        while (mm) {
            const int src = __ffs(mm) - 1;
            mm &= mm - 1;
            // every warp-per-point item of a launch shares the launch's flat depth
            cx<double> s = keldysh_sum<R, RFMAX, GS>(ws, ws.upt + src * NU, n, n_max, d, dv, tab, item_col<R>(I), inv_h,
                                                     s0, I.L, RFMAX, lane, sub, I.split);
            if (lane == src) {
                cx<double> cval = times_i_pow(s, n);
                myval = mk<double>(w * cval.re, w * cval.im);
            }
            __syncwarp();
        }
        double sr = myval.re, cr = 0.0, si = myval.im, ci = 0.0;
        warp_reduce_pair(sr, cr);
        warp_reduce_pair(si, ci);
        if (lane == 0) {
            double *pp = I.partials + 4 * (size_t)local;
            pp[0] = sr;
            pp[1] = si;
            pp[2] = cr;
            pp[3] = ci;
            I.inside[local] = sub == 0 ? __popc(mask) : 0u;  // a point counts once, in subtree 0
        }
    }
}

// ----------------------------------------------------------------------------
// One-point-per-lane kernel for small orders (items whose tuning asks for it):
// persistent warps pull chunks of 32 Sobol' indices, every lane generates,
// warps and sums its own point entirely in registers; no shared memory.
// ----------------------------------------------------------------------------
template <class R, int N>
__device__ __forceinline__ cx<double> lane_point(const ItemDev &I, int k, uint64_t i, bool &inside) {
    double u[N + 1];
    double uprev = I.t, prod = 1.0, tn = 1.0, jt = 1.0;
    u[0] = I.t;
#pragma unroll
    for (int m = 0; m < N; ++m) {
        uint32_t y = point_word(I.lat_z, I.lat_m, m, i, I.shifts[k * N + m]);
        double v, omx, jac;
        point_gap<R>(I, m, y, v, omx, jac);
        uprev = uprev - v;
        u[m + 1] = uprev;
        prod *= omx;
        tn *= I.tau;
        jt *= jac;
    }
    inside = uprev > 0.0;
    if (!inside) return mk<double>(0.0, 0.0);
    const double w = tn / prod * jt;
    const double inv_h = 1.0 / I.h;
    const cx<R> d = mk<R>((R)I.g0_re, (R)I.g0_im);
    const cx<R> dv = mk<R>((R)I.g0_re, (R)(I.g0_im - I.alpha));
    cx<double> s = lane_keldysh_sum<R, N>(u, d, dv, item_table<R>(I), item_col<R>(I), inv_h, I.T * inv_h, I.L);
    cx<double> c = times_i_pow(s, N);
    return mk<double>(w * c.re, w * c.im);
}

template <class R>
__global__ void __launch_bounds__(128) lane_kernel(const ItemDev *__restrict__ items, int n_items,
                                                   long long total_chunks, unsigned long long *counter) {
    const int lane = threadIdx.x & 31;
    while (true) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(counter, 1ull);
        c = __shfl_sync(FULL, c, 0);
        if ((long long)c >= total_chunks) break;
        int it = 0;
        while (it + 1 < n_items && items[it + 1].chunk_begin <= (long long)c) ++it;
        const ItemDev &I = items[it];
        const long long local = (long long)c - I.chunk_begin;
        const int k = (int)(local / I.chunks_per_shift);
        const long long blk = local - (long long)k * I.chunks_per_shift;
        const long long idx = blk * kChunk + lane;
        bool inside = false;
        cx<double> v = mk<double>(0.0, 0.0);
        if (idx < I.n_points) {
            const uint64_t i = (uint64_t)(I.first_index + idx);
            switch (I.order) {
                case 1: v = lane_point<R, 1>(I, k, i, inside); break;
                case 2: v = lane_point<R, 2>(I, k, i, inside); break;
                case 3: v = lane_point<R, 3>(I, k, i, inside); break;
                default: v = lane_point<R, 4>(I, k, i, inside); break;
            }
        }
        const unsigned mask = __ballot_sync(FULL, inside);
        double sr = v.re, cr = 0.0, si = v.im, ci = 0.0;
        warp_reduce_pair(sr, cr);
        warp_reduce_pair(si, ci);
        if (lane == 0) {
            double *pp = I.partials + 4 * (size_t)local;
            pp[0] = sr;
            pp[1] = si;
            pp[2] = cr;
            pp[3] = ci;
            I.inside[local] = __popc(mask);
        }
    }
}

// Per shifted sequence: compensated sum of its chunk partials in a fixed order.
// out[2*g], out[2*g+1] = sum_i w_i c_n(u_i) (complex, not divided by N);
// counts[g] = in-domain points.  One block of 256 threads per sequence.
__global__ void reduce_kernel(const ItemDev *__restrict__ items, int n_items, double *out,
                              unsigned long long *counts) {
    __shared__ double s_re[256], c_re[256], s_im[256], c_im[256];
    __shared__ unsigned long long cnt[256];
    int g = blockIdx.x;
    int it = 0, base = 0;
    while (it < n_items && g >= base + items[it].n_shifts) {
        base += items[it].n_shifts;
        ++it;
    }
    if (it >= n_items) return;
    const ItemDev &I = items[it];
    const int k = g - base;
    const double *pp = I.partials + 4 * (size_t)k * I.chunks_per_shift;
    const unsigned int *ins = I.inside + (size_t)k * I.chunks_per_shift;
    Acc<double> ar, ai;
    ar.init();
    ai.init();
    unsigned long long cn = 0;
    for (int q = threadIdx.x; q < I.chunks_per_shift; q += blockDim.x) {
        ar.add(pp[4 * q]);
        ar.add(pp[4 * q + 2]);
        ai.add(pp[4 * q + 1]);
        ai.add(pp[4 * q + 3]);
        cn += ins[q];
    }
    s_re[threadIdx.x] = ar.s;
    c_re[threadIdx.x] = ar.c;
    s_im[threadIdx.x] = ai.s;
    c_im[threadIdx.x] = ai.c;
    cnt[threadIdx.x] = cn;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            double t, e;
            two_sum(s_re[threadIdx.x], s_re[threadIdx.x + o], t, e);
            s_re[threadIdx.x] = t;
            c_re[threadIdx.x] = c_re[threadIdx.x] + c_re[threadIdx.x + o] + e;
            two_sum(s_im[threadIdx.x], s_im[threadIdx.x + o], t, e);
            s_im[threadIdx.x] = t;
            c_im[threadIdx.x] = c_im[threadIdx.x] + c_im[threadIdx.x + o] + e;
            cnt[threadIdx.x] += cnt[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * g] = s_re[0] + c_re[0];
        out[2 * g + 1] = s_im[0] + c_im[0];
        counts[g] = cnt[0];
    }
}

// ----------------------------------------------------------------------------
// Check kernels
// ----------------------------------------------------------------------------
__global__ void sobol_kernel(int order, uint64_t first, uint64_t count, const uint32_t *shift, uint32_t *out,
                             const uint32_t *lat_z, int lat_m) {
    uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (q >= count) return;
    for (int m = 0; m < order; ++m)
        out[q * order + m] = point_word(lat_z, lat_m, m, first + q, shift ? shift[m] : 0u);
}

__global__ void warp_kernel(int order, uint64_t first, uint64_t count, const uint32_t *shift, double t, double tau,
                            double *u, double *w, int32_t *inside, const uint32_t *lat_z, int lat_m) {
    uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (q >= count) return;
    double uprev = t, prod = 1.0;
    for (int m = 0; m < order; ++m) {
        uint32_t y = point_word(lat_z, lat_m, m, first + q, shift ? shift[m] : 0u);
        double x = (double)y * 0x1p-32;
        uprev = uprev - (-tau * log1p(-x));
        u[q * order + m] = uprev;
        prod *= (1.0 - x);
    }
    w[q] = pow(tau, (double)order) / prod;
    inside[q] = uprev > 0.0;
}

// One warp per caller point.
// One warp per caller point, grid-stride over the points.
template <class R, int RF, bool GS>
__global__ void integrand_kernel(ItemDev I, uint64_t count, const double *u, double *out, int n_max, cx<R> *gstack) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint64_t wid = blockIdx.x * (uint64_t)(blockDim.x >> 5) + warp;
    cx<R> *gst = nullptr;
    if (GS) gst = gstack + wid * gstack_entries<R>(n_max, RF);
    WarpSmem<R> ws = carve<R>(smem_raw + (size_t)warp * warp_smem_bytes<R>(n_max, RF, GS), n_max, RF, gst);
    const int n = I.order;
    const cx<R> d = mk<R>((R)I.g0_re, (R)I.g0_im);
    const cx<R> dv = mk<R>((R)I.g0_re, (R)(I.g0_im - I.alpha));
    const double inv_h = 1.0 / I.h;
    for (uint64_t q = wid; q < count; q += (uint64_t)gridDim.x * (blockDim.x >> 5)) {
        if (lane <= n) ws.upt[lane] = lane == 0 ? I.t : u[q * n + lane - 1];
        __syncwarp();
        cx<double> s = keldysh_sum<R, RF, GS>(ws, ws.upt, n, n_max, d, dv, item_table<R>(I), item_col<R>(I), inv_h,
                                          I.T * inv_h, I.L, RF, lane);
        if (lane == 0) {
            cx<double> cval = times_i_pow(s, n);
            out[2 * q] = cval.re;
            out[2 * q + 1] = cval.im;
        }
        __syncwarp();
    }
}

// ----------------------------------------------------------------------------
// Green-function table: contour-deformed Fourier integral (App. E).
//   g^<(tau) = (i/2pi) Int_{-inf}^{0} e^{-i w tau} A(w) dw,   A(w) = 2 Gamma / ((w-eps)^2 + Gamma^2)
// For tau > 0 the half line (-inf, w_m] is replaced by the vertical ray
// w = w_m - i y, y in [0, inf) (no pole crossed for w_m < eps), on which the
// exponential decays without oscillating; the rest [w_m, 0] stays on the real
// axis.  Ray: exp-sinh rule y = exp(pi/2 sinh s); segment: composite 16-point
// Gauss-Legendre.  g^> = g^< - i exp(-i eps tau - Gamma tau) (sum rule).
// One warp per node with tau > 0; the node at -h/2 is the mirror image.
// ----------------------------------------------------------------------------
__device__ __forceinline__ cx<double> lorentz(cx<double> z, double eps, double gam) {
    // 2 gam / ((z - eps)^2 + gam^2)
    cx<double> q = mk<double>(z.re - eps, z.im);
    cx<double> den = mk<double>(q.re * q.re - q.im * q.im + gam * gam, 2.0 * q.re * q.im);
    cx<double> r = crcp(den);
    return mk<double>(2.0 * gam * r.re, 2.0 * gam * r.im);
}

__global__ void gf_table_kernel(dbl4 *tab, float4 *tab32, int L, double T, double h, double eps, double gam,
                                int panels) {
    const int lane = threadIdx.x & 31;
    const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // 0 .. L/2-1 -> node L/2 + q
    if (q >= L / 2) return;
    const int node = L / 2 + q;
    const double tau = -T + (double)node * h;
    const double wm = fmin(eps, 0.0) - 3.0 * gam;
    double ar = 0.0, ai = 0.0;  // integral of e^{-i w tau} A(w) dw along the contour
    // ray: Int = i Int_0^inf e^{-i wm tau} e^{-y tau} A(wm - i y) dy
    {
        const double hs = 1.0 / 32.0;
        const int ns = 289;  // s in [-4.5, 4.5]
        double rr = 0.0, ri = 0.0;
        for (int j = lane; j < ns; j += 32) {
            double s = -4.5 + hs * j;
            double y = exp(1.5707963267948966 * sinh(s));
            double dy = y * 1.5707963267948966 * cosh(s);
            double e = exp(-y * tau) * dy;
            cx<double> a = lorentz(mk<double>(wm, -y), eps, gam);
            rr += e * a.re;
            ri += e * a.im;
        }
        rr *= hs;
        ri *= hs;
        // multiply by i e^{-i wm tau}
        double sn, cs;
        sincos(wm * tau, &sn, &cs);
        cx<double> ph = mk<double>(sn, cs);  // i * (cos - i sin) = sin + i cos
        cx<double> v = cmul(ph, mk<double>(rr, ri));
        ar += v.re;
        ai += v.im;
    }
    // segment [wm, 0]
    {
        const double len = -wm;
        const double pw = len / panels;
        for (int j = lane; j < panels * 16; j += 32) {
            int pnl = j >> 4, g = j & 15;
            double w = wm + pw * (pnl + 0.5 * (c_gl_x[g] + 1.0));
            double wt = 0.5 * pw * c_gl_w[g];
            double sn, cs;
            sincos(w * tau, &sn, &cs);
            cx<double> a = lorentz(mk<double>(w, 0.0), eps, gam);
            // e^{-i w tau} A = (cs - i sn) * a.re (A real on the axis)
            ar += wt * cs * a.re;
            ai -= wt * sn * a.re;
        }
    }
    // warp sum
    for (int o = 16; o > 0; o >>= 1) {
        ar += __shfl_xor_sync(FULL, ar, o);
        ai += __shfl_xor_sync(FULL, ai, o);
    }
    if (lane == 0) {
        const double inv2pi = 0.15915494309189535;
        // g^< = (i / 2pi) (ar + i ai) = (-ai + i ar) / 2pi
        double glr = -ai * inv2pi, gli = ar * inv2pi;
        double sn, cs;
        sincos(eps * tau, &sn, &cs);
        double dec = exp(-gam * tau);
        // -i e^{-i eps tau} e^{-gam tau} = -i (cs - i sn) dec = (-sn - i cs) dec
        double ggr = glr - sn * dec, ggi = gli - cs * dec;
        tab[q + 1] = make_double4_32a(glr, gli, ggr, ggi);
        tab32[q + 1] = make_float4((float)glr, (float)gli, (float)ggr, (float)ggi);
        if (q == 0) {  // node at -h/2: g(-tau) = -conj g(tau)
            tab[0] = make_double4_32a(-glr, gli, -ggr, ggi);
            tab32[0] = make_float4((float)-glr, (float)gli, (float)-ggr, (float)ggi);
        }
    }
}

// ----------------------------------------------------------------------------
// Finite-bandwidth leads (App. E): semicircular hybridisation of half-width D
// shared by two leads, symmetric bias V, T = 0.  With w = D sin(theta):
//   Gamma(w) = Gamma cos(theta),  Delta(w) = Gamma (sin(theta) - i cos(theta)),
//   g^R = 1 / (w - E_d - Delta),  f_L = theta(V/2 - w),  f_R = theta(-V/2 - w),
//   g^<_00 =  i Gamma(w) |g^R|^2 (f_L + f_R),
//   g^>_00 = -i Gamma(w) |g^R|^2 (2 - f_L - f_R),
//   gamma g^<_01 =  i f_R Gamma(w) g^R + (Delta^* / 2) g^<_00,
//   gamma g^>_01 = -i (1 - f_R) Gamma(w) g^R + (Delta^* / 2) g^>_00
// (lead R, which holds site 1, sits at -V/2; gamma G_01 = G_00 Delta_R by the
// Dyson equation and the Langreth rule).  g(tau) = Int dw/2pi e^{-i w tau} g(w)
// = Int dtheta (D cos(theta) / 2pi) e^{-i w(theta) tau} g(w(theta)): the
// square-root edges disappear and every integrand is smooth in theta between
// the Fermi steps, so each segment takes composite 16-point Gauss-Legendre.
// ----------------------------------------------------------------------------
struct LeadSeg {
    double a, b;   // theta range
    int panels;
    int first;     // first quadrature node of the segment
    double fL, fR; // Fermi factors on the segment
};

struct LeadQuad {
    LeadSeg seg[3];
    int n_seg;
    double gam, Ed, D;
};

// Quadrature node j: w_j and the four spectral values times weight x dw/dtheta / 2pi.
__global__ void lead_spectrum_kernel(LeadQuad q, int nq, double *w_out, dbl4 *s00, dbl4 *s01) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nq) return;
    int sg = 0;
    while (sg + 1 < q.n_seg && j >= q.seg[sg + 1].first) ++sg;
    const LeadSeg S = q.seg[sg];
    const int r = j - S.first;
    const int pnl = r >> 4, g = r & 15;
    const double pw = (S.b - S.a) / S.panels;
    const double th = S.a + pw * (pnl + 0.5 * (c_gl_x[g] + 1.0));
    const double wt = 0.5 * pw * c_gl_w[g];
    double sn, cs;
    sincos(th, &sn, &cs);
    const double w = q.D * sn;
    const double G = q.gam * cs;
    // g^R = 1 / (w - E_d - Gamma sin + i Gamma cos)
    const cx<double> gR = crcp(mk<double>(w - q.Ed - q.gam * sn, G));
    const double a2 = gR.re * gR.re + gR.im * gR.im;
    const double jac = wt * q.D * cs * 0.15915494309189535;
    const double lt = G * a2 * (S.fL + S.fR), gt = G * a2 * (2.0 - S.fL - S.fR);
    const cx<double> gl = mk<double>(0.0, lt), gg = mk<double>(0.0, -gt);
    const cx<double> dh = mk<double>(0.5 * q.gam * sn, 0.5 * q.gam * cs);  // Delta^* / 2
    // i f_R G g^R = f_R G (-gR.im + i gR.re)
    const cx<double> cl = mk<double>(-S.fR * G * gR.im + (dh.re * gl.re - dh.im * gl.im),
                                     S.fR * G * gR.re + (dh.re * gl.im + dh.im * gl.re));
    // -i (1 - f_R) G g^R = (1 - f_R) G (gR.im - i gR.re)
    const cx<double> cg = mk<double>((1.0 - S.fR) * G * gR.im + (dh.re * gg.re - dh.im * gg.im),
                                     -(1.0 - S.fR) * G * gR.re + (dh.re * gg.im + dh.im * gg.re));
    w_out[j] = w;
    s00[j] = make_double4_32a(jac * gl.re, jac * gl.im, jac * gg.re, jac * gg.im);
    s01[j] = make_double4_32a(jac * cl.re, jac * cl.im, jac * cg.re, jac * cg.im);
}

// One warp per output: nodes q = 0 .. L-1 (tau = -T + q h) and q = L (tau = 0).
// Dot tables go to the half table (nodes L/2-1 .. L-1), dot-lead tables to the
// column table (nodes 0 .. L/2); tau = 0 gives g^<_00(0) and gamma g^<_01(0).
__global__ void lead_table_kernel(int nq, const double *__restrict__ wq, const dbl4 *__restrict__ s00,
                                  const dbl4 *__restrict__ s01, int L, double T, double h, dbl4 *tab, float4 *tab32,
                                  dbl4 *col, float4 *col32, double *zero) {
    const int lane = threadIdx.x & 31;
    const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q > L) return;
    const double tau = q == L ? 0.0 : -T + (double)q * h;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int j = lane; j < nq; j += 32) {
        double sn, cs;
        sincos(wq[j] * tau, &sn, &cs);  // e^{-i w tau} = cs - i sn
        const dbl4 a = s00[j], b = s01[j];
        acc[0] += cs * a.x + sn * a.y;
        acc[1] += cs * a.y - sn * a.x;
        acc[2] += cs * a.z + sn * a.w;
        acc[3] += cs * a.w - sn * a.z;
        acc[4] += cs * b.x + sn * b.y;
        acc[5] += cs * b.y - sn * b.x;
        acc[6] += cs * b.z + sn * b.w;
        acc[7] += cs * b.w - sn * b.z;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] += __shfl_xor_sync(FULL, acc[c], o);
    if (lane != 0) return;
    if (q == L) {
        zero[0] = acc[0];
        zero[1] = acc[1];
        zero[2] = acc[4];
        zero[3] = acc[5];
        return;
    }
    if (q >= L / 2 - 1) {
        tab[q - (L / 2 - 1)] = make_double4_32a(acc[0], acc[1], acc[2], acc[3]);
        tab32[q - (L / 2 - 1)] = make_float4((float)acc[0], (float)acc[1], (float)acc[2], (float)acc[3]);
    }
    if (col && q <= L / 2) {
        col[q] = make_double4_32a(acc[4], acc[5], acc[6], acc[7]);
        col32[q] = make_float4((float)acc[4], (float)acc[5], (float)acc[6], (float)acc[7]);
    }
}

// ----------------------------------------------------------------------------
// host launchers
// ----------------------------------------------------------------------------
static void gauss_legendre16(double *x, double *w) {
    const int n = 16;
    for (int i = 0; i < n; ++i) {
        long double z = cosl(3.14159265358979323846264338327950288L * (i + 0.75L) / (n + 0.5L));
        long double pp = 0;
        for (int it = 0; it < 100; ++it) {
            long double p1 = 1, p2 = 0;
            for (int j = 1; j <= n; ++j) {
                long double p3 = p2;
                p2 = p1;
                p1 = ((2 * j - 1) * z * p2 - (j - 1) * p3) / j;
            }
            pp = n * (z * p1 - p2) / (z * z - 1);
            long double z1 = z;
            z = z1 - p1 / pp;
            if (fabsl(z - z1) < 1e-19L) break;
        }
        x[i] = (double)z;
        w[i] = (double)(2.0L / ((1 - z * z) * pp * pp));
    }
}

int upload_direction_numbers() {
    uint32_t dirs[kMaxOrder * 32];
    direction_numbers(kMaxOrder, dirs);
    cudaError_t e = cudaMemcpyToSymbol(c_dirs, dirs, sizeof(dirs));
    if (e != cudaSuccess) return cuda_error(e, "upload direction numbers");
    double gx[16], gw[16];
    gauss_legendre16(gx, gw);
    e = cudaMemcpyToSymbol(c_gl_x, gx, sizeof(gx));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_gl_w, gw, sizeof(gw));
    if (e != cudaSuccess) return cuda_error(e, "upload quadrature rule");
    return QQMC_OK;
}

int launch_gf_table(const Problem &pr, cudaStream_t s) {
    const qqmc_params &p = pr.params;
    double wm = fmin(p.eps_d, 0.0) - 3.0 * p.gamma;
    int panels = 64 + (int)ceil(-wm * (p.t_max + 4.0 / p.gamma));
    if (panels > 8192) panels = 8192;
    int warps = pr.L / 2;
    int threads = 128;
    int blocks = (warps * 32 + threads - 1) / threads;
    gf_table_kernel<<<blocks, threads, 0, s>>>(pr.d_table, pr.d_table32, pr.L, p.t_max, pr.h, p.eps_d, p.gamma,
                                               panels);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "gf_table_kernel launch");
    return QQMC_OK;
}

// Builds the dot (and, for the current, dot-lead) tables of finite-bandwidth
// leads; returns g^<_00(0) and gamma g^<_01(0) in zero[0..3] (host).  Panels:
// at most 2 radians of phase D T per panel and a quarter of the resonance
// width Gamma / D.
int launch_lead_table(Problem &pr, cudaStream_t s, double *zero) {
    const qqmc_params &p = pr.params;
    const double D = p.half_bandwidth, V = p.bias;
    LeadQuad q{};
    q.gam = p.gamma;
    q.Ed = p.eps_d;
    q.D = D;
    const double pi2 = 1.5707963267948966;
    double br[4];
    double fl[3], fr[3];
    int nb = 0;
    br[nb++] = -pi2;
    if (0.5 * V < D && V > 0.0) {
        br[nb++] = asin(-0.5 * V / D);
        br[nb++] = asin(0.5 * V / D);
        fl[0] = 1; fr[0] = 1;  // w < -V/2
        fl[1] = 1; fr[1] = 0;  // -V/2 < w < V/2
        fl[2] = 0; fr[2] = 0;  // w > V/2
    } else if (0.5 * V < D) {  // V = 0: one Fermi step at w = 0
        br[nb++] = 0.0;
        fl[0] = 1; fr[0] = 1;
        fl[1] = 0; fr[1] = 0;
    } else {  // the bias window covers the band
        fl[0] = 1; fr[0] = 0;
    }
    br[nb++] = pi2;
    double dth = fmin(fmin(2.0 / (D * p.t_max), 0.25 * p.gamma / D), 0.05);
    long long nq = 0;
    q.n_seg = nb - 1;
    for (int sg = 0; sg < q.n_seg; ++sg) {
        q.seg[sg].a = br[sg];
        q.seg[sg].b = br[sg + 1];
        long long pn = (long long)ceil((br[sg + 1] - br[sg]) / dth);
        if (pn < 1) pn = 1;
        q.seg[sg].panels = (int)(pn > (1 << 22) ? (1 << 22) : pn);
        q.seg[sg].first = (int)nq;
        q.seg[sg].fL = fl[sg];
        q.seg[sg].fR = fr[sg];
        nq += 16 * pn;
    }
    if (nq > (1ll << 24))
        return set_error(QQMC_E_INVAL, "half_bandwidth x t_max too large for the lead-table quadrature");
    double *d_w = nullptr, *d_zero = nullptr;
    dbl4 *d_s00 = nullptr, *d_s01 = nullptr;
    cudaError_t e = cudaMalloc(&d_w, nq * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&d_s00, nq * sizeof(dbl4));
    if (e == cudaSuccess) e = cudaMalloc(&d_s01, nq * sizeof(dbl4));
    if (e == cudaSuccess) e = cudaMalloc(&d_zero, 4 * sizeof(double));
    if (e == cudaSuccess) {
        lead_spectrum_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, s>>>(q, (int)nq, d_w, d_s00, d_s01);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const long long threads = 32ll * (pr.L + 1);
        lead_table_kernel<<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(
            (int)nq, d_w, d_s00, d_s01, pr.L, p.t_max, pr.h, pr.d_table, pr.d_table32, pr.d_col, pr.d_col32, d_zero);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(zero, d_zero, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_w);
    cudaFree(d_s00);
    cudaFree(d_s01);
    cudaFree(d_zero);
    if (e != cudaSuccess) return cuda_error(e, "lead table build");
    return QQMC_OK;
}

size_t detsum_smem_bytes(int n_max, int precision, const Tuning &tune) {
    size_t per = precision == QQMC_PREC_FP64 ? warp_smem_bytes<double>(n_max, tune.flat_min)
                                             : warp_smem_bytes<float>(n_max, tune.flat_min);
    return per * tune.warps_per_block;
}

// The tree stack is split (wide top levels in device memory) where it does not
// fit in shared memory, and from the order set by qqmc_set_stack_policy
// (default: from order 11 in both precisions, measured fastest on GB300): a large
// shared-memory stack limits the warps per SM, while the wide levels are built
// only a few times per point.
constexpr int kGsDefault[2] = {11, 11};
static std::atomic<int> g_gs_min_order[2] = {{kGsDefault[0]}, {kGsDefault[1]}};  // read by plans on any thread

void set_stack_policy(int precision, int min_order) {
    const int p = precision == QQMC_PREC_FP64 ? 0 : 1;
    g_gs_min_order[p].store(min_order <= 0 ? kGsDefault[p] : min_order);
}

template <class R>
static bool stack_in_global(int n_max, int rf_min) {
    return warp_smem_bytes<R>(n_max, rf_min) > kSmemMax || n_max >= g_gs_min_order[sizeof(R) == 8 ? 0 : 1].load();
}

template <class R, int F, bool GS>
static cudaError_t launch_detsum_t(const ItemDev *d_items, int n_items, long long total_chunks,
                                   unsigned long long *d_counter, int n_max, int wpb, int rf_min, void *gstack,
                                   long long gstack_warps, cudaStream_t s) {
    // fewer warps per block when the shared memory of the requested shape does not fit
    const size_t per_warp = warp_smem_bytes<R>(n_max, rf_min, GS);
    if (per_warp > kSmemMax) return cudaErrorInvalidConfiguration;
    while (wpb > 1 && per_warp * wpb > kSmemMax) --wpb;
    size_t smem = per_warp * wpb;
    cudaError_t e =
        cudaFuncSetAttribute(detsum_kernel<R, F, GS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, detsum_kernel<R, F, GS>, wpb * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long want = (total_chunks + wpb - 1) / wpb;
    long long grid = (long long)sms * per_sm;
    if (grid > want) grid = want;
    if (GS) {
        if (!gstack) return cudaErrorInvalidValue;
        if (grid > gstack_warps / wpb) grid = gstack_warps / wpb;
    }
    if (grid < 1) return cudaErrorInvalidConfiguration;
    detsum_kernel<R, F, GS><<<(unsigned)grid, wpb * 32, smem, s>>>(d_items, n_items, total_chunks, d_counter, n_max,
                                                                    rf_min, static_cast<cx<R> *>(gstack));
    return cudaGetLastError();
}

template <class R, int F>
static cudaError_t launch_detsum_f(const ItemDev *d_items, int n_items, long long total_chunks,
                                   unsigned long long *d_counter, int n_max, int wpb, int rf_min, void *gstack,
                                   long long gstack_warps, cudaStream_t s) {
    // without a device-memory buffer (the allocation-free entry) the shared-memory stack serves where it fits
    if (stack_in_global<R>(n_max, rf_min) && (gstack || warp_smem_bytes<R>(n_max, rf_min) > kSmemMax))
        return launch_detsum_t<R, F, true>(d_items, n_items, total_chunks, d_counter, n_max, wpb, rf_min, gstack,
                                           gstack_warps, s);
    return launch_detsum_t<R, F, false>(d_items, n_items, total_chunks, d_counter, n_max, wpb, rf_min, nullptr, 0, s);
}

static int clamp_rf_min(const Tuning &tune) {
    return tune.flat_min < 2 ? 2 : (tune.flat_min > tune.flat ? tune.flat : tune.flat_min);
}

template <class R>
static long long gstack_warps_t(int n_max, int rf_min, size_t *bytes_per_warp) {
    *bytes_per_warp = 0;
    if (!stack_in_global<R>(n_max, rf_min)) return 0;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t per_warp = warp_smem_bytes<R>(n_max, rf_min, true);
    long long per_sm = (long long)(kSmemMax / per_warp);  // resident warps, bound by shared memory
    if (per_sm > 64) per_sm = 64;                          // and by the SM's warp slots
    *bytes_per_warp = gstack_entries<R>(n_max, rf_min) * sizeof(cx<R>);
    return (long long)sms * (per_sm < 1 ? 1 : per_sm);
}

bool detsum_stack_fits_shared(int n_max, int precision, const Tuning &tune) {
    const int rf_min = clamp_rf_min(tune);
    return precision == QQMC_PREC_FP64 ? warp_smem_bytes<double>(n_max, rf_min) <= kSmemMax
                                       : warp_smem_bytes<float>(n_max, rf_min) <= kSmemMax;
}

long long detsum_gstack_warps(int n_max, int precision, const Tuning &tune, size_t *bytes_per_warp) {
    const int rf_min = clamp_rf_min(tune);
    return precision == QQMC_PREC_FP64 ? gstack_warps_t<double>(n_max, rf_min, bytes_per_warp)
                                       : gstack_warps_t<float>(n_max, rf_min, bytes_per_warp);
}

cudaError_t launch_detsum(const ItemDev *d_items, int n_items, long long total_chunks, unsigned long long *d_counter,
                          int n_max, int precision, const Tuning &tune, void *gstack, long long gstack_warps,
                          cudaStream_t s) {
    const int wpb = tune.warps_per_block;
    const int rf_min = clamp_rf_min(tune);
#define QQMC_DETSUM(RT, F)                                                                                        \
    launch_detsum_f<RT, F>(d_items, n_items, total_chunks, d_counter, n_max, wpb, rf_min, gstack, gstack_warps, s)
    if (precision == QQMC_PREC_FP64) {
        switch (tune.flat) {
            case 2: return QQMC_DETSUM(double, 2);
            case 3: return QQMC_DETSUM(double, 3);
            case 4: return QQMC_DETSUM(double, 4);
            default: return QQMC_DETSUM(double, 5);
        }
    }
    switch (tune.flat) {
        case 2: return QQMC_DETSUM(float, 2);
        case 3: return QQMC_DETSUM(float, 3);
        case 4: return QQMC_DETSUM(float, 4);
        default: return QQMC_DETSUM(float, 5);
    }
#undef QQMC_DETSUM
}

template <class R>
static cudaError_t launch_lane_t(const ItemDev *d_items, int n_items, long long total_chunks,
                                 unsigned long long *d_counter, cudaStream_t s) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lane_kernel<R>, 128, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long want = (total_chunks + 3) / 4;
    long long grid = (long long)sms * per_sm;
    if (grid > want) grid = want;
    if (grid < 1) grid = 1;
    lane_kernel<R><<<(unsigned)grid, 128, 0, s>>>(d_items, n_items, total_chunks, d_counter);
    return cudaGetLastError();
}

cudaError_t launch_lane(const ItemDev *d_items, int n_items, long long total_chunks, unsigned long long *d_counter,
                        int precision, cudaStream_t s) {
    if (n_items < 1 || total_chunks < 1) return cudaSuccess;
    return precision == QQMC_PREC_FP64 ? launch_lane_t<double>(d_items, n_items, total_chunks, d_counter, s)
                                       : launch_lane_t<float>(d_items, n_items, total_chunks, d_counter, s);
}

cudaError_t launch_reduce(const ItemDev *d_items, int n_items, int total_shifts, double *d_out,
                          unsigned long long *d_counts, cudaStream_t s) {
    reduce_kernel<<<total_shifts, 256, 0, s>>>(d_items, n_items, d_out, d_counts);
    return cudaGetLastError();
}

cudaError_t launch_sobol(int order, uint64_t first, uint64_t count, const uint32_t *d_shift, uint32_t *d_out,
                         const uint32_t *d_lat_z, int lat_m, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    unsigned blocks = (unsigned)((count + 255) / 256);
    sobol_kernel<<<blocks, 256, 0, s>>>(order, first, count, d_shift, d_out, d_lat_z, lat_m);
    return cudaGetLastError();
}

cudaError_t launch_warp(int order, uint64_t first, uint64_t count, const uint32_t *d_shift, double t, double tau,
                        double *d_u, double *d_w, int32_t *d_inside, const uint32_t *d_lat_z, int lat_m,
                        cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    unsigned blocks = (unsigned)((count + 255) / 256);
    warp_kernel<<<blocks, 256, 0, s>>>(order, first, count, d_shift, t, tau, d_u, d_w, d_inside, d_lat_z, lat_m);
    return cudaGetLastError();
}

template <class R, int F, bool GS>
static cudaError_t launch_integrand_t(const ItemDev &item, uint64_t count, const double *d_u, double *d_out,
                                      cudaStream_t s) {
    const size_t per_warp = warp_smem_bytes<R>(item.order, F, GS);
    if (per_warp > kSmemMax) return cudaErrorInvalidConfiguration;
    const int wpb = per_warp * 2 <= kSmemMax ? 2 : 1;
    size_t smem = per_warp * wpb;
    cudaError_t e =
        cudaFuncSetAttribute(integrand_kernel<R, F, GS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    uint64_t blocks = (count + wpb - 1) / wpb;
    cx<R> *gstack = nullptr;
    if (GS) {  // check path: a bounded number of warps, each with its own slice of device memory
        if (blocks > 304) blocks = 304;
        e = cudaMalloc(&gstack, blocks * wpb * gstack_entries<R>(item.order, F) * sizeof(cx<R>));
        if (e != cudaSuccess) return e;
    }
    integrand_kernel<R, F, GS><<<(unsigned)blocks, wpb * 32, smem, s>>>(item, count, d_u, d_out, item.order, gstack);
    e = cudaGetLastError();
    if (GS) {
        cudaError_t e2 = cudaStreamSynchronize(s);
        cudaFree(gstack);
        if (e == cudaSuccess) e = e2;
    }
    return e;
}

template <class R, int F>
static cudaError_t launch_integrand_f(const ItemDev &item, uint64_t count, const double *d_u, double *d_out,
                                      cudaStream_t s) {
    if (stack_in_global<R>(item.order, F)) return launch_integrand_t<R, F, true>(item, count, d_u, d_out, s);
    return launch_integrand_t<R, F, false>(item, count, d_u, d_out, s);
}

cudaError_t launch_integrand(const ItemDev &item, uint64_t count, const double *d_u, double *d_out, int precision,
                             const Tuning &tune, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    if (precision == QQMC_PREC_FP64) {
        switch (tune.flat) {
            case 2: return launch_integrand_f<double, 2>(item, count, d_u, d_out, s);
            case 3: return launch_integrand_f<double, 3>(item, count, d_u, d_out, s);
            case 4: return launch_integrand_f<double, 4>(item, count, d_u, d_out, s);
            default: return launch_integrand_f<double, 5>(item, count, d_u, d_out, s);
        }
    }
    switch (tune.flat) {
        case 2: return launch_integrand_f<float, 2>(item, count, d_u, d_out, s);
        case 3: return launch_integrand_f<float, 3>(item, count, d_u, d_out, s);
        case 4: return launch_integrand_f<float, 4>(item, count, d_u, d_out, s);
        default: return launch_integrand_f<float, 5>(item, count, d_u, d_out, s);
    }
}

}  // namespace qqmc
