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
#include <type_traits>

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
// rounding stays below 1e-14 of the Keldysh-sum scale, and the lanes' shares
// are combined with two-sum (per point in warp_total, or weighted and summed
// over a work unit's points with add_weighted in the integration kernel).
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

// (s, c) += w z: the product's rounding error by FMA (error-free product), the
// sum by two-sum, both errors into c.
__device__ __forceinline__ void add_weighted(double w, double z, double &s, double &c) {
    const double p = w * z;
    const double e = fma(w, z, -p);
    double t, f;
    two_sum(s, p, t, f);
    s = t;
    c += f + e;
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

// Vertex times as the kernels keep them, one 8-byte slot per vertex (u_0 = t
// first).  FP64: the time u itself.  Mixed: the mesh position x = u / h split
// into its integer part and an FP32 fraction, so that a pair's position
// s = x_j - x_k + T / h takes integer and FP32 operations only (the FP64 pipe
// runs at 1/64 of the FP32 rate on this part).  With h = 2T / (L - 1), T / h
// is (L - 1) / 2 exactly: integer part (L - 1) / 2, fraction 0 or 1/2.  The
// fraction carries 24 bits, so the interpolation weight is exact to ~1e-7,
// the rounding of the FP32 blend itself.
struct VP32 {
    int k;
    float f;
};

template <class R>
__device__ __forceinline__ void store_time(double *slot, double u, double inv_h) {
    if constexpr (sizeof(R) == 8) {
        *slot = u;
    } else {
        const double x = u * inv_h;
        const double kx = floor(x);
        VP32 v;
        v.k = (int)kx;
        v.f = (float)(x - kx);
        *reinterpret_cast<VP32 *>(slot) = v;
    }
}

// Node index and weight of position K + phi (phi in (-1, 2)) clamped to [kmin, kmax].
__device__ __forceinline__ int mesh_node(int K, float phi, int kmin, int kmax, float &fr) {
    int k = K + (phi >= 1.0f ? 1 : 0) - (phi < 0.0f ? 1 : 0);
    k = k < kmin ? kmin : (k > kmax ? kmax : k);
    fr = phi + (float)(K - k);
    return k;
}

// Pair values of vertices j < k (u_j > u_k) from the stored times.
template <class R>
__device__ __forceinline__ void interp_pair_u(const typename TabT<R>::V *tab, double inv_h, double s0, int L,
                                              const double *u, int j, int k, cx<R> &gl, cx<R> &gg) {
    if constexpr (sizeof(R) == 8) {
        interp_pair<R>(tab, inv_h, s0, L, u[j] - u[k], gl, gg);
    } else {
        const VP32 a = *reinterpret_cast<const VP32 *>(u + j), b = *reinterpret_cast<const VP32 *>(u + k);
        const int kmin = L / 2 - 1;
        float fr;
        const int q = mesh_node(a.k - b.k + (L - 1) / 2, (a.f - b.f) + ((L - 1) & 1 ? 0.5f : 0.0f), kmin, L - 2, fr);
        const float g = 1.0f - fr;
        const float4 lo = tab[q - kmin], hi = tab[q - kmin + 1];
        gl = mk<R>(fmaf(fr, hi.x, g * lo.x), fmaf(fr, hi.y, g * lo.y));
        gg = mk<R>(fmaf(fr, hi.z, g * lo.z), fmaf(fr, hi.w, g * lo.w));
    }
}

// Measurement-column values of vertex k from the stored times (tau = u_k - t).
template <class R>
__device__ __forceinline__ void interp_col_u(const typename TabT<R>::V *col, double inv_h, double s0, int L,
                                             const double *u, int k, cx<R> &cl, cx<R> &cg) {
    if constexpr (sizeof(R) == 8) {
        interp_col<R>(col, inv_h, s0, L, u[k] - u[0], cl, cg);
    } else {
        const VP32 a = *reinterpret_cast<const VP32 *>(u + k), b = *reinterpret_cast<const VP32 *>(u);
        float fr;
        const int q = mesh_node(a.k - b.k + (L - 1) / 2, (a.f - b.f) + ((L - 1) & 1 ? 0.5f : 0.0f), 0, L / 2 - 1, fr);
        const float g = 1.0f - fr;
        const float4 lo = col[q], hi = col[q + 1];
        cl = mk<R>(fmaf(fr, hi.x, g * lo.x), fmaf(fr, hi.y, g * lo.y));
        cg = mk<R>(fmaf(fr, hi.z, g * lo.z), fmaf(fr, hi.w, g * lo.w));
    }
}

// ----------------------------------------------------------------------------
// Complex helpers and the leaf formula shared by both Keldysh-sum trees.
// ----------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ cx<R> sel(int bit, cx<R> one, cx<R> zero) {
    return mk<R>(bit ? one.re : zero.re, bit ? one.im : zero.im);
}
template <class R>
__device__ __forceinline__ cx<R> cneg(cx<R> a) {
    return mk<R>(-a.re, -a.im);
}
template <class R>
__device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) {
    return mk<R>(a.re - b.re, a.im - b.im);
}
// c + a * b
template <class R>
__device__ __forceinline__ cx<R> cfma(cx<R> c, cx<R> a, cx<R> b) {
    return mk<R>(fmaR(a.re, b.re, fmaR(-a.im, b.im, c.re)), fmaR(a.re, b.im, fmaR(a.im, b.re, c.im)));
}

// Leaf term after a lone last vertex p: with pivot pv and the copies' entries,
//   det' = det pv,   S_cc = m_cc - m_cp m_pc / pv   (c = copy 0, 1),
//   det'^2 (S_00 - S_11) = det^2 pv (pv (m_00 - m_11) - (m_0p m_p0 - m_1p m_p1)):
// no reciprocal, so a vanishing pivot (det M_down = 0) gives a zero term.
template <class R>
__device__ __forceinline__ cx<R> leaf_term(cx<R> m00, cx<R> m11, cx<R> m0p, cx<R> mp0, cx<R> m1p, cx<R> mp1, cx<R> pv,
                                           cx<R> det) {
    const cx<R> q = cfms(cmul(m0p, mp0), m1p, mp1);  // m0p mp0 - m1p mp1
    const cx<R> r = cfms(q, pv, csub(m00, m11));      // q - pv (m00 - m11)
    return cmul(cmul(det, det), cmul(pv, cneg(r)));
}

template <class R>
__device__ __forceinline__ void two_sum_r(R a, R b, R &s, R &e) {
    s = a + b;
    R z = s - a;
    e = (a - (s - z)) + (b - z);
}

// Float-float or double-double style butterfly of the lane accumulators over
// groups of W lanes (W = 32: the warp, 16: each half-warp): combines the
// (s, c) pairs with two-sum in R; every lane gets its group's pair.
template <class R, int W = 32>
__device__ __forceinline__ Acc<R> group_pair(Acc<R> acc) {
    R s = acc.s, c = acc.c;
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) {
        R s2 = __shfl_xor_sync(FULL, s, o);
        R c2 = __shfl_xor_sync(FULL, c, o);
        R t, e;
        int lo = ((threadIdx.x & 31) & o) == 0;
        if (lo) two_sum_r<R>(s, s2, t, e); else two_sum_r<R>(s2, s, t, e);
        s = t;
        c = lo ? (c + c2) + e : (c2 + c) + e;
    }
    Acc<R> r;
    r.s = s;
    r.c = c;
    return r;
}

// The pair's value s + c in double.
template <class R>
__device__ __forceinline__ double pair_value(Acc<R> a) {
    return (double)a.s + (double)a.c;
}

template <class R>
__device__ __forceinline__ double warp_total(Acc<R> acc) {
    return pair_value<R>(group_pair<R>(acc));
}

// What a Keldysh-sum tree returns: the warp total in double (kOutTotal), the
// lane's own share in double (kOutShare: the shares sum to the total, for
// callers that weight and accumulate shares per lane), or the warp total as
// the unevaluated pairs in R (kOutPair: for callers that convert it later).
constexpr int kOutTotal = 0, kOutShare = 1, kOutPair = 2;

template <class R>
struct PairSum {
    Acc<R> re, im;
};
template <class R, int OUT>
struct SumOut {
    using type = cx<double>;
};
template <class R>
struct SumOut<R, kOutPair> {
    using type = PairSum<R>;
};

template <class R, int OUT>
__device__ __forceinline__ typename SumOut<R, OUT>::type tree_result(Acc<R> ar, Acc<R> ai) {
    if constexpr (OUT == kOutPair) {
        PairSum<R> r;
        r.re = group_pair<R>(ar);
        r.im = group_pair<R>(ai);
        return r;
    } else if constexpr (OUT == kOutShare) {
        return mk<double>(pair_value<R>(ar), pair_value<R>(ai));
    } else {
        return mk<double>(warp_total<R>(ar), warp_total<R>(ai));
    }
}

// Mixed path: a work unit's sum of the lanes' FP64 values (re, im) as an FP64
// (sum, compensation) pair per part, with the butterfly on the FP32 pipe.  The
// values are scaled by one power of two (the largest magnitude in the warp then
// lies in [2^63, 2^64), so 32 of them stay far from the FP32 limit and the
// smallest that matter far above its underflow), split into float-float pairs
// (about 48 bits), combined with group_pair and scaled back.  FP64 instructions
// cost 64 FP32 instructions' issue here: this takes 18 of them per unit where
// the FP64 butterfly takes 80.  A NaN or infinity stays one.
__device__ __forceinline__ void unit_pairs_ff(double re, double im, double &sr, double &cr, double &si, double &ci) {
    const int er = (__double2hiint(re) >> 20) & 0x7ff, ei = (__double2hiint(im) >> 20) & 0x7ff;
    const int e = (int)__reduce_max_sync(FULL, (unsigned)(er > ei ? er : ei));
    int k = e == 0x7ff ? 0 : 1023 + 63 - e;  // scale by 2^k, |k| <= 1022
    k = k > 1022 ? 1022 : k;
    const double up = __hiloint2double((k + 1023) << 20, 0), down = __hiloint2double((1023 - k) << 20, 0);
    auto split = [&](double x) {
        const double xs = x * up;
        Acc<float> a;
        a.s = (float)xs;
        a.c = (float)(xs - (double)a.s);
        return group_pair<float>(a);
    };
    const Acc<float> pr = split(re), pi = split(im);
    sr = (double)pr.s * down;
    cr = (double)pr.c * down;
    si = (double)pi.s * down;
    ci = (double)pi.c * down;
}

// ----------------------------------------------------------------------------
// Single-vertex Schur tree (the fast path): one vertex per tree level with
// its 1x1 pivot.  Pivots are the ratios of consecutive leading minors of
// M_down, the first being the vertex diagonal g^<(0) - i alpha itself; the
// plans use this tree for problems whose vertex diagonal is well away from
// zero and the pair-block tree (namespace pairs) otherwise.
// ----------------------------------------------------------------------------
namespace single {

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
    double *upt;    // [32][n_max+1] point times of the chunk (u_0 = t; store_time form); device memory with the split stack
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
        if (Rl < kTreeLeaf && 2 * bfs_entries(Rl, RF) > e) e = 2 * bfs_entries(Rl, RF);  // two points
        m = e > m ? e : m;
    }
    return m;
}

// The shared-memory part of the tree stack: the levels that live there, and at
// least the two level-0 matrices of a two-point pass (orders <= kTreeLeaf + 1).
__host__ __device__ inline size_t stack_smem_entries(int n_max, int gs_level) {
    const size_t lv = gs_level ? stack_entries_split(n_max, false, gs_level) : stack_entries(n_max);
    const size_t n2 = n_max < kTreeLeaf + 1 ? n_max : kTreeLeaf + 1;
    const size_t two = 2 * (2 * n2) * (2 * n2);
    return lv > two ? lv : two;
}

// The mixed-precision path builds sibling leaves in pairs (one depth-first step
// for two leaves: its steps are latency-bound); the FP64 path, bound by its
// FP64 pipe, gains nothing from it and keeps the shared memory for warps.
template <class R>
__host__ __device__ constexpr bool twin_leaves() { return sizeof(R) == 4; }

// Orders whose tree has no depth-first level and whose choice paths fill at
// most half a warp run two points per warp (keldysh_sum2): orders <= kTreeLeaf
// (at most 16 paths, one per lane), and in FP32 with a flat depth of
// kTreeLeaf also order kTreeLeaf + 1 (the paired flat phase: 16 lanes, two
// paths each).  Both points' breadth-first levels are built together.
template <class R, int RFMAX>
__host__ __device__ inline bool two_point_order(int n) {
    return n <= kTreeLeaf || (n == kTreeLeaf + 1 && twin_leaves<R>() && RFMAX >= kTreeLeaf);
}

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
    size_t c = stack_smem_entries(n_max, gs_level) + pair_entries(n_max) +
               n_max + 1 + sib_entries<R>(n_max) + 4 * (size_t)n_max + bfs_max_entries(n_max, RF) + wide;
    size_t bytes = (c * sizeof(cx<R>) + 15) & ~(size_t)15;
    if (!gs_level) bytes += 32 * (size_t)(n_max + 1) * sizeof(double);
    return (bytes + 127) & ~(size_t)127;
}

// Split-stack boundary: the widest levels go to device memory, two rows at a
// time, until a warp's shared memory lets the SM hold the warps its bound pipe
// needs (FP64: 24 KB, 9 warps per SM at order 10 with the point times in
// device memory; re-tuned benchmark step 2326 ms, against 2332 at 28 KB, 2362
// at 32 KB and 2511 at 36 KB with the point times in shared memory; mixed: 12).
// Never the tree leaf (S = 12) or its parent (S = 14): the last depth-first
// step and the breadth-first and flat phases work in shared memory only.
template <class R>
__host__ __device__ inline int gs_level_of(int n_max, int RF) {
    const size_t budget = sizeof(R) == 8 ? 24 * 1024 : 18 * 1024;
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
    p += stack_smem_entries(n_max, w.gs_level);
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

// Flat phase for the two choice paths that differ only in the last vertex:
// `path` holds the Keldysh indices of the first F - 1 remaining vertices and
// the lane carries both rows and columns of the last one (register indices F
// and F + 1) through the first F - 1 eliminations, then closes each path with
// its own leaf term.  Per path this shares all but the leaf, about a third of
// flat_phase's flops and loads at F = 5; the entries joining the two copies
// of the last vertex are never used and never built.  The terms equal
// flat_phase's for the same paths, operation for operation.
template <class R, int F>
__device__ __forceinline__ void flat_pair(const cx<R> *E, cx<R> detD, int parity, int path, Acc<R> &acc_re,
                                          Acc<R> &acc_im) {
    static_assert(F >= 2, "the paired flat phase needs a vertex before the last");
    constexpr int S = 2 * F + 2;
    constexpr int M = F + 2;  // 2 copies, vertices 1 .. F-2, both indices of vertex F-1
    auto used = [](int x, int y) { return x == y || !((x < 2 && y < 2) || (x >= F && y >= F)); };
    int idx[M];
    idx[0] = 0;
    idx[1] = 1;
#pragma unroll
    for (int q = 1; q < F - 1; ++q) idx[q + 1] = 2 + 2 * q + ((path >> q) & 1);
    idx[F] = 2 * F;
    idx[F + 1] = 2 * F + 1;
    const int p0 = 2 + (path & 1);
    cx<R> piv = E[p0 * S + p0];
    detD = cmul(detD, piv);
    cx<R> ip = crcp(piv);
    cx<R> m[M][M];
    cx<R> prow[M];
#pragma unroll
    for (int y = 0; y < M; ++y) prow[y] = cmul(E[p0 * S + idx[y]], ip);
#pragma unroll
    for (int x = 0; x < M; ++x) {
        cx<R> cf = E[idx[x] * S + p0];
#pragma unroll
        for (int y = 0; y < M; ++y)
            if (used(x, y)) m[x][y] = cfms(E[idx[x] * S + idx[y]], cf, prow[y]);
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
                if (!(y < 2 || y > p) || !used(x, y)) continue;
                m[x][y] = cfms(m[x][y], m[x][p], m[p][y]);
            }
        }
    }
    parity ^= __popc(path) & 1;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int L = F + c;
        cx<R> term = leaf_term(m[0][0], m[1][1], m[0][L], m[L][0], m[1][L], m[L][1], m[L][L], detD);
        if (parity ^ c) term = mk<R>(-term.re, -term.im);
        acc_re.add(term.re);
        acc_im.add(term.im);
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
// every load of the step is issued at once and the lane mapping needs no
// division.  FP64 (pivot_slots<R>()): a depth-first node's two pivot
// reciprocals (for a = 0, 1) are formed once, when the node is built, by the
// lanes that compute the pivots, and kept in the cross slots (2, 3) and (3, 2),
// which join the first vertex's two copies and are never read as entries; a
// step loads its reciprocal with the rest, and both children of a node share
// it (one reciprocal per node instead of one per child: FP64 benchmark step
// 1.5 % faster, results bit-identical).  FP32 forms the reciprocal in the step:
// the two-lane branch at the end of the step measured 5-10 % slower there.
//
// Children of 2T = 12, 14 or 16 rows (the deep, frequent steps): lanes 0-15
// take the even rows, lanes 16-31 the odd rows, column c2 = lane & 15.
template <class R>
__host__ __device__ constexpr bool pivot_slots() { return sizeof(R) == 8; }

template <class R, int T>
__device__ __forceinline__ void expand_one_t(const cx<R> *__restrict__ in, int a, cx<R> *__restrict__ out,
                                             const cx<R> *detD_in, cx<R> *detD_out, int lane, bool rcp_child) {
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
    // the pivot's reciprocal: from its row's cross slot, or formed here
    const cx<R> ip = pivot_slots<R>() ? in[pr * S + 5 - pr] : crcp(piv);
    if (lane == 0) *detD_out = cmul(*detD_in, piv);
    if (act) {
        const cx<R> w = cmul(prc, ip);
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const cx<R> v = cfms(ev[t], cv[t], w);
            if constexpr (pivot_slots<R>()) {
                // row 2 + rsub of the child: its cross entry (2 + rsub, 3 - rsub) is never read as
                // an entry; for an inner node it holds the reciprocal of the diagonal entry instead
                if (t == 1 && rcp_child && c2 == 3 - rsub) continue;
                out[(rsub + 2 * t) * S2 + c2] = v;
                if (t == 1 && rcp_child && c2 == 2 + rsub) out[(2 + rsub) * S2 + 3 - rsub] = crcp(v);
            } else {
                out[(rsub + 2 * t) * S2 + c2] = v;
            }
        }
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
    const cx<R> ip0 = pivot_slots<R>() ? in[2 * S + 3] : crcp(piv0);  // the pivots' reciprocals
    const cx<R> ip1 = pivot_slots<R>() ? in[3 * S + 2] : crcp(piv1);
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
                                                const cx<R> *detD_in, cx<R> *detD_out, int lane, bool rcp_child) {
    constexpr int NB = sizeof(R) == 4 ? 8 : 4;  // rows per batch (FP64: register budget)
    const int S2 = S - 2;
    const int pr = 2 + a;
    const cx<R> piv = in[pr * S + pr];
    const cx<R> ip = pivot_slots<R>() ? in[pr * S + 5 - pr] : crcp(piv);
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
            for (int t = 0; t < NB; ++t) {
                const int r2 = r0 + t;
                if (r2 >= S2) continue;
                const cx<R> v = cfms(ev[t], cv[t], w);
                const bool slot = pivot_slots<R>() && rcp_child && (r2 == 2 || r2 == 3);
                if (slot && lane == (r2 ^ 1)) continue;  // the cross slot, written below
                out[r2 * S2 + lane] = v;
                if (slot && lane == r2) out[r2 * S2 + (r2 ^ 1)] = crcp(v);
            }
        }
    }
    __syncwarp();
}

template <class R>
__device__ __forceinline__ void expand_one(const cx<R> *__restrict__ in, int S, int a, cx<R> *__restrict__ out,
                                           const cx<R> *detD_in, cx<R> *detD_out, int lane, bool rcp_child) {
    switch (S - 2) {
        case 12: expand_one_t<R, 6>(in, a, out, detD_in, detD_out, lane, rcp_child); break;
        case 14: expand_one_t<R, 7>(in, a, out, detD_in, detD_out, lane, rcp_child); break;
        case 16: expand_one_t<R, 8>(in, a, out, detD_in, detD_out, lane, rcp_child); break;
        default: expand_one_wide<R>(in, S, a, out, detD_in, detD_out, lane, rcp_child); break;
    }
}

// The pivot reciprocals of a depth-first node built by the general step, which
// leaves the cross slots unbuilt: 1 / E(2,2) into E(2,3), 1 / E(3,3) into E(3,2).
template <class R>
__device__ __forceinline__ void fill_pivot_slots(cx<R> *E, int S, int lane) {
    if (lane < 2) E[(2 + lane) * S + 3 - lane] = crcp(E[(2 + lane) * S + 2 + lane]);
    __syncwarp();
}

// Steps 1 and 2 of the Keldysh sum of one point whose times are in u[0..n]:
// its pair values into P and Rr, then level 0 of the tree into `out`
// (2n x 2n).  slots: also form vertex 2's two pivot reciprocals in level 0's
// cross slots (FP64 trees with depth-first levels, see expand_one_t).
template <class R>
__device__ __forceinline__ void build_level0(const WarpSmem<R> &ws, const double *u, int n, cx<R> d, cx<R> dv,
                                             const typename TabT<R>::V *tab, const typename TabT<R>::V *col,
                                             double inv_h, double s0, int L, cx<R> *__restrict__ out, bool slots,
                                             int lane) {
    // 1. pair interpolation, 0 <= j < k <= n
    const int npairs = n * (n + 1) / 2;
    for (int p = lane; p < npairs; p += 32) {
        int k = (int)((1.0f + sqrtf(8.0f * p + 1.0f)) * 0.5f);
        while (k * (k - 1) / 2 > p) --k;
        while ((k + 1) * k / 2 <= p) ++k;
        int j = p - k * (k - 1) / 2;
        cx<R> gl, gg;
        interp_pair_u<R>(tab, inv_h, s0, L, u, j, k, gl, gg);
        const int ok = p - j + k - 1;  // vertex k's block: (k-1)(k+2)/2
        ws.P[ok + j] = gg;
        ws.Rr[ok + j] = gl;
        if (j == 0) {  // measurement column of vertex k: g^<(u_k - t), g^>(u_k - t) for the charge
            cx<R> c0 = nconj(gl), c1 = nconj(gg);
            if (col) interp_col_u<R>(col, inv_h, s0, L, u, k, c0, c1);
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
            cx<R> *o = out + (2 * bx) * S0 + 2 * by;
            const cx<R> o00 = cfms(b00, left0, right0), o11 = cfms(b11, left1, right1);
            o[0] = o00;
            o[S0 + 1] = o11;
            if (slots && bx == 1 && by == 1) {  // pivot reciprocals (expand_one_t)
                o[1] = crcp(o00);
                o[S0] = crcp(o11);
            } else {
                o[1] = cfms(b01, left0, right1);
                o[S0] = cfms(b10, left1, right0);
            }
            by += sr;
            bx += sq;
            if (by >= n) {
                by -= n;
                ++bx;
            }
        }
    }
}

// Keldysh sum for one point whose times are in u[0..n] (u_0 = t).
// Returns sum_{a_2..a_n} (-1)^{a_2+..+a_n} det M_down^2 (S00(0) - S00(1)),
// i.e. sum_a (-1)^{|a|} det M_up det M_down (without the i^n factor).
// The depth-first walk covers the subtree `sub` of 2^split: the first `split`
// tree levels follow the bits of sub (split <= levels); split = 0: whole tree.
// OUT: the form of the result (kOutTotal, kOutShare, kOutPair).
template <class R, int RFMAX, bool GS, int OUT = kOutTotal>
__device__ typename SumOut<R, OUT>::type keldysh_sum(const WarpSmem<R> &ws, const double *u, int n, int n_max,
                                                     cx<R> d, cx<R> dv,
                                  const typename TabT<R>::V *tab, const typename TabT<R>::V *col, double inv_h,
                                  double s0, int L, int RF, int lane, int sub = 0, int split = 0) {
    // 1. pair interpolation, 0 <= j < k <= n, and 2. level 0 (build_level0)
    const int R0 = n - 1;
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
    build_level0<R>(ws, u, n, d, dv, tab, col, inv_h, s0, L, level(0), pivot_slots<R>() && levels >= 1, lane);
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
            const bool inner = l + 1 < levels;  // the child is a depth-first node in turn, not a leaf
            if (S - 2 <= 32) {
                expand_one<R>(level(l), S, a, level(l + 1), ws.detD + l, ws.detD + l + 1, lane, inner);
            } else {
                expand_level<R>(level(l), S, 1, a, level(l + 1), ws.detD + l, ws.detD + l + 1, ws.wrow, ws.bip,
                                lane);
                if (pivot_slots<R>() && inner) fill_pivot_slots<R>(level(l + 1), S - 2, lane);
            }
        }
        if (twin)  // the leaves' parent has 2 kTreeLeaf + 4 rows
            expand_both_t<R, kTreeLeaf + 1>(level_smem(levels - 1), level_smem(levels), ws.sib,
                                            ws.detD + levels - 1, ws.detD + levels, ws.detD + levels + 1, lane);
        if constexpr (twin_leaves<R>() && RFMAX >= kTreeLeaf) {
            // both leaves at once, flat on all kTreeLeaf vertices: half-warp h resolves leaf h,
            // two choice paths per lane (the last vertex's two indices)
            if (twin && B == 0) {
                const int h = lane >> 4;
                const cx<R> *E = h ? ws.sib : level_smem(levels);
                flat_pair<R, kTreeLeaf>(E, ws.detD[levels + h], __popc(b + h) & 1, lane & 15, ar, ai);
                __syncwarp();
                continue;
            }
        }
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
    return tree_result<R, OUT>(ar, ai);
}

// Keldysh sums of two points at once (two_point_order(n)): the points whose
// times are in ua and ub get level 0 side by side at the bottom of the stack,
// and their trees run as one tree with a top bit h = the point.  Half-warp h
// resolves point h: at order kTreeLeaf + 1 (FP32, flat kTreeLeaf) its leaf
// with the paired flat phase; at lower orders the breadth-first levels build
// both points' nodes together (2, 4, ... parents) and lane 16 h + (node, path)
// takes one path (at most 16 per point).  Each point's sum is the total of its
// half-warp; both are returned to every lane in the form OUT, as keldysh_sum's
// (kOutShare: each lane's own share of its half's point, in sa).
template <class R, int RFMAX, int OUT = kOutTotal>
__device__ void keldysh_sum2(const WarpSmem<R> &ws, const double *ua, const double *ub, int n, cx<R> d, cx<R> dv,
                             const typename TabT<R>::V *tab, const typename TabT<R>::V *col, double inv_h, double s0,
                             int L, int RF, int lane, typename SumOut<R, OUT>::type &sa,
                             typename SumOut<R, OUT>::type &sb) {
    const int S0 = 2 * n;
    build_level0<R>(ws, ua, n, d, dv, tab, col, inv_h, s0, L, ws.stack, false, lane);
    __syncwarp();  // P, Rr and lr are rebuilt for the second point
    build_level0<R>(ws, ub, n, d, dv, tab, col, inv_h, s0, L, ws.stack + S0 * S0, false, lane);
    if (lane < 2) ws.detD[lane] = dv;
    __syncwarp();
    const int Rleaf = n - 1;
    Acc<R> ar, ai;
    ar.init();
    ai.init();
    bool paired = false;
    if constexpr (twin_leaves<R>() && RFMAX >= kTreeLeaf) {
        if (Rleaf == kTreeLeaf) {
            const int h = lane >> 4;
            flat_pair<R, kTreeLeaf>(ws.stack + h * S0 * S0, dv, 0, lane & 15, ar, ai);
            paired = true;
        }
    }
    if (!paired) {
        const int B = Rleaf > RF ? Rleaf - RF : 0;
        const int Rf = Rleaf - B;
        const cx<R> *E = ws.stack;
        int S = S0;
        const cx<R> *ndet = ws.detD;
        cx<R> *dbuf = ws.bdet;
        size_t bo = 0;
        for (int lb = 0; lb < B; ++lb) {
            const int nparent = 2 << lb;
            cx<R> *out = ws.bfs + bo;
            expand_level<R>(E, S, 2 * nparent, 0, out, ndet, dbuf, ws.wrow, ws.bip, lane);
            bo += (size_t)(2 * nparent) * (S - 2) * (S - 2);
            E = out;
            S -= 2;
            ndet = dbuf;
            dbuf = (dbuf == ws.bdet) ? ws.bdet + 32 : ws.bdet;
        }
        const int hl = lane & 15;  // half-warp h = lane >> 4 takes point h
        if (hl < (1 << Rleaf)) {
            const int nb = hl >> Rf;                  // the node's breadth-first choices
            const int node = ((lane >> 4) << B) | nb;  // its index in the last level
            flat_dispatch<R, RFMAX>(Rf, E + (size_t)node * S * S, ndet[node], __popc(nb) & 1, hl & ((1 << Rf) - 1),
                                    ar, ai);
        }
    }
    __syncwarp();
    if constexpr (OUT == kOutShare) {  // the lane's share of its half-warp's point, in sa
        sa = tree_result<R, kOutShare>(ar, ai);
        sb = mk<double>(0.0, 0.0);
    } else {
        const Acc<R> hr = group_pair<R, 16>(ar), hi = group_pair<R, 16>(ai);
        auto from = [&](int src) {  // half-warp src / 16's pair, from its first lane
            PairSum<R> p;
            p.re.s = __shfl_sync(FULL, hr.s, src);
            p.re.c = __shfl_sync(FULL, hr.c, src);
            p.im.s = __shfl_sync(FULL, hi.s, src);
            p.im.c = __shfl_sync(FULL, hi.c, src);
            return p;
        };
        const PairSum<R> pa = from(0), pb = from(16);
        if constexpr (OUT == kOutPair) {
            sa = pa;
            sb = pb;
        } else {
            sa = mk<double>(pair_value<R>(pa.re), pair_value<R>(pa.im));
            sb = mk<double>(pair_value<R>(pb.re), pair_value<R>(pb.im));
        }
    }
}

}  // namespace single

namespace pairs {

// ----------------------------------------------------------------------------
// Pair-block Schur tree for the Keldysh sum.
//
// Every vertex diagonal of M_down is g^<(0) - i alpha.  With alpha at the
// occupation Im g^<(0) (the Hartree-cancelling choice of App. E) that diagonal
// is zero, and at particle-hole symmetry M_down is then skew-symmetric for
// every Keldysh index vector (g^>(tau) = conj g^<(tau)), so every odd leading
// minor vanishes.  The tree therefore eliminates the vertices two at a time,
// (1,2), (3,4), ..., with 2x2 block pivots B whose determinants are the even
// leading minors, and resolves a lone last vertex (odd n) without a reciprocal.
//
// A node with R remaining vertices is an S x S matrix, S = 2R + 2: rows and
// columns 0, 1 are the two copies of the measurement row/column (a_1 = 0, 1),
// row 2 + 2i + a is the i-th remaining vertex with Keldysh index a.  Entries
// joining a row to its own other copy are never read and not formed.
//
//   root    vertices 1, 2 eliminated from the pair values for a_2 = s (two
//           roots), R_r = n - 2 vertices left;
//   levels  depth first, one vertex pair (a_{2l+1}, a_{2l+2}) per level, four
//           children per node, down to a leaf of at most kLeafMax vertices;
//   leaf    breadth-first pair levels (all four children of every node), then
//           each lane resolves the last F vertices of one node along one
//           choice path in registers (2^F paths per node).
// For n <= 6 both roots form one leaf group and there is no walk.
// ----------------------------------------------------------------------------
constexpr int kLeafMax = 6;

struct TreeShape {
    int Rr;     // vertices left after the root block, n - 2
    int dfl;    // depth-first pair levels below the root
    int Rleaf;  // vertices left at a leaf
    int g;      // 1: both roots form one leaf group (no walk)
    int lbits;  // bits of a leaf's index: a_2, then two per depth-first level
};

__host__ __device__ inline TreeShape tree_shape(int n) {
    TreeShape t;
    t.Rr = n > 2 ? n - 2 : 0;
    t.dfl = t.Rr > kLeafMax ? (t.Rr - kLeafMax + 1) / 2 : 0;
    t.Rleaf = t.Rr - 2 * t.dfl;
    t.g = t.Rr <= 4 ? 1 : 0;
    t.lbits = t.g ? 0 : 1 + 2 * t.dfl;
    return t;
}

// Breadth-first pair levels below a leaf of Rleaf vertices for the tuned flat
// depth RF; each lane then resolves F = Rleaf - 2 B vertices (RF - 1 <= F <= RF).
__host__ __device__ inline int bfs_levels(int Rleaf, int RF) { return Rleaf > RF ? (Rleaf - RF + 1) / 2 : 0; }

__host__ __device__ inline size_t zmax(size_t a, size_t b) { return a > b ? a : b; }

// entries of tree level l (the root level holds both roots when g = 1)
__host__ __device__ inline size_t level_entries(const TreeShape &t, int l) {
    const size_t S = 2 * (size_t)(t.Rr - 2 * l) + 2;
    return (l == 0 && t.g ? 2 : 1) * S * S;
}

// Tree-stack entries of order n: all levels (part 0), or with the split stack
// the levels of S <= gs_level (part 1, shared memory) or S > gs_level (part 2,
// device memory).
__host__ __device__ inline size_t stack_entries_n(int n, int part, int gs_level) {
    if (n < 3) return 0;
    const TreeShape t = tree_shape(n);
    size_t tot = 0;
    for (int l = 0; l <= t.dfl; ++l) {
        const int S = 2 * (t.Rr - 2 * l) + 2;
        if (part == 0 || ((S > gs_level) == (part == 2))) tot += level_entries(t, l);
    }
    return tot;
}

// a launch serves every order up to n_max with one layout
__host__ __device__ inline size_t stack_cap(int n_max, int part, int gs_level) {
    size_t m = 0;
    for (int n = 3; n <= n_max; ++n) m = zmax(m, stack_entries_n(n, part, gs_level));
    return m;
}

// Buffers of the breadth-first levels and of the general pair step.
struct LeafBufs {
    size_t bfs;   // all breadth-first levels of one leaf group
    size_t wrow;  // scaled pivot rows, 2 per child column
    size_t bip;   // B^-1 per child (4 entries)
    size_t half;  // nodes of the widest breadth-first level (det buffer: two levels)
};

__host__ __device__ inline LeafBufs leaf_bufs(int n_max, int RF) {
    LeafBufs m = {0, 0, 0, 0};
    for (int n = 3; n <= n_max; ++n) {
        const TreeShape t = tree_shape(n);
        const int B = bfs_levels(t.Rleaf, RF);
        size_t nodes = (size_t)1 << t.g, bfs = 0;
        for (int b = 1; b <= B; ++b) {
            nodes *= 4;
            const size_t S = 2 * (size_t)(t.Rleaf - 2 * b) + 2;
            bfs += nodes * S * S;
            m.wrow = zmax(m.wrow, 2 * nodes * S);
            m.bip = zmax(m.bip, 4 * nodes);
            m.half = zmax(m.half, nodes);
        }
        m.bfs = zmax(m.bfs, bfs);
        for (int l = 1; l <= t.dfl; ++l) {  // depth-first children wider than a warp: the general step
            const size_t S = 2 * (size_t)(t.Rr - 2 * l) + 2;
            if (S > 32) {
                m.wrow = zmax(m.wrow, 2 * S);
                m.bip = zmax(m.bip, 4);
            }
        }
    }
    return m;
}

// packed pair values with the measurement column (P and Rr: blocks of k + 1
// entries for the vertices k = 1 .. n_max)
__host__ __device__ inline size_t pair_entries(int n_max) { return (size_t)n_max * (n_max + 3); }

// Shared memory of one warp.  gs_level = 0: the whole tree stack and the point
// times in shared memory.  gs_level > 0 (split stack): the levels wider than
// gs_level and the point times in a per-warp slice of device memory.
template <class R>
__host__ __device__ inline size_t warp_smem_bytes_at(int n_max, int RF, int gs_level) {
    const LeafBufs lb = leaf_bufs(n_max, RF);
    size_t c = (gs_level ? stack_cap(n_max, 1, gs_level) : stack_cap(n_max, 0, 0)) + pair_entries(n_max) +
               n_max + 2 + 8 * (size_t)n_max + 20 * (size_t)tree_shape(n_max).dfl + lb.bfs + lb.wrow + lb.bip +
               2 * lb.half;
    size_t bytes = (c * sizeof(cx<R>) + 15) & ~(size_t)15;
    if (!gs_level) bytes += 32 * (size_t)(n_max + 1) * sizeof(double);
    return (bytes + 127) & ~(size_t)127;
}

// Split-stack boundary: the widest levels go to device memory, two rows at a
// time, until a warp's shared memory lets the SM hold the warps its bound pipe
// needs (FP64: 6 warps keep GB300's two FP64 lanes per SM busy; mixed: 12).
// Never a leaf (S <= 14) or its parent (S <= 18): the last depth-first step and
// the breadth-first and flat phases work in shared memory only.
template <class R>
__host__ __device__ inline int gs_level_of(int n_max, int RF) {
    const size_t budget = sizeof(R) == 8 ? 36 * 1024 : 18 * 1024;
    int lev = 2 * n_max;
    while (lev > 18 && warp_smem_bytes_at<R>(n_max, RF, lev) > budget) lev -= 2;
    return lev;
}

// Shared memory of one warp; with the split stack (gs) the wide top levels of
// the tree live in a per-warp slice of device memory (FP64 orders whose whole
// stack exceeds the 227 KB a block can address, and the orders the stack
// policy names).
template <class R>
__host__ __device__ inline size_t warp_smem_bytes(int n_max, int RF, bool gs = false) {
    return warp_smem_bytes_at<R>(n_max, RF, gs ? gs_level_of<R>(n_max, RF) : 0);
}

// Device-memory slice of one warp with the split stack: the wide levels, one
// spare entry, and the point times of the chunk.
template <class R>
__host__ __device__ inline size_t gstack_entries(int n_max, int RF) {
    return stack_cap(n_max, 2, gs_level_of<R>(n_max, RF)) + 1 +
           (32 * (size_t)(n_max + 1) * sizeof(double) + sizeof(cx<R>) - 1) / sizeof(cx<R>);
}

template <class R>
struct WarpSmem {
    cx<R> *stack;   // tree levels with S <= gs_level (every level without the split stack)
    cx<R> *gstack;  // split stack: the levels with S > gs_level in device memory, or null
    cx<R> *P;       // vertex k's block at o_k = (k-1)(k+2)/2: P[o_k + j] = g^>(u_j - u_k), 0 <= j < k,
                    // and P[o_k + k] = measurement-column entry (k, a_k = 1)
    cx<R> *Rr;      // Rr[o_k + j] = g^<(u_j - u_k); Rr[o_k + k] = column entry (k, a_k = 0)
    cx<R> *detD;    // det M_down of the eliminated vertices per tree level (level 0: both roots when g = 1)
    cx<R> *lr;      // root: per block index L(., 0), L(., 1), B^-1 R(., 0), B^-1 R(., 1) (8 entries)
    cx<R> *piv;     // per depth-first parent level: its four children's B^-1 and det B (node_pivots)
    cx<R> *bfs;     // breadth-first levels (all nodes of one level contiguous)
    cx<R> *wrow;    // general pair step: B^-1 (row p; row q) per child column
    cx<R> *bip;     // general pair step: B^-1 per child
    cx<R> *bdet;    // det M_down per breadth-first node, two levels of `half` nodes
    int half;
    double *upt;    // [32][n_max+1] point times of the chunk (u_0 = t; store_time form); device memory with the split stack
    int gs_level;   // split stack: levels with S > gs_level in device memory
};

template <class R>
__device__ __forceinline__ WarpSmem<R> carve(unsigned char *base, int n_max, int RF, cx<R> *gstack = nullptr) {
    WarpSmem<R> w;
    const LeafBufs lb = leaf_bufs(n_max, RF);
    cx<R> *p = reinterpret_cast<cx<R> *>(base);
    w.gstack = gstack;
    w.gs_level = gstack ? gs_level_of<R>(n_max, RF) : 0;
    w.stack = p;
    p += gstack ? stack_cap(n_max, 1, w.gs_level) : stack_cap(n_max, 0, 0);
    const int npair = n_max * (n_max + 3) / 2;
    w.P = p;
    p += npair;
    w.Rr = p;
    p += npair;
    w.detD = p;
    p += n_max + 2;
    w.lr = p;
    p += 8 * n_max;
    w.piv = p;
    p += 20 * tree_shape(n_max).dfl;
    w.bfs = p;
    p += lb.bfs;
    w.wrow = p;
    p += lb.wrow;
    w.bip = p;
    p += lb.bip;
    w.bdet = p;
    p += 2 * lb.half;
    w.half = (int)lb.half;
    size_t off = (reinterpret_cast<unsigned char *>(p) - base + 15) & ~(size_t)15;
    w.upt = gstack ? reinterpret_cast<double *>(gstack + stack_cap(n_max, 2, w.gs_level) + 1)
                   : reinterpret_cast<double *>(base + off);
    return w;
}

// packed offset of vertex k's block
__device__ __forceinline__ int vblk(int k) { return (int)((unsigned)((k - 1) * (k + 2)) >> 1); }

// Leaf term after the last vertex pair (p, q), also without a reciprocal:
//   delta = det B,  x_c = (m_cp, m_cq) adj(B) (m_pc, m_qc)^T,
//   det'^2 (S_00 - S_11) = det^2 delta (delta (m_00 - m_11) - (x_0 - x_1)).
template <class R>
__device__ __forceinline__ cx<R> leaf_pair(cx<R> m00, cx<R> m11, cx<R> m0p, cx<R> m0q, cx<R> mp0, cx<R> mq0,
                                           cx<R> m1p, cx<R> m1q, cx<R> mp1, cx<R> mq1, cx<R> mpp, cx<R> mpq,
                                           cx<R> mqp, cx<R> mqq, cx<R> det) {
    const cx<R> del = cfms(cmul(mpp, mqq), mpq, mqp);
    // adj(B) (m_pc; m_qc) = (mqq m_pc - mpq m_qc; mpp m_qc - mqp m_pc)
    const cx<R> v00 = cfms(cmul(mqq, mp0), mpq, mq0), v01 = cfms(cmul(mpp, mq0), mqp, mp0);
    const cx<R> v10 = cfms(cmul(mqq, mp1), mpq, mq1), v11 = cfms(cmul(mpp, mq1), mqp, mp1);
    const cx<R> x0 = cfma(cmul(m0p, v00), m0q, v01);
    const cx<R> x1 = cfma(cmul(m1p, v10), m1q, v11);
    const cx<R> r = cfms(csub(x0, x1), del, csub(m00, m11));  // (x0 - x1) - delta (m00 - m11)
    return cmul(cmul(det, det), cmul(del, cneg(r)));
}

// Register tail of a path: m is M x M (copies 0, 1 and M - 2 <= 3 vertices).
template <class R, int M>
__device__ __forceinline__ cx<R> reg_tail(cx<R> (&m)[M][M], cx<R> det) {
    if constexpr (M == 3) {
        return leaf_term(m[0][0], m[1][1], m[0][2], m[2][0], m[1][2], m[2][1], m[2][2], det);
    } else if constexpr (M == 4) {
        return leaf_pair(m[0][0], m[1][1], m[0][2], m[0][3], m[2][0], m[3][0], m[1][2], m[1][3], m[2][1], m[3][1],
                         m[2][2], m[2][3], m[3][2], m[3][3], det);
    } else {
        static_assert(M == 5, "at most three vertices after the first pair");
        // pair (2, 3) with its pivot, then the lone vertex 4
        const cx<R> del = cfms(cmul(m[2][2], m[3][3]), m[2][3], m[3][2]);
        det = cmul(det, del);
        const cx<R> id = crcp(del);
        const int keep[3] = {0, 1, 4};
        cx<R> w0[3], w1[3], t[3][3];
#pragma unroll
        for (int y = 0; y < 3; ++y) {
            const cx<R> e2 = m[2][keep[y]], e3 = m[3][keep[y]];
            w0[y] = cmul(cfms(cmul(m[3][3], e2), m[2][3], e3), id);
            w1[y] = cmul(cfms(cmul(m[2][2], e3), m[3][2], e2), id);
        }
#pragma unroll
        for (int x = 0; x < 3; ++x)
#pragma unroll
            for (int y = 0; y < 3; ++y) {
                if (x < 2 && y < 2 && x != y) continue;
                t[x][y] = cfms(cfms(m[keep[x]][keep[y]], m[keep[x]][2], w0[y]), m[keep[x]][3], w1[y]);
            }
        return leaf_term(t[0][0], t[1][1], t[0][2], t[2][0], t[1][2], t[2][1], t[2][2], det);
    }
}

// Flat phase: one lane resolves the F remaining vertices of node matrix E
// (S = 2F + 2) along the choice path `path` (bit q = Keldysh index of the q-th
// remaining vertex) and returns its (unsigned) leaf term.  F <= 2: the leaf
// formulas straight from E.  F >= 3: the first pair is eliminated with its
// pivot while the rows and columns of the path are gathered into registers.
template <class R, int F>
__device__ __forceinline__ cx<R> flat_term(const cx<R> *E, cx<R> det, int path) {
    constexpr int S = 2 * F + 2;
    const int p = 2 + (path & 1);
    if constexpr (F == 1) {
        return leaf_term(E[0], E[S + 1], E[p], E[p * S], E[S + p], E[p * S + 1], E[p * S + p], det);
    } else {
        const int q = 4 + ((path >> 1) & 1);
        if constexpr (F == 2) {
            return leaf_pair(E[0], E[S + 1], E[p], E[q], E[p * S], E[q * S], E[S + p], E[S + q], E[p * S + 1],
                             E[q * S + 1], E[p * S + p], E[p * S + q], E[q * S + p], E[q * S + q], det);
        } else {
            constexpr int M = F;  // copies + the F - 2 vertices after the first pair
            int idx[M];
            idx[0] = 0;
            idx[1] = 1;
#pragma unroll
            for (int r = 2; r < M; ++r) idx[r] = 2 + 2 * r + ((path >> r) & 1);
            const cx<R> bpp = E[p * S + p], bpq = E[p * S + q], bqp = E[q * S + p], bqq = E[q * S + q];
            const cx<R> del = cfms(cmul(bpp, bqq), bpq, bqp);
            det = cmul(det, del);
            const cx<R> id = crcp(del);
            cx<R> w0[M], w1[M], m[M][M];
#pragma unroll
            for (int y = 0; y < M; ++y) {
                const cx<R> epy = E[p * S + idx[y]], eqy = E[q * S + idx[y]];
                w0[y] = cmul(cfms(cmul(bqq, epy), bpq, eqy), id);
                w1[y] = cmul(cfms(cmul(bpp, eqy), bqp, epy), id);
            }
#pragma unroll
            for (int x = 0; x < M; ++x) {
                const cx<R> exp = E[idx[x] * S + p], exq = E[idx[x] * S + q];
#pragma unroll
                for (int y = 0; y < M; ++y) {
                    if (x < 2 && y < 2 && x != y) continue;  // copy cross terms are never used
                    m[x][y] = cfms(cfms(E[idx[x] * S + idx[y]], exp, w0[y]), exq, w1[y]);
                }
            }
            return reg_tail<R, M>(m, det);
        }
    }
}

template <class R, int RFMAX>
__device__ __forceinline__ cx<R> flat_dispatch(int F, const cx<R> *E, cx<R> det, int path) {
    switch (F) {  // 1 <= F <= RFMAX
        case 1: return flat_term<R, 1>(E, det, path);
        case 2: return flat_term<R, 2>(E, det, path);
        case 3: if (RFMAX >= 3) return flat_term<R, (RFMAX >= 3 ? 3 : 2)>(E, det, path); break;
        case 4: if (RFMAX >= 4) return flat_term<R, (RFMAX >= 4 ? 4 : 2)>(E, det, path); break;
        default: if (RFMAX >= 5) return flat_term<R, (RFMAX >= 5 ? 5 : 2)>(E, det, path); break;
    }
    return mk<R>(0, 0);
}

// Root for a_2 = s: vertices 1 and 2 eliminated with the pivot block
// B = [[dv, M(1,2)], [M(2,1), dv]] (M(1,2) and M(2,1) follow a_2; vertex 1's own
// index only reaches the measurement row and column, so the two copies carry
// it).  Block index i: 0 = the copies, i >= 1 = vertex i + 2 with both indices.
// Entry (x, y) = base(x, y) - L_x . B^-1 R_y with L_x = (M(x,1), M(x,2)) and
// R_y = (M(1,y), M(2,y)).  Writes the S x S root (S = 2n - 2) and det B.
template <class R>
__device__ void build_root(const WarpSmem<R> &ws, int n, int s, cx<R> d, cx<R> dv, cx<R> *__restrict__ out,
                           cx<R> *det_out, int lane) {
    const int nb = n - 1, S = 2 * nb;
    const cx<R> m12 = sel<R>(s, ws.Rr[3], ws.P[3]);
    const cx<R> m21 = nconj(sel<R>(s, ws.P[3], ws.Rr[3]));
    const cx<R> del = cfms(cmul(dv, dv), m12, m21);
    const cx<R> id = crcp(del);
    if (lane < nb) {
        cx<R> l00, l01, l10, l11, r00, r01, r10, r11;  // l_a = L(i, a), r_b = R(i, b), two components each
        if (lane == 0) {
            l00 = ws.P[0];  // M(0,1), a_1 = 0
            l10 = ws.Rr[0];
            l01 = l11 = sel<R>(s, ws.Rr[2], ws.P[2]);  // M(0,2)
            r00 = ws.Rr[1];  // M(1,0), a_1 = 0
            r10 = ws.P[1];
            r01 = r11 = sel<R>(s, ws.P[4], ws.Rr[4]);  // M(2,0)
        } else {
            const int o = vblk(lane + 2);
            l00 = nconj(ws.Rr[o + 1]);  // M(v,1), a_v = 0
            l10 = nconj(ws.P[o + 1]);
            l01 = nconj(ws.Rr[o + 2]);  // M(v,2)
            l11 = nconj(ws.P[o + 2]);
            r00 = ws.P[o + 1];  // M(1,v), a_v = 0
            r10 = ws.Rr[o + 1];
            r01 = ws.P[o + 2];  // M(2,v)
            r11 = ws.Rr[o + 2];
        }
        // B^-1 = (1 / delta) [[dv, -M12], [-M21, dv]]
        cx<R> *lr = ws.lr + 8 * lane;
        lr[0] = l00;
        lr[1] = l01;
        lr[2] = l10;
        lr[3] = l11;
        lr[4] = cmul(cfms(cmul(dv, r00), m12, r01), id);
        lr[5] = cmul(cfms(cmul(dv, r01), m21, r00), id);
        lr[6] = cmul(cfms(cmul(dv, r10), m12, r11), id);
        lr[7] = cmul(cfms(cmul(dv, r11), m21, r10), id);
    }
    __syncwarp();
    // lane -> block (bx, by), stepped by 32 blocks without divisions.  The base entry follows
    // the later vertex's index: above the diagonal (row 0: the measurement row) the column's,
    // below it (column 0: the measurement column, stored as is) the row's.
    const int sq = 32 / nb, sr = 32 - sq * nb;
    int bx = lane / nb, by = lane - bx * nb;
    for (int bid = lane; bid < nb * nb; bid += 32) {
        const bool up = bx < by, diag = bx == by;
        const int v = bx + 2, w = by + 2;
        const int idx = up ? vblk(w) + (bx ? v : 0) : vblk(v) + (by ? w : v);
        const cx<R> vP = ws.P[diag ? 0 : idx], vR = ws.Rr[diag ? 0 : idx];
        const cx<R> *lx = ws.lr + 8 * bx, *wy = ws.lr + 8 * by + 4;
        const R sg = (!up && by) ? R(-1) : R(1);  // lower entries of vertex pairs: -conj
        const cx<R> lo0 = mk<R>(sg * vR.re, vR.im), lo1 = mk<R>(sg * vP.re, vP.im);
        const cx<R> dd = bx == 0 ? d : dv;
        const cx<R> b00 = diag ? dd : (up ? vP : lo0), b01 = up ? vR : lo0;
        const cx<R> b10 = up ? vP : lo1, b11 = diag ? dd : (up ? vR : lo1);
        cx<R> *o = out + (2 * bx) * S + 2 * by;
        o[0] = cfms(cfms(b00, lx[0], wy[0]), lx[1], wy[1]);
        o[S + 1] = cfms(cfms(b11, lx[2], wy[2]), lx[3], wy[3]);
        if (!diag) {
            o[1] = cfms(cfms(b01, lx[0], wy[2]), lx[1], wy[3]);
            o[S] = cfms(cfms(b10, lx[2], wy[0]), lx[3], wy[1]);
        }
        by += sr;
        bx += sq;
        if (by >= nb) {
            by -= nb;
            ++bx;
        }
    }
    if (lane == 0) *det_out = del;
    __syncwarp();
}

// Pivot data of the four children of a node (S x S, vertex pair in rows 2-3 and
// 4-5), once per node: child (a, b) has the block B = E[{p,q},{p,q}], p = 2 + a,
// q = 4 + b, and pv[5 (2a + b) + 0..3] = B^-1 (row major), pv[5 (2a + b) + 4] =
// det B.  Four lanes work; the depth-first steps to the node's children read it.
template <class R>
__device__ __forceinline__ void node_pivots(const cx<R> *__restrict__ E, int S, cx<R> *pv, int lane) {
    if (lane < 4) {
        const int p = 2 + (lane >> 1), q = 4 + (lane & 1);
        const cx<R> bpp = E[p * S + p], bpq = E[p * S + q], bqp = E[q * S + p], bqq = E[q * S + q];
        const cx<R> del = cfms(cmul(bpp, bqq), bpq, bqp);
        const cx<R> id = crcp(del);
        cx<R> *o = pv + 5 * lane;
        o[0] = cmul(bqq, id);
        o[1] = cneg(cmul(bpq, id));
        o[2] = cneg(cmul(bqp, id));
        o[3] = cmul(bpp, id);
        o[4] = del;
    }
    __syncwarp();
}

// One child of a depth-first pair step: the vertices in rows 2-3 and 4-5 of
// the S x S parent fixed to (a, b), pivot block B = E[{p,q},{p,q}] (p = 2 + a,
// q = 4 + b) with B^-1 and det B in pv (node_pivots); the (S - 4) x (S - 4)
// child keeps parent rows/columns 0, 1, 6, 7, ...  Entry E_xy - E_xp W0_y -
// E_xq W1_y with (W0; W1) = B^-1 (E_p.; E_q.).  A step is latency-bound, so
// every load is issued first.  Children of 2T = 12, 14 or 16 rows: lanes 0-15
// take the even rows, lanes 16-31 the odd rows, column c2 = lane & 15.
template <class R, int T>
__device__ __forceinline__ void pair_one_t(const cx<R> *__restrict__ in, int a, int b, const cx<R> *pv,
                                           cx<R> *__restrict__ out, const cx<R> *detD_in, cx<R> *detD_out,
                                           int lane) {
    constexpr int S2 = 2 * T, S = S2 + 4;
    const int p = 2 + a, q = 4 + b;
    const int c2 = lane & 15, rsub = lane >> 4;
    const bool act = c2 < S2;
    const int c = c2 < 2 ? c2 : c2 + 4;
    const cx<R> b00 = pv[0], b01 = pv[1], b10 = pv[2], b11 = pv[3];
    cx<R> epc = mk<R>(0, 0), eqc = mk<R>(0, 0), ev[T], ep[T], eq[T];
#pragma unroll
    for (int t = 0; t < T; ++t) ev[t] = ep[t] = eq[t] = mk<R>(0, 0);
    if (act) {
        epc = in[p * S + c];
        eqc = in[q * S + c];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int r2 = rsub + 2 * t;
            const int r = r2 < 2 ? r2 : r2 + 4;
            ev[t] = in[r * S + c];
            ep[t] = in[r * S + p];
            eq[t] = in[r * S + q];
        }
    }
    if (lane == 0) *detD_out = cmul(*detD_in, pv[4]);
    if (act) {
        const cx<R> w0 = cfma(cmul(b00, epc), b01, eqc);
        const cx<R> w1 = cfma(cmul(b10, epc), b11, eqc);
#pragma unroll
        for (int t = 0; t < T; ++t) out[(rsub + 2 * t) * S2 + c2] = cfms(cfms(ev[t], ep[t], w0), eq[t], w1);
    }
    __syncwarp();
}

// Wider children (S - 4 = 18 .. 32 rows): lane = column, rows in batches
// (eight in FP32, four in FP64) with the batch's loads issued first.
template <class R>
__device__ __forceinline__ void pair_one_wide(const cx<R> *__restrict__ in, int S, int a, int b, const cx<R> *pv,
                                              cx<R> *__restrict__ out, const cx<R> *detD_in, cx<R> *detD_out,
                                              int lane) {
    constexpr int NB = sizeof(R) == 4 ? 8 : 4;  // rows per batch (FP64: register budget)
    const int S2 = S - 4;
    const int p = 2 + a, q = 4 + b;
    if (lane == 0) *detD_out = cmul(*detD_in, pv[4]);
    if (lane < S2) {
        const int c = lane < 2 ? lane : lane + 4;
        const cx<R> epc = in[p * S + c], eqc = in[q * S + c];
        const cx<R> w0 = cfma(cmul(pv[0], epc), pv[1], eqc);
        const cx<R> w1 = cfma(cmul(pv[2], epc), pv[3], eqc);
        for (int r0 = 0; r0 < S2; r0 += NB) {
            cx<R> ev[NB], ep[NB], eq[NB];
#pragma unroll
            for (int t = 0; t < NB; ++t) {
                const int r2 = r0 + t < S2 ? r0 + t : S2 - 1;  // a clamped duplicate of the last row
                const int r = r2 < 2 ? r2 : r2 + 4;
                ev[t] = in[r * S + c];
                ep[t] = in[r * S + p];
                eq[t] = in[r * S + q];
            }
#pragma unroll
            for (int t = 0; t < NB; ++t)
                if (r0 + t < S2) out[(r0 + t) * S2 + lane] = cfms(cfms(ev[t], ep[t], w0), eq[t], w1);
        }
    }
    __syncwarp();
}

// General cooperative pair step.  nchild = 4 nparent children of the S x S
// parents (contiguous in `in`): child j from parent j >> 2 with
// (a, b) = ((j >> 1) & 1, j & 1); or one child (nchild = 1) with (a1, b1).  The
// (S-4) x (S-4) children are contiguous in `out`.  Breadth-first levels, and
// depth-first children wider than a warp.
template <class R>
__device__ void pair_level(const cx<R> *__restrict__ in, int S, int nchild, int a1, int b1, cx<R> *__restrict__ out,
                           const cx<R> *detD_in, cx<R> *detD_out, cx<R> *__restrict__ wrow, cx<R> *binv, int lane,
                           const cx<R> *pv = nullptr) {
    const int S2 = S - 4;
    if (pv) {  // one child whose pivot data the node already holds
        if (lane < 4) binv[lane] = pv[lane];
        if (lane == 0) detD_out[0] = cmul(detD_in[0], pv[4]);
    }
    // pivot blocks: B^-1 and the running det M_down per child
    for (int j = lane; j < (pv ? 0 : nchild); j += 32) {
        const int a = nchild == 1 ? a1 : (j >> 1) & 1, b = nchild == 1 ? b1 : j & 1;
        const int pj = nchild == 1 ? 0 : j >> 2;
        const cx<R> *E = in + (size_t)pj * S * S;
        const int p = 2 + a, q = 4 + b;
        const cx<R> bpp = E[p * S + p], bpq = E[p * S + q], bqp = E[q * S + p], bqq = E[q * S + q];
        const cx<R> del = cfms(cmul(bpp, bqq), bpq, bqp);
        const cx<R> id = crcp(del);
        binv[4 * j] = cmul(bqq, id);
        binv[4 * j + 1] = cneg(cmul(bpq, id));
        binv[4 * j + 2] = cneg(cmul(bqp, id));
        binv[4 * j + 3] = cmul(bpp, id);
        detD_out[j] = cmul(detD_in[pj], del);
    }
    __syncwarp();
    // scaled pivot rows (W0; W1) = B^-1 (row p; row q) on the child's columns
    for (int e = lane; e < nchild * S2; e += 32) {
        const int j = e / S2, c2 = e - j * S2;
        const int a = nchild == 1 ? a1 : (j >> 1) & 1, b = nchild == 1 ? b1 : j & 1;
        const int pj = nchild == 1 ? 0 : j >> 2;
        const cx<R> *E = in + (size_t)pj * S * S;
        const int p = 2 + a, q = 4 + b, c = c2 < 2 ? c2 : c2 + 4;
        const cx<R> epc = E[p * S + c], eqc = E[q * S + c];
        const cx<R> *bi = binv + 4 * j;
        wrow[2 * e] = cfma(cmul(bi[0], epc), bi[1], eqc);
        wrow[2 * e + 1] = cfma(cmul(bi[2], epc), bi[3], eqc);
    }
    __syncwarp();
    // Only entries that are ever read are built: a choice path takes one copy of every vertex (and
    // one measurement copy per determinant), so the entry joining row r2 to its row's other copy,
    // column r2 ^ 1, is never used.  lane -> (child j, row r2, used column cc of W = S2 - 1) stepped
    // by 32 entries without divisions.
    const int W = S2 - 1;
    const int dr = 32 / W, dc = 32 - dr * W;
    int r2 = lane / W, cc = lane - r2 * W, j = 0;
    while (r2 >= S2) {
        r2 -= S2;
        ++j;
    }
    const int total = nchild * S2 * W;
    for (int e = lane; e < total; e += 32) {
        const int c2 = cc < (r2 ^ 1) ? cc : cc + 1;
        const int a = nchild == 1 ? a1 : (j >> 1) & 1, b = nchild == 1 ? b1 : j & 1;
        const int pj = nchild == 1 ? 0 : j >> 2;
        const int p = 2 + a, q = 4 + b;
        const int r = r2 < 2 ? r2 : r2 + 4;
        const int c = c2 < 2 ? c2 : c2 + 4;
        const cx<R> *E = in + (size_t)pj * S * S;
        const cx<R> *wr = wrow + 2 * (j * S2 + c2);
        out[((size_t)j * S2 + r2) * S2 + c2] = cfms(cfms(E[r * S + c], E[r * S + p], wr[0]), E[r * S + q], wr[1]);
        cc += dc;
        r2 += dr;
        if (cc >= W) {
            cc -= W;
            ++r2;
        }
        while (r2 >= S2) {
            r2 -= S2;
            ++j;
        }
    }
    __syncwarp();
}

// One depth-first pair step from an S x S parent.
// pv: the parent's pivot data for this child (node_pivots).
template <class R>
__device__ __forceinline__ void pair_step(const WarpSmem<R> &ws, const cx<R> *in, int S, int a, int b,
                                          const cx<R> *pv, cx<R> *out, const cx<R> *detD_in, cx<R> *detD_out,
                                          int lane) {
    switch (S - 4) {
        case 12: pair_one_t<R, 6>(in, a, b, pv, out, detD_in, detD_out, lane); break;
        case 14: pair_one_t<R, 7>(in, a, b, pv, out, detD_in, detD_out, lane); break;
        case 16: pair_one_t<R, 8>(in, a, b, pv, out, detD_in, detD_out, lane); break;
        default:
            if (S - 4 <= 32)
                pair_one_wide<R>(in, S, a, b, pv, out, detD_in, detD_out, lane);
            else
                pair_level<R>(in, S, 1, a, b, out, detD_in, detD_out, ws.wrow, ws.bip, lane, pv);
            break;
    }
}

// Below a leaf group (1 << g matrices of Rleaf vertices at E, dets at ndet):
// B breadth-first pair levels, then the per-lane flat phase over the
// nodes x 2^F choice paths.  tpar: parity of the Keldysh indices fixed above.
template <class R, int RFMAX>
__device__ __forceinline__ void leaf_group(const WarpSmem<R> &ws, const cx<R> *E, const cx<R> *ndet, int g,
                                           int Rleaf, int B, int F, int tpar, Acc<R> &ar, Acc<R> &ai, int lane) {
    int S = 2 * Rleaf + 2;
    int nodes = 1 << g;
    cx<R> *dbuf = ws.bdet;
    size_t bo = 0;
    for (int lb = 0; lb < B; ++lb) {
        cx<R> *out = ws.bfs + bo;
        pair_level<R>(E, S, 4 * nodes, 0, 0, out, ndet, dbuf, ws.wrow, ws.bip, lane);
        bo += (size_t)(4 * nodes) * (S - 4) * (S - 4);
        E = out;
        S -= 4;
        nodes *= 4;
        ndet = dbuf;
        dbuf = (dbuf == ws.bdet) ? ws.bdet + ws.half : ws.bdet;
    }
    const int combos = nodes << F;
    for (int cb = lane; cb < combos; cb += 32) {
        const int node = cb >> F, path = cb & ((1 << F) - 1);
        cx<R> term = flat_dispatch<R, RFMAX>(F, E + (size_t)node * S * S, ndet[node], path);
        if ((tpar ^ __popc(node) ^ __popc(path)) & 1) term = cneg(term);
        ar.add(term.re);
        ai.add(term.im);
    }
    __syncwarp();
}

// Keldysh sum for one point whose times are in u[0..n] (u_0 = t).
// Returns sum_{a_2..a_n} (-1)^{a_2+..+a_n} det M_down^2 (S00(0) - S00(1)),
// i.e. sum_a (-1)^{|a|} det M_up det M_down (without the i^n factor).
// The depth-first walk covers the subtree `sub` of 2^split: the first `split`
// bits of the leaf index (a_2, then two per level) follow sub; split = 0: the
// whole tree.
template <class R, int RFMAX, bool GS, int OUT = kOutTotal>
__device__ typename SumOut<R, OUT>::type keldysh_sum(const WarpSmem<R> &ws, const double *u, int n, int n_max,
                                                     cx<R> d, cx<R> dv,
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
        interp_pair_u<R>(tab, inv_h, s0, L, u, j, k, gl, gg);
        const int ok = p - j + k - 1;  // vertex k's block: (k-1)(k+2)/2
        ws.P[ok + j] = gg;
        ws.Rr[ok + j] = gl;
        if (j == 0) {  // measurement column of vertex k: g^<(u_k - t), g^>(u_k - t) for the charge
            cx<R> c0 = nconj(gl), c1 = nconj(gg);
            if (col) interp_col_u<R>(col, inv_h, s0, L, u, k, c0, c1);
            ws.Rr[ok + k] = c0;
            ws.P[ok + k] = c1;
        }
    }
    __syncwarp();
    Acc<R> ar, ai;
    ar.init();
    ai.init();
    if (n <= 2) {
        // orders 1 and 2 in closed form (every lane computes it, lane 0 adds it)
        cx<R> term;
        if (n == 1) {  // det M_up(a_1) = d dv - M(0,1) M(1,0), det M_down = dv
            term = cmul(dv, csub(cmul(ws.Rr[0], ws.P[1]), cmul(ws.P[0], ws.Rr[1])));
        } else {  // the root pair is the last pair
            const cx<R> one = mk<R>(1, 0);
            term = mk<R>(0, 0);
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const cx<R> m12 = sel<R>(s, ws.Rr[3], ws.P[3]), m21 = nconj(sel<R>(s, ws.P[3], ws.Rr[3]));
                const cx<R> m02 = sel<R>(s, ws.Rr[2], ws.P[2]), m20 = sel<R>(s, ws.P[4], ws.Rr[4]);
                const cx<R> t = leaf_pair(d, d, ws.P[0], m02, ws.Rr[1], m20, ws.Rr[0], m02, ws.P[1], m20, dv, m12,
                                          m21, dv, one);
                term = s ? csub(term, t) : t;
            }
        }
        if (lane == 0) {
            ar.add(term.re);
            ai.add(term.im);
        }
    } else {
        const TreeShape ts = tree_shape(n);
        const int B = bfs_levels(ts.Rleaf, RF);
        const int F = ts.Rleaf - 2 * B;
        const int Sr = 2 * ts.Rr + 2;
        // tree levels: [0, lg) in device memory (split stack, S > gs_level), the rest in shared memory
        int lg = 0;
        if (GS)
            while (lg <= ts.dfl && Sr - 4 * lg > ws.gs_level) ++lg;
        auto level = [&](int l) -> cx<R> * {
            const bool dev = GS && l < lg;
            size_t off = 0;
            for (int j = dev ? 0 : lg; j < l; ++j) off += level_entries(ts, j);
            return (dev ? ws.gstack : ws.stack) + off;
        };
        // Depth-first walk over the leaves (one leaf group, both roots, when g = 1).  Each code
        // path below has one call site, which keeps the inlined kernel small.
        const int free_bits = ts.g ? 0 : ts.lbits - split;
        const int nleaf = 1 << free_bits;
        for (int bl = 0; bl < nleaf; ++bl) {
            const int b = (sub << free_bits) | bl;  // leaf index: the subtree's fixed prefix, then bl
            int from = 0;
            if (bl) {  // rebuild from the level of the highest index bit that changed
                const int pos = __ffs(b) - 1;
                from = pos == ts.lbits - 1 ? 0 : (ts.lbits - pos) >> 1;
            }
            for (int l = from; l <= ts.dfl; ++l) {
                cx<R> *E = level(l);
                const int S = Sr - 4 * l;
                if (l == 0) {
                    for (int r = 0; r <= ts.g; ++r)  // a_2 = the top leaf-index bit, or both roots
                        build_root<R>(ws, n, ts.g ? r : (b >> (ts.lbits - 1)) & 1, d, dv, E + r * Sr * Sr,
                                      ws.detD + r, lane);
                } else {
                    const int a = (b >> (ts.lbits - 2 * l)) & 1, c = (b >> (ts.lbits - 2 * l - 1)) & 1;
                    pair_step<R>(ws, level(l - 1), S + 4, a, c, ws.piv + 20 * (l - 1) + 5 * (2 * a + c), E,
                                 ws.detD + l - 1, ws.detD + l, lane);
                }
                if (l < ts.dfl) node_pivots<R>(E, S, ws.piv + 20 * l, lane);
            }
            leaf_group<R, RFMAX>(ws, level(ts.dfl), ws.detD + ts.dfl, ts.g, ts.Rleaf, B, F,
                                 ts.g ? 0 : __popc(b) & 1, ar, ai, lane);
        }
    }
    return tree_result<R, OUT>(ar, ai);
}


}  // namespace pairs

// The two trees behind one interface for the determinant kernels.
struct SingleTree {
    template <class R>
    using Smem = single::WarpSmem<R>;
    template <class R>
    __host__ __device__ static size_t smem_bytes(int n_max, int RF, bool gs) {
        return single::warp_smem_bytes<R>(n_max, RF, gs);
    }
    template <class R>
    __host__ __device__ static size_t gstack_entries(int n_max, int RF) {
        return single::gstack_entries<R>(n_max, RF);
    }
    template <class R>
    __device__ static Smem<R> carve(unsigned char *base, int n_max, int RF, cx<R> *gstack) {
        return single::carve<R>(base, n_max, RF, gstack);
    }
    template <class R, int RFMAX, bool GS, int OUT = kOutTotal>
    __device__ static typename SumOut<R, OUT>::type sum(const Smem<R> &ws, const double *u, int n, int n_max, cx<R> d, cx<R> dv,
                                     const typename TabT<R>::V *tab, const typename TabT<R>::V *col, double inv_h,
                                     double s0, int L, int RF, int lane, int sub = 0, int split = 0) {
        return single::keldysh_sum<R, RFMAX, GS, OUT>(ws, u, n, n_max, d, dv, tab, col, inv_h, s0, L, RF, lane, sub,
                                                 split);
    }
    // depth-first levels above the tree leaf (5 vertices), one bit of the leaf index each
    static int leaf_bits(int n) { return n - 1 > single::kTreeLeaf ? n - 1 - single::kTreeLeaf : 0; }
};

struct PairTree {
    template <class R>
    using Smem = pairs::WarpSmem<R>;
    template <class R>
    __host__ __device__ static size_t smem_bytes(int n_max, int RF, bool gs) {
        return pairs::warp_smem_bytes<R>(n_max, RF, gs);
    }
    template <class R>
    __host__ __device__ static size_t gstack_entries(int n_max, int RF) {
        return pairs::gstack_entries<R>(n_max, RF);
    }
    template <class R>
    __device__ static Smem<R> carve(unsigned char *base, int n_max, int RF, cx<R> *gstack) {
        return pairs::carve<R>(base, n_max, RF, gstack);
    }
    template <class R, int RFMAX, bool GS, int OUT = kOutTotal>
    __device__ static typename SumOut<R, OUT>::type sum(const Smem<R> &ws, const double *u, int n, int n_max, cx<R> d, cx<R> dv,
                                     const typename TabT<R>::V *tab, const typename TabT<R>::V *col, double inv_h,
                                     double s0, int L, int RF, int lane, int sub = 0, int split = 0) {
        return pairs::keldysh_sum<R, RFMAX, GS, OUT>(ws, u, n, n_max, d, dv, tab, col, inv_h, s0, L, RF, lane, sub,
                                                split);
    }
    static int leaf_bits(int n) { return pairs::tree_shape(n).lbits; }
};

// One point per lane (small orders), registers only: the lane interpolates its
// own pairs, and for each a_2 and every choice path of vertices 3..N builds the
// path's N x N matrix -- rows/columns {copy a_1 = 0, copy a_1 = 1, vertices
// 3..N with their chosen Keldysh index}, vertices 1 and 2 already eliminated
// with their pivot block -- from the pair values, then resolves the rest with
// the leaf formulas.  All loops are unrolled, so every array index is static.
template <class R, int N>
__device__ __forceinline__ cx<double> lane_keldysh_sum(const double *u, cx<R> d, cx<R> dv,
                                                       const typename TabT<R>::V *tab,
                                                       const typename TabT<R>::V *col, double inv_h, double s0,
                                                       int L) {
    cx<R> P[N + 1][N + 1], Rr[N + 1][N + 1];  // P[j][k] = g^>(u_j - u_k), Rr[j][k] = g^<(u_j - u_k), j < k
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
    Acc<R> ar, ai;
    ar.init();
    ai.init();
    if constexpr (N == 1) {  // det M_up(a_1) = d dv - M(0,1) M(1,0), det M_down = dv
        const cx<R> term = cmul(dv, csub(cmul(Rr[0][1], C1[1]), cmul(P[0][1], C0[1])));
        ar.add(term.re);
        ai.add(term.im);
    } else {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const cx<R> m12 = sel<R>(s, Rr[1][2], P[1][2]), m21 = nconj(sel<R>(s, P[1][2], Rr[1][2]));
            const cx<R> m02 = sel<R>(s, Rr[0][2], P[0][2]), m20 = sel<R>(s, C1[2], C0[2]);
            const cx<R> del = cfms(cmul(dv, dv), m12, m21);
            if constexpr (N == 2) {  // the root pair is the last pair
                const cx<R> term =
                    pairs::leaf_pair(d, d, P[0][1], m02, C0[1], m20, Rr[0][1], m02, C1[1], m20, dv, m12, m21, dv, mk<R>(1, 0));
                ar.add(s ? -term.re : term.re);
                ai.add(s ? -term.im : term.im);
            } else {
                const cx<R> id = crcp(del);
                constexpr int M = N;  // copies + vertices 3..N at positions 2..N-1
#pragma unroll
                for (int path = 0; path < (1 << (N - 2)); ++path) {
                    cx<R> l0[M], l1[M], w0[M], w1[M], m[M][M];
#pragma unroll
                    for (int x = 0; x < M; ++x) {
                        cx<R> r0, r1;
                        if (x < 2) {
                            l0[x] = sel<R>(x, Rr[0][1], P[0][1]);  // M(0,1) with a_1 = x
                            l1[x] = m02;
                            r0 = sel<R>(x, C1[1], C0[1]);  // M(1,0) with a_1 = x
                            r1 = m20;
                        } else {
                            const int v = x + 1, a = (path >> (x - 2)) & 1;
                            l0[x] = nconj(sel<R>(a, P[1][v], Rr[1][v]));
                            l1[x] = nconj(sel<R>(a, P[2][v], Rr[2][v]));
                            r0 = sel<R>(a, Rr[1][v], P[1][v]);
                            r1 = sel<R>(a, Rr[2][v], P[2][v]);
                        }
                        // B^-1 (r0; r1), B^-1 = (1 / delta) [[dv, -M12], [-M21, dv]]
                        w0[x] = cmul(cfms(cmul(dv, r0), m12, r1), id);
                        w1[x] = cmul(cfms(cmul(dv, r1), m21, r0), id);
                    }
#pragma unroll
                    for (int x = 0; x < M; ++x)
#pragma unroll
                        for (int y = 0; y < M; ++y) {
                            if (x < 2 && y < 2 && x != y) continue;  // copy cross terms are never used
                            cx<R> base;
                            if (x == y) {
                                base = x < 2 ? d : dv;
                            } else if (x < 2) {  // measurement row, vertex y + 1
                                base = sel<R>((path >> (y - 2)) & 1, Rr[0][y + 1], P[0][y + 1]);
                            } else if (y < 2) {  // vertex x + 1, measurement column
                                base = sel<R>((path >> (x - 2)) & 1, C1[x + 1], C0[x + 1]);
                            } else if (x < y) {  // upper: index of the column vertex
                                base = sel<R>((path >> (y - 2)) & 1, Rr[x + 1][y + 1], P[x + 1][y + 1]);
                            } else {  // lower: index of the row vertex
                                base = nconj(sel<R>((path >> (x - 2)) & 1, P[y + 1][x + 1], Rr[y + 1][x + 1]));
                            }
                            m[x][y] = cfms(cfms(base, l0[x], w0[y]), l1[x], w1[y]);
                        }
                    cx<R> term;
                    if constexpr (N == 3) {
                        term = leaf_term(m[0][0], m[1][1], m[0][2], m[2][0], m[1][2], m[2][1], m[2][2], del);
                    } else {
                        static_assert(N == 4, "one point per lane serves orders 1..4");
                        term = pairs::leaf_pair(m[0][0], m[1][1], m[0][2], m[0][3], m[2][0], m[3][0], m[1][2], m[1][3],
                                         m[2][1], m[3][1], m[2][2], m[2][3], m[3][2], m[3][3], del);
                    }
                    if ((s + __popc(path)) & 1) term = cneg(term);
                    ar.add(term.re);
                    ai.add(term.im);
                }
            }
        }
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

// The item owning global work unit c: the last item whose chunk_begin <= c
// (items are laid out with ascending chunk_begin), by bisection.
__device__ __forceinline__ int item_of(const ItemDev *__restrict__ items, int n_items, long long c) {
    int lo = 0, hi = n_items;  // items[lo].chunk_begin <= c < items[hi].chunk_begin
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (items[mid].chunk_begin <= c) lo = mid; else hi = mid;
    }
    return lo;
}

// Device clock (ns) for the execution span of a launch: span[0] = earliest warp
// start, span[1] = latest warp exit, over every launch that shares the span.
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// A work unit's in-domain count carries this bit when its partial sum is not
// finite (NaN or infinite: non-finite tables, or an overflow).
constexpr unsigned kNonFinite = 0x80000000u;

__device__ __forceinline__ unsigned unit_flag(double a, double b, double c, double d) {
    return (isfinite(a) && isfinite(b) && isfinite(c) && isfinite(d)) ? 0u : kNonFinite;
}

// ----------------------------------------------------------------------------
// Hot-path kernel: persistent warps pull chunks of 32 Sobol' indices.
// ----------------------------------------------------------------------------
template <class Tree, class R, int RFMAX, bool GS>
__device__ __forceinline__ void detsum_body(const ItemDev *__restrict__ items, int n_items, long long total_chunks,
                                            unsigned long long *counter, int n_max, int rf_min, cx<R> *gstack,
                                            unsigned long long *span) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    if (span && lane == 0) atomicMin(span, gtimer());
    cx<R> *gst = nullptr;
    if (GS)
        gst = gstack +
              ((size_t)blockIdx.x * (blockDim.x >> 5) + warp) * Tree::template gstack_entries<R>(n_max, rf_min);
    const auto ws = Tree::template carve<R>(
        smem_raw + (size_t)warp * Tree::template smem_bytes<R>(n_max, rf_min, GS), n_max, rf_min, gst);
    const int NU = n_max + 1;
    while (true) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(counter, 1ull);
        c = __shfl_sync(FULL, c, 0);
        if ((long long)c >= total_chunks) break;
        const ItemDev &I = items[item_of(items, n_items, (long long)c)];
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
        const double inv_h = 1.0 / I.h;
        if (valid) {
            const uint64_t i = (uint64_t)(I.first_index + idx);
            double uprev = I.t, prod = 1.0;
            store_time<R>(ws.upt + lane * NU, I.t, inv_h);
            double jt = 1.0;
            for (int m = 0; m < n; ++m) {
                uint32_t y = point_word(I.lat_z, I.lat_m, m, i, I.shifts[k * n + m]);
                double v, omx, jac;
                point_gap<R>(I, m, y, v, omx, jac);
                uprev = uprev - v;
                store_time<R>(ws.upt + lane * NU + 1 + m, uprev, inv_h);
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
        // FP64: each lane adds w_i times its own share of every point's Keldysh sum (error-free
        // product, two-sum) and the warp reduces once per unit, instead of a two-sum butterfly per
        // point.  Mixed: the warp forms each point's total as FP32 pairs, the point's own lane keeps
        // it, every lane converts and weights its point in FP64 once per unit, and the unit's values
        // are summed as float-float pairs (unit_pairs_ff): an FP64 instruction costs 64 FP32
        // instructions' issue here, so none runs per point.
        constexpr int kOut = sizeof(R) == 8 ? kOutShare : kOutPair;
        using Out = typename SumOut<R, kOut>::type;
        PairSum<R> own;  // mixed: this lane's point total
        own.re.init();
        own.im.init();
        double sr = 0.0, cr = 0.0, si = 0.0, ci = 0.0;
        const cx<R> d = mk<R>((R)I.g0_re, (R)I.g0_im);
        const cx<R> dv = mk<R>((R)I.g0_re, (R)(I.g0_im - I.alpha));
        const typename TabT<R>::V *tab = item_table<R>(I);
        const double s0 = I.T * inv_h;
        unsigned mm = mask;
        if constexpr (std::is_same<Tree, SingleTree>::value) {
            if (I.split == 0 && single::two_point_order<R, RFMAX>(n)) {
                while (__popc(mm) >= 2) {  // two points per pass (keldysh_sum2), a lone last one below
                    const int a = __ffs(mm) - 1;
                    mm &= mm - 1;
                    const int b = __ffs(mm) - 1;
                    mm &= mm - 1;
                    Out sa, sb;
                    single::keldysh_sum2<R, RFMAX, kOut>(ws, ws.upt + a * NU, ws.upt + b * NU, n, d, dv, tab,
                                                         item_col<R>(I), inv_h, s0, I.L, RFMAX, lane, sa, sb);
                    if constexpr (kOut == kOutShare) {
                        const double wp = __shfl_sync(FULL, w, (lane >> 4) ? b : a);
                        const cx<double> sh = times_i_pow(sa, n);
                        add_weighted(wp, sh.re, sr, cr);
                        add_weighted(wp, sh.im, si, ci);
                    } else {
                        if (lane == a) own = sa;
                        if (lane == b) own = sb;
                    }
                    __syncwarp();
                }
            }
        }
        while (mm) {
            const int src = __ffs(mm) - 1;
            mm &= mm - 1;
            // every warp-per-point item of a launch shares the launch's flat depth
            const Out s = Tree::template sum<R, RFMAX, GS, kOut>(ws, ws.upt + src * NU, n, n_max, d, dv, tab,
                                                                 item_col<R>(I), inv_h, s0, I.L, RFMAX, lane, sub,
                                                                 I.split);
            if constexpr (kOut == kOutShare) {
                const double wp = __shfl_sync(FULL, w, src);
                const cx<double> sh = times_i_pow(s, n);
                add_weighted(wp, sh.re, sr, cr);
                add_weighted(wp, sh.im, si, ci);
            } else if (lane == src) {
                own = s;
            }
            __syncwarp();
        }
        if constexpr (kOut == kOutPair) {
            if ((mask >> lane) & 1u) {  // the lane's point was in the domain
                const cx<double> cval = times_i_pow(mk<double>(pair_value<R>(own.re), pair_value<R>(own.im)), n);
                sr = w * cval.re;
                si = w * cval.im;
            }
            unit_pairs_ff(sr, si, sr, cr, si, ci);
        } else {
            warp_reduce_pair(sr, cr);
            warp_reduce_pair(si, ci);
        }
        if (lane == 0) {
            double *pp = I.partials + 4 * (size_t)local;
            pp[0] = sr;
            pp[1] = si;
            pp[2] = cr;
            pp[3] = ci;
            // a point counts once, in subtree 0
            I.inside[local] = (sub == 0 ? __popc(mask) : 0u) | unit_flag(sr, si, cr, ci);
        }
    }
    if (span && lane == 0) atomicMax(span + 1, gtimer());
}

#define QQMC_DETSUM_PARAMS                                                                                   \
    const ItemDev *__restrict__ items, int n_items, long long total_chunks, unsigned long long *counter,   \
        int n_max, int rf_min, cx<R> *gstack, unsigned long long *span
#define QQMC_DETSUM_ARGS items, n_items, total_chunks, counter, n_max, rf_min, gstack, span

template <class Tree, class R, int RFMAX, bool GS>
__global__ void detsum_kernel(QQMC_DETSUM_PARAMS) {
    detsum_body<Tree, R, RFMAX, GS>(QQMC_DETSUM_ARGS);
}

// The single-vertex tree's FP32 flat-5 kernel (paired flat phase) with a
// register cap: left alone the compiler hoists the leaf gathers into ~240
// registers.  128 registers (10 values spilled) with the stack in shared
// memory: up to 16 resident warps, and measured 1 % faster than the
// spill-free cap even where shared memory holds the SM to 14 warps (order 10).
// With the split stack (orders >= 11) the tight cap spills 18 values and costs
// 4-5 %, so there the 144-register instance runs unless 128 registers buy
// more resident warps.
constexpr int kFlat5Regs = 144;
constexpr int kFlat5RegsTight = 128;
template <class Tree, class R, int RFMAX, bool GS>
__global__ void __maxnreg__(kFlat5Regs) detsum_kernel_capped(QQMC_DETSUM_PARAMS) {
    detsum_body<Tree, R, RFMAX, GS>(QQMC_DETSUM_ARGS);
}
template <class Tree, class R, int RFMAX, bool GS>
__global__ void __maxnreg__(kFlat5RegsTight) detsum_kernel_tight(QQMC_DETSUM_PARAMS) {
    detsum_body<Tree, R, RFMAX, GS>(QQMC_DETSUM_ARGS);
}
#undef QQMC_DETSUM_PARAMS
#undef QQMC_DETSUM_ARGS

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
                                                   long long total_chunks, unsigned long long *counter,
                                                   unsigned long long *span) {
    const int lane = threadIdx.x & 31;
    if (span && lane == 0) atomicMin(span, gtimer());
    while (true) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(counter, 1ull);
        c = __shfl_sync(FULL, c, 0);
        if ((long long)c >= total_chunks) break;
        const ItemDev &I = items[item_of(items, n_items, (long long)c)];
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
        if constexpr (sizeof(R) == 4) {
            unit_pairs_ff(v.re, v.im, sr, cr, si, ci);
        } else {
            warp_reduce_pair(sr, cr);
            warp_reduce_pair(si, ci);
        }
        if (lane == 0) {
            double *pp = I.partials + 4 * (size_t)local;
            pp[0] = sr;
            pp[1] = si;
            pp[2] = cr;
            pp[3] = ci;
            I.inside[local] = __popc(mask) | unit_flag(sr, si, cr, ci);
        }
    }
    if (span && lane == 0) atomicMax(span + 1, gtimer());
}

// Per shifted sequence: compensated sum of its chunk partials in a fixed order.
// out[2*g], out[2*g+1] = sum_i w_i c_n(u_i) (complex, not divided by N);
// counts[g] = in-domain points; bad[g] (if bad is not null) = work units whose
// partial sum was not finite.  One block of 256 threads per sequence: each
// thread sums its strided share of the units with two-sum, then the block
// combines the (sum, compensation) pairs in a fixed tree, also with two-sum.
struct TwoSum {
    double s, c;
    __device__ __forceinline__ void add(double x) {
        double t, e;
        two_sum(s, x, t, e);
        s = t;
        c += e;
    }
};

__global__ void reduce_kernel(const ItemDev *__restrict__ items, int n_items, double *out,
                              unsigned long long *counts, unsigned int *bad) {
    __shared__ double s_re[256], c_re[256], s_im[256], c_im[256];
    __shared__ unsigned long long cnt[256];
    __shared__ unsigned int nbad[256];
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
    TwoSum ar = {0.0, 0.0}, ai = {0.0, 0.0};
    unsigned long long cn = 0;
    unsigned int nb = 0;
    for (int q = threadIdx.x; q < I.chunks_per_shift; q += blockDim.x) {
        ar.add(pp[4 * q]);
        ar.add(pp[4 * q + 2]);
        ai.add(pp[4 * q + 1]);
        ai.add(pp[4 * q + 3]);
        const unsigned int v = ins[q];
        cn += v & ~kNonFinite;
        nb += v >> 31;
    }
    s_re[threadIdx.x] = ar.s;
    c_re[threadIdx.x] = ar.c;
    s_im[threadIdx.x] = ai.s;
    c_im[threadIdx.x] = ai.c;
    cnt[threadIdx.x] = cn;
    nbad[threadIdx.x] = nb;
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
            nbad[threadIdx.x] += nbad[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * g] = s_re[0] + c_re[0];
        out[2 * g + 1] = s_im[0] + c_im[0];
        counts[g] = cnt[0];
        if (bad) bad[g] = nbad[0];
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
template <class Tree, class R, int RF, bool GS>
__global__ void integrand_kernel(ItemDev I, uint64_t count, const double *u, double *out, int n_max, cx<R> *gstack) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint64_t wid = blockIdx.x * (uint64_t)(blockDim.x >> 5) + warp;
    cx<R> *gst = nullptr;
    if (GS) gst = gstack + wid * Tree::template gstack_entries<R>(n_max, RF);
    const auto ws = Tree::template carve<R>(smem_raw + (size_t)warp * Tree::template smem_bytes<R>(n_max, RF, GS),
                                            n_max, RF, gst);
    const int n = I.order;
    const cx<R> d = mk<R>((R)I.g0_re, (R)I.g0_im);
    const cx<R> dv = mk<R>((R)I.g0_re, (R)(I.g0_im - I.alpha));
    const double inv_h = 1.0 / I.h;
    for (uint64_t q = wid; q < count; q += (uint64_t)gridDim.x * (blockDim.x >> 5)) {
        if (lane <= n) store_time<R>(ws.upt + lane, lane == 0 ? I.t : u[q * n + lane - 1], inv_h);
        __syncwarp();
        cx<double> s = Tree::template sum<R, RF, GS>(ws, ws.upt, n, n_max, d, dv, item_table<R>(I), item_col<R>(I),
                                                     inv_h, I.T * inv_h, I.L, RF, lane);
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

// Every kernel of the library prefers the largest shared-memory carveout, the
// one the determinant kernels need: an SM runs blocks of different kernels side
// by side only while they agree on its L1 / shared-memory split, so small
// kernels (table builds, one-point-per-lane items, reductions) of another
// launch can start next to running determinant blocks instead of waiting for
// the SM to drain.
template <class K>
static void prefer_shared(K kernel) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
}

int launch_gf_table(const Problem &pr, cudaStream_t s) {
    const qqmc_params &p = pr.params;
    double wm = fmin(p.eps_d, 0.0) - 3.0 * p.gamma;
    int panels = 64 + (int)ceil(-wm * (p.t_max + 4.0 / p.gamma));
    if (panels > 8192) panels = 8192;
    int warps = pr.L / 2;
    int threads = 128;
    int blocks = (warps * 32 + threads - 1) / threads;
    prefer_shared(gf_table_kernel);
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
    // stream-ordered temporaries: no device-wide synchronisation with other streams' work
    cudaError_t e = cudaMallocAsync(&d_w, nq * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_s00, nq * sizeof(dbl4), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_s01, nq * sizeof(dbl4), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_zero, 4 * sizeof(double), s);
    if (e == cudaSuccess) {
        prefer_shared(lead_spectrum_kernel);
        prefer_shared(lead_table_kernel);
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
    if (d_w) cudaFreeAsync(d_w, s);
    if (d_s00) cudaFreeAsync(d_s00, s);
    if (d_s01) cudaFreeAsync(d_s01, s);
    if (d_zero) cudaFreeAsync(d_zero, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return cuda_error(e, "lead table build");
    return QQMC_OK;
}

int tree_leaf_bits(int order, bool pairs) { return pairs ? PairTree::leaf_bits(order) : SingleTree::leaf_bits(order); }

// The tree stack is split (wide top levels in device memory) where it does not
// fit in shared memory, and from the order set by qqmc_set_stack_policy
// (default, measured fastest on GB300 with the single-vertex tree: FP64 from
// order 5, so that the point times leave shared memory and 9 warps fit an SM;
// mixed from order 11, whose latency-bound steps want every level close): a
// large shared-memory stack limits the warps per SM, while the wide levels are
// built only a few times per point.
constexpr int kGsDefault[2] = {5, 11};
static std::atomic<int> g_gs_min_order[2] = {{kGsDefault[0]}, {kGsDefault[1]}};  // read by plans on any thread

void set_stack_policy(int precision, int min_order) {
    const int p = precision == QQMC_PREC_FP64 ? 0 : 1;
    g_gs_min_order[p].store(min_order <= 0 ? kGsDefault[p] : min_order);
}

template <class Tree, class R>
static bool stack_in_global(int n_max, int rf_min) {
    return Tree::template smem_bytes<R>(n_max, rf_min, false) > kSmemMax ||
           n_max >= g_gs_min_order[sizeof(R) == 8 ? 0 : 1].load();
}

template <class Tree, class R, int F>
constexpr bool flat5_capped() {
    return std::is_same<Tree, SingleTree>::value && sizeof(R) == 4 && F == 5;
}

// The kernel of one (tree, precision, flat depth, stack) shape: for the
// single-vertex tree's FP32 flat 5 a register-capped instance (above), the
// plain one otherwise.  Sets the kernel's shared-memory attributes.
template <class Tree, class R, int F, bool GS>
static cudaError_t detsum_entry(int wpb, size_t smem, void (**out)(const ItemDev *, int, long long,
                                                                    unsigned long long *, int, int, cx<R> *,
                                                                    unsigned long long *)) {
    auto prepare = [&](auto k, int *per_sm) {
        prefer_shared(k);
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, wpb * 32, smem);
        return e;
    };
    int per_sm = 0;
    if constexpr (flat5_capped<Tree, R, F>() && !GS) {
        *out = detsum_kernel_tight<Tree, R, F, GS>;
        return prepare(detsum_kernel_tight<Tree, R, F, GS>, &per_sm);
    } else if constexpr (flat5_capped<Tree, R, F>()) {
        cudaError_t e = prepare(detsum_kernel_capped<Tree, R, F, GS>, &per_sm);
        if (e != cudaSuccess) return e;
        *out = detsum_kernel_capped<Tree, R, F, GS>;
        int per_sm_tight = 0;
        e = prepare(detsum_kernel_tight<Tree, R, F, GS>, &per_sm_tight);
        if (e != cudaSuccess) return e;
        if (per_sm_tight > per_sm) *out = detsum_kernel_tight<Tree, R, F, GS>;
        return cudaSuccess;
    } else {
        *out = detsum_kernel<Tree, R, F, GS>;
        return prepare(detsum_kernel<Tree, R, F, GS>, &per_sm);
    }
}

template <class Tree, class R, int F, bool GS>
static cudaError_t launch_detsum_t(const ItemDev *d_items, int n_items, long long total_chunks,
                                   unsigned long long *d_counter, int n_max, int wpb, int rf_min, void *gstack,
                                   long long gstack_warps, unsigned long long *span, cudaStream_t s) {
    // fewer warps per block when the shared memory of the requested shape does not fit
    const size_t per_warp = Tree::template smem_bytes<R>(n_max, rf_min, GS);
    if (per_warp > kSmemMax) return cudaErrorInvalidConfiguration;
    while (wpb > 1 && per_warp * wpb > kSmemMax) --wpb;
    size_t smem = per_warp * wpb;
    void (*kern)(const ItemDev *, int, long long, unsigned long long *, int, int, cx<R> *,
                 unsigned long long *) = nullptr;
    cudaError_t e = detsum_entry<Tree, R, F, GS>(wpb, smem, &kern);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, wpb * 32, smem);
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
    kern<<<(unsigned)grid, wpb * 32, smem, s>>>(d_items, n_items, total_chunks, d_counter, n_max, rf_min,
                                                static_cast<cx<R> *>(gstack), span);
    return cudaGetLastError();
}

template <class Tree, class R, int F>
static cudaError_t launch_detsum_f(const ItemDev *d_items, int n_items, long long total_chunks,
                                   unsigned long long *d_counter, int n_max, int wpb, int rf_min, void *gstack,
                                   long long gstack_warps, unsigned long long *span, cudaStream_t s) {
    // without a device-memory buffer (the allocation-free entry) the shared-memory stack serves where it fits
    if (stack_in_global<Tree, R>(n_max, rf_min) &&
        (gstack || Tree::template smem_bytes<R>(n_max, rf_min, false) > kSmemMax))
        return launch_detsum_t<Tree, R, F, true>(d_items, n_items, total_chunks, d_counter, n_max, wpb, rf_min,
                                                 gstack, gstack_warps, span, s);
    return launch_detsum_t<Tree, R, F, false>(d_items, n_items, total_chunks, d_counter, n_max, wpb, rf_min,
                                              nullptr, 0, span, s);
}

static int clamp_rf_min(const Tuning &tune) {
    return tune.flat_min < 2 ? 2 : (tune.flat_min > tune.flat ? tune.flat : tune.flat_min);
}

template <class Tree, class R>
static long long gstack_warps_t(int n_max, int rf_min, size_t *bytes_per_warp) {
    *bytes_per_warp = 0;
    if (!stack_in_global<Tree, R>(n_max, rf_min)) return 0;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t per_warp = Tree::template smem_bytes<R>(n_max, rf_min, true);
    long long per_sm = (long long)(kSmemMax / per_warp);  // resident warps, bound by shared memory
    if (per_sm > 64) per_sm = 64;                          // and by the SM's warp slots
    *bytes_per_warp = Tree::template gstack_entries<R>(n_max, rf_min) * sizeof(cx<R>);
    return (long long)sms * (per_sm < 1 ? 1 : per_sm);
}

template <class Tree>
static bool stack_fits_t(int n_max, int precision, int rf_min) {
    return precision == QQMC_PREC_FP64 ? Tree::template smem_bytes<double>(n_max, rf_min, false) <= kSmemMax
                                       : Tree::template smem_bytes<float>(n_max, rf_min, false) <= kSmemMax;
}

bool detsum_stack_fits_shared(int n_max, int precision, const Tuning &tune, bool pairs) {
    const int rf_min = clamp_rf_min(tune);
    return pairs ? stack_fits_t<PairTree>(n_max, precision, rf_min) : stack_fits_t<SingleTree>(n_max, precision, rf_min);
}

template <class Tree>
static long long gstack_warps_p(int n_max, int precision, int rf_min, size_t *bytes_per_warp) {
    return precision == QQMC_PREC_FP64 ? gstack_warps_t<Tree, double>(n_max, rf_min, bytes_per_warp)
                                       : gstack_warps_t<Tree, float>(n_max, rf_min, bytes_per_warp);
}

long long detsum_gstack_warps(int n_max, int precision, const Tuning &tune, bool pairs, size_t *bytes_per_warp) {
    const int rf_min = clamp_rf_min(tune);
    return pairs ? gstack_warps_p<PairTree>(n_max, precision, rf_min, bytes_per_warp)
                 : gstack_warps_p<SingleTree>(n_max, precision, rf_min, bytes_per_warp);
}

template <class Tree>
static cudaError_t launch_detsum_tree(const ItemDev *d_items, int n_items, long long total_chunks,
                                      unsigned long long *d_counter, int n_max, int precision, const Tuning &tune,
                                      void *gstack, long long gstack_warps, unsigned long long *span,
                                      cudaStream_t s) {
    const int wpb = tune.warps_per_block;
    const int rf_min = clamp_rf_min(tune);
#define QQMC_DETSUM(RT, F)                                                                                         \
    launch_detsum_f<Tree, RT, F>(d_items, n_items, total_chunks, d_counter, n_max, wpb, rf_min, gstack,          \
                                 gstack_warps, span, s)
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

cudaError_t launch_detsum(const ItemDev *d_items, int n_items, long long total_chunks, unsigned long long *d_counter,
                          int n_max, int precision, const Tuning &tune, bool pairs, void *gstack,
                          long long gstack_warps, unsigned long long *span, cudaStream_t s) {
    return pairs ? launch_detsum_tree<PairTree>(d_items, n_items, total_chunks, d_counter, n_max, precision, tune,
                                                gstack, gstack_warps, span, s)
                 : launch_detsum_tree<SingleTree>(d_items, n_items, total_chunks, d_counter, n_max, precision, tune,
                                                  gstack, gstack_warps, span, s);
}

template <class R>
static cudaError_t launch_lane_t(const ItemDev *d_items, int n_items, long long total_chunks,
                                 unsigned long long *d_counter, unsigned long long *span, cudaStream_t s) {
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
    prefer_shared(lane_kernel<R>);
    lane_kernel<R><<<(unsigned)grid, 128, 0, s>>>(d_items, n_items, total_chunks, d_counter, span);
    return cudaGetLastError();
}

cudaError_t launch_lane(const ItemDev *d_items, int n_items, long long total_chunks, unsigned long long *d_counter,
                        int precision, unsigned long long *span, cudaStream_t s) {
    if (n_items < 1 || total_chunks < 1) return cudaSuccess;
    return precision == QQMC_PREC_FP64 ? launch_lane_t<double>(d_items, n_items, total_chunks, d_counter, span, s)
                                       : launch_lane_t<float>(d_items, n_items, total_chunks, d_counter, span, s);
}

cudaError_t launch_reduce(const ItemDev *d_items, int n_items, int total_shifts, double *d_out,
                          unsigned long long *d_counts, unsigned int *d_bad, cudaStream_t s) {
    prefer_shared(reduce_kernel);
    reduce_kernel<<<total_shifts, 256, 0, s>>>(d_items, n_items, d_out, d_counts, d_bad);
    return cudaGetLastError();
}

__global__ void store_item_kernel(ItemDev item, ItemDev *dst, unsigned long long *counter) {
    *dst = item;
    *counter = 0ull;
}

cudaError_t launch_store_item(const ItemDev &item, ItemDev *d_item, unsigned long long *d_counter, cudaStream_t s) {
    prefer_shared(store_item_kernel);
    store_item_kernel<<<1, 1, 0, s>>>(item, d_item, d_counter);
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

template <class Tree, class R, int F, bool GS>
static cudaError_t launch_integrand_t(const ItemDev &item, uint64_t count, const double *d_u, double *d_out,
                                      cudaStream_t s) {
    const size_t per_warp = Tree::template smem_bytes<R>(item.order, F, GS);
    if (per_warp > kSmemMax) return cudaErrorInvalidConfiguration;
    const int wpb = per_warp * 2 <= kSmemMax ? 2 : 1;
    size_t smem = per_warp * wpb;
    auto kern = integrand_kernel<Tree, R, F, GS>;
    prefer_shared(kern);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    uint64_t blocks = (count + wpb - 1) / wpb;
    cx<R> *gstack = nullptr;
    if (GS) {  // check path: a bounded number of warps, each with its own slice of device memory
        if (blocks > 304) blocks = 304;
        e = cudaMalloc(&gstack, blocks * wpb * Tree::template gstack_entries<R>(item.order, F) * sizeof(cx<R>));
        if (e != cudaSuccess) return e;
    }
    kern<<<(unsigned)blocks, wpb * 32, smem, s>>>(item, count, d_u, d_out, item.order, gstack);
    e = cudaGetLastError();
    if (GS) {
        cudaError_t e2 = cudaStreamSynchronize(s);
        cudaFree(gstack);
        if (e == cudaSuccess) e = e2;
    }
    return e;
}

template <class Tree, class R, int F>
static cudaError_t launch_integrand_f(const ItemDev &item, uint64_t count, const double *d_u, double *d_out,
                                      cudaStream_t s) {
    if (stack_in_global<Tree, R>(item.order, F)) return launch_integrand_t<Tree, R, F, true>(item, count, d_u, d_out, s);
    return launch_integrand_t<Tree, R, F, false>(item, count, d_u, d_out, s);
}

template <class Tree>
static cudaError_t launch_integrand_tree(const ItemDev &item, uint64_t count, const double *d_u, double *d_out,
                                         int precision, const Tuning &tune, cudaStream_t s) {
    if (precision == QQMC_PREC_FP64) {
        switch (tune.flat) {
            case 2: return launch_integrand_f<Tree, double, 2>(item, count, d_u, d_out, s);
            case 3: return launch_integrand_f<Tree, double, 3>(item, count, d_u, d_out, s);
            case 4: return launch_integrand_f<Tree, double, 4>(item, count, d_u, d_out, s);
            default: return launch_integrand_f<Tree, double, 5>(item, count, d_u, d_out, s);
        }
    }
    switch (tune.flat) {
        case 2: return launch_integrand_f<Tree, float, 2>(item, count, d_u, d_out, s);
        case 3: return launch_integrand_f<Tree, float, 3>(item, count, d_u, d_out, s);
        case 4: return launch_integrand_f<Tree, float, 4>(item, count, d_u, d_out, s);
        default: return launch_integrand_f<Tree, float, 5>(item, count, d_u, d_out, s);
    }
}

cudaError_t launch_integrand(const ItemDev &item, uint64_t count, const double *d_u, double *d_out, int precision,
                             const Tuning &tune, bool pairs, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    return pairs ? launch_integrand_tree<PairTree>(item, count, d_u, d_out, precision, tune, s)
                 : launch_integrand_tree<SingleTree>(item, count, d_u, d_out, precision, tune, s);
}

}  // namespace qqmc
