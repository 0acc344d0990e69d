/*
 * ORACLE -- test infrastructure only.
 *
 * Plain, slow, obviously-correct CPU restatement of the quantum quasi-Monte
 * Carlo (QQMC) estimator for the order-n coefficient of the equal-time lesser
 * function G^<_{0i}(t,t) of the Anderson single-level dot: i = 0 gives the
 * charge Q_n, i = 1 (dot-lead) the current I_n (App. E).  Only tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this code; the product never does.  It shares
 * no source with the CUDA path.
 *
 * Everything is complex128 (C99 `double complex`).  Each function names the
 * passage of the paper it follows:
 *   - Keldysh Green function of two contour points: App. E, Eq. (integral_gf)
 *     and the 2x2 matrix g[(x,u,a),(x',u',a')] below it (g^T, g^<, g^>, g^Tbar).
 *   - Wick determinants and the Keldysh index sum: App. E, Eq. (integral_gf).
 *   - Product model warp with h(v) = exp(-v/tau): Eq. (warper1d), App. D
 *     Eq. (x_of_v_simple), App. F Eq. (hi_expo); points with u_n < 0 give 0
 *     (App. F, change of variables u -> v).
 *   - Estimator F_n(N) = (C/N) sum_i f_n(u_i)/p_n(u_i): Eq. (warped_int2),
 *     App. B (main computing loop), with C = int p_n = tau^n.
 *   - Sobol' points (Gray-code order) with a digital shift: main text below
 *     Eq. (warped_int2) and App. H (digitally shifted generators).
 *   - Or a rank-1 lattice with N = 2^m points and a random shift (the lattice
 *     rules the paper cites as the alternative low-discrepancy family):
 *     x_i = frac(i z / N + Delta), held as 32-bit fixed point, so the point
 *     word is ((i z_d mod 2^m) << (32 - m)) + S_d mod 2^32; optionally followed
 *     by the baker's (tent) transform x -> 1 - |2x - 1| (Hickernell 2002), which
 *     keeps the uniform measure and lets lattice rules integrate non-periodic
 *     functions at their higher rate.
 *
 * The determinant of every Keldysh configuration is formed independently by
 * LU factorisation with partial pivoting; there is no reuse between
 * configurations.  Sums over points use Neumaier's compensated summation.
 *
 * Tables: g^<(tau_k), g^>(tau_k) on L uniform nodes tau_k = -T + k*2T/(L-1),
 * k = 0..L-1, stored as interleaved (re, im) doubles; interpolation is linear
 * in re and im separately with k = clamp(floor((tau+T)/h), 0, L-2).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define ORACLE_MAX_ORDER 22

/* ---- table interpolation (plain definition of linear interpolation) ---- */
static cplx table_at(const double *tab, int L, double T, double tau) {
    double h = 2.0 * T / (double)(L - 1);
    double s = (tau + T) / h;
    double kf = floor(s);
    int k = (int)kf;
    if (k < 0) k = 0;
    if (k > L - 2) k = L - 2;
    double f = s - (double)k;
    cplx a = tab[2 * k] + I * tab[2 * k + 1];
    cplx b = tab[2 * k + 2] + I * tab[2 * k + 3];
    return (1.0 - f) * a + f * b;
}

typedef struct {
    const double *gl; /* g^< table, interleaved complex, L entries */
    const double *gg; /* g^> table */
    int L;
    double T;         /* table covers [-T, T] */
    cplx gl0;         /* g^<(0): the equal-time value of the measurement pair */
    cplx dv;          /* diagonal of a vertex: g^<(0) - i alpha (App. E, quadratic shift alpha) */
    /* Current (i = 1): the measurement column point sits on lead site 1, so the
     * entries of column 0 are dot-lead functions.  cl, cg: gamma g^<_{01},
     * gamma g^>_{01} on the same mesh; c0 = gamma g^<_{01}(0).  cl == NULL for
     * the charge. */
    const double *cl, *cg;
    cplx c0;
} gf_t;

/* col: NULL (charge) or [gamma g^<_01 (2L doubles) | gamma g^>_01 (2L) | re, im of gamma g^<_01(0)]. */
static gf_t make_gf(const double *gl, const double *gg, int L, double T, double gl0_re, double gl0_im,
                    double alpha, const double *col) {
    gf_t g = {gl, gg, L, T, gl0_re + I * gl0_im, gl0_re + I * (gl0_im - alpha), NULL, NULL, 0.0};
    if (col) {
        g.cl = col;
        g.cg = col + 2 * L;
        g.c0 = col[4 * L] + I * col[4 * L + 1];
    }
    return g;
}

/*
 * Keldysh Green function between two contour points (time u, Keldysh index a)
 * and (u', a'), App. E: the 2x2 matrix [[g^T, g^<], [g^>, g^Tbar]]_{a a'} with
 *   g^T(u,u')    = theta(u-u') g^>(u-u') + theta(u'-u) g^<(u-u'),
 *   g^Tbar(u,u') = theta(u'-u) g^>(u-u') + theta(u-u') g^<(u-u').
 * `same` marks a point paired with itself: 1 = the measurement pair, whose
 * entry is g^<(0); 2 = a vertex on the diagonal, g^<(0) shifted by -i alpha
 * (App. E: every diagonal except the one of the measurement point).
 * `lead`: the second point is on lead site 1 (current measurement column):
 * the dot-lead tables replace the dot-dot ones.
 */
static cplx keldysh_g(const gf_t *g, double u, int a, double up, int ap, int same, int lead) {
    const double *tl = lead ? g->cl : g->gl;
    const double *tg = lead ? g->cg : g->gg;
    if (same == 1) return lead ? g->c0 : g->gl0;
    if (same == 2) return g->dv;
    double tau = u - up;
    if (a == 0 && ap == 1) return table_at(tl, g->L, g->T, tau);
    if (a == 1 && ap == 0) return table_at(tg, g->L, g->T, tau);
    int later = (u > up); /* theta(u - u') */
    if (a == 0) /* time ordered */
        return later ? table_at(tg, g->L, g->T, tau) : table_at(tl, g->L, g->T, tau);
    /* anti-time ordered */
    return later ? table_at(tl, g->L, g->T, tau) : table_at(tg, g->L, g->T, tau);
}

/* Determinant by Doolittle LU factorisation with partial pivoting (row swaps
 * flip the sign).  A is m x m, row-major, overwritten. */
static cplx det_lu(cplx *A, int m) {
    cplx det = 1.0;
    for (int c = 0; c < m; ++c) {
        int p = c;
        double best = cabs(A[c * m + c]);
        for (int r = c + 1; r < m; ++r) {
            double v = cabs(A[r * m + c]);
            if (v > best) { best = v; p = r; }
        }
        if (best == 0.0) return 0.0;
        if (p != c) {
            for (int j = 0; j < m; ++j) {
                cplx tmp = A[c * m + j];
                A[c * m + j] = A[p * m + j];
                A[p * m + j] = tmp;
            }
            det = -det;
        }
        cplx piv = A[c * m + c];
        det *= piv;
        for (int r = c + 1; r < m; ++r) {
            cplx l = A[r * m + c] / piv;
            for (int j = c + 1; j < m; ++j) A[r * m + j] -= l * A[c * m + j];
        }
    }
    return det;
}

/*
 * Order-n integrand of App. E Eq. (integral_gf) at vertex times u[0..n-1]
 * (any order; the theta functions decide), measurement time t:
 *   c(u) = i^n * sum_{a in {0,1}^n} (-1)^{sum a}
 *          [[(0,t,0), U_1..U_n ; (i,t,1), U_1..U_n]] * [[U_1..U_n ; U_1..U_n]]
 * with U_k = (0, u_k, a_k); i = 1 (current) when g->cl is set, else 0.  The left Wick determinant is the spin-up one
 * ((n+1)x(n+1), row 0 / column 0 = the measurement points), the right one is
 * spin-down (n x n).  Both are formed from scratch for every a.
 * Also returns sum_a |term| (before the i^n factor) in *abs_sum if non-NULL,
 * and in *had_sum if non-NULL the sum over a of the Hadamard bounds of both
 * determinants (|det A| <= product of the Euclidean norms of A's rows): the
 * scale of the rounding error of a determinant, which stays finite where the
 * determinant itself vanishes.
 * With alpha != 0 the vertex diagonals are shifted (see keldysh_g).
 */
static double hadamard(const cplx *A, int m) {
    double h = 1.0;
    for (int r = 0; r < m; ++r) {
        double s = 0.0;
        for (int c = 0; c < m; ++c) s += creal(A[r * m + c]) * creal(A[r * m + c]) + cimag(A[r * m + c]) * cimag(A[r * m + c]);
        h *= sqrt(s);
    }
    return h;
}

static cplx integrand(const gf_t *g, int n, const double *u, double t, double *abs_sum, double *had_sum) {
    cplx up[(ORACLE_MAX_ORDER + 1) * (ORACLE_MAX_ORDER + 1)];
    cplx dn[ORACLE_MAX_ORDER * ORACLE_MAX_ORDER];
    int a[ORACLE_MAX_ORDER];
    double re_acc = 0.0, re_c = 0.0, im_acc = 0.0, im_c = 0.0, asum = 0.0, hsum = 0.0;
    uint32_t nconf = 1u << n;
    int m = n + 1;
    for (uint32_t conf = 0; conf < nconf; ++conf) {
        int parity = 0;
        for (int k = 0; k < n; ++k) { a[k] = (conf >> k) & 1; parity ^= a[k]; }
        /* spin-up: row points A_0=(t,0), A_j=U_j ; column points B_0=(t,1), B_k=U_k */
        for (int r = 0; r < m; ++r) {
            double ur = (r == 0) ? t : u[r - 1];
            int ar = (r == 0) ? 0 : a[r - 1];
            for (int c = 0; c < m; ++c) {
                double uc = (c == 0) ? t : u[c - 1];
                int ac = (c == 0) ? 1 : a[c - 1];
                up[r * m + c] = keldysh_g(g, ur, ar, uc, ac, r == c ? (r == 0 ? 1 : 2) : 0,
                                          c == 0 && g->cl != NULL);
            }
        }
        for (int r = 0; r < n; ++r)
            for (int c = 0; c < n; ++c)
                dn[r * n + c] = keldysh_g(g, u[r], a[r], u[c], a[c], r == c ? 2 : 0, 0);
        if (had_sum) hsum += hadamard(up, m) * hadamard(dn, n);
        cplx term = det_lu(up, m) * det_lu(dn, n);
        if (parity) term = -term;
        asum += cabs(term);
        /* Neumaier sum of the 2^n terms */
        double x = creal(term), s = re_acc + x;
        re_c += (fabs(re_acc) >= fabs(x)) ? (re_acc - s) + x : (x - s) + re_acc;
        re_acc = s;
        x = cimag(term); s = im_acc + x;
        im_c += (fabs(im_acc) >= fabs(x)) ? (im_acc - s) + x : (x - s) + im_acc;
        im_acc = s;
    }
    cplx sum = (re_acc + re_c) + I * (im_acc + im_c);
    cplx in = 1.0;
    for (int k = 0; k < n; ++k) in *= I;
    if (abs_sum) *abs_sum = asum;
    if (had_sum) *had_sum = hsum;
    return in * sum;
}

/* ------------------------------ exported API ------------------------------ */

/* Integrand at `count` points; u is count x n row-major (any time order).
 * out: 2*count doubles (re, im) of c(u); abs_out (optional): sum_a |term|;
 * had_out (optional): sum_a of the Hadamard bounds of the two determinants.
 * col: NULL for the charge, else the dot-lead tables (see make_gf). */
int oracle_integrand(int n, int64_t count, const double *u, double t,
                     const double *gl, const double *gg, int L, double T,
                     double gl0_re, double gl0_im, double *out, double *abs_out, double alpha,
                     const double *col, double *had_out) {
    if (n < 0 || n > ORACLE_MAX_ORDER || L < 2 || count < 0) return -1;
    gf_t g = make_gf(gl, gg, L, T, gl0_re, gl0_im, alpha, col);
    for (int64_t i = 0; i < count; ++i) {
        double as, hs;
        cplx v = integrand(&g, n, u + i * n, t, &as, had_out ? &hs : NULL);
        out[2 * i] = creal(v);
        out[2 * i + 1] = cimag(v);
        if (abs_out) abs_out[i] = as;
        if (had_out) had_out[i] = hs;
    }
    return 0;
}

/* Unshifted Sobol' integers in Gray-code order for point indices i0..i0+count-1:
 * X_{i,d} = XOR over the set bits j of gray(i) = i ^ (i>>1) of V[d*32 + j].
 * out: count x n uint32, row-major. */
int oracle_sobol(int n, int64_t i0, int64_t count, const uint32_t *V, uint32_t *out) {
    for (int64_t q = 0; q < count; ++q) {
        uint64_t i = (uint64_t)(i0 + q);
        uint64_t gray = i ^ (i >> 1);
        for (int d = 0; d < n; ++d) {
            uint32_t x = 0;
            for (int j = 0; j < 32; ++j)
                if ((gray >> j) & 1u) x ^= V[d * 32 + j];
            out[q * n + d] = x;
        }
    }
    return 0;
}

/* Point-family code: 0 = Sobol', m = lattice of 2^m points, 64 + m = the same followed by the tent map. */
static int bad_family(int code) { return code < 0 || (code > 32 && (code < 65 || code > 96)); }

/* Baker's transform on a 32-bit fixed-point word: x' = 2x below 1/2, 2 - 2x
 * above (the single word 2^31, which would give exactly 1, is kept at 1 - 2^-32). */
static uint32_t tent_word(uint32_t w) {
    if (w < 0x80000000u) return w << 1;
    uint64_t v = (1ull << 33) - 2ull * (uint64_t)w;
    return v > 0xffffffffull ? 0xffffffffu : (uint32_t)v;
}

/* Shifted point words of index i: Sobol' (digital shift, XOR) when lattice_m
 * == 0, else the rank-1 lattice with generating vector V[0..n-1] and N = 2^m
 * (shift added modulo 2^32); lattice_m + 64 selects the lattice followed by
 * the baker's transform. */
static void point_words(int n, int64_t i, const uint32_t *V, const uint32_t *S, int lattice_m, uint32_t *X) {
    int tent = 0;
    if (lattice_m >= 64) {
        tent = 1;
        lattice_m -= 64;
    }
    if (lattice_m == 0) {
        oracle_sobol(n, i, 1, V, X);
        for (int d = 0; d < n; ++d) X[d] ^= S[d];
        return;
    }
    uint64_t mask = (1ull << lattice_m) - 1ull;
    for (int d = 0; d < n; ++d) {
        uint64_t r = ((uint64_t)i * (uint64_t)V[d]) & mask;
        X[d] = (uint32_t)((r << (32 - lattice_m)) + (uint64_t)S[d]);
        if (tent) X[d] = tent_word(X[d]);
    }
}

/*
 * Partial QQMC estimate over point indices [i0, i1) of one digitally shifted
 * Sobol' sequence (or one randomly shifted lattice, see point_words): returns
 * sum_i w_i c(u_i) (Neumaier-compensated, re/im) and the number of points
 * inside the domain.
 *   x_m = (shifted point word of dimension m-1) * 2^-32,
 *   v_m = -tau * log1p(-x_m)          (inverse CDF of h(v) = exp(-v/tau)),
 *   u_0 = t, u_m = u_{m-1} - v_m,     in domain iff u_n > 0,
 *   w   = C / p_n(u) with C = tau^n and p_n = prod_m exp(-v_m / tau).
 * result: [sum_re, sum_im, comp_re, comp_im]; *n_in: in-domain count.
 */
int oracle_estimate(int n, int64_t i0, int64_t i1, const uint32_t *V, const uint32_t *S,
                    double t, double tau, const double *gl, const double *gg, int L,
                    double T, double gl0_re, double gl0_im, double *result, int64_t *n_in, double alpha,
                    const double *col, int lattice_m) {
    if (n < 1 || n > ORACLE_MAX_ORDER || L < 2 || bad_family(lattice_m)) return -1;
    gf_t g = make_gf(gl, gg, L, T, gl0_re, gl0_im, alpha, col);
    double re_acc = 0.0, re_c = 0.0, im_acc = 0.0, im_c = 0.0;
    int64_t inside = 0;
    uint32_t X[ORACLE_MAX_ORDER];
    double u[ORACLE_MAX_ORDER];
    for (int64_t i = i0; i < i1; ++i) {
        point_words(n, i, V, S, lattice_m, X);
        double uprev = t, vsum = 0.0;
        for (int m = 0; m < n; ++m) {
            double x = (double)X[m] * 0x1p-32;
            double v = -tau * log1p(-x);
            vsum += v;
            u[m] = uprev - v;
            uprev = u[m];
        }
        if (!(u[n - 1] > 0.0)) continue;
        ++inside;
        double C = pow(tau, (double)n);
        double p = exp(-vsum / tau);
        double w = C / p;
        cplx val = w * integrand(&g, n, u, t, NULL, NULL);
        double x = creal(val), s = re_acc + x;
        re_c += (fabs(re_acc) >= fabs(x)) ? (re_acc - s) + x : (x - s) + re_acc;
        re_acc = s;
        x = cimag(val); s = im_acc + x;
        im_c += (fabs(im_acc) >= fabs(x)) ? (im_acc - s) + x : (x - s) + im_acc;
        im_acc = s;
    }
    result[0] = re_acc;
    result[1] = im_acc;
    result[2] = re_c;
    result[3] = im_c;
    *n_in = inside;
    return 0;
}

/* Warped points only (for the domain / weight checks): u (count x n), w, flag. */
int oracle_warp(int n, int64_t i0, int64_t count, const uint32_t *V, const uint32_t *S,
                double t, double tau, double *u_out, double *w_out, int32_t *inside, int lattice_m) {
    uint32_t X[ORACLE_MAX_ORDER];
    if (bad_family(lattice_m)) return -1;
    for (int64_t q = 0; q < count; ++q) {
        point_words(n, i0 + q, V, S, lattice_m, X);
        double uprev = t, vsum = 0.0;
        for (int m = 0; m < n; ++m) {
            double x = (double)X[m] * 0x1p-32;
            double v = -tau * log1p(-x);
            vsum += v;
            u_out[q * n + m] = uprev - v;
            uprev = u_out[q * n + m];
        }
        w_out[q] = pow(tau, (double)n) / exp(-vsum / tau);
        inside[q] = (u_out[q * n + n - 1] > 0.0);
    }
    return 0;
}

/* Shifted point words (count x n) of either point family; for the pins. */
int oracle_points(int n, int64_t i0, int64_t count, const uint32_t *V, const uint32_t *S, int lattice_m,
                  uint32_t *out) {
    if (n < 1 || n > ORACLE_MAX_ORDER || bad_family(lattice_m)) return -1;
    for (int64_t q = 0; q < count; ++q) point_words(n, i0 + q, V, S, lattice_m, out + q * n);
    return 0;
}

/* Exposed for the pins: determinant of an m x m complex matrix (interleaved
 * re/im, row-major; copied, not modified) and table interpolation at tau. */
int oracle_det(int m, const double *A, double *out) {
    cplx M[(ORACLE_MAX_ORDER + 1) * (ORACLE_MAX_ORDER + 1)];
    if (m < 1 || m > ORACLE_MAX_ORDER + 1) return -1;
    for (int i = 0; i < m * m; ++i) M[i] = A[2 * i] + I * A[2 * i + 1];
    cplx d = det_lu(M, m);
    out[0] = creal(d);
    out[1] = cimag(d);
    return 0;
}

int oracle_table_at(const double *tab, int L, double T, int64_t count, const double *tau, double *out) {
    for (int64_t i = 0; i < count; ++i) {
        cplx v = table_at(tab, L, T, tau[i]);
        out[2 * i] = creal(v);
        out[2 * i + 1] = cimag(v);
    }
    return 0;
}

/*
 * Learned warp (App. F, learning h from the integrand): w_m in [0,1) has a
 * piecewise-constant density on `cells` equal cells with cumulative values
 * cdf[m*(cells+1) + k].  x -> w: the cell k with cdf[k] <= x < cdf[k+1]
 * (scanned from below), w = (k + (x - cdf[k]) / (cdf[k+1] - cdf[k])) / cells,
 * dw/dx = 1 / (cells (cdf[k+1] - cdf[k])).  Then v = -tau log(1 - w) as in the
 * plain warp, and the weight is C/p_n(u) times prod_m dw_m/dx_m.
 */
static double learned_w(const double *cdf, int cells, double x, double *jac) {
    int k = 0;
    while (k + 1 < cells && cdf[k + 1] <= x) ++k;
    double dc = cdf[k + 1] - cdf[k];
    *jac = 1.0 / ((double)cells * dc);
    return ((double)k + (x - cdf[k]) / dc) / (double)cells;
}

int oracle_estimate_proj(int n, int64_t i0, int64_t i1, const uint32_t *V, const uint32_t *S, double t,
                         double tau, const double *cdf, int cells, const double *gl, const double *gg, int L,
                         double T, double gl0_re, double gl0_im, double *result, int64_t *n_in,
                         double alpha, const double *col, int lattice_m) {
    if (n < 1 || n > ORACLE_MAX_ORDER || L < 2 || cells < 1 || bad_family(lattice_m)) return -1;
    gf_t g = make_gf(gl, gg, L, T, gl0_re, gl0_im, alpha, col);
    double re_acc = 0.0, re_c = 0.0, im_acc = 0.0, im_c = 0.0;
    int64_t inside = 0;
    uint32_t X[ORACLE_MAX_ORDER];
    double u[ORACLE_MAX_ORDER];
    for (int64_t i = i0; i < i1; ++i) {
        point_words(n, i, V, S, lattice_m, X);
        double uprev = t, vsum = 0.0, jt = 1.0;
        for (int m = 0; m < n; ++m) {
            double x = (double)X[m] * 0x1p-32;
            double jac;
            double w = learned_w(cdf + (size_t)m * (cells + 1), cells, x, &jac);
            double v = -tau * log1p(-w);
            vsum += v;
            jt *= jac;
            u[m] = uprev - v;
            uprev = u[m];
        }
        if (!(u[n - 1] > 0.0)) continue;
        ++inside;
        double wgt = pow(tau, (double)n) / exp(-vsum / tau) * jt;
        cplx val = wgt * integrand(&g, n, u, t, NULL, NULL);
        double x = creal(val), s = re_acc + x;
        re_c += (fabs(re_acc) >= fabs(x)) ? (re_acc - s) + x : (x - s) + re_acc;
        re_acc = s;
        x = cimag(val); s = im_acc + x;
        im_c += (fabs(im_acc) >= fabs(x)) ? (im_acc - s) + x : (x - s) + im_acc;
        im_acc = s;
    }
    result[0] = re_acc;
    result[1] = im_acc;
    result[2] = re_c;
    result[3] = im_c;
    *n_in = inside;
    return 0;
}
