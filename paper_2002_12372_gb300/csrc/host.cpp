// Host-side generators of the product path: Sobol' direction words, digital
// shift words, error reporting.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "qqmc_internal.h"

namespace qqmc {

static thread_local std::string g_last_error;

int set_error(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int cuda_error(cudaError_t e, const char *what) {
    return set_error(QQMC_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Joe & Kuo (2008) primitive polynomials and initial direction values for
// Sobol' dimensions 2..kMaxOrder (dimension 1 is the van der Corput
// sequence).  Each row: degree s, coefficient word a (bits a_1..a_{s-1},
// a_1 most significant), initial values m_1..m_s.
struct JoeKuo {
    int s;
    int a;
    int m[8];
};
static const JoeKuo kJoeKuo[] = {
    {1, 0, {1}},
    {2, 1, {1, 3}},
    {3, 1, {1, 3, 1}},
    {3, 2, {1, 1, 1}},
    {4, 1, {1, 1, 3, 3}},
    {4, 4, {1, 3, 5, 13}},
    {5, 2, {1, 1, 5, 5, 17}},
    {5, 4, {1, 1, 5, 5, 5}},
    {5, 7, {1, 1, 7, 11, 19}},
    {5, 11, {1, 1, 5, 1, 1}},
    {5, 13, {1, 1, 1, 3, 11}},
    {5, 14, {1, 3, 5, 5, 31}},
    {6, 1, {1, 3, 3, 9, 7, 49}},
    {6, 13, {1, 1, 1, 15, 21, 21}},
    {6, 16, {1, 3, 1, 13, 27, 49}},
    {6, 19, {1, 1, 1, 15, 7, 5}},
    {6, 22, {1, 3, 1, 15, 13, 25}},
    {6, 25, {1, 1, 5, 5, 19, 61}},
    {7, 1, {1, 3, 7, 11, 23, 15, 103}},
    {7, 4, {1, 3, 7, 13, 13, 15, 69}},
    {7, 7, {1, 1, 3, 13, 7, 35, 63}},
};

// V[d][j] = m_{j+1} * 2^{31-j}: the j-th direction word of dimension d.
void direction_numbers(int n_dims, uint32_t *out) {
    for (int d = 0; d < n_dims; ++d) {
        uint32_t *V = out + 32 * d;
        if (d == 0) {
            for (int j = 0; j < 32; ++j) V[j] = 1u << (31 - j);
            continue;
        }
        const JoeKuo &jk = kJoeKuo[d - 1];
        uint64_t m[33];
        for (int i = 1; i <= jk.s; ++i) m[i] = (uint64_t)jk.m[i - 1];
        // m_i = 2 a_1 m_{i-1} ^ 4 a_2 m_{i-2} ^ ... ^ 2^{s-1} a_{s-1} m_{i-s+1} ^ 2^s m_{i-s} ^ m_{i-s}
        for (int i = jk.s + 1; i <= 32; ++i) {
            uint64_t v = m[i - jk.s] ^ (m[i - jk.s] << jk.s);
            for (int k = 1; k < jk.s; ++k) {
                int ak = (jk.a >> (jk.s - 1 - k)) & 1;
                if (ak) v ^= m[i - k] << k;
            }
            m[i] = v;
        }
        for (int j = 0; j < 32; ++j) V[j] = (uint32_t)(m[j + 1] << (31 - j));
    }
}

uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void shift_words(uint64_t seed, int n_shifts, int n_dims, uint32_t *out) {
    for (int k = 0; k < n_shifts; ++k)
        for (int d = 0; d < n_dims; ++d)
            out[k * n_dims + d] = (uint32_t)(splitmix64(seed ^ ((uint64_t)k * 65536u + (uint64_t)d)) >> 32);
}

}  // namespace qqmc

namespace qqmc {

// Parabola-map resummation (see qqmc_resum_parabola).  U = |p| artanh^2(sqrt W)
// = |p| sum_{m>=1} c_m W^m with c_m = sum_{j=0}^{m-1} 1 / ((2j+1)(2(m-1-j)+1)).
static double resum_value(const double *a, int n, double p, double U, int invert, double *tail) {
    double f[QQMC_MAX_ORDER + 1];
    if (invert) {  // power series of 1 / F
        f[0] = 1.0 / a[0];
        for (int k = 1; k <= n; ++k) {
            double acc = 0.0;
            for (int j = 1; j <= k; ++j) acc += a[j] * f[k - j];
            f[k] = -acc / a[0];
        }
    } else {
        for (int k = 0; k <= n; ++k) f[k] = a[k];
    }
    const double ap = fabs(p);
    double c[QQMC_MAX_ORDER + 1];
    c[0] = 0.0;
    for (int m = 1; m <= n; ++m) {
        double acc = 0.0;
        for (int j = 0; j <= m - 1; ++j) acc += 1.0 / ((2.0 * j + 1.0) * (2.0 * (m - 1 - j) + 1.0));
        c[m] = ap * acc;
    }
    // b(W) = sum_k f_k U(W)^k, truncated at W^n
    double b[QQMC_MAX_ORDER + 1], pw[QQMC_MAX_ORDER + 1], tmp[QQMC_MAX_ORDER + 1];
    for (int k = 0; k <= n; ++k) {
        b[k] = 0.0;
        pw[k] = 0.0;
    }
    pw[0] = 1.0;  // U(W)^0
    b[0] = f[0];
    for (int k = 1; k <= n; ++k) {
        for (int i = 0; i <= n; ++i) tmp[i] = 0.0;
        for (int i = 0; i <= n; ++i)
            if (pw[i] != 0.0)
                for (int m = 1; i + m <= n; ++m) tmp[i + m] += pw[i] * c[m];
        for (int i = 0; i <= n; ++i) {
            pw[i] = tmp[i];
            b[i] += f[k] * pw[i];
        }
    }
    const double th = tanh(sqrt(U / ap));
    const double W = th * th;
    double val = 0.0, Wk = 1.0, last = 0.0;
    for (int k = 0; k <= n; ++k) {
        last = b[k] * Wk;
        val += last;
        Wk *= W;
    }
    if (tail) *tail = fabs(last);
    return invert ? 1.0 / val : val;
}

}  // namespace qqmc

extern "C" int qqmc_resum_parabola(const double *a, const double *a_err, int n, double p, double U, int invert,
                                   double *value, double *err, double *tail) {
    if (!a || !value || n < 0 || n > qqmc::kMaxOrder || !(p < 0.0) || !(U >= 0.0) || !isfinite(p) || !isfinite(U))
        return qqmc::set_error(QQMC_E_INVAL, "qqmc_resum_parabola: need a, value, 0 <= n <= QQMC_MAX_ORDER, p < 0, U >= 0");
    if (invert && a[0] == 0.0) return qqmc::set_error(QQMC_E_INVAL, "qqmc_resum_parabola: 1/F needs a_0 != 0");
    double t = 0.0;
    const double v = qqmc::resum_value(a, n, p, U, invert, &t);
    *value = v;
    if (tail) *tail = t;
    if (err) {  // linear propagation of the coefficient errors (central differences)
        double e2 = 0.0;
        if (a_err) {
            double ac[qqmc::kMaxOrder + 1];
            for (int k = 0; k <= n; ++k) ac[k] = a[k];
            for (int k = 0; k <= n; ++k) {
                if (!(a_err[k] > 0.0)) continue;
                const double hstep = a_err[k];
                ac[k] = a[k] + hstep;
                const double vp = qqmc::resum_value(ac, n, p, U, invert, nullptr);
                ac[k] = a[k] - hstep;
                const double vm = qqmc::resum_value(ac, n, p, U, invert, nullptr);
                ac[k] = a[k];
                const double d = 0.5 * (vp - vm);
                e2 += d * d;
            }
        }
        *err = sqrt(e2);
    }
    return QQMC_OK;
}

namespace qqmc {

// In-place radix-2 complex DFT, X[f] = sum_n x[n] exp(-2 pi i f n / L) (inv: +i, no 1/L).
static void fft(std::vector<double> &re, std::vector<double> &im, bool inv) {
    const size_t L = re.size();
    for (size_t i = 1, j = 0; i < L; ++i) {
        size_t bit = L >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            std::swap(re[i], re[j]);
            std::swap(im[i], im[j]);
        }
    }
    for (size_t len = 2; len <= L; len <<= 1) {
        const double ang = (inv ? 2.0 : -2.0) * M_PI / (double)len;
        for (size_t i = 0; i < L; i += len) {
            for (size_t k = 0; k < len / 2; ++k) {
                const double wr = cos(ang * (double)k), wi = sin(ang * (double)k);
                const size_t a = i + k, b = a + len / 2;
                const double tr = re[b] * wr - im[b] * wi, ti = re[b] * wi + im[b] * wr;
                re[b] = re[a] - tr;
                im[b] = im[a] - ti;
                re[a] += tr;
                im[a] += ti;
            }
        }
    }
}

// omega(x) = 2 pi^2 B_2(x), B_2(x) = x^2 - x + 1/6: the kernel of the shift-averaged worst-case
// error of a rank-1 lattice in the weighted Korobov space of smoothness 2.
static inline double omega(double x) { return 2.0 * M_PI * M_PI * (x * x - x + 1.0 / 6.0); }

}  // namespace qqmc

// Component-by-component construction for N = 2^m (see qqmc.h).  For each new
// component the criterion of every candidate z is T(z) = sum_k p_k omega({k z / N}),
// p the running product over the earlier components.  Grouping k = 2^j k' (k' odd)
// turns the sum into one sum per modulus M = 2^(m-j) over the odd residues, a group
// {+-5^a}; omega is symmetric, so each sum is a cyclic correlation of length M/4 in
// the exponent a, done by FFT: O(N log N) per component.
extern "C" int qqmc_lattice_cbc(int log2_n, int dims, const double *gamma, uint32_t *z) {
    if (!z || !gamma || log2_n < 3 || log2_n > 24 || dims < 1 || dims > qqmc::kMaxOrder)
        return qqmc::set_error(QQMC_E_INVAL, "qqmc_lattice_cbc: need 3 <= log2_n <= 24, 1 <= dims <= QQMC_MAX_ORDER");
    for (int d = 0; d < dims; ++d)
        if (!(gamma[d] > 0.0) || !isfinite(gamma[d])) return qqmc::set_error(QQMC_E_INVAL, "weights must be > 0");
    const int m = log2_n;
    const uint64_t N = 1ull << m;
    // a_N(r): exponent of odd r = +-5^a mod N
    std::vector<uint32_t> expo(N, 0);
    {
        uint64_t r = 1;
        for (uint64_t a = 0; a < N / 4; ++a) {
            expo[r] = (uint32_t)a;
            expo[N - r] = (uint32_t)a;
            r = (r * 5) & (N - 1);
        }
    }
    std::vector<double> p(N);
    for (uint64_t k = 0; k < N; ++k) p[k] = 1.0 + gamma[0] * qqmc::omega((double)k / (double)N);
    z[0] = 1;
    std::vector<double> T(N / 4);  // T indexed by a_N(z) (z and -z share it)
    for (int d = 1; d < dims; ++d) {
        std::fill(T.begin(), T.end(), p[0] * qqmc::omega(0.0));
        for (int j = 0; j < m; ++j) {
            const uint64_t M = N >> j;  // modulus; odd k' < M, k = 2^j k'
            if (M == 2) {  // k' = 1: omega(1/2) for every z
                const double v = p[(uint64_t)1 << j] * qqmc::omega(0.5);
                for (auto &t : T) t += v;
                continue;
            }
            if (M == 4) {  // k' z = 1 or 3 mod 4: omega(1/4) = omega(3/4)
                const double v = (p[(uint64_t)1 << j] + p[(uint64_t)3 << j]) * qqmc::omega(0.25);
                for (auto &t : T) t += v;
                continue;
            }
            const uint64_t Lj = M / 4;
            std::vector<double> qr(Lj), qi(Lj, 0.0), wr(Lj), wi(Lj, 0.0);
            uint64_t r = 1;
            for (uint64_t b = 0; b < Lj; ++b) {  // Q(b) = q(5^b) + q(-5^b), W(b) = omega(5^b / M)
                qr[b] = p[r << j] + p[(M - r) << j];
                wr[b] = qqmc::omega((double)r / (double)M);
                r = (r * 5) & (M - 1);
            }
            qqmc::fft(qr, qi, false);
            qqmc::fft(wr, wi, false);
            for (uint64_t f = 0; f < Lj; ++f) {  // A^ = W^ conj(Q^)
                const double ar = wr[f] * qr[f] + wi[f] * qi[f], ai = wi[f] * qr[f] - wr[f] * qi[f];
                wr[f] = ar;
                wi[f] = ai;
            }
            qqmc::fft(wr, wi, true);
            for (uint64_t a = 0; a < N / 4; ++a) T[a] += wr[a % Lj] / (double)Lj;
        }
        // smallest odd z <= N/2 whose criterion is within rounding of the minimum
        double lo = T[expo[1]];
        for (uint64_t c = 3; c <= N / 2; c += 2) lo = T[expo[c]] < lo ? T[expo[c]] : lo;
        const double tol = 1e-12 * fabs(lo) + 1e-300;
        uint64_t best = 1;
        for (uint64_t c = 1; c <= N / 2; c += 2)
            if (T[expo[c]] <= lo + tol) {
                best = c;
                break;
            }
        z[d] = (uint32_t)best;
        for (uint64_t k = 0; k < N; ++k)
            p[k] *= 1.0 + gamma[d] * qqmc::omega((double)((k * best) & (N - 1)) / (double)N);
    }
    return QQMC_OK;
}

extern "C" int qqmc_last_error(char *buf, size_t len) {
    if (!buf || len == 0) return QQMC_E_INVAL;
    size_t n = qqmc::g_last_error.size();
    if (n >= len) n = len - 1;
    memcpy(buf, qqmc::g_last_error.data(), n);
    buf[n] = '\0';
    return QQMC_OK;
}

extern "C" int qqmc_direction_numbers(int n_dims, uint32_t *out) {
    if (!out || n_dims < 1 || n_dims > qqmc::kMaxOrder)
        return qqmc::set_error(QQMC_E_INVAL, "qqmc_direction_numbers: n_dims must be in 1..QQMC_MAX_ORDER");
    qqmc::direction_numbers(n_dims, out);
    return QQMC_OK;
}

extern "C" int qqmc_shift_words(uint64_t seed, int n_shifts, int n_dims, uint32_t *out) {
    if (!out || n_shifts < 1 || n_dims < 1) return qqmc::set_error(QQMC_E_INVAL, "qqmc_shift_words: bad arguments");
    qqmc::shift_words(seed, n_shifts, n_dims, out);
    return QQMC_OK;
}
