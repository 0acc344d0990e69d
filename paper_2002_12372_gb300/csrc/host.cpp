// Host-side generators of the product path: Sobol' direction words, digital
// shift words, error reporting.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <string>

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
