// C ABI: problems, single and batched integrations, inspection calls.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "qqmc_internal.h"

using namespace qqmc;

struct qqmc_problem : public qqmc::Problem {};

namespace qqmc {

// ---------------------------------------------------------------- device init
static std::mutex g_init_mu;
static bool g_init_done[64];
static cudaStream_t g_table_stream[64];

static int ensure_device() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return set_error(QQMC_E_CUDA, "device index out of range");
    std::lock_guard<std::mutex> lk(g_init_mu);
    if (g_init_done[dev]) return QQMC_OK;
    int rc = upload_direction_numbers();
    if (rc != QQMC_OK) return rc;
    // Table builds get their own non-blocking stream at the highest priority, so that a problem
    // created while long integrations run (a server admitting a new round) neither waits for
    // them nor queues its kernel behind their pending blocks.
    int least = 0, greatest = 0;
    e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&g_table_stream[dev], cudaStreamNonBlocking, greatest);
    if (e != cudaSuccess) return cuda_error(e, "table stream");
    g_init_done[dev] = true;
    return QQMC_OK;
}

static cudaStream_t table_stream() {
    int dev = 0;
    cudaGetDevice(&dev);
    return dev >= 0 && dev < 64 ? g_table_stream[dev] : nullptr;
}

// ---------------------------------------------------------------- tuning
static std::mutex g_tune_mu;
static Tuning g_tune[2][2][kMaxOrder + 1];  // [precision][pair tree][order]
static bool g_tune_set[2][2][kMaxOrder + 1];

static Tuning default_tuning(int precision, int order) {
    Tuning t;
    // FP64: breadth-first expansion below the tree leaf, 2 vertices per lane
    // (the FP64 pipe is the bound, so fewer flops win; measured best on GB300
    // at orders 11..16); mixed: 5 vertices per lane in registers (the
    // cooperative steps are latency-bound in FP32).
    (void)order;
    t.flat = precision == QQMC_PREC_FP64 ? 2 : 5;
    t.flat_min = t.flat;
    t.warps_per_block = precision == QQMC_PREC_FP64 ? 2 : 4;
    return t;
}

Tuning get_tuning(int precision, int order, bool pairs) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const int p = precision == QQMC_PREC_FP64 ? 0 : 1, t = pairs ? 1 : 0;
    if (order >= 1 && order <= kMaxOrder && g_tune_set[p][t][order]) return g_tune[p][t][order];
    return default_tuning(precision, order);
}

bool use_pairs(const Problem &P, int precision) {
    if (P.elimination == QQMC_ELIM_PAIRS) return true;
    if (P.elimination == QQMC_ELIM_SINGLE) return false;
    const double dv = hypot(P.g0_re, P.g0_im - P.params.alpha);  // |g^<(0) - i alpha|
    const double scale = fmax(hypot(P.g0_re, P.g0_im), hypot(P.g0_re, P.g0_im - 1.0));  // g^>(0) = g^<(0) - i
    return dv < (precision == QQMC_PREC_FP64 ? 0.01 : 0.25) * scale;
}

}  // namespace qqmc

namespace qqmc {

bool valid_params(const qqmc_params *p, std::string &why) {
    if (!p) { why = "params is NULL"; return false; }
    if (!(p->gamma > 0) || !isfinite(p->gamma)) { why = "gamma must be > 0"; return false; }
    if (!isfinite(p->eps_d)) { why = "eps_d must be finite"; return false; }
    if (!(p->t_max > 0) || !isfinite(p->t_max)) { why = "t_max must be > 0"; return false; }
    if (!(p->tau > 0) || !isfinite(p->tau)) { why = "tau must be > 0"; return false; }
    if (!isfinite(p->alpha)) { why = "alpha must be finite"; return false; }
    if (p->n_table < 4 || p->n_table > (1 << 20) || (p->n_table & 1)) {
        why = "n_table must be even and in 4..2^20";
        return false;
    }
    if (p->observable != QQMC_OBS_CHARGE && p->observable != QQMC_OBS_CURRENT) {
        why = "observable must be QQMC_OBS_CHARGE or QQMC_OBS_CURRENT";
        return false;
    }
    if (!(p->half_bandwidth >= 0) || !isfinite(p->half_bandwidth)) { why = "half_bandwidth must be >= 0"; return false; }
    if (!(p->bias >= 0) || !isfinite(p->bias)) { why = "bias must be >= 0"; return false; }
    if (p->half_bandwidth == 0.0 && p->bias != 0.0) {
        why = "a bias needs finite-bandwidth leads (half_bandwidth > 0)";
        return false;
    }
    if (p->half_bandwidth == 0.0 && p->observable == QQMC_OBS_CURRENT) {
        why = "the current needs finite-bandwidth leads (half_bandwidth > 0)";
        return false;
    }
    if (p->half_bandwidth > 0.0 && !(fabs(p->eps_d) + p->gamma < p->half_bandwidth)) {
        why = "|eps_d| + gamma must be below half_bandwidth (no bound state outside the band)";
        return false;
    }
    return true;
}

// Order-0 value of the observable: Q_0 = -2i g^<(0) = 2 <n>, I_0 = -4 Re gamma g^<_01(0).
double order0_value(const Problem &pr) {
    return pr.params.observable == QQMC_OBS_CURRENT ? -4.0 * pr.c0_re : 2.0 * pr.g0_im;
}

}  // namespace qqmc

static int alloc_problem(const qqmc_params *p, qqmc_problem **out) {
    std::string why;
    if (!out) return set_error(QQMC_E_INVAL, "out is NULL");
    *out = nullptr;
    if (!valid_params(p, why)) return set_error(QQMC_E_INVAL, "qqmc params: " + why);
    int rc = ensure_device();
    if (rc != QQMC_OK) return rc;
    qqmc_problem *pr = new (std::nothrow) qqmc_problem();
    if (!pr) return set_error(QQMC_E_NOMEM, "host allocation failed");
    pr->params = *p;
    pr->L = p->n_table;
    pr->h = 2.0 * p->t_max / (double)(p->n_table - 1);
    cudaGetDevice(&pr->device);
    size_t nh = (size_t)pr->L / 2 + 1;
    cudaError_t e = cudaMalloc(&pr->d_table, nh * sizeof(dbl4));
    if (e == cudaSuccess) e = cudaMalloc(&pr->d_table32, nh * sizeof(float4));
    if (e == cudaSuccess && p->observable == QQMC_OBS_CURRENT) {
        e = cudaMalloc(&pr->d_col, nh * sizeof(dbl4));
        if (e == cudaSuccess) e = cudaMalloc(&pr->d_col32, nh * sizeof(float4));
    }
    if (e != cudaSuccess) {
        cudaFree(pr->d_table);
        cudaFree(pr->d_table32);
        cudaFree(pr->d_col);
        delete pr;
        return set_error(QQMC_E_NOMEM, std::string("device allocation of the tables failed: ") + cudaGetErrorString(e));
    }
    *out = pr;
    return QQMC_OK;
}

extern "C" int qqmc_create_problem(const qqmc_params *p, qqmc_problem **out) {
    qqmc_problem *pr = nullptr;
    int rc = alloc_problem(p, &pr);  // validates p and initialises the device
    if (rc != QQMC_OK) return rc;
    cudaStream_t ts = table_stream();
    if (p->half_bandwidth > 0.0) {  // semicircular leads: numerical tables, g^<(0) from the same quadrature
        double zero[4] = {0, 0, 0, 0};
        rc = launch_lead_table(*pr, ts, zero);
        pr->g0_re = zero[0];
        pr->g0_im = zero[1];
        pr->c0_re = zero[2];
        pr->c0_im = zero[3];
    } else {
        pr->g0_re = 0.0;
        pr->g0_im = 0.5 - atan(p->eps_d / p->gamma) / M_PI;
        rc = launch_gf_table(*pr, ts);
        if (rc == QQMC_OK) {
            cudaError_t e = cudaStreamSynchronize(ts);
            if (e != cudaSuccess) rc = cuda_error(e, "table build");
        }
    }
    if (rc != QQMC_OK) {
        qqmc_destroy_problem(pr);
        return rc;
    }
    *out = pr;
    return QQMC_OK;
}

extern "C" int qqmc_create_problem_tables(const qqmc_params *p, const double *gl, const double *gg, double g0_re,
                                          double g0_im, qqmc_problem **out) {
    if (!gl || !gg) return set_error(QQMC_E_INVAL, "tables are NULL");
    if (!isfinite(g0_re) || !isfinite(g0_im)) return set_error(QQMC_E_INVAL, "g0 must be finite");
    if (p && p->observable != QQMC_OBS_CHARGE)
        return set_error(QQMC_E_INVAL, "caller tables start as a charge problem; qqmc_set_current_tables switches it");
    qqmc_problem *pr = nullptr;
    int rc = alloc_problem(p, &pr);
    if (rc != QQMC_OK) return rc;
    pr->g0_re = g0_re;
    pr->g0_im = g0_im;
    const int L = pr->L;
    const int k0 = L / 2 - 1;
    std::vector<dbl4> h(L / 2 + 1);
    std::vector<float4> h32(L / 2 + 1);
    for (int q = 0; q <= L / 2; ++q) {
        int k = k0 + q;
        h[q] = make_double4_32a(gl[2 * k], gl[2 * k + 1], gg[2 * k], gg[2 * k + 1]);
        h32[q] = make_float4((float)gl[2 * k], (float)gl[2 * k + 1], (float)gg[2 * k], (float)gg[2 * k + 1]);
    }
    cudaError_t e = cudaMemcpy(pr->d_table, h.data(), h.size() * sizeof(dbl4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pr->d_table32, h32.data(), h32.size() * sizeof(float4), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        qqmc_destroy_problem(pr);
        return cuda_error(e, "table upload");
    }
    *out = pr;
    return QQMC_OK;
}

extern "C" int qqmc_set_current_tables(qqmc_problem *pr, const double *cl, const double *cg, double c0_re,
                                       double c0_im) {
    if (!pr || !cl || !cg) return set_error(QQMC_E_INVAL, "qqmc_set_current_tables: NULL argument");
    if (!isfinite(c0_re) || !isfinite(c0_im)) return set_error(QQMC_E_INVAL, "c0 must be finite");
    const int L = pr->L;
    const size_t nh = (size_t)L / 2 + 1;
    std::vector<dbl4> h(nh);
    std::vector<float4> h32(nh);
    for (int k = 0; k <= L / 2; ++k) {
        h[k] = make_double4_32a(cl[2 * k], cl[2 * k + 1], cg[2 * k], cg[2 * k + 1]);
        h32[k] = make_float4((float)cl[2 * k], (float)cl[2 * k + 1], (float)cg[2 * k], (float)cg[2 * k + 1]);
    }
    cudaError_t e = cudaSuccess;
    if (!pr->d_col) {
        e = cudaMalloc(&pr->d_col, nh * sizeof(dbl4));
        if (e == cudaSuccess) e = cudaMalloc(&pr->d_col32, nh * sizeof(float4));
        if (e != cudaSuccess) {
            cudaFree(pr->d_col);
            pr->d_col = nullptr;
            pr->d_col32 = nullptr;
            return set_error(QQMC_E_NOMEM, "device allocation of the dot-lead tables failed");
        }
    }
    e = cudaMemcpy(pr->d_col, h.data(), nh * sizeof(dbl4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pr->d_col32, h32.data(), nh * sizeof(float4), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "dot-lead table upload");
    pr->c0_re = c0_re;
    pr->c0_im = c0_im;
    pr->params.observable = QQMC_OBS_CURRENT;
    return QQMC_OK;
}

extern "C" int qqmc_set_stack_policy(int precision, int min_order) {
    if (precision != QQMC_PREC_FP64 && precision != QQMC_PREC_MIXED)
        return set_error(QQMC_E_INVAL, "precision must be QQMC_PREC_FP64 or QQMC_PREC_MIXED");
    set_stack_policy(precision, min_order);
    return QQMC_OK;
}

extern "C" int qqmc_set_lattice(qqmc_problem *pr, int log2_n, const uint32_t *z, int dims, int bakers) {
    if (!pr) return set_error(QQMC_E_INVAL, "problem is NULL");
    if (!z) {  // back to Sobol'
        cudaFree(pr->d_lat_z);
        pr->d_lat_z = nullptr;
        pr->lat_m = pr->lat_dims = 0;
        return QQMC_OK;
    }
    if (log2_n < 1 || log2_n > 32 || dims < 1 || dims > kMaxOrder)
        return set_error(QQMC_E_INVAL, "qqmc_set_lattice: need 1 <= log2_n <= 32 and 1 <= dims <= QQMC_MAX_ORDER");
    for (int d = 0; d < dims; ++d)
        if (!(z[d] & 1u)) return set_error(QQMC_E_INVAL, "qqmc_set_lattice: components must be odd (units mod 2^m)");
    if (!pr->d_lat_z) {
        cudaError_t e = cudaMalloc(&pr->d_lat_z, sizeof(uint32_t) * kMaxOrder);
        if (e != cudaSuccess) {
            pr->d_lat_z = nullptr;
            return set_error(QQMC_E_NOMEM, "device allocation of the lattice failed");
        }
    }
    cudaError_t e = cudaMemcpy(pr->d_lat_z, z, sizeof(uint32_t) * dims, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "lattice upload");
    pr->lat_m = log2_n + (bakers ? 64 : 0);
    pr->lat_dims = dims;
    return QQMC_OK;
}

extern "C" int qqmc_problem_current_tables(const qqmc_problem *pr, double *cl, double *cg, double *c0) {
    if (!pr) return set_error(QQMC_E_INVAL, "problem is NULL");
    if (pr->params.observable != QQMC_OBS_CURRENT || !pr->d_col)
        return set_error(QQMC_E_INVAL, "problem has no dot-lead tables (charge observable)");
    const int L = pr->L;
    std::vector<dbl4> h(L / 2 + 1);
    cudaError_t e = cudaMemcpy(h.data(), pr->d_col, h.size() * sizeof(dbl4), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "dot-lead table download");
    for (int k = 0; k <= L / 2; ++k) {
        if (cl) { cl[2 * k] = h[k].x; cl[2 * k + 1] = h[k].y; }
        if (cg) { cg[2 * k] = h[k].z; cg[2 * k + 1] = h[k].w; }
    }
    if (c0) { c0[0] = pr->c0_re; c0[1] = pr->c0_im; }
    return QQMC_OK;
}

extern "C" int qqmc_destroy_problem(qqmc_problem *pr) {
    if (!pr) return QQMC_OK;
    cudaFree(pr->d_table);
    cudaFree(pr->d_table32);
    cudaFree(pr->d_col);
    cudaFree(pr->d_col32);
    cudaFree(pr->d_lat_z);
    for (int n = 0; n <= kMaxOrder; ++n) cudaFree(pr->d_proj[n]);
    delete pr;
    return QQMC_OK;
}

extern "C" int qqmc_problem_tables(const qqmc_problem *pr, double *gl, double *gg, double *g0) {
    if (!pr) return set_error(QQMC_E_INVAL, "problem is NULL");
    const int L = pr->L;
    std::vector<dbl4> h(L / 2 + 1);
    cudaError_t e = cudaMemcpy(h.data(), pr->d_table, h.size() * sizeof(dbl4), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "table download");
    const int k0 = L / 2 - 1;
    for (int k = 0; k < L; ++k) {
        dbl4 v;
        if (k >= k0) {
            v = h[k - k0];
        } else {  // mirror: node k is -tau of node L-1-k
            dbl4 m = h[(L - 1 - k) - k0];
            v = make_double4_32a(-m.x, m.y, -m.z, m.w);
        }
        if (gl) { gl[2 * k] = v.x; gl[2 * k + 1] = v.y; }
        if (gg) { gg[2 * k] = v.z; gg[2 * k + 1] = v.w; }
    }
    if (g0) { g0[0] = pr->g0_re; g0[1] = pr->g0_im; }
    return QQMC_OK;
}

// ---------------------------------------------------------------- plans
struct qqmc_plan {
    std::vector<qqmc_item> items;   // caller order
    std::vector<ItemDev> hitems;    // device order: highest order first (longest work first)
    std::vector<int> perm;          // device position -> caller index
    int n_warp = 0;                 // items [0, n_warp) run one warp per point, the rest one lane per point
    long long chunks_lane = 0;
    // Warp-per-point items in groups of equal tuned shape (flat depth), one
    // persistent launch per group with shared memory sized for its own
    // highest order; every item runs with its own order's flat depth.
    struct Group {
        int first = 0, count = 0, n_max = 0;
        long long chunks = 0;
        Tuning tune{};
        bool pairs = false;          // the pair-block tree (else the single-vertex tree)
        long long gstack_warps = 0;  // warps with a device-memory stack slice, fixed at creation
    };
    std::vector<Group> groups;
    int precision = 0;
    int n_max = 0;
    long long total_chunks = 0;
    int total_shifts = 0;
    ItemDev *d_items = nullptr;
    uint32_t *d_shifts = nullptr;
    double *d_partials = nullptr;
    unsigned int *d_inside = nullptr;
    unsigned long long *d_counter = nullptr;
    double *d_out = nullptr;
    unsigned long long *d_counts = nullptr;
    unsigned int *d_bad = nullptr;  // per shift: work units whose partial sum was not finite
    void *d_gstack = nullptr;       // FP64 tree stack in device memory (orders whose stack exceeds shared memory)
    long long gstack_warps = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ek0 = nullptr, ek1 = nullptr;
    bool kernel_timed = false;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t gstream = nullptr;
    bool launched = false;
    int device = 0;
};

static void free_plan(qqmc_plan *pl) {
    if (!pl) return;
    if (pl->gexec) cudaGraphExecDestroy(pl->gexec);
    cudaFree(pl->d_items);
    cudaFree(pl->d_shifts);
    cudaFree(pl->d_partials);
    cudaFree(pl->d_inside);
    cudaFree(pl->d_counter);
    cudaFree(pl->d_out);
    cudaFree(pl->d_counts);
    cudaFree(pl->d_bad);
    cudaFree(pl->d_gstack);
    if (pl->ev0) cudaEventDestroy(pl->ev0);
    if (pl->ev1) cudaEventDestroy(pl->ev1);
    if (pl->ek0) cudaEventDestroy(pl->ek0);
    if (pl->ek1) cudaEventDestroy(pl->ek1);
    delete pl;
}

extern "C" int qqmc_plan_create(const qqmc_item *items, int n_items, int precision, qqmc_plan **out) {
    if (!out) return set_error(QQMC_E_INVAL, "out is NULL");
    *out = nullptr;
    if (!items || n_items < 1 || n_items > 65536) return set_error(QQMC_E_INVAL, "n_items must be in 1..65536");
    if (precision != QQMC_PREC_FP64 && precision != QQMC_PREC_MIXED)
        return set_error(QQMC_E_INVAL, "precision must be QQMC_PREC_FP64 or QQMC_PREC_MIXED");
    for (int i = 0; i < n_items; ++i) {
        const qqmc_item &it = items[i];
        if (!it.problem) return set_error(QQMC_E_INVAL, "item has no problem");
        if (it.order < 1 || it.order > kMaxOrder) return set_error(QQMC_E_RANGE, "order outside 1..QQMC_MAX_ORDER");
        if (it.n_points < 1 || it.n_points > (1ull << QQMC_MAX_POINTS_LOG2))
            return set_error(QQMC_E_INVAL, "n_points must be in 1..2^30");
        if (it.n_shifts < 1 || it.n_shifts > 1024) return set_error(QQMC_E_INVAL, "n_shifts must be in 1..1024");
        if (it.first_index > (1ull << 40)) return set_error(QQMC_E_INVAL, "first_index too large");
        const Problem *P = it.problem;
        if (P->d_lat_z && (it.order > P->lat_dims || it.first_index + it.n_points > (1ull << (P->lat_m & 63))))
            return set_error(QQMC_E_INVAL, "item outside its problem's lattice (order > its dimension or index >= N)");
    }
    int rc = ensure_device();
    if (rc != QQMC_OK) return rc;
    qqmc_plan *pl = new (std::nothrow) qqmc_plan();
    if (!pl) return set_error(QQMC_E_NOMEM, "host allocation failed");
    cudaGetDevice(&pl->device);
    pl->items.assign(items, items + n_items);
    pl->precision = precision;
    size_t shift_words_total = 0, chunk_total = 0;
    // Work units.  A chunk is 32 consecutive point indices of one shift.  Items with few chunks are
    // cut finer until an item has about kTargetUnits units (the persistent grid needs work for every
    // warp; the chunks alone would leave most of it idle):
    //  1. a chunk's points go to 2^pbits units of 32 >> pbits points each (pbits <= 5), which costs
    //     nothing but the point generation of the idle lanes;
    //  2. then each point's Keldysh tree goes to 2^split units, each a subtree with the first `split`
    //     bits of its leaf index fixed (a_2, then two per depth-first level).  Such a unit repeats
    //     the pair interpolation, the root and its subtree's fixed prefix, so a subtree keeps at
    //     least 2^kMinSubtreeLevels leaves, which holds that repeated work to a few per cent.
    // The cut depends on the item alone (batched and single runs agree bit for bit).
    constexpr long long kTargetUnits = 1 << 14;
    constexpr int kMinSubtreeLevels = 4;
    // the Keldysh-sum tree of each item (the problem's elimination order at this precision)
    std::vector<char> pv(n_items);
    for (int i = 0; i < n_items; ++i) pv[i] = use_pairs(*items[i].problem, precision);
    auto lane_mode = [&](int i) {
        return items[i].order <= kLaneMaxOrder && get_tuning(precision, items[i].order, pv[i]).flat == 1;
    };
    std::vector<char> lmv(n_items);
    std::vector<int> pbits_of(n_items, 0), split_of(n_items, 0);
    for (int i = 0; i < n_items; ++i) {
        const qqmc_item &it = items[i];
        lmv[i] = lane_mode(i);
        if (lmv[i]) continue;  // one point per lane: no cut
        const int levels = tree_leaf_bits(it.order, pv[i]);  // bits of the tree's leaf index
        const long long units = (long long)((it.n_points + kChunk - 1) / kChunk) * it.n_shifts;
        int pb = 0, sp = 0;
        while (pb < 5 && (units << pb) < kTargetUnits) ++pb;
        while (sp < levels - kMinSubtreeLevels && (units << (pb + sp)) < kTargetUnits) ++sp;
        pbits_of[i] = pb;
        split_of[i] = sp;
    }
    for (int i = 0; i < n_items; ++i) {
        const qqmc_item &it = items[i];
        pl->n_max = it.order > pl->n_max ? it.order : pl->n_max;
        shift_words_total += (size_t)it.n_shifts * it.order;
        size_t cps = ((it.n_points + kChunk - 1) / kChunk) << (pbits_of[i] + split_of[i]);
        chunk_total += cps * it.n_shifts;
        pl->total_shifts += it.n_shifts;
    }
    pl->total_chunks = (long long)chunk_total;
    cudaError_t e = cudaMalloc(&pl->d_items, sizeof(ItemDev) * n_items);
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_shifts, sizeof(uint32_t) * shift_words_total);
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_partials, sizeof(double) * 4 * chunk_total);
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_inside, sizeof(unsigned int) * chunk_total);
    // work counters (one per launch) and, after them, the execution span of the determinant launches
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_counter, (kMaxOrder + 4) * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_out, sizeof(double) * 2 * pl->total_shifts);
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_counts, sizeof(unsigned long long) * pl->total_shifts);
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_bad, sizeof(unsigned int) * pl->total_shifts);
    if (e != cudaSuccess) {
        free_plan(pl);
        return set_error(QQMC_E_NOMEM, std::string("device allocation of the plan failed: ") + cudaGetErrorString(e));
    }
    // Device order: the warp-per-point items grouped by tree and their order's
    // tuned flat depth (groups holding higher orders first), then the
    // one-point-per-lane items (orders <= 4 whose tuning asks for it); within a
    // group highest order first, then more points first, so the longest items
    // start early and the persistent grid drains evenly.  Each launch has its own
    // chunk numbering.
    auto flat_of = [&](int i) {
        const int f = get_tuning(precision, items[i].order, pv[i]).flat;
        return f < 2 ? 2 : f;
    };
    auto key_of = [&](int i) { return 6 * pv[i] + flat_of(i); };  // launch group: (tree, flat depth)
    int group_top[12] = {};  // highest order per group
    for (int i = 0; i < n_items; ++i)
        if (!lmv[i] && items[i].order > group_top[key_of(i)]) group_top[key_of(i)] = items[i].order;
    pl->perm.resize(n_items);
    for (int i = 0; i < n_items; ++i) pl->perm[i] = i;
    std::stable_sort(pl->perm.begin(), pl->perm.end(), [&](int a, int b) {
        if (lmv[a] != lmv[b]) return !lmv[a];
        if (!lmv[a]) {
            const int fa = key_of(a), fb = key_of(b);
            if (group_top[fa] != group_top[fb]) return group_top[fa] > group_top[fb];
            if (fa != fb) return fa > fb;
        }
        if (items[a].order != items[b].order) return items[a].order > items[b].order;
        return items[a].n_points > items[b].n_points;
    });
    std::vector<uint32_t> hs(shift_words_total);
    size_t so = 0, co = 0;
    long long cl = 0;
    pl->hitems.resize(n_items);
    for (int q = 0; q < n_items; ++q) {
        const int ci = pl->perm[q];
        const qqmc_item &it = items[ci];
        const bool lm = lmv[ci];
        const qqmc_problem *pr = it.problem;
        if (it.shift_words)
            memcpy(hs.data() + so, it.shift_words, sizeof(uint32_t) * it.n_shifts * it.order);
        else
            shift_words(pr->params.seed, it.n_shifts, it.order, hs.data() + so);
        ItemDev &d = pl->hitems[q];
        d.table = pr->d_table;
        d.table32 = pr->d_table32;
        d.shifts = pl->d_shifts + so;
        d.pbits = pbits_of[ci];
        d.split = split_of[ci];
        size_t cps = ((it.n_points + kChunk - 1) / kChunk) << (d.pbits + d.split);  // work units per shift
        d.partials = pl->d_partials + 4 * co;
        d.inside = pl->d_inside + co;
        d.g0_re = pr->g0_re;
        d.g0_im = pr->g0_im;
        d.t = pr->params.t_max;
        d.tau = pr->params.tau;
        d.T = pr->params.t_max;
        d.h = pr->h;
        d.first_index = (long long)it.first_index;
        d.n_points = (long long)it.n_points;
        d.order = it.order;
        d.n_shifts = it.n_shifts;
        d.L = pr->L;
        d.chunks_per_shift = (int)cps;
        d.flat = lm ? 1 : flat_of(ci);
        d.alpha = pr->params.alpha;
        d.col = pr->params.observable == QQMC_OBS_CURRENT ? pr->d_col : nullptr;
        d.col32 = pr->params.observable == QQMC_OBS_CURRENT ? pr->d_col32 : nullptr;
        d.lat_z = pr->d_lat_z;
        d.lat_m = pr->lat_m;
        d.proj = pr->d_proj[it.order];
        d.proj_cells = pr->proj_cells[it.order];
        if (lm) {
            d.chunk_begin = cl;
            cl += (long long)cps * it.n_shifts;
        } else {
            if (pl->groups.empty() || pl->groups.back().tune.flat != d.flat ||
                pl->groups.back().pairs != (pv[ci] != 0)) {
                qqmc_plan::Group g;
                g.first = q;
                g.n_max = it.order;  // highest order first within a group
                g.pairs = pv[ci] != 0;
                g.tune = get_tuning(precision, it.order, g.pairs);
                g.tune.flat = g.tune.flat_min = d.flat;
                pl->groups.push_back(g);
            }
            qqmc_plan::Group &g = pl->groups.back();
            d.chunk_begin = g.chunks;
            g.chunks += (long long)cps * it.n_shifts;
            ++g.count;
            ++pl->n_warp;
        }
        so += (size_t)it.n_shifts * it.order;
        co += cps * it.n_shifts;
    }
    pl->chunks_lane = cl;
    // the groups launch one after another on the plan's stream and share one tree-stack buffer
    // (each group keeps the warp count it was sized for, so a later change of the stack policy
    // cannot make a launch index past the buffer)
    size_t gs_bytes = 0;
    for (auto &g : pl->groups) {
        size_t bpw = 0;
        const long long w = detsum_gstack_warps(g.n_max, precision, g.tune, g.pairs, &bpw);
        g.gstack_warps = w;
        if ((size_t)w * bpw > gs_bytes) gs_bytes = (size_t)w * bpw;
        if (w > pl->gstack_warps) pl->gstack_warps = w;
    }
    if (gs_bytes > 0) {
        e = cudaMalloc(&pl->d_gstack, gs_bytes);
        if (e != cudaSuccess) {
            free_plan(pl);
            return set_error(QQMC_E_NOMEM, "device allocation of the tree stack failed");
        }
    }
    e = cudaMemcpy(pl->d_shifts, hs.data(), sizeof(uint32_t) * shift_words_total, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(pl->d_items, pl->hitems.data(), sizeof(ItemDev) * n_items, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaEventCreate(&pl->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&pl->ev1);
    if (e == cudaSuccess) e = cudaEventCreate(&pl->ek0);
    if (e == cudaSuccess) e = cudaEventCreate(&pl->ek1);
    if (e != cudaSuccess) {
        free_plan(pl);
        return cuda_error(e, "plan upload");
    }
    *out = pl;
    return QQMC_OK;
}

static unsigned long long *plan_span(const qqmc_plan *pl) { return pl->d_counter + kMaxOrder + 2; }

static cudaError_t enqueue_plan(qqmc_plan *pl, cudaStream_t s, bool timed) {
    const int ng = (int)pl->groups.size();
    cudaError_t e = cudaMemsetAsync(pl->d_counter, 0, (ng + 1) * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(plan_span(pl), 0xff, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(plan_span(pl) + 1, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (timed && (e = cudaEventRecord(pl->ek0, s)) != cudaSuccess) return e;
    for (int gi = 0; gi < ng; ++gi) {
        const auto &g = pl->groups[gi];
        // a group's share of the device-memory stack (the buffer holds the largest group's need);
        // a group sized without one gets none, and then runs the shared-memory stack or fails cleanly
        const long long w = g.gstack_warps;
        e = launch_detsum(pl->d_items + g.first, g.count, g.chunks, pl->d_counter + gi, g.n_max, pl->precision, g.tune,
                          g.pairs, w > 0 ? pl->d_gstack : nullptr, w, plan_span(pl), s);
        if (e != cudaSuccess) return e;
    }
    const int n_lane = (int)pl->items.size() - pl->n_warp;
    if (n_lane > 0) {
        e = launch_lane(pl->d_items + pl->n_warp, n_lane, pl->chunks_lane, pl->d_counter + ng, pl->precision,
                        plan_span(pl), s);
        if (e != cudaSuccess) return e;
    }
    if (timed && (e = cudaEventRecord(pl->ek1, s)) != cudaSuccess) return e;
    return launch_reduce(pl->d_items, (int)pl->items.size(), pl->total_shifts, pl->d_out, pl->d_counts, pl->d_bad, s);
}

extern "C" int qqmc_plan_launch(qqmc_plan *pl, void *stream, int use_graph) {
    if (!pl) return set_error(QQMC_E_INVAL, "plan is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaEventRecord(pl->ev0, s);
    if (e != cudaSuccess) return cuda_error(e, "event record");
    if (use_graph) {
        if (!pl->gexec || pl->gstream != s) {
            if (pl->gexec) {
                cudaGraphExecDestroy(pl->gexec);
                pl->gexec = nullptr;
            }
            cudaStream_t cs = s;
            bool own = false;
            if (cs == 0) {  // the legacy stream cannot be captured: capture on a private stream
                e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
                if (e != cudaSuccess) return cuda_error(e, "stream create");
                own = true;
            }
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e2 = enqueue_plan(pl, cs, false);
                e = cudaStreamEndCapture(cs, &g);
                if (e2 != cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&pl->gexec, g, 0);
            if (g) cudaGraphDestroy(g);
            if (own) cudaStreamDestroy(cs);
            if (e != cudaSuccess) return cuda_error(e, "graph capture");
            pl->gstream = s;
        }
        e = cudaGraphLaunch(pl->gexec, s);
        pl->kernel_timed = false;
    } else {
        e = enqueue_plan(pl, s, true);
        pl->kernel_timed = true;
    }
    if (e != cudaSuccess) return cuda_error(e, "plan launch");
    e = cudaEventRecord(pl->ev1, s);
    if (e != cudaSuccess) return cuda_error(e, "event record");
    pl->launched = true;
    return QQMC_OK;
}

extern "C" int qqmc_plan_kernel_count(const qqmc_plan *pl) {
    if (!pl) return 0;
    return 1 + (int)pl->groups.size() + ((int)pl->items.size() > pl->n_warp ? 1 : 0);
}

extern "C" int qqmc_plan_timing(const qqmc_plan *pl, double *kernel_ms, double *total_ms) {
    if (!pl || !pl->launched) return set_error(QQMC_E_INVAL, "plan is NULL or was not launched");
    cudaError_t e = cudaEventSynchronize(pl->ev1);
    if (e != cudaSuccess) return cuda_error(e, "plan execution");
    float a = 0.f, k = 0.f;
    cudaEventElapsedTime(&a, pl->ev0, pl->ev1);
    if (pl->kernel_timed) cudaEventElapsedTime(&k, pl->ek0, pl->ek1);
    if (kernel_ms) *kernel_ms = k;
    if (total_ms) *total_ms = a;
    return QQMC_OK;
}

static void finish_result(const qqmc_item &it, const double *S, const unsigned long long *cnt,
                          const unsigned int *bad, float ms, qqmc_result *r) {
    const int K = it.n_shifts;
    const double N = (double)it.n_points;
    double mean = 0.0, imax = 0.0;
    uint64_t nin = 0, nbad = 0;
    std::vector<double> q(K);
    const bool current = it.problem->params.observable == QQMC_OBS_CURRENT;
    for (int k = 0; k < K; ++k) {
        // charge: Q = -2i S / N (real part; the imaginary part is zero in exact arithmetic);
        // current: I = -4 Re S / N (the other component, -4 Im S / N, is reported as "imag")
        q[k] = current ? -4.0 * S[2 * k] / N : 2.0 * S[2 * k + 1] / N;
        double qi = current ? -4.0 * S[2 * k + 1] / N : -2.0 * S[2 * k] / N;
        mean += q[k];
        imax = fabs(qi) > imax ? fabs(qi) : imax;
        nin += cnt[k];
        nbad += bad[k];
    }
    mean /= K;
    double var = 0.0;
    for (int k = 0; k < K; ++k) var += (q[k] - mean) * (q[k] - mean);
    r->order = it.order;
    r->n_shifts = K;
    r->n_points = it.n_points;
    r->q_mean = mean;
    r->q_err = K > 1 ? sqrt(var / (K - 1)) / sqrt((double)K) : 0.0;
    r->q_imag_absmax = imax;
    r->n_in_domain = nin;
    r->device_ms = ms;
    r->n_nonfinite = nbad;
}

extern "C" int qqmc_plan_results(qqmc_plan *pl, qqmc_result *results, double *per_shift) {
    if (!pl) return set_error(QQMC_E_INVAL, "plan is NULL");
    if (!pl->launched) return set_error(QQMC_E_INVAL, "plan was not launched");
    cudaError_t e = cudaEventSynchronize(pl->ev1);
    if (e != cudaSuccess) return cuda_error(e, "plan execution");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, pl->ev0, pl->ev1);
    std::vector<double> S(2 * (size_t)pl->total_shifts);
    std::vector<unsigned long long> cnt(pl->total_shifts);
    std::vector<unsigned int> bad(pl->total_shifts);
    e = cudaMemcpy(S.data(), pl->d_out, sizeof(double) * S.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(cnt.data(), pl->d_counts, sizeof(unsigned long long) * cnt.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(bad.data(), pl->d_bad, sizeof(unsigned int) * bad.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "result download");
    uint64_t nbad = 0;
    int first_bad = -1;
    // per-shift outputs are in device order; caller offsets for per_shift
    const size_t n_items = pl->items.size();
    std::vector<size_t> user_off(n_items + 1, 0);
    for (size_t i = 0; i < n_items; ++i) user_off[i + 1] = user_off[i] + pl->items[i].n_shifts;
    size_t g = 0;
    for (size_t q = 0; q < n_items; ++q) {
        const int i = pl->perm[q];
        const qqmc_item &it = pl->items[i];
        for (int k = 0; k < it.n_shifts; ++k) {
            nbad += bad[g + k];
            if (bad[g + k] && first_bad < 0) first_bad = i;
        }
        if (results) finish_result(it, S.data() + 2 * g, cnt.data() + g, bad.data() + g, ms, &results[i]);
        if (per_shift)
            for (int k = 0; k < it.n_shifts; ++k) {
                per_shift[2 * (user_off[i] + k)] = S[2 * (g + k)] / (double)it.n_points;
                per_shift[2 * (user_off[i] + k) + 1] = S[2 * (g + k) + 1] / (double)it.n_points;
            }
        g += it.n_shifts;
    }
    if (nbad)
        return set_error(QQMC_E_NONFINITE, std::to_string(nbad) + " work unit(s) gave a NaN or infinite integrand sum "
                                           "(first affected item " + std::to_string(first_bad) +
                                           "); check the Green-function tables");
    return QQMC_OK;
}

extern "C" int qqmc_plan_device_span(const qqmc_plan *pl, uint64_t *start_ns, uint64_t *end_ns) {
    if (!pl || !pl->launched || !start_ns || !end_ns)
        return set_error(QQMC_E_INVAL, "qqmc_plan_device_span: plan not launched or NULL output");
    cudaError_t e = cudaEventSynchronize(pl->ev1);
    if (e != cudaSuccess) return cuda_error(e, "plan execution");
    unsigned long long v[2];
    e = cudaMemcpy(v, plan_span(pl), sizeof(v), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "span download");
    *start_ns = v[0];
    *end_ns = v[1];
    return QQMC_OK;
}

extern "C" int qqmc_plan_chunk_sums(const qqmc_plan *pl, int item, int shift, const int64_t *chunk, int count,
                                    double *out) {
    if (!pl || !pl->launched) return set_error(QQMC_E_INVAL, "plan is NULL or was not launched");
    if (item < 0 || item >= (int)pl->items.size() || !chunk || !out || count < 0)
        return set_error(QQMC_E_INVAL, "qqmc_plan_chunk_sums: bad item or buffers");
    int q = 0;
    while (pl->perm[q] != item) ++q;
    const ItemDev &d = pl->hitems[q];
    if (shift < 0 || shift >= d.n_shifts) return set_error(QQMC_E_INVAL, "qqmc_plan_chunk_sums: bad shift");
    cudaError_t e = cudaEventSynchronize(pl->ev1);
    if (e != cudaSuccess) return cuda_error(e, "plan execution");
    const int nsub = 1 << (d.pbits + d.split);  // a chunk's sum is split over its work units
    std::vector<double> buf(4 * (size_t)nsub);
    for (int i = 0; i < count; ++i) {
        if (chunk[i] < 0 || chunk[i] >= (int64_t)(d.chunks_per_shift >> (d.pbits + d.split)))
            return set_error(QQMC_E_INVAL, "qqmc_plan_chunk_sums: chunk index out of range");
        const double *src = d.partials + 4 * ((size_t)shift * d.chunks_per_shift + (size_t)chunk[i] * nsub);
        e = cudaMemcpy(buf.data(), src, 4 * sizeof(double) * nsub, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_error(e, "chunk download");
        for (int c = 0; c < 4; ++c) {
            double acc = 0.0;
            for (int j = 0; j < nsub; ++j) acc += buf[4 * j + c];
            out[4 * i + c] = acc;
        }
    }
    return QQMC_OK;
}

extern "C" int qqmc_plan_destroy(qqmc_plan *pl) {
    free_plan(pl);
    return QQMC_OK;
}

extern "C" int qqmc_integrate(qqmc_problem *pr, int order, uint64_t n_points, int n_shifts, int precision,
                              const uint32_t *shift_words, double *per_shift, qqmc_result *out) {
    if (!pr) return set_error(QQMC_E_INVAL, "problem is NULL");
    qqmc_item it;
    it.problem = pr;
    it.order = order;
    it.n_shifts = n_shifts;
    it.n_points = n_points;
    it.first_index = 0;
    it.shift_words = shift_words;
    qqmc_plan *pl = nullptr;
    int rc = qqmc_plan_create(&it, 1, precision, &pl);
    if (rc != QQMC_OK) return rc;
    rc = qqmc_plan_launch(pl, nullptr, 0);
    if (rc == QQMC_OK) rc = qqmc_plan_results(pl, out, per_shift);
    qqmc_plan_destroy(pl);
    return rc;
}

// precision argument of the tuning calls: QQMC_PREC_* | optionally QQMC_TUNE_PAIRS
static bool tuning_target(int arg, int *precision, int *tree) {
    *precision = arg & ~QQMC_TUNE_PAIRS;
    *tree = (arg & QQMC_TUNE_PAIRS) ? 1 : 0;
    return *precision == QQMC_PREC_FP64 || *precision == QQMC_PREC_MIXED;
}

extern "C" int qqmc_set_tuning(int precision, int order, int warps_per_block, int flat_vertices) {
    int prec = 0, t = 0;
    if (!tuning_target(precision, &prec, &t) || order < 1 || order > kMaxOrder)
        return set_error(QQMC_E_INVAL, "qqmc_set_tuning: bad precision or order");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const int p = prec == QQMC_PREC_FP64 ? 0 : 1;
    if (warps_per_block <= 0 || flat_vertices <= 0) {
        g_tune_set[p][t][order] = false;
        return QQMC_OK;
    }
    if (warps_per_block > 16 || flat_vertices > 5)
        return set_error(QQMC_E_INVAL, "qqmc_set_tuning: warps_per_block in 1..16, flat_vertices in 1..5");
    g_tune[p][t][order].warps_per_block = warps_per_block;
    g_tune[p][t][order].flat = flat_vertices;
    g_tune[p][t][order].flat_min = flat_vertices;
    g_tune_set[p][t][order] = true;
    return QQMC_OK;
}

extern "C" int qqmc_get_tuning(int precision, int order, int *wpb, int *flat) {
    int prec = 0, t = 0;
    if (!tuning_target(precision, &prec, &t) || order < 1 || order > kMaxOrder || !wpb || !flat)
        return set_error(QQMC_E_INVAL, "qqmc_get_tuning: bad arguments");
    Tuning tu = get_tuning(prec, order, t != 0);
    *wpb = tu.warps_per_block;
    *flat = tu.flat;
    return QQMC_OK;
}

extern "C" int qqmc_set_elimination(qqmc_problem *pr, int mode) {
    if (!pr) return set_error(QQMC_E_INVAL, "qqmc_set_elimination: problem is NULL");
    if (mode != QQMC_ELIM_AUTO && mode != QQMC_ELIM_PAIRS && mode != QQMC_ELIM_SINGLE)
        return set_error(QQMC_E_INVAL, "qqmc_set_elimination: mode must be QQMC_ELIM_AUTO, _PAIRS or _SINGLE");
    pr->elimination = mode;
    return QQMC_OK;
}

extern "C" int qqmc_elimination(const qqmc_problem *pr, int precision) {
    if (!pr || (precision != QQMC_PREC_FP64 && precision != QQMC_PREC_MIXED))
        return set_error(QQMC_E_INVAL, "qqmc_elimination: NULL problem or bad precision");
    return use_pairs(*pr, precision) ? QQMC_ELIM_PAIRS : QQMC_ELIM_SINGLE;
}

// ---------------------------------------------------------------- inspection
template <class T>
struct DevBuf {
    T *p = nullptr;
    cudaError_t alloc(size_t n) { return cudaMalloc(&p, sizeof(T) * (n ? n : 1)); }
    ~DevBuf() { cudaFree(p); }
};

extern "C" int qqmc_sobol_points(int order, uint64_t first, uint64_t count, const uint32_t *shift, uint32_t *out) {
    if (order < 1 || order > kMaxOrder) return set_error(QQMC_E_RANGE, "order outside 1..QQMC_MAX_ORDER");
    if (!out || count > (1ull << 28)) return set_error(QQMC_E_INVAL, "bad output or count");
    if (count == 0) return QQMC_OK;
    int rc = ensure_device();
    if (rc != QQMC_OK) return rc;
    DevBuf<uint32_t> d_out, d_shift;
    cudaError_t e = d_out.alloc(count * order);
    if (e == cudaSuccess && shift) {
        e = d_shift.alloc(order);
        if (e == cudaSuccess) e = cudaMemcpy(d_shift.p, shift, sizeof(uint32_t) * order, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = launch_sobol(order, first, count, shift ? d_shift.p : nullptr, d_out.p, nullptr, 0, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, d_out.p, sizeof(uint32_t) * count * order, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "qqmc_sobol_points");
    return QQMC_OK;
}

extern "C" int qqmc_warp_points(const qqmc_problem *pr, int order, uint64_t first, uint64_t count,
                                const uint32_t *shift, double *u, double *w, int32_t *inside) {
    if (!pr) return set_error(QQMC_E_INVAL, "problem is NULL");
    if (order < 1 || order > kMaxOrder) return set_error(QQMC_E_RANGE, "order outside 1..QQMC_MAX_ORDER");
    if (!u || !w || !inside || count > (1ull << 26)) return set_error(QQMC_E_INVAL, "bad output or count");
    if (count == 0) return QQMC_OK;
    int rc = ensure_device();
    if (rc != QQMC_OK) return rc;
    DevBuf<uint32_t> d_shift;
    DevBuf<double> d_u, d_w;
    DevBuf<int32_t> d_in;
    cudaError_t e = d_u.alloc(count * order);
    if (e == cudaSuccess) e = d_w.alloc(count);
    if (e == cudaSuccess) e = d_in.alloc(count);
    if (e == cudaSuccess && shift) {
        e = d_shift.alloc(order);
        if (e == cudaSuccess) e = cudaMemcpy(d_shift.p, shift, sizeof(uint32_t) * order, cudaMemcpyHostToDevice);
    }
    if (pr->d_lat_z && (order > pr->lat_dims || first + count > (1ull << (pr->lat_m & 63))))
        return set_error(QQMC_E_INVAL, "points outside the problem's lattice (order > its dimension or index >= N)");
    if (e == cudaSuccess)
        e = launch_warp(order, first, count, shift ? d_shift.p : nullptr, pr->params.t_max, pr->params.tau, d_u.p,
                        d_w.p, d_in.p, pr->d_lat_z, pr->lat_m, 0);
    if (e == cudaSuccess) e = cudaMemcpy(u, d_u.p, sizeof(double) * count * order, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(w, d_w.p, sizeof(double) * count, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(inside, d_in.p, sizeof(int32_t) * count, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "qqmc_warp_points");
    return QQMC_OK;
}

extern "C" int qqmc_integrand(const qqmc_problem *pr, int order, uint64_t count, const double *u, int precision,
                              double *out) {
    if (!pr) return set_error(QQMC_E_INVAL, "problem is NULL");
    if (order < 1 || order > kMaxOrder) return set_error(QQMC_E_RANGE, "order outside 1..QQMC_MAX_ORDER");
    if (precision != QQMC_PREC_FP64 && precision != QQMC_PREC_MIXED)
        return set_error(QQMC_E_INVAL, "precision must be QQMC_PREC_FP64 or QQMC_PREC_MIXED");
    if (!u || !out || count > (1ull << 24)) return set_error(QQMC_E_INVAL, "bad input, output or count");
    const double t = pr->params.t_max;
    for (uint64_t q = 0; q < count; ++q) {
        double prev = t;
        for (int m = 0; m < order; ++m) {
            double v = u[q * order + m];
            if (!(v < prev) || !(v > 0.0)) return set_error(QQMC_E_INVAL, "points must satisfy t_max > u_1 > ... > u_n > 0");
            prev = v;
        }
    }
    if (count == 0) return QQMC_OK;
    int rc = ensure_device();
    if (rc != QQMC_OK) return rc;
    DevBuf<double> d_u, d_out;
    cudaError_t e = d_u.alloc(count * order);
    if (e == cudaSuccess) e = d_out.alloc(2 * count);
    if (e == cudaSuccess) e = cudaMemcpy(d_u.p, u, sizeof(double) * count * order, cudaMemcpyHostToDevice);
    ItemDev it{};
    it.table = pr->d_table;
    it.table32 = pr->d_table32;
    it.g0_re = pr->g0_re;
    it.g0_im = pr->g0_im;
    it.t = t;
    it.tau = pr->params.tau;
    it.T = t;
    it.h = pr->h;
    it.L = pr->L;
    it.order = order;
    it.alpha = pr->params.alpha;
    it.col = pr->params.observable == QQMC_OBS_CURRENT ? pr->d_col : nullptr;
    it.col32 = pr->params.observable == QQMC_OBS_CURRENT ? pr->d_col32 : nullptr;
    const bool pairs = use_pairs(*pr, precision);
    Tuning tu = get_tuning(precision, order, pairs);
    if (tu.flat < 2) tu.flat = tu.flat_min = 2;  // the check kernel runs one warp per point
    it.flat = tu.flat;
    if (e == cudaSuccess) e = launch_integrand(it, count, d_u.p, d_out.p, precision, tu, pairs, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, d_out.p, sizeof(double) * 2 * count, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "qqmc_integrand");
    return QQMC_OK;
}

// ---------------------------------------------------------------- learned warp
extern "C" int qqmc_set_projection(qqmc_problem *pr, int order, const double *cdf, int cells) {
    if (!pr) return set_error(QQMC_E_INVAL, "problem is NULL");
    if (order < 1 || order > kMaxOrder) return set_error(QQMC_E_RANGE, "order outside 1..QQMC_MAX_ORDER");
    if (!cdf || cells <= 0) {  // back to the plain exponential warp
        cudaFree(pr->d_proj[order]);
        pr->d_proj[order] = nullptr;
        pr->proj_cells[order] = 0;
        return QQMC_OK;
    }
    if (cells > (1 << 20)) return set_error(QQMC_E_INVAL, "cells must be <= 2^20");
    for (int m = 0; m < order; ++m) {
        const double *c = cdf + (size_t)m * (cells + 1);
        if (c[0] != 0.0 || c[cells] != 1.0)
            return set_error(QQMC_E_INVAL, "each CDF must start at 0 and end at 1");
        for (int k = 0; k < cells; ++k)
            if (!(c[k + 1] >= c[k])) return set_error(QQMC_E_INVAL, "each CDF must be non-decreasing");
    }
    int rc = ensure_device();
    if (rc != QQMC_OK) return rc;
    double *d = nullptr;
    const size_t bytes = sizeof(double) * order * (size_t)(cells + 1);
    cudaError_t e = cudaMalloc(&d, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(d, cdf, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_error(e, "projection table upload");
    }
    cudaFree(pr->d_proj[order]);
    pr->d_proj[order] = d;
    pr->proj_cells[order] = cells;
    return QQMC_OK;
}

extern "C" int qqmc_learn_projection(qqmc_problem *pr, int order, uint64_t M, int n_bins, double lambda,
                                     double floor_frac, int cells, double *cdf_out) {
    if (!pr) return set_error(QQMC_E_INVAL, "problem is NULL");
    if (order < 1 || order > kMaxOrder) return set_error(QQMC_E_RANGE, "order outside 1..QQMC_MAX_ORDER");
    if (M < 1 || M > (1ull << 24) || n_bins < 1 || n_bins > 65536 || !(lambda > 0) || !(floor_frac >= 0) ||
        !(floor_frac < 1) || cells < 1 || cells > (1 << 20))
        return set_error(QQMC_E_INVAL, "qqmc_learn_projection: bad M, n_bins, lambda, floor or cells");
    int rc = ensure_device();
    if (rc != QQMC_OK) return rc;
    const int n = order;
    // 1. M points of the learning sequence (Sobol' shifted by the words of shift index 65535),
    //    plain exponential warp, host FP64
    std::vector<uint32_t> V(32 * kMaxOrder), S(n);
    direction_numbers(kMaxOrder, V.data());
    for (int d = 0; d < n; ++d)
        S[d] = (uint32_t)(splitmix64(pr->params.seed ^ ((uint64_t)65535 * 65536u + (uint64_t)d)) >> 32);
    const double t = pr->params.t_max, tau = pr->params.tau;
    std::vector<double> xs((size_t)M * n), wts, us;
    std::vector<uint64_t> idx_in;
    for (uint64_t a = 0; a < M; ++a) {
        const uint64_t g = a ^ (a >> 1);
        double uprev = t, prod = 1.0, tn = 1.0;
        std::vector<double> u(n);
        for (int d = 0; d < n; ++d) {
            uint32_t X = 0;
            for (int j = 0; j < 32; ++j)
                if ((g >> j) & 1u) X ^= V[32 * d + j];
            const double x = (double)(X ^ S[d]) * 0x1p-32;
            xs[a * n + d] = x;
            uprev -= -tau * log1p(-x);
            u[d] = uprev;
            prod *= (1.0 - x);
            tn *= tau;
        }
        if (uprev > 0.0) {
            idx_in.push_back(a);
            wts.push_back(tn / prod);
            us.insert(us.end(), u.begin(), u.end());
        }
    }
    // 2. integrand at the in-domain points on the device (FP64, same code as the integration)
    const uint64_t nin = idx_in.size();
    std::vector<double> c(2 * nin);
    if (nin) {
        double *d_u = nullptr, *d_c = nullptr;
        cudaError_t e = cudaMalloc(&d_u, sizeof(double) * us.size());
        if (e == cudaSuccess) e = cudaMalloc(&d_c, sizeof(double) * c.size());
        if (e == cudaSuccess) e = cudaMemcpy(d_u, us.data(), sizeof(double) * us.size(), cudaMemcpyHostToDevice);
        ItemDev it{};
        it.table = pr->d_table;
        it.table32 = pr->d_table32;
        it.g0_re = pr->g0_re;
        it.g0_im = pr->g0_im;
        it.t = t;
        it.tau = tau;
        it.T = t;
        it.h = pr->h;
        it.L = pr->L;
        it.order = n;
        it.alpha = pr->params.alpha;
        it.col = pr->params.observable == QQMC_OBS_CURRENT ? pr->d_col : nullptr;
        it.col32 = nullptr;
        const bool pairs = use_pairs(*pr, QQMC_PREC_FP64);
        Tuning tu = get_tuning(QQMC_PREC_FP64, n, pairs);
        if (tu.flat < 2) tu.flat = tu.flat_min = 2;
        it.flat = tu.flat;
        if (e == cudaSuccess) e = launch_integrand(it, nin, d_u, d_c, QQMC_PREC_FP64, tu, pairs, 0);
        if (e == cudaSuccess) e = cudaMemcpy(c.data(), d_c, sizeof(double) * c.size(), cudaMemcpyDeviceToHost);
        cudaFree(d_u);
        cudaFree(d_c);
        if (e != cudaSuccess) return cuda_error(e, "qqmc_learn_projection sampling");
    }
    // 3. projection of |integrand| onto each dimension (histogram of N_b bins)
    std::vector<double> hist((size_t)n * n_bins, 0.0);
    for (uint64_t q = 0; q < nin; ++q) {
        const double val = wts[q] * hypot(c[2 * q], c[2 * q + 1]) / (double)M;
        const uint64_t a = idx_in[q];
        for (int d = 0; d < n; ++d) {
            int b = (int)(xs[a * n + d] * n_bins);
            b = b < 0 ? 0 : (b >= n_bins ? n_bins - 1 : b);
            hist[(size_t)d * n_bins + b] += val;
        }
    }
    // 4. Gaussian kernel smoothing onto the cells, floor, cumulative distribution
    std::vector<double> cdf((size_t)n * (cells + 1));
    for (int d = 0; d < n; ++d) {
        std::vector<double> h(cells);
        double hmax = 0.0;
        for (int k = 0; k < cells; ++k) {
            const double z = (k + 0.5) / cells;
            double num = 0.0, den = 0.0;
            for (int l = 0; l < n_bins; ++l) {
                const double y = (l + 0.5) / n_bins;
                const double K = exp(-(z - y) * (z - y) / (lambda * lambda));
                num += K * hist[(size_t)d * n_bins + l];
                den += K;
            }
            h[k] = den > 0 ? num / den : 0.0;
            hmax = h[k] > hmax ? h[k] : hmax;
        }
        double tot = 0.0;
        for (int k = 0; k < cells; ++k) {
            if (hmax <= 0.0) h[k] = 1.0;  // no signal: uniform
            else if (h[k] < floor_frac * hmax) h[k] = floor_frac * hmax;
            tot += h[k];
        }
        double *cd = cdf.data() + (size_t)d * (cells + 1);
        cd[0] = 0.0;
        double acc = 0.0;
        for (int k = 0; k < cells; ++k) {
            acc += h[k];
            cd[k + 1] = acc / tot;
        }
        cd[cells] = 1.0;
    }
    rc = qqmc_set_projection(pr, order, cdf.data(), cells);
    if (rc != QQMC_OK) return rc;
    if (cdf_out) memcpy(cdf_out, cdf.data(), sizeof(double) * cdf.size());
    return QQMC_OK;
}
