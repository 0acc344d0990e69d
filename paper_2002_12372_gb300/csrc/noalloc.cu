// Allocation-free variant of one order-n integration.
//
// qqmc_integrate / the plans allocate their scratch (work counter, chunk
// partial sums, in-domain counts, item descriptor) with cudaMalloc.  Some
// callers cannot allocate device memory at the point where they integrate:
// a host framework that owns the whole device through its own memory pool,
// or a real-time loop that must not enter the driver's allocator.  For them
// qqmc_integrate_noalloc runs the same determinant and reduction kernels with
// all scratch taken from one fixed array compiled into this library.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <string>

#include "qqmc_internal.h"

using namespace qqmc;

namespace {

// Every GPU that loads the library holds this array until the process exits.
constexpr size_t kScratchBytes = 16u << 20;  // 16 MiB
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Scratch layout: [item descriptor | counter | counts | partials | inside].
constexpr size_t kItemOff = 0;
constexpr size_t kCounterOff = 256;
constexpr size_t kCountsOff = 512;                       // n_shifts x uint64 (used when the caller passes none)
constexpr size_t kPartialsOff = kCountsOff + 1024 * 8;  // chunks x 4 doubles
constexpr size_t kPerChunk = 4 * sizeof(double) + sizeof(unsigned int);
constexpr size_t kMaxChunks = (kScratchBytes - kPartialsOff) / kPerChunk;
static_assert(sizeof(ItemDev) <= kCounterOff - kItemOff, "the item descriptor overlaps the work counter");
static_assert(kCounterOff % 8 == 0 && kCountsOff % 8 == 0 && kPartialsOff % 8 == 0,
              "scratch areas must be 8-byte aligned");

std::mutex g_mu;
unsigned char *g_dev_ptr[64];  // device address of g_scratch, per device
bool g_ready[64];

// Once per device, with that device current: the device address of the array
// (in host code the symbol names a host-side stand-in, not device memory) and
// the constant tables of the kernels.
int setup_device(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return set_error(QQMC_E_CUDA, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ready[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(static scratch)");
        int rc = upload_direction_numbers();
        if (rc != QQMC_OK) return rc;
        g_dev_ptr[dev] = static_cast<unsigned char *>(p);
        g_ready[dev] = true;
    }
    *out = g_dev_ptr[dev];
    return QQMC_OK;
}

}  // namespace

extern "C" int qqmc_integrate_noalloc(const qqmc_problem *pr, int order, uint64_t n_points, int n_shifts,
                                      int precision, const uint32_t *d_shift_words, double *d_sums,
                                      unsigned long long *d_counts, void *stream) {
    const Problem *P = reinterpret_cast<const Problem *>(pr);
    if (!P) return set_error(QQMC_E_INVAL, "qqmc_integrate_noalloc: problem is NULL");
    if (order < 1 || order > kMaxOrder) return set_error(QQMC_E_RANGE, "order outside 1..QQMC_MAX_ORDER");
    if (precision != QQMC_PREC_FP64 && precision != QQMC_PREC_MIXED)
        return set_error(QQMC_E_INVAL, "precision must be QQMC_PREC_FP64 or QQMC_PREC_MIXED");
    if (!d_shift_words || !d_sums) return set_error(QQMC_E_INVAL, "shift words and sums must be device pointers");
    if (n_points < 1 || n_shifts < 1 || n_shifts > 1024)
        return set_error(QQMC_E_INVAL, "n_points must be >= 1 and n_shifts in 1..1024");
    const uint64_t cps = (n_points + kChunk - 1) / kChunk;
    if (cps > kMaxChunks || cps * (uint64_t)n_shifts > kMaxChunks)
        return set_error(QQMC_E_INVAL,
                         "qqmc_integrate_noalloc: n_shifts * ceil(n_points / 32) exceeds the static scratch (" +
                             std::to_string(kMaxChunks) + " chunks of 32 points)");
    int dev = 0;
    cudaError_t de = cudaGetDevice(&dev);
    if (de != cudaSuccess) return cuda_error(de, "cudaGetDevice");
    if (dev != P->device)
        return set_error(QQMC_E_INVAL, "qqmc_integrate_noalloc: the problem's tables are on device " +
                                           std::to_string(P->device) + " but device " + std::to_string(dev) +
                                           " is current");
    unsigned char *base = nullptr;
    int rc = setup_device(&base);
    if (rc != QQMC_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    ItemDev it{};
    it.table = P->d_table;
    it.table32 = P->d_table32;
    it.shifts = d_shift_words;
    it.partials = reinterpret_cast<double *>(base + kPartialsOff);
    it.inside = reinterpret_cast<unsigned int *>(base + kPartialsOff + cps * n_shifts * 4 * sizeof(double));
    it.g0_re = P->g0_re;
    it.g0_im = P->g0_im;
    it.t = P->params.t_max;
    it.tau = P->params.tau;
    it.T = P->params.t_max;
    it.h = P->h;
    it.first_index = 0;
    it.n_points = (long long)n_points;
    it.chunk_begin = 0;
    it.order = order;
    it.n_shifts = n_shifts;
    it.L = P->L;
    it.chunks_per_shift = (int)cps;
    it.alpha = P->params.alpha;
    it.col = P->params.observable == QQMC_OBS_CURRENT ? P->d_col : nullptr;
    it.col32 = P->params.observable == QQMC_OBS_CURRENT ? P->d_col32 : nullptr;
    it.lat_z = P->d_lat_z;
    it.lat_m = P->lat_m;
    if (P->d_lat_z && (order > P->lat_dims || n_points > (1ull << (P->lat_m & 63))))
        return set_error(QQMC_E_INVAL, "points outside the problem's lattice (order > its dimension or index >= N)");
    it.proj = P->d_proj[order];
    it.proj_cells = P->proj_cells[order];
    const bool pairs = use_pairs(*P, precision);
    Tuning tu = get_tuning(precision, order, pairs);
    it.flat = tu.flat;
    if (it.flat < 2 && order > 4) it.flat = 2;
    if (tu.flat < 2) tu.flat = tu.flat_min = 2;
    if (!(it.flat == 1 && order <= kLaneMaxOrder) && !detsum_stack_fits_shared(order, precision, tu, pairs))
        return set_error(QQMC_E_INVAL,
                         "qqmc_integrate_noalloc: this order's FP64 tree stack needs device memory; use the mixed "
                         "precision or qqmc_integrate");

    ItemDev *d_item = reinterpret_cast<ItemDev *>(base + kItemOff);
    unsigned long long *d_counter = reinterpret_cast<unsigned long long *>(base + kCounterOff);
    unsigned long long *counts = d_counts ? d_counts : reinterpret_cast<unsigned long long *>(base + kCountsOff);

    // The descriptor travels as a kernel argument (copied when the launch is enqueued), so
    // the call reads no host memory after it returns and makes no pageable copy.
    cudaError_t e = launch_store_item(it, d_item, d_counter, s);
    if (e == cudaSuccess) {
        if (it.flat == 1 && order <= kLaneMaxOrder)
            e = launch_lane(d_item, 1, (long long)(cps * n_shifts), d_counter, precision, nullptr, s);
        else
            e = launch_detsum(d_item, 1, (long long)(cps * n_shifts), d_counter, order, precision, tu, pairs, nullptr,
                              0, nullptr, s);
    }
    if (e == cudaSuccess) e = launch_reduce(d_item, 1, n_shifts, d_sums, counts, nullptr, s);
    if (e != cudaSuccess) return cuda_error(e, "qqmc_integrate_noalloc");
    return QQMC_OK;
}
