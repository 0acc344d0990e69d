// Internal declarations shared by the QQMC library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/qqmc.h"

namespace qqmc {

using dbl4 = double4_32a;  // 32-byte aligned: one 256-bit load per table node

constexpr int kMaxOrder = QQMC_MAX_ORDER;
constexpr int kChunk = 32;  // Sobol' indices per work chunk (one per lane)

// Device-resident problem: half table of (g^<, g^>) on the nodes with tau >= -h/2.
struct Problem {
    qqmc_params params;
    int L = 0;
    double h = 0;        // node spacing 2 t_max / (L - 1)
    double g0_re = 0, g0_im = 0;
    dbl4 *d_table = nullptr;  // [L/2 + 1]: (gl.re, gl.im, gg.re, gg.im) at nodes k = L/2-1 .. L-1
    float4 *d_table32 = nullptr; // same, FP32 (mixed precision)
    int device = 0;
    double *d_proj[kMaxOrder + 1] = {};  // learned warp per order: [order][proj_cells[order] + 1]
    int proj_cells[kMaxOrder + 1] = {};
    // current observable: dot-lead tables gamma g^<_01, gamma g^>_01 at nodes k = 0 .. L/2
    dbl4 *d_col = nullptr;
    float4 *d_col32 = nullptr;
    double c0_re = 0, c0_im = 0;  // gamma g^<_01(0)
    // rank-1 lattice point set (instead of Sobol'): generating vector and log2 of its size
    uint32_t *d_lat_z = nullptr;
    int lat_m = 0;       // log2 N, plus 64 when the baker's transform follows the shift
    int lat_dims = 0;
    int elimination = QQMC_ELIM_AUTO;  // Keldysh-sum tree: QQMC_ELIM_* (qqmc_set_elimination)
};

// Whether a problem's Keldysh sums run on the pair-block tree (else the
// single-vertex tree), for the given precision: QQMC_ELIM_AUTO picks pairs when
// the vertex diagonal dv = g^<(0) - i alpha is small against the scale of the
// Green function at tau = 0, max(|g^<(0)|, |g^>(0)|) with g^>(0) = g^<(0) - i.
bool use_pairs(const Problem &P, int precision);

// One item as the device sees it.
struct ItemDev {
    const dbl4 *table;
    const float4 *table32;
    const uint32_t *shifts;  // [n_shifts][order]
    double *partials;        // [n_shifts * chunks_per_shift][4]: sum.re, sum.im, comp.re, comp.im
    unsigned int *inside;    // [n_shifts * chunks_per_shift]: in-domain count per chunk
    double g0_re, g0_im, t, tau, T, h;
    long long first_index;
    long long n_points;
    long long chunk_begin;   // first global chunk of this item
    int order, n_shifts, L;
    int chunks_per_shift;    // work units per shift: point chunks << (pbits + split)
    int pbits;               // a chunk's 32 points in 2^pbits units of 32 >> pbits points
    int split;               // each point's Keldysh tree in 2^split subtrees (separate work units)
    int flat;                // vertices resolved per lane for this item (its order's tuning)
    const double *proj;      // learned warp: [order][proj_cells + 1] CDF per dimension, or null (plain)
    int proj_cells;
    double alpha;            // quadratic shift: vertex diagonals are g^<(0) - i alpha
    const dbl4 *col;         // current: dot-lead column table [L/2 + 1] at nodes 0 .. L/2, else null
    const float4 *col32;
    const uint32_t *lat_z;   // rank-1 lattice generating vector, or null (Sobol')
    int lat_m;               // lattice size 2^(lat_m & 63); lat_m >= 64: baker's transform
};

struct Tuning {
    int warps_per_block;
    int flat;      // largest flat depth of the launch (kernel template)
    int flat_min;  // smallest flat depth (sizes the breadth-first buffers)
};

// Error reporting (thread-local message).
int set_error(int code, const std::string &msg);
int cuda_error(cudaError_t e, const char *what);

// Host-side generators (product side).
void direction_numbers(int n_dims, uint32_t *out);  // [n_dims][32]
uint64_t splitmix64(uint64_t x);
void shift_words(uint64_t seed, int n_shifts, int n_dims, uint32_t *out);

// Kernel launchers (kernels.cu).
int upload_direction_numbers();
int launch_gf_table(const Problem &pr, cudaStream_t s);
int launch_lead_table(Problem &pr, cudaStream_t s, double *zero);
// span (may be null): [earliest warp start, latest warp exit] of the launch in device-clock ns,
// merged with atomicMin / atomicMax (the caller initialises it to [~0, 0]).
// pairs: the pair-block tree, else the single-vertex tree (every item of a launch uses one tree).
cudaError_t launch_detsum(const ItemDev *d_items, int n_items, long long total_chunks, unsigned long long *d_counter,
                          int n_max, int precision, const Tuning &tune, bool pairs, void *gstack,
                          long long gstack_warps, unsigned long long *span, cudaStream_t s);
// Warps (and bytes per warp) of device memory the determinant launch needs for
// its tree stack; 0 when the stack fits in shared memory.
long long detsum_gstack_warps(int n_max, int precision, const Tuning &tune, bool pairs, size_t *bytes_per_warp);
void set_stack_policy(int precision, int min_order);
bool detsum_stack_fits_shared(int n_max, int precision, const Tuning &tune, bool pairs);
cudaError_t launch_lane(const ItemDev *d_items, int n_items, long long total_chunks, unsigned long long *d_counter,
                        int precision, unsigned long long *span, cudaStream_t s);
constexpr int kLaneMaxOrder = 4;  // orders that may run one point per lane
// Bits of the leaf index of an order's Keldysh tree (single-vertex tree: one
// per depth-first level; pair tree: a_2, then two per depth-first pair level);
// work units may fix a prefix of them.
int tree_leaf_bits(int order, bool pairs);
// d_bad (may be null): per shift, the work units whose partial sum was not finite.
cudaError_t launch_reduce(const ItemDev *d_items, int n_items, int total_shifts, double *d_out, unsigned long long *d_counts,
                          unsigned int *d_bad, cudaStream_t s);
// One thread writes the item descriptor (a kernel argument) to d_item and zeroes the work counter.
cudaError_t launch_store_item(const ItemDev &item, ItemDev *d_item, unsigned long long *d_counter, cudaStream_t s);
cudaError_t launch_sobol(int order, uint64_t first, uint64_t count, const uint32_t *d_shift, uint32_t *d_out,
                         const uint32_t *d_lat_z, int lat_m, cudaStream_t s);
cudaError_t launch_warp(int order, uint64_t first, uint64_t count, const uint32_t *d_shift, double t, double tau,
                        double *d_u, double *d_w, int32_t *d_inside, const uint32_t *d_lat_z, int lat_m,
                        cudaStream_t s);
cudaError_t launch_integrand(const ItemDev &item, uint64_t count, const double *d_u, double *d_out, int precision,
                             const Tuning &tune, bool pairs, cudaStream_t s);
// Launch shape of an order's determinant kernel, per precision and tree.
Tuning get_tuning(int precision, int order, bool pairs);
bool valid_params(const qqmc_params *p, std::string &why);
double order0_value(const Problem &pr);

}  // namespace qqmc
