// Internal declarations shared by the CUDA translation units of libsph_gb300.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/sph.h"

namespace sph {

// Support of the cubic spline in units of the smoothing length (Dehnen & Aly
// 2012): H = GAMMA_K h.  With eta = 1.2348 this gives ~48 neighbours.
constexpr float GAMMA_K = 1.825742f;
constexpr double GAMMA_K_D = 1.825742;
constexpr float KERNEL_NORM = 2.5464790894703255f;  // 8 / pi
constexpr int MORTON_BITS = 10;                       // per axis inside a top-level cell
constexpr int KEY_MORTON_BITS = 3 * MORTON_BITS;
constexpr int MAX_BINS = 64;
constexpr int WARPS_PER_BLOCK = 8;
constexpr int LEAF_MAX_LIMIT = 64;
constexpr int CHUNK = 16;          // most leaves in a chunk (at most 32: one warp ballot)
constexpr int WG_MAX = 32;         // particles per work group of the pair loops (one per lane)

// Device-resident state of the context: the integer timeline, the sizes of
// the cell structure, work queues, error flags and counters.  Everything a
// kernel needs that can change between steps lives here, so a captured CUDA
// graph stays valid across steps and rebuilds.
struct DevState {
  long long ti;          // current tick
  long long ti_next;     // next tick (set by the bins kernel)
  unsigned int epoch;    // incremented by every mark, stamps active cells
  int m_act;             // largest active bin at ti (63 at tick 0)
  // cell structure (written at build)
  int nc;                // cells per axis
  int n_cells;           // nc^3
  int n_leaves;
  int n_chunks;          // octree nodes of up to CHUNK leaves of one cell (see launch_chunks)
  int n_groups;          // work groups: runs of consecutive leaves of one cell, <= WG_MAX particles
  int n_active_groups;   // work groups holding active particles (light ones from the front of
                         // q_group, heavy ones from its back; see n_heavy_groups)
  int n_heavy_groups;    // active work groups whose estimated cost is well above the mean
  int test_stall;        // testing: density launches whose first warp still has to stall
  int test_bad_group;    // testing (checks build): density launches still to plant a bad group
  unsigned long long group_cost_sum;  // sum over work groups of group_cost (written at build)
  double w;              // cell width
  // queues (written by mark)
  int n_active_leaves;   // leaves holding active particles
  int n_active_cells;    // cells holding active particles
  int n_drift_chunks;    // leaf chunks of the cells within one cell of an active cell
  int n_bin_groups;      // plain form: active work groups holding particles of one bin
  int n_bin_coop;        // plain form: those the force loop shares (back of q_bin)
  int n_wake;            // limiter: inactive particles asked to wake in this step (q_wake)
  // persistent-kernel work heads
  int head_density, head_force, head_drift, head_kick;
  int head_open, head_bins, head_misc;
  int head_coop_force;        // force loop: shared work groups taken so far
  int head_grad;              // gradient loop (velocity divergence and curl)
  unsigned int blocks_done;   // blocks of the closing kernel of a step that have finished
  // errors
  unsigned int halt;      // a step-invalidating error happened: kernels return
  int first_error;        // first SPH_ERR_* code recorded
  unsigned long long err_count[16];
  // first failed bounds check (a library built with SPH_CHECKS)
  int check_site;         // sph_check_site (0: none)
  float m_uniform;        // the particles' common mass (0: the masses differ), set at build
  long long check_index, check_bound;
  // rebuild criterion
  unsigned int excursion_bits;  // max distance (float bits) of a particle outside its cell
  unsigned int Hmax_bits;       // max kernel support H (float bits) over all particles
  unsigned int want_h_bits;     // largest h an iteration wanted beyond the cell limit
  int dens_split;               // parts per work group of the last whole-step density launch
  // counters of the step in progress (reset when a step starts, added to the
  // totals when it completes, so a halted attempt leaves no trace)
  unsigned long long s_pairs_density, s_pairs_force, s_cand_density, s_cand_force;
  unsigned long long s_iters_density, s_active_particles;
  unsigned long long s_gathers_density, s_list_overflows, s_evals_density;
  // totals over completed steps
  unsigned long long pairs_density, pairs_force, cand_density, cand_force;
  unsigned long long iters_density, active_particles;
  unsigned long long gathers_density, list_overflows, evals_density;
  unsigned long long steps;
  unsigned long long wakes;   // limiter: inactive particles whose steps were cut
  // time-bin occupancy
  int bin_count[MAX_BINS];
  // smallest and largest particle mass (float bits), found at each cell build
  unsigned int m_lo_bits, m_hi_bits;
};

// Pointers and constants handed to every kernel (by value).
struct View {
  long long n;
  // caller particle arrays (cell order after a build)
  double *x, *y, *z;
  float *vx, *vy, *vz, *ax, *ay, *az, *A, *Adot, *h, *rho, *f, *P, *c, *vsig, *m;
  int8_t *bin;
  long long *ti_begin, *ti_end, *ti_drift;
  uint8_t *active;
  int32_t *ngb_density, *ngb_force;
  float *div_v, *curl_v;     // velocity divergence and |curl| (variants; may be null)
  int8_t *ngb_bin;           // limiter: smallest bin among the force neighbours (step scratch)
  int32_t *wake_bin;         // limiter: smallest bin an active neighbour asks an inactive
                             // particle down to (WAKE_NONE: none; reset once applied)
  int32_t *q_wake;           // limiter: the particles with a request, in request order
  // cell structure
  int32_t *cell_start;       // [n_cells + 1] first particle of each cell
  int32_t *cell_leaf_start;  // [n_cells + 1] first leaf of each cell
  unsigned int *cell_stamp;  // [n_cells] epoch at which the cell was last marked active
  unsigned int *cell_rel_stamp;  // [n_cells] epoch at which the cell was queued for drift
  int32_t *cell_chunk_start; // [n_cells + 1] first chunk of each cell
  int32_t *chunk_cell;       // [n_chunks] cell of each chunk
  int32_t *chunk_leaf_start; // [n_chunks + 1] first leaf of each chunk (at most CHUNK leaves)
  int32_t *leaf_chunk;       // [n_leaves] chunk of each leaf
  float4 *chunk_lo;          // chunk bbox min, cell frame; w = max H in the chunk
  float4 *chunk_hi;          // chunk bbox max, cell frame
  int32_t *leaf_start;       // [n_leaves + 1] first particle of each leaf
  int32_t *leaf_cell;        // [n_leaves]
  uint32_t *leaf_k;          // [n_leaves] Morton-grid corner of the leaf inside its cell:
                             // kx | ky << 10 | kz << 20, in units of w / 1024
  float4 *leaf_lo;           // bbox min (cell-relative), w = max H in the leaf
  float4 *leaf_hi;           // bbox max (cell-relative)
  uint8_t *leaf_min_bin;     // smallest bin in the leaf
  unsigned long long *leaf_bin_mask;  // bins present in the leaf
  int32_t *pcell;            // [n] cell of each particle
  int32_t *pleaf;            // [n] leaf of each particle
  int32_t *group_leaf0;      // [n_groups + 1] first leaf of each work group
  int32_t *group_cell;       // [n_groups] cell of each work group
  int32_t *group_cost;       // [n_groups] estimated neighbour records of one search (at build)
  // FP32 records read by the pair loops (cell-relative positions)
  float4 *rec_xm;  // x, y, z, m
  float4 *rec_xH;  // x, y, z, H
  float4 *rec_v;   // predicted v, m
  float4 *rec_h;   // rho, f P / rho^2, c, 1 / H
  // queues
  int32_t *q_active;         // leaves holding active particles
  int32_t *q_act_cells;      // cells holding active particles
  int32_t *q_drift;          // chunks to drift (cells next to an active cell)
  int32_t *q_group;          // work groups holding active particles: light ones at
                             // [0, n_active_groups), heavy ones at n_groups - 1 - k
  int32_t *q_bin;            // plain form: active work groups holding particles of one bin
                             // (light ones at [0, n_bin_groups), heavy ones from the back)
  // neighbour lists of the density loop: squared distance and mass of every
  // candidate within a particle's search radius (with equal masses the squared
  // distance alone, 4-byte entries in the first half of the area), list_cap
  // entries per lane,
  // one area per warp of the launch's blocks (a launch has at most list_blocks
  // blocks; entry k of lane s of warp w of block b at
  // nbr[((b * 8 + w) * list_cap + k) * 32 + s]): the area of a warp is reused
  // by its next work group, so the lists stay in L2.
  float2 *nbr;
  DevState *ds;
  // parameters
  double box, eta, gamma, alpha, cfl, h_tol, dt_min;
  long long wait_limit;      // polls of a bounded barrier wait (0: the default)
  float search_margin;       // a density search reaches search_margin x the support
  int list_cap, list_blocks;  // neighbour-list entries per lane; blocks with list areas
  int stage_depth;           // staging buffers per warp (1..3)
  int balsara, predict, limiter;  // variants of the scheme (0/1)
  double heavy_factor;       // heavy work group: estimated cost > heavy_factor x mean
  int coop_max_groups;       // steps with at most this many active groups: all cooperative
                             // (force loop)
  int h_max_iter, bin_cap, leaf_max, G, drift_all;
  int uniform_mass;          // every particle has the same mass (found at the last cell build)
  int grid_util;             // blocks of the grid-stride utility kernels
};

// Reverse-mode work arrays of one step, in the order of the backward pass's
// own cell build (FP64 accumulators; see sph_adjoint.cu).
struct AdjWork {
  const int32_t *perm;           // backward-build slot -> caller index
  double *xb, *yb, *zb;          // d loss / d position at the step's tick
  double *vpxb, *vpyb, *vpzb;    // d loss / d predicted velocity
  double *hb, *rhob, *fb;        // d loss / d h, rho, f as the force loop saw them
  double *Qb, *cb;               // d loss / d (f P / rho^2), d c; then d A_pred, d u
  double *axb, *ayb, *azb, *Adotb;  // d loss / d a, Adot computed by this step
  double *ka, *kb, *km;          // density-adjoint coefficients of the active particles
};

// address of a DevState field on the device, computed on the host
#define SPH_DS_FIELD(ds, field) \
  (reinterpret_cast<decltype(&((DevState *)nullptr)->field)>( \
      reinterpret_cast<char *>(ds) + offsetof(DevState, field)))

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void record_error(DevState *ds, int code, unsigned long long count,
                                             bool halt) {
  atomicCAS(&ds->first_error, 0, code);
  atomicAdd(&ds->err_count[code & 15], count);
  if (halt) atomicExch(&ds->halt, 1u);
}

// No wake request (the limiter's waking of inactive neighbours): the byte
// pattern 0x7f of a cudaMemset, above every bin.
constexpr int32_t WAKE_NONE = 0x7f7f7f7f;

// Device bounds checks.  SPH_IN(ds, i, n, site) is true when 0 <= i < n.  In
// a library compiled with -DSPH_CHECKS a false result records SPH_ERR_BOUNDS
// (halting the step) and, for the first failure, the site, index and bound;
// the caller then skips the access.  (ds may be null: the access is skipped
// and nothing is recorded.)  Without SPH_CHECKS the test compiles
// away (always true).
#ifdef SPH_CHECKS
static __device__ __noinline__ bool check_failed(DevState *ds, int site, long long i, long long n) {
  if (!ds) return false;  // (a caller without a device state: the access is skipped)
  if (atomicCAS(&ds->check_site, 0, site) == 0) {
    ds->check_index = i;
    ds->check_bound = n;
  }
  record_error(ds, SPH_ERR_BOUNDS, 1, true);
  return false;
}
#define SPH_IN(ds, i, n, site)                                                           \
  ((unsigned long long)(long long)(i) < (unsigned long long)(long long)(n) ||          \
   ::sph::check_failed((ds), (site), (long long)(i), (long long)(n)))
#else
#define SPH_IN(ds, i, n, site) true
#endif

__device__ __forceinline__ void atomic_max_float_pos(unsigned int *addr, float v) {
  // non-negative floats order like their bit patterns
  atomicMax(addr, __float_as_uint(fmaxf(v, 0.0f)));
}

// Morton-grid corner of a leaf: integer coordinates (0..1023 per axis) inside
// its cell.  Positions in the FP32 records are relative to this corner, so
// their precision follows the leaf's size, not the cell's; the offset between
// two leaves is an exact integer number of grid steps.
__host__ __device__ __forceinline__ int leaf_kx(uint32_t k) { return (int)(k & 1023u); }
__host__ __device__ __forceinline__ int leaf_ky(uint32_t k) { return (int)((k >> 10) & 1023u); }
__host__ __device__ __forceinline__ int leaf_kz(uint32_t k) { return (int)((k >> 20) & 1023u); }

__device__ __forceinline__ int wrap_cell(int c, int nc) {
  return c < 0 ? c + nc : (c >= nc ? c - nc : c);
}

// k-th entry of the active work-group queue: the heavy groups first (they
// start in the first wave of a persistent kernel), then the light ones.
__device__ __forceinline__ int active_group(const View &v, const DevState *ds, int k) {
  const int nh = ds->n_heavy_groups;
  return k < nh ? v.q_group[ds->n_groups - 1 - k] : v.q_group[k - nh];
}

// Whether this step hands every active work group to a whole block (one lane
// per particle, few active groups: warps would otherwise idle).
__device__ __forceinline__ bool all_coop(const View &v, const DevState *ds) {
  return v.G == 1 && ds->n_active_groups + ds->n_heavy_groups <= v.coop_max_groups;
}

// Number of integer bins active at tick ti: particles on bin b are active
// when ti is a multiple of 2^b, i.e. b <= ctz(ti) (every bin at tick 0).
__host__ __device__ __forceinline__ int max_active_bin(long long ti) {
  if (ti == 0) return MAX_BINS - 1;
#ifdef __CUDA_ARCH__
  return __ffsll(ti) - 1;
#else
  return __builtin_ctzll((unsigned long long)ti);
#endif
}

// Host-side count of kernel launches issued by the library (graph replays add
// the kernels of the captured graph); reported by sph_get_counters.
void note_launches(int n);

// ---------------------------------------------------------------------------
// launchers implemented in the .cu files (all asynchronous on `st`)
// ---------------------------------------------------------------------------
// sph_cells.cu
cudaError_t launch_reduce_hmax(const View &v, float *out_max, cudaStream_t st);
cudaError_t launch_mass_range(const View &v, cudaStream_t st);
// (bad: a device counter, incremented per particle with a non-finite position
// or an h that is not a positive finite number)
cudaError_t launch_cell_keys(const View &v, int nc, double w, unsigned long long *keys,
                             unsigned int *vals, unsigned int *bad, cudaStream_t st);
cudaError_t radix_sort_pairs(unsigned long long *keys, unsigned int *vals,
                             unsigned long long *keys_alt, unsigned int *vals_alt, int n,
                             int nbits, unsigned int *hist, unsigned int *scan_tmp,
                             int n_hist_max, bool *result_in_alt, cudaStream_t st,
                             DevState *ds);  // ds: where a failed bounds check is recorded (may be null)
cudaError_t exclusive_scan_u32(const unsigned int *in, unsigned int *out, int n,
                               unsigned int *tmp, cudaStream_t st);
cudaError_t launch_gather(void *dst, const void *src, const unsigned int *idx, long long n,
                          int elem_bytes, cudaStream_t st, DevState *ds);
cudaError_t launch_cell_start(const unsigned long long *sorted_keys, long long n, int n_cells,
                              int32_t *cell_start, int32_t *pcell, cudaStream_t st);
// Leaves of every cell in particle order (leaf_start[n_leaves] = n), their
// cells and corners, and the first leaf of every cell (cell_leaf_start[n_cells]
// = n_leaves).  Scratch: lead (n bytes), nodes (n int2), work (n/4096 + 12
// words); *n_leaves points at the device count.
cudaError_t launch_leaves(const unsigned long long *sorted_keys, const int32_t *cell_start,
                          int n_cells, long long n, int leaf_max, uint8_t *lead, int2 *nodes,
                          unsigned int *work, unsigned int *scan_tmp, int32_t *leaf_start,
                          int32_t *leaf_cell, uint32_t *leaf_k, int32_t *cell_leaf_start,
                          int grid, const unsigned int **n_leaves, cudaStream_t st);
cudaError_t launch_bin_histogram(const View &v, cudaStream_t st);
cudaError_t launch_groups(const int32_t *cell_leaf_start, const int32_t *leaf_start, int n_cells,
                          int n_leaves_max, unsigned int *counts, unsigned int *offsets,
                          unsigned int *scan_tmp, int32_t *group_leaf0, int32_t *group_cell,
                          int32_t *pleaf, int n_leaves_host, cudaStream_t st);
cudaError_t launch_chunks(const unsigned long long *sorted_keys, const int32_t *leaf_start,
                          const int32_t *cell_leaf_start, int n_cells, int n_leaves,
                          unsigned long long *leaf_keys, uint8_t *lead, int2 *nodes,
                          unsigned int *work, unsigned int *scan_tmp, uint32_t *corner_tmp,
                          int32_t *chunk_leaf_start, int32_t *chunk_cell,
                          int32_t *cell_chunk_start, int32_t *leaf_chunk, int grid,
                          const unsigned int **n_chunks, cudaStream_t st);
// sph_integrate.cu
cudaError_t launch_refresh_all(const View &v, cudaStream_t st);
cudaError_t launch_mark(const View &v, long long ti_or_neg, cudaStream_t st);
cudaError_t launch_drift(const View &v, cudaStream_t st);
cudaError_t launch_kick(const View &v, int phase, cudaStream_t st);
cudaError_t launch_bins(const View &v, long long *ti_next_out, int count_step, cudaStream_t st);
cudaError_t launch_mark_bin(const View &v, int bin, cudaStream_t st);
// closing kick, new bins, opening kick and the next tick of a step, one launch
cudaError_t launch_close_step(const View &v, cudaStream_t st);
// sph_pairs.cu
cudaError_t launch_density(const View &v, int flags, int bin_filter, bool persistent,
                           int grid, cudaStream_t st);
cudaError_t launch_force(const View &v, int bin_filter, bool persistent, int grid,
                         cudaStream_t st);
cudaError_t launch_entropy_from_u(const View &v, cudaStream_t st);
int persistent_blocks_per_sm(int G, bool density);
cudaError_t launch_group_cost(const View &v, int grid, cudaStream_t st);
// velocity divergence and curl of the active particles (after their density)
cudaError_t launch_gradient(const View &v, int grid, cudaStream_t st);
// sph_adjoint.cu
cudaError_t launch_adj_prepare(const sph_particles &pre, const sph_particles &post,
                               const sph_particles &W, const sph_adjoint &adj, long long ti,
                               int first, double dt_min, double box, double gamma,
                               cudaStream_t st);
cudaError_t launch_adj_step(const View &v, const AdjWork &w, const sph_particles &pre,
                            const sph_particles &post, const sph_adjoint &adj, long long ti,
                            int first, int grid_pairs, cudaStream_t st);
cudaError_t launch_grid_density(const sph_particles &p, int n_grid, long long ti, double dt_min,
                                double box, double *rho_g, const double *rho_bar,
                                const sph_adjoint *adj, cudaStream_t st);
cudaError_t launch_state_copy(const sph_particles &src, const sph_particles &dst,
                              const int32_t *perm, cudaStream_t st);
int adj_blocks_per_sm();

}  // namespace sph
