// C ABI of libsph_gb300 (declared in include/sph.h): the context, the cell
// build, the individual hot-path calls and the two forms of a full
// kick-drift-kick step (plain per-bin launches, and the batched form with
// persistent pair-loop kernels replayed from a CUDA graph).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "sph_internal.cuh"
#include "sph_diag.cuh"

#include <atomic>

using namespace sph;

namespace sph {
static std::atomic<unsigned long long> g_launches{0};
// set while this thread captures a step into a graph: its launches are graph
// nodes, counted when the graph is replayed, not launches
static thread_local bool t_capturing = false;
void note_launches(int n) {
  if (!t_capturing) g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed);
}
}  // namespace sph

namespace {

constexpr int NC_MAX = 255;  // cells per axis (the exclusive scan covers <= 2^24 entries)

struct Buffers {
  // sort
  unsigned long long *keys[2] = {nullptr, nullptr};
  unsigned int *vals[2] = {nullptr, nullptr};
  unsigned int *hist = nullptr;
  unsigned int *scan_tmp = nullptr;
  int n_hist_max = 0;
  void *scratch = nullptr;  // 8 bytes per particle, permutation staging
  int32_t *perm = nullptr;  // composed permutation since the first build
  int32_t *perm_tmp = nullptr;
  int32_t *pcell = nullptr;
  // leaves (at most one per particle)
  int32_t *leaf_start = nullptr, *leaf_cell = nullptr;
  uint32_t *leaf_k = nullptr;
  // chunks: octree nodes of at most CHUNK leaves (at most one per particle)
  int32_t *chunk_cell = nullptr, *chunk_leaf_start = nullptr, *leaf_chunk = nullptr;
  float4 *chunk_lo = nullptr, *chunk_hi = nullptr;
  float4 *leaf_lo = nullptr, *leaf_hi = nullptr;
  uint8_t *leaf_min_bin = nullptr;
  unsigned long long *leaf_bin_mask = nullptr;
  int32_t *q_active = nullptr, *q_drift = nullptr, *q_bin = nullptr, *q_group = nullptr;
  // work groups of the pair loops
  int32_t *pleaf = nullptr, *group_leaf0 = nullptr, *group_cell = nullptr, *group_cost = nullptr;
  // records
  float4 *rec_xm = nullptr, *rec_xH = nullptr, *rec_v = nullptr, *rec_h = nullptr;
  // cells (grown on demand)
  long long cell_cap = 0;
  int32_t *cell_start = nullptr, *cell_leaf_start = nullptr, *cell_chunk_start = nullptr;
  unsigned int *cell_stamp = nullptr, *cell_rel_stamp = nullptr;
  int32_t *q_act_cells = nullptr;
  unsigned int *leaf_counts = nullptr, *leaf_offsets = nullptr;
  // neighbour lists of the density loop: list_cap entries per lane of every
  // warp of a persistent density launch
  float2 *nbr = nullptr;
  int8_t *ngb_bin = nullptr;  // limiter: smallest neighbour bin of each active particle
  int32_t *wake_bin = nullptr, *q_wake = nullptr;  // limiter: wake requests and their queue
  // state
  DevState *ds = nullptr;
  float *d_hmax = nullptr;
  double *diag = nullptr;  // diagnostics: block partials, then the result
  unsigned int *d_bad = nullptr;  // invalid-input count of the last cell build
  DevState *h_ds = nullptr;  // pinned host mirror
};

// Reverse-mode scratch (allocated on the first sph_step_bwd): a second
// context whose cells are built over internal copies of the step's particles,
// those copies, and the FP64 work arrays.
struct AdjBuffers {
  sph_ctx *sub = nullptr;
  double *x = nullptr, *y = nullptr, *z = nullptr;
  float *f32 = nullptr;       // 15 float arrays of n_max
  int8_t *bin = nullptr;
  int64_t *ti = nullptr;      // ti_begin, ti_end, ti_drift
  uint8_t *active = nullptr;
  double *work = nullptr;     // ADJ_WORK_ARRAYS double arrays of n_max
  int grid_pairs = 0;
};
constexpr int ADJ_WORK_ARRAYS = 18;  // the FP64 arrays of AdjWork

}  // namespace

struct sph_ctx {
  sph_params prm;
  long long n_max = 0;
  int device = 0;
  int num_sms = 0;
  int grid_util = 0;
  int grid_dens = 0, grid_force = 0;
  int list_blocks = 0;  // blocks a density launch may have (each warp has a list area)
  Buffers b;
  bool built = false;
  bool entropy_ready = false;  // the first density pass has converted u to A
  int nc = 0;
  double w = 0.0;
  int n_leaves = 0;
  float h_floor = 0.0f;  // after an h overflow: the next build sizes cells for this h
  long long alloc_version = 0;
  long long rebuilds = 0, redone = 0;
  long long steps_seen = 0;    // device step counter at the last sph_step_sync
  int pending = 0;             // steps enqueued since the last sph_step_sync
  bool init_pending = false;   // the entropy-initialising step is enqueued, not yet confirmed
  // optional CUDA-event timing of the pair-loop launches (0 density, 1 force)
  bool prof_on = false;
  cudaEvent_t prof_ev[2][64][2] = {};
  int prof_n[2] = {0, 0};
  double prof_ms[2] = {0.0, 0.0};
  long long prof_launches[2] = {0, 0};
  // captured batched step
  cudaGraphExec_t graph = nullptr;
  cudaStream_t cap_stream = nullptr;
  long long graph_version = -1;
  bool graph_profiled = false;
  bool uniform_mass = false;   // every particle has the same mass (last cell build)
  float m_uniform = 0.0f;      // that mass (0: the masses differ)
  bool graph_uniform = false;  // uniform_mass when the graph was captured
  int graph_kernels = 0;       // kernel nodes in the captured step
  sph_particles graph_p;
  AdjBuffers *adj = nullptr;
};

namespace {

#define SPH_CUDA(call)                          \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return SPH_ERR_CUDA; \
  } while (0)

template <typename T>
int dalloc(T **p, size_t count) {
  if (count == 0) count = 1;
  if (cudaMalloc((void **)p, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return SPH_ERR_NOMEM;
  }
  return SPH_OK;
}

template <typename T>
void dfree(T *&p) {
  if (p) cudaFree((void *)p);
  p = nullptr;
}

#define SPH_TRY(x)               \
  do {                           \
    int r_ = (x);                \
    if (r_ != SPH_OK) return r_; \
  } while (0)

cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }

bool valid_params(const sph_params *p) {
  if (!p) return false;
  if (!(p->box > 0) || !(p->eta > 0) || !(p->gamma > 1.0) || !(p->alpha_visc >= 0)) return false;
  if (!(p->cfl > 0) || !(p->h_tol > 0) || p->h_max_iter < 1 || p->bin_cap < 0 || p->bin_cap > 62)
    return false;
  if (!(p->dt_min > 0) || !(p->cell_margin >= 1.0)) return false;
  if (p->leaf_max < 1 || p->leaf_max > WG_MAX) return false;
  int G = p->threads_per_particle;
  if (G != 1 && G != 2 && G != 4 && G != 8 && G != 16 && G != 32) return false;
  if (p->n_cells_override < 0 || p->n_cells_override > NC_MAX) return false;
  if (std::isnan(p->heavy_factor) || p->coop_max_groups < -1) return false;
  if (p->list_cap < 32 || p->list_cap > 4096) return false;
  if (!(p->search_margin >= 1.0 && p->search_margin <= 2.0)) return false;
  if (p->staging_depth < 1 || p->staging_depth > 3) return false;
  if (p->wait_limit < 0 || p->test_stall < 0 || p->test_bad_group < 0) return false;
#ifndef SPH_CHECKS
  if (p->test_bad_group != 0) return false;  // only a checks build may plant a bad index
#endif
  const int vars[3] = {p->balsara, p->predict_inactive, p->limiter};
  for (int f : vars)
    if (f != 0 && f != 1) return false;
  if ((p->balsara || p->predict_inactive || p->limiter) && G != 1) return false;
  return true;
}

bool valid_particles(const sph_ctx *ctx, const sph_particles *p) {
  if (!p || p->n < 0 || p->n > ctx->n_max) return false;
  if (p->n == 0) return true;
  const void *req[] = {p->x,  p->y,  p->z,   p->vx,  p->vy,   p->vz,       p->ax,     p->ay,
                       p->az, p->A,  p->Adot, p->h,  p->rho,  p->f,        p->P,      p->c,
                       p->vsig, p->m, p->bin, p->ti_begin, p->ti_end, p->ti_drift, p->active};
  for (const void *q : req)
    if (!q) return false;
  // the variants that use the velocity divergence keep it per particle
  if ((ctx->prm.balsara || ctx->prm.predict_inactive) && (!p->div_v || !p->curl_v)) return false;
  return true;
}

View make_view(const sph_ctx *ctx, const sph_particles *p) {
  View v;
  std::memset(&v, 0, sizeof(v));
  v.n = p ? p->n : 0;
  if (p) {
    v.x = p->x; v.y = p->y; v.z = p->z;
    v.vx = p->vx; v.vy = p->vy; v.vz = p->vz;
    v.ax = p->ax; v.ay = p->ay; v.az = p->az;
    v.A = p->A; v.Adot = p->Adot; v.h = p->h; v.rho = p->rho; v.f = p->f; v.P = p->P;
    v.c = p->c; v.vsig = p->vsig; v.m = p->m; v.bin = p->bin;
    v.ti_begin = reinterpret_cast<long long *>(p->ti_begin);
    v.ti_end = reinterpret_cast<long long *>(p->ti_end);
    v.ti_drift = reinterpret_cast<long long *>(p->ti_drift);
    v.active = p->active;
    v.ngb_density = p->ngb_density;
    v.ngb_force = p->ngb_force;
    v.div_v = p->div_v;
    v.curl_v = p->curl_v;
  }
  const Buffers &b = ctx->b;
  v.cell_start = b.cell_start;
  v.cell_leaf_start = b.cell_leaf_start;
  v.cell_chunk_start = b.cell_chunk_start;
  v.chunk_cell = b.chunk_cell;
  v.chunk_leaf_start = b.chunk_leaf_start;
  v.leaf_chunk = b.leaf_chunk;
  v.chunk_lo = b.chunk_lo;
  v.chunk_hi = b.chunk_hi;
  v.cell_stamp = b.cell_stamp;
  v.cell_rel_stamp = b.cell_rel_stamp;
  v.leaf_start = b.leaf_start;
  v.leaf_cell = b.leaf_cell;
  v.leaf_k = b.leaf_k;
  v.leaf_lo = b.leaf_lo;
  v.leaf_hi = b.leaf_hi;
  v.leaf_min_bin = b.leaf_min_bin;
  v.leaf_bin_mask = b.leaf_bin_mask;
  v.pcell = b.pcell;
  v.rec_xm = b.rec_xm;
  v.rec_xH = b.rec_xH;
  v.rec_v = b.rec_v;
  v.rec_h = b.rec_h;
  v.q_active = b.q_active;
  v.q_group = b.q_group;
  v.pleaf = b.pleaf;
  v.group_leaf0 = b.group_leaf0;
  v.group_cell = b.group_cell;
  v.group_cost = b.group_cost;
  v.q_act_cells = b.q_act_cells;
  v.q_drift = b.q_drift;
  v.q_bin = b.q_bin;
  v.ds = b.ds;
  const sph_params &q = ctx->prm;
  v.box = q.box;
  v.eta = q.eta;
  v.gamma = q.gamma;
  v.alpha = q.alpha_visc;
  v.cfl = q.cfl;
  v.h_tol = q.h_tol;
  v.dt_min = q.dt_min;
  v.heavy_factor = q.heavy_factor;
  // (a step with few groups leaves warps idle; measured on the 2.1M clustered
  // set, sharing each group among a block pays up to ~2 groups per block)
  v.coop_max_groups = q.coop_max_groups < 0 ? 2 * ctx->grid_dens : q.coop_max_groups;
  v.h_max_iter = q.h_max_iter;
  v.bin_cap = q.bin_cap;
  v.leaf_max = q.leaf_max;
  v.G = q.threads_per_particle;
  v.drift_all = q.drift_all;
  v.uniform_mass = ctx->uniform_mass ? 1 : 0;
  v.grid_util = ctx->grid_util;
  v.nbr = b.nbr;
  v.list_cap = q.list_cap;
  v.list_blocks = ctx->list_blocks;
  v.search_margin = (float)q.search_margin;
  v.stage_depth = q.staging_depth;
  v.wait_limit = q.wait_limit;
  v.balsara = q.balsara;
  v.predict = q.predict_inactive;
  v.limiter = q.limiter;
  v.ngb_bin = b.ngb_bin;
  v.wake_bin = b.wake_bin;
  v.q_wake = b.q_wake;
  return v;
}

int ensure_cells(sph_ctx *ctx, long long n_cells) {
  Buffers &b = ctx->b;
  if (n_cells <= b.cell_cap) return SPH_OK;
  cudaDeviceSynchronize();
  dfree(b.cell_start);
  dfree(b.cell_leaf_start);
  dfree(b.cell_chunk_start);
  dfree(b.cell_stamp);
  dfree(b.cell_rel_stamp);
  dfree(b.q_act_cells);
  dfree(b.leaf_counts);
  dfree(b.leaf_offsets);
  long long cap = std::max<long long>(n_cells, b.cell_cap * 2);
  cap = std::min<long long>(cap, (long long)NC_MAX * NC_MAX * NC_MAX);
  cap = std::max(cap, n_cells);
  SPH_TRY(dalloc(&b.cell_start, cap + 1));
  SPH_TRY(dalloc(&b.cell_leaf_start, cap + 1));
  SPH_TRY(dalloc(&b.cell_chunk_start, cap + 1));
  SPH_TRY(dalloc(&b.cell_stamp, cap));
  SPH_TRY(dalloc(&b.cell_rel_stamp, cap));
  SPH_TRY(dalloc(&b.q_act_cells, cap));
  SPH_TRY(dalloc(&b.leaf_counts, cap + 1));
  SPH_TRY(dalloc(&b.leaf_offsets, cap + 1));
  SPH_CUDA(cudaMemset(b.cell_stamp, 0, sizeof(unsigned int) * cap));
  SPH_CUDA(cudaMemset(b.cell_rel_stamp, 0, sizeof(unsigned int) * cap));
  b.cell_cap = cap;
  ctx->alloc_version++;
  return SPH_OK;
}

int read_state(sph_ctx *ctx, cudaStream_t st) {
  SPH_CUDA(cudaMemcpyAsync(ctx->b.h_ds, ctx->b.ds, sizeof(DevState), cudaMemcpyDeviceToHost, st));
  SPH_CUDA(cudaStreamSynchronize(st));
  return SPH_OK;
}

// Event record on `st`; inside a stream capture it becomes an event-record
// node of the graph, so every replay records it.
void record_event(cudaEvent_t ev, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
  else cudaEventRecord(ev, st);
}

void prof_begin(sph_ctx *ctx, int kind, cudaStream_t st) {
  if (ctx->prof_on && ctx->prof_n[kind] < 64) record_event(ctx->prof_ev[kind][ctx->prof_n[kind]][0], st);
}

void prof_end(sph_ctx *ctx, int kind, cudaStream_t st) {
  if (ctx->prof_on && ctx->prof_n[kind] < 64) {
    record_event(ctx->prof_ev[kind][ctx->prof_n[kind]][1], st);
    ctx->prof_n[kind]++;
  }
}

// after a synchronisation: add the recorded launch durations
void prof_collect(sph_ctx *ctx) {
  for (int k = 0; k < 2; k++) {
    for (int i = 0; i < ctx->prof_n[k]; i++) {
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, ctx->prof_ev[k][i][0], ctx->prof_ev[k][i][1]) == cudaSuccess) {
        ctx->prof_ms[k] += ms;
        ctx->prof_launches[k]++;
      } else {
        cudaGetLastError();
      }
    }
    ctx->prof_n[k] = 0;
  }
}

int permute_array(sph_ctx *ctx, void *arr, int elem, long long n, const unsigned int *perm,
                  cudaStream_t st) {
  if (!arr) return SPH_OK;
  SPH_CUDA(launch_gather(ctx->b.scratch, arr, perm, n, elem, st, ctx->b.ds));
  SPH_CUDA(cudaMemcpyAsync(arr, ctx->b.scratch, (size_t)n * elem, cudaMemcpyDeviceToDevice, st));
  return SPH_OK;
}

int build_cells(sph_ctx *ctx, sph_particles *p, cudaStream_t st) {
  if (!valid_particles(ctx, p)) return SPH_ERR_ARG;
  Buffers &b = ctx->b;
  const long long n = p->n;
  if (!ctx->built && n > 0) {
    // the composed permutation starts as the identity
    std::vector<int32_t> id((size_t)n);
    for (long long k = 0; k < n; k++) id[(size_t)k] = (int32_t)k;
    SPH_CUDA(cudaMemcpyAsync(b.perm, id.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
    SPH_CUDA(cudaStreamSynchronize(st));
  }
  View v = make_view(ctx, p);
  // cells per axis from the largest support
  int nc = ctx->prm.n_cells_override;
  if (nc <= 0) {
    SPH_CUDA(launch_reduce_hmax(v, b.d_hmax, st));
    float hmax = 0.0f;
    SPH_CUDA(cudaMemcpyAsync(&hmax, b.d_hmax, sizeof(float), cudaMemcpyDeviceToHost, st));
    SPH_CUDA(cudaStreamSynchronize(st));
    if (n > 0 && !(hmax > 0.0f && std::isfinite(hmax))) return SPH_ERR_ARG;
    hmax = std::max(hmax, ctx->h_floor);
    double Hmax = GAMMA_K_D * (double)hmax;
    double ncd = n > 0 ? std::floor(ctx->prm.box / (ctx->prm.cell_margin * Hmax)) : 3.0;
    nc = (int)std::max(3.0, std::min((double)NC_MAX, ncd));
  }
  const long long n_cells = (long long)nc * nc * nc;
  SPH_TRY(ensure_cells(ctx, n_cells));
  v = make_view(ctx, p);
  const double w = ctx->prm.box / (double)nc;
  // keys, stable radix sort, permutation of every particle array
  SPH_CUDA(cudaMemsetAsync(b.d_bad, 0, sizeof(unsigned int), st));
  SPH_CUDA(launch_cell_keys(v, nc, w, b.keys[0], b.vals[0], b.d_bad, st));
  if (n > 0) {
    // non-finite positions or h: rejected before anything is reordered
    unsigned int bad = 0;
    SPH_CUDA(cudaMemcpyAsync(&bad, b.d_bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    SPH_CUDA(cudaStreamSynchronize(st));
    if (bad) return SPH_ERR_ARG;
  }
  int cell_bits = 1;
  while ((1LL << cell_bits) < n_cells) cell_bits++;
  bool alt = false;
  SPH_CUDA(radix_sort_pairs(b.keys[0], b.vals[0], b.keys[1], b.vals[1], (int)n,
                            KEY_MORTON_BITS + cell_bits, b.hist, b.scan_tmp, b.n_hist_max, &alt,
                            st, b.ds));
  unsigned long long *skeys = alt ? b.keys[1] : b.keys[0];
  unsigned int *perm = alt ? b.vals[1] : b.vals[0];
  SPH_TRY(permute_array(ctx, p->x, 8, n, perm, st));
  SPH_TRY(permute_array(ctx, p->y, 8, n, perm, st));
  SPH_TRY(permute_array(ctx, p->z, 8, n, perm, st));
  float *f32[] = {p->vx, p->vy, p->vz, p->ax, p->ay, p->az, p->A, p->Adot, p->h,
                  p->rho, p->f, p->P, p->c, p->vsig, p->m};
  for (float *a : f32) SPH_TRY(permute_array(ctx, a, 4, n, perm, st));
  SPH_TRY(permute_array(ctx, p->bin, 1, n, perm, st));
  SPH_TRY(permute_array(ctx, p->ti_begin, 8, n, perm, st));
  SPH_TRY(permute_array(ctx, p->ti_end, 8, n, perm, st));
  SPH_TRY(permute_array(ctx, p->ti_drift, 8, n, perm, st));
  SPH_TRY(permute_array(ctx, p->ngb_density, 4, n, perm, st));
  SPH_TRY(permute_array(ctx, p->ngb_force, 4, n, perm, st));
  SPH_TRY(permute_array(ctx, p->div_v, 4, n, perm, st));
  SPH_TRY(permute_array(ctx, p->curl_v, 4, n, perm, st));
  if (n > 0) {
    SPH_CUDA(launch_gather(b.perm_tmp, b.perm, perm, n, 4, st, b.ds));
    SPH_CUDA(cudaMemcpyAsync(b.perm, b.perm_tmp, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st));
    SPH_CUDA(cudaMemsetAsync(p->active, 0, (size_t)n, st));
  }
  // cells and leaves
  SPH_CUDA(launch_cell_start(skeys, n, (int)n_cells, b.cell_start, b.pcell, st));
  // (scratch: the marks in b.scratch, the node lists in the sort's spare key
  // buffer, the counters in the histogram)
  const unsigned int *d_n_leaves = nullptr;
  SPH_CUDA(launch_leaves(skeys, b.cell_start, (int)n_cells, n, ctx->prm.leaf_max,
                         (uint8_t *)b.scratch, (int2 *)(alt ? b.keys[0] : b.keys[1]), b.hist,
                         b.scan_tmp, b.leaf_start, b.leaf_cell, b.leaf_k, b.cell_leaf_start,
                         2 * ctx->grid_util, &d_n_leaves, st));
  SPH_CUDA(cudaMemcpyAsync(SPH_DS_FIELD(b.ds, n_leaves), d_n_leaves, sizeof(int),
                           cudaMemcpyDeviceToDevice, st));
  int n_leaves_h = 0;
  SPH_CUDA(cudaMemcpyAsync(&n_leaves_h, d_n_leaves, sizeof(int), cudaMemcpyDeviceToHost, st));
  SPH_CUDA(cudaStreamSynchronize(st));
  // work groups and the leaf of each particle
  SPH_CUDA(launch_groups(b.cell_leaf_start, b.leaf_start, (int)n_cells, (int)n, b.leaf_counts,
                         b.leaf_offsets, b.scan_tmp, b.group_leaf0, b.group_cell, b.pleaf, n_leaves_h,
                         st));
  SPH_CUDA(cudaMemcpyAsync(SPH_DS_FIELD(b.ds, n_groups), b.leaf_offsets + n_cells, sizeof(int),
                           cudaMemcpyDeviceToDevice, st));
  // chunks: octree nodes of at most CHUNK leaves (scratch free again by now:
  // the leaves' first keys in the spare key buffer, the node lists in the
  // sorted keys' buffer, the marks in b.scratch, the counters in the
  // histogram, the unused corners in b.vals[0])
  const unsigned int *d_n_chunks = nullptr;
  SPH_CUDA(launch_chunks(skeys, b.leaf_start, b.cell_leaf_start, (int)n_cells, n_leaves_h,
                         alt ? b.keys[0] : b.keys[1], (uint8_t *)b.scratch,
                         reinterpret_cast<int2 *>(skeys), b.hist, b.scan_tmp,
                         reinterpret_cast<uint32_t *>(b.vals[0]), b.chunk_leaf_start, b.chunk_cell,
                         b.cell_chunk_start, b.leaf_chunk, 2 * ctx->grid_util, &d_n_chunks, st));
  SPH_CUDA(cudaMemcpyAsync(SPH_DS_FIELD(b.ds, n_chunks), d_n_chunks, sizeof(int),
                           cudaMemcpyDeviceToDevice, st));
  // device state of the new structure
  int ncs[2] = {nc, (int)n_cells};
  SPH_CUDA(cudaMemcpyAsync(SPH_DS_FIELD(b.ds, nc), &ncs[0], sizeof(int), cudaMemcpyHostToDevice, st));
  SPH_CUDA(cudaMemcpyAsync(SPH_DS_FIELD(b.ds, n_cells), &ncs[1], sizeof(int), cudaMemcpyHostToDevice, st));
  SPH_CUDA(cudaMemcpyAsync(SPH_DS_FIELD(b.ds, w), &w, sizeof(double), cudaMemcpyHostToDevice, st));
  SPH_CUDA(cudaMemsetAsync(SPH_DS_FIELD(b.ds, n_active_leaves), 0, sizeof(int), st));
  SPH_CUDA(cudaMemsetAsync(SPH_DS_FIELD(b.ds, n_active_groups), 0, sizeof(int), st));
  SPH_CUDA(cudaMemsetAsync(SPH_DS_FIELD(b.ds, excursion_bits), 0, sizeof(unsigned int), st));
  SPH_CUDA(cudaMemsetAsync(SPH_DS_FIELD(b.ds, Hmax_bits), 0, sizeof(unsigned int), st));
  SPH_CUDA(cudaMemsetAsync(SPH_DS_FIELD(b.ds, want_h_bits), 0, sizeof(unsigned int), st));
  SPH_CUDA(launch_bin_histogram(v, st));
  SPH_CUDA(launch_refresh_all(v, st));
  // cost estimate of every work group (only heavy-group scheduling uses it)
  if (ctx->prm.heavy_factor > 0.0) SPH_CUDA(launch_group_cost(v, ctx->grid_dens, st));
  // equal masses: the density loop sums the kernel alone (rho = m sum w)
  SPH_CUDA(launch_mass_range(v, st));
  int nl = 0;
  unsigned int mr[2] = {0u, 0u};
  SPH_CUDA(cudaMemcpyAsync(&nl, SPH_DS_FIELD(b.ds, n_leaves), sizeof(int), cudaMemcpyDeviceToHost, st));
  SPH_CUDA(cudaMemcpyAsync(mr, SPH_DS_FIELD(b.ds, m_lo_bits), 2 * sizeof(unsigned int),
                           cudaMemcpyDeviceToHost, st));
  SPH_CUDA(cudaStreamSynchronize(st));
  ctx->n_leaves = nl;
  {
    float lo, hi;
    std::memcpy(&lo, &mr[0], sizeof(float));
    std::memcpy(&hi, &mr[1], sizeof(float));
    ctx->m_uniform = (n > 0 && mr[0] == mr[1] && lo > 0.0f && std::isfinite(lo)) ? lo : 0.0f;
    (void)hi;
  }
  ctx->uniform_mass = ctx->m_uniform > 0.0f;
  SPH_CUDA(cudaMemcpyAsync(SPH_DS_FIELD(b.ds, m_uniform), &ctx->m_uniform, sizeof(float),
                           cudaMemcpyHostToDevice, st));
  SPH_CUDA(cudaStreamSynchronize(st));  // (the build is complete on return, as before)
  ctx->h_floor = 0.0f;
  ctx->nc = nc;
  ctx->w = w;
  // no wake request survives a reordering (a halted step may have left some)
  SPH_CUDA(cudaMemsetAsync(b.wake_bin, 0x7f, sizeof(int32_t) * (size_t)ctx->n_max, st));
  ctx->built = true;
  ctx->rebuilds++;
  return SPH_OK;
}

// --- pieces of a step ------------------------------------------------------
int batched_body(sph_ctx *ctx, const View &v, int flags, cudaStream_t st) {
  SPH_CUDA(launch_mark(v, -1, st));
  SPH_CUDA(launch_drift(v, st));
  prof_begin(ctx, 0, st);
  SPH_CUDA(launch_density(v, flags, -1, true, ctx->grid_dens, st));
  prof_end(ctx, 0, st);
  if (flags & SPH_DENSITY_INIT_ENTROPY) SPH_CUDA(launch_entropy_from_u(v, st));
  if (v.balsara || v.predict) SPH_CUDA(launch_gradient(v, ctx->grid_force, st));
  prof_begin(ctx, 1, st);
  SPH_CUDA(launch_force(v, -1, true, ctx->grid_force, st));
  prof_end(ctx, 1, st);
  SPH_CUDA(launch_close_step(v, st));
  return SPH_OK;
}

int plain_body(sph_ctx *ctx, const View &v, int flags, cudaStream_t st) {
  SPH_CUDA(launch_mark(v, -1, st));
  SPH_CUDA(launch_drift(v, st));
  SPH_TRY(read_state(ctx, st));
  const DevState &h = *ctx->b.h_ds;
  int bins[MAX_BINS], nb = 0;
  for (int b = 0; b <= std::min(h.m_act, MAX_BINS - 1); b++)
    if (h.bin_count[b] > 0) bins[nb++] = b;
  // one density launch per active bin, the grid sized from the bin's queue
  for (int k = 0; k < nb; k++) {
    SPH_CUDA(launch_mark_bin(v, bins[k], st));
    int nq[2] = {0, 0};  // groups taken one per warp, heavy groups taken one per block
    SPH_CUDA(cudaMemcpyAsync(nq, SPH_DS_FIELD(v.ds, n_bin_groups), 2 * sizeof(int),
                             cudaMemcpyDeviceToHost, st));
    SPH_CUDA(cudaStreamSynchronize(st));
    // the bin's groups, one per warp, pulled from a head by at most the
    // persistent grid's blocks (each warp has its own neighbour-list area)
    const int want = (nq[0] + nq[1] + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
    prof_begin(ctx, 0, st);
    SPH_CUDA(launch_density(v, flags, bins[k], true, std::min(want, ctx->list_blocks), st));
    prof_end(ctx, 0, st);
  }
  if (flags & SPH_DENSITY_INIT_ENTROPY) SPH_CUDA(launch_entropy_from_u(v, st));
  if (v.balsara || v.predict) SPH_CUDA(launch_gradient(v, ctx->grid_force, st));
  for (int k = 0; k < nb; k++) {
    SPH_CUDA(launch_mark_bin(v, bins[k], st));
    int nq[2] = {0, 0};
    SPH_CUDA(cudaMemcpyAsync(nq, SPH_DS_FIELD(v.ds, n_bin_groups), 2 * sizeof(int),
                             cudaMemcpyDeviceToHost, st));
    SPH_CUDA(cudaStreamSynchronize(st));
    const int ncb = std::min(nq[1], ctx->list_blocks);
    prof_begin(ctx, 1, st);
    SPH_CUDA(launch_force(v, bins[k], false,
                          ncb + (nq[0] + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK, st));
    prof_end(ctx, 1, st);
  }
  SPH_CUDA(launch_close_step(v, st));
  return SPH_OK;
}

// After a halted step: rebuild with wider cells when the cells overflowed.
int recover(sph_ctx *ctx, sph_particles *p, cudaStream_t st, bool *redo) {
  *redo = false;
  SPH_TRY(read_state(ctx, st));
  const DevState &h = *ctx->b.h_ds;
  if (!h.halt) return SPH_OK;
  if (h.first_error != SPH_ERR_CELL_OVERFLOW) return h.first_error ? h.first_error : SPH_ERR_CUDA;
  // the cells are too small for the supports: rebuild.  When an h iteration
  // wanted to grow past the cell, size the new cells for the h it wanted.
  float want_h, Hmax;
  std::memcpy(&want_h, &h.want_h_bits, sizeof(float));
  std::memcpy(&Hmax, &h.Hmax_bits, sizeof(float));
  if (ctx->nc <= 3 && (double)Hmax > ctx->w)
    return SPH_ERR_CELL_OVERFLOW;  // even three cells per axis are narrower than a support
  if (want_h > 0.0f) {
    if (ctx->nc <= 3 || ctx->prm.n_cells_override > 0)
      return SPH_ERR_CELL_OVERFLOW;  // the box cannot hold three cells of this support
    ctx->h_floor = want_h * 1.05f;
  }
  SPH_CUDA(cudaMemsetAsync(SPH_DS_FIELD(ctx->b.ds, halt), 0, sizeof(unsigned int), st));
  SPH_CUDA(cudaMemsetAsync(SPH_DS_FIELD(ctx->b.ds, first_error), 0, sizeof(int), st));
  SPH_CUDA(cudaMemsetAsync(SPH_DS_FIELD(ctx->b.ds, err_count), 0, sizeof(h.err_count), st));
  SPH_TRY(build_cells(ctx, p, st));
  ctx->redone++;
  *redo = true;
  return SPH_OK;
}

int capture_graph(sph_ctx *ctx, sph_particles *p) {
  if (ctx->graph) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
  }
  View v = make_view(ctx, p);
  cudaGraph_t g = nullptr;
  const int saved_n[2] = {ctx->prof_n[0], ctx->prof_n[1]};
  ctx->prof_n[0] = ctx->prof_n[1] = 0;  // the graph records into slot 0 of each kind
  SPH_CUDA(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
  t_capturing = true;
  int r = batched_body(ctx, v, 0, ctx->cap_stream);
  t_capturing = false;
  cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
  // the kernels of one replay: the graph's kernel nodes
  ctx->graph_kernels = 0;
  size_t n_nodes = 0;
  if (e == cudaSuccess && r == SPH_OK && cudaGraphGetNodes(g, nullptr, &n_nodes) == cudaSuccess) {
    std::vector<cudaGraphNode_t> nodes(n_nodes);
    if (n_nodes && cudaGraphGetNodes(g, nodes.data(), &n_nodes) == cudaSuccess) {
      for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
          ctx->graph_kernels++;
      }
    }
  }
  ctx->prof_n[0] = saved_n[0];
  ctx->prof_n[1] = saved_n[1];
  ctx->graph_profiled = ctx->prof_on;
  ctx->graph_uniform = ctx->uniform_mass;
  if (r != SPH_OK) {
    if (g) cudaGraphDestroy(g);
    return r;
  }
  if (e != cudaSuccess) return SPH_ERR_CUDA;
  e = cudaGraphInstantiate(&ctx->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return SPH_ERR_CUDA;
  ctx->graph_version = ctx->alloc_version;
  ctx->graph_p = *p;
  return SPH_OK;
}

bool valid_adjoint(const sph_adjoint *a, long long n) {
  if (!a || a->n != n) return false;
  if (n == 0) return true;
  const void *req[] = {a->x, a->y, a->z, a->vx, a->vy, a->vz, a->ax, a->ay, a->az,
                       a->A, a->Adot, a->h, a->rho, a->f};
  for (const void *q : req)
    if (!q) return false;
  return true;
}

void free_adj(AdjBuffers *a) {
  if (a->sub) sph_destroy(a->sub);
  dfree(a->x); dfree(a->y); dfree(a->z); dfree(a->f32); dfree(a->bin); dfree(a->ti);
  dfree(a->active); dfree(a->work);
  delete a;
}

int ensure_adj(sph_ctx *ctx) {
  if (ctx->adj) return SPH_OK;
  AdjBuffers *a = new (std::nothrow) AdjBuffers();
  if (!a) return SPH_ERR_NOMEM;
  const long long n = std::max<long long>(ctx->n_max, 1);
  int r = sph_create(&ctx->prm, ctx->n_max, &a->sub);
  if (r == SPH_OK &&
      ((r = dalloc(&a->x, n)) || (r = dalloc(&a->y, n)) || (r = dalloc(&a->z, n)) ||
       (r = dalloc(&a->f32, 15 * n)) || (r = dalloc(&a->bin, n)) || (r = dalloc(&a->ti, 3 * n)) ||
       (r = dalloc(&a->active, n)) || (r = dalloc(&a->work, (long long)ADJ_WORK_ARRAYS * n)))) {
  }
  if (r == SPH_OK) {
    const int nb = adj_blocks_per_sm();
    if (nb <= 0) r = SPH_ERR_CUDA;
    a->grid_pairs = ctx->num_sms * nb;
  }
  if (r != SPH_OK) {
    free_adj(a);
    return r;
  }
  ctx->adj = a;
  return SPH_OK;
}

sph_particles adj_particles(const AdjBuffers &a, long long n_max, long long n) {
  sph_particles W;
  std::memset(&W, 0, sizeof(W));
  W.n = n;
  W.x = a.x; W.y = a.y; W.z = a.z;
  float *f[15];
  for (int k = 0; k < 15; k++) f[k] = a.f32 + (size_t)k * n_max;
  W.vx = f[0]; W.vy = f[1]; W.vz = f[2]; W.ax = f[3]; W.ay = f[4]; W.az = f[5];
  W.A = f[6]; W.Adot = f[7]; W.h = f[8]; W.rho = f[9]; W.f = f[10]; W.P = f[11];
  W.c = f[12]; W.vsig = f[13]; W.m = f[14];
  W.bin = a.bin;
  W.ti_begin = a.ti; W.ti_end = a.ti + n_max; W.ti_drift = a.ti + 2 * n_max;
  W.active = a.active;
  return W;
}

AdjWork adj_work(const AdjBuffers &a, long long n_max, const int32_t *perm) {
  AdjWork w;
  double *d[ADJ_WORK_ARRAYS];
  for (int k = 0; k < ADJ_WORK_ARRAYS; k++) d[k] = a.work + (size_t)k * n_max;
  w.perm = perm;
  w.xb = d[0]; w.yb = d[1]; w.zb = d[2];
  w.vpxb = d[3]; w.vpyb = d[4]; w.vpzb = d[5];
  w.hb = d[6]; w.rhob = d[7]; w.fb = d[8]; w.Qb = d[9]; w.cb = d[10];
  w.axb = d[11]; w.ayb = d[12]; w.azb = d[13]; w.Adotb = d[14];
  w.ka = d[15]; w.kb = d[16]; w.km = d[17];
  return w;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void sph_default_params(sph_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->box = 1.0;
  p->eta = 1.2348;
  p->gamma = 5.0 / 3.0;
  p->alpha_visc = 0.8;
  p->cfl = 0.1;
  p->h_tol = 1e-6;
  p->h_max_iter = 30;
  p->bin_cap = 20;
  p->dt_min = 1e-6;
  p->t_begin = 0.0;
  p->cell_margin = 2.0;
  p->leaf_max = 8;
  p->threads_per_particle = 1;
  p->drift_all = 0;
  p->n_cells_override = 0;
  p->heavy_factor = 2.0;
  p->coop_max_groups = -1;
  p->list_cap = 512;
  p->search_margin = 1.02;
  p->staging_depth = 1;
  p->wait_limit = 0;
  p->test_stall = 0;
  p->test_bad_group = 0;
  p->balsara = 0;
  p->predict_inactive = 0;
  p->limiter = 0;
}

const char *sph_strerror(int code) {
  switch (code) {
    case SPH_OK: return "ok";
    case SPH_ERR_ARG: return "invalid argument";
    case SPH_ERR_CUDA: return "CUDA runtime error";
    case SPH_ERR_H_NOCONV: return "smoothing length did not converge";
    case SPH_ERR_CELL_OVERFLOW: return "kernel support outgrew the cell width (rebuild needed)";
    case SPH_ERR_DT_TOO_SMALL: return "time step below dt_min";
    case SPH_ERR_TIMEOUT: return "bounded device wait timed out";
    case SPH_ERR_NOMEM: return "device allocation failed";
    case SPH_ERR_NOT_BUILT: return "cells not built";
    case SPH_ERR_BOUNDS: return "device bounds check failed";
    default: return "unknown error";
  }
}

int sph_create(const sph_params *params, int64_t n_max, sph_ctx **out) {
  if (!out || !valid_params(params) || n_max < 0 || n_max > (1LL << 30)) return SPH_ERR_ARG;
  *out = nullptr;
  sph_ctx *ctx = new (std::nothrow) sph_ctx();
  if (!ctx) return SPH_ERR_NOMEM;
  ctx->prm = *params;
  ctx->n_max = n_max;
  int r = SPH_OK;
  do {
    if (cudaGetDevice(&ctx->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device) !=
            cudaSuccess) {
      r = SPH_ERR_CUDA;
      break;
    }
    ctx->grid_util = ctx->num_sms * 4;
    const int G = params->threads_per_particle;
    ctx->grid_dens = ctx->num_sms * persistent_blocks_per_sm(G, true);
    ctx->grid_force = ctx->num_sms * persistent_blocks_per_sm(G, false);
    if (ctx->grid_dens == 0 || ctx->grid_force == 0) {
      r = SPH_ERR_CUDA;  // the pair kernels cannot be resident with their shared memory
      break;
    }
    Buffers &b = ctx->b;
    const long long n = std::max<long long>(n_max, 1);
    const long long n_tiles = (n + 4095) / 4096;
    b.n_hist_max = (int)(256 * n_tiles);
    if ((r = dalloc(&b.keys[0], n)) || (r = dalloc(&b.keys[1], n)) || (r = dalloc(&b.vals[0], n)) ||
        (r = dalloc(&b.vals[1], n)) || (r = dalloc(&b.hist, b.n_hist_max)) ||
        (r = dalloc(&b.scan_tmp, 4096)) || (r = dalloc((char **)&b.scratch, 8 * n)) ||
        (r = dalloc(&b.perm, n)) || (r = dalloc(&b.perm_tmp, n)) || (r = dalloc(&b.pcell, n)) ||
        (r = dalloc(&b.leaf_start, n + 1)) || (r = dalloc(&b.leaf_cell, n)) || (r = dalloc(&b.leaf_k, n)) ||
        (r = dalloc(&b.chunk_cell, n)) || (r = dalloc(&b.chunk_leaf_start, n + 1)) ||
        (r = dalloc(&b.leaf_chunk, n)) || (r = dalloc(&b.chunk_lo, n)) || (r = dalloc(&b.chunk_hi, n)) ||
        (r = dalloc(&b.leaf_lo, n)) || (r = dalloc(&b.leaf_hi, n)) ||
        (r = dalloc(&b.leaf_min_bin, n)) || (r = dalloc(&b.leaf_bin_mask, n)) ||
        (r = dalloc(&b.q_active, n)) || (r = dalloc(&b.q_drift, n)) || (r = dalloc(&b.q_bin, n)) ||
        (r = dalloc(&b.q_group, n)) || (r = dalloc(&b.pleaf, n)) || (r = dalloc(&b.group_leaf0, n + 1)) ||
        (r = dalloc(&b.group_cell, n)) || (r = dalloc(&b.group_cost, n)) ||
        (r = dalloc(&b.rec_xm, n)) || (r = dalloc(&b.rec_xH, n)) || (r = dalloc(&b.rec_v, n)) ||
        (r = dalloc(&b.rec_h, n)) || (r = dalloc(&b.ds, 1)) || (r = dalloc(&b.d_hmax, 1)) ||
        (r = dalloc(&b.diag, (long long)(DIAG_BLOCKS + 1) * DIAG_FIELDS)) ||
        (r = dalloc(&b.d_bad, 1)))
      break;
    if (cudaMallocHost((void **)&b.h_ds, sizeof(DevState)) != cudaSuccess) {
      r = SPH_ERR_NOMEM;
      break;
    }
    if (cudaMemset(b.ds, 0, sizeof(DevState)) != cudaSuccess ||
        cudaMemcpy(SPH_DS_FIELD(b.ds, test_stall), &params->test_stall, sizeof(int),
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(SPH_DS_FIELD(b.ds, test_bad_group), &params->test_bad_group, sizeof(int),
                   cudaMemcpyHostToDevice) != cudaSuccess) {
      r = SPH_ERR_CUDA;
      break;
    }
    // neighbour lists of the density loop: by particle, and for the blocks
    // that share a work group (those of a persistent launch; a per-bin launch
    // uses at most as many)
    ctx->list_blocks = ctx->grid_dens;
    if ((r = dalloc(&b.ngb_bin, n)) || (r = dalloc(&b.wake_bin, n)) ||
        (r = dalloc(&b.q_wake, n)) ||
        (r = dalloc(&b.nbr, (long long)ctx->list_blocks * WARPS_PER_BLOCK * 32 * params->list_cap)))
      break;
    // no neighbour bin known yet: no limit (a bins call without a force pass);
    // no wake request
    if (cudaMemset(b.ngb_bin, 127, (size_t)n) != cudaSuccess ||
        cudaMemset(b.wake_bin, 0x7f, sizeof(int32_t) * (size_t)n) != cudaSuccess) {
      r = SPH_ERR_CUDA;
      break;
    }
    if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      r = SPH_ERR_CUDA;
      break;
    }
  } while (0);
  if (r != SPH_OK) {
    sph_destroy(ctx);
    return r;
  }
  *out = ctx;
  return SPH_OK;
}

int sph_destroy(sph_ctx *ctx) {
  if (!ctx) return SPH_ERR_ARG;
  cudaDeviceSynchronize();
  if (ctx->adj) {
    free_adj(ctx->adj);
    ctx->adj = nullptr;
  }
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  for (auto &kind : ctx->prof_ev)
    for (auto &pair : kind)
      for (auto &ev : pair)
        if (ev) cudaEventDestroy(ev);
  Buffers &b = ctx->b;
  dfree(b.keys[0]); dfree(b.keys[1]); dfree(b.vals[0]); dfree(b.vals[1]);
  dfree(b.hist); dfree(b.scan_tmp);
  if (b.scratch) cudaFree(b.scratch);
  dfree(b.perm); dfree(b.perm_tmp); dfree(b.pcell);
  dfree(b.leaf_start); dfree(b.leaf_cell); dfree(b.leaf_k);
  dfree(b.chunk_cell); dfree(b.chunk_leaf_start); dfree(b.leaf_chunk); dfree(b.chunk_lo); dfree(b.chunk_hi); dfree(b.leaf_lo); dfree(b.leaf_hi);
  dfree(b.leaf_min_bin); dfree(b.leaf_bin_mask);
  dfree(b.q_active); dfree(b.q_drift); dfree(b.q_bin); dfree(b.q_group);
  dfree(b.pleaf); dfree(b.group_leaf0); dfree(b.group_cell); dfree(b.group_cost);
  dfree(b.rec_xm); dfree(b.rec_xH); dfree(b.rec_v); dfree(b.rec_h);
  dfree(b.cell_start); dfree(b.cell_leaf_start); dfree(b.cell_stamp); dfree(b.cell_rel_stamp);
  dfree(b.q_act_cells); dfree(b.leaf_counts); dfree(b.leaf_offsets);
  dfree(b.ds); dfree(b.d_hmax); dfree(b.diag); dfree(b.d_bad);
  dfree(b.nbr); dfree(b.ngb_bin); dfree(b.wake_bin); dfree(b.q_wake);
  if (b.h_ds) cudaFreeHost(b.h_ds);
  delete ctx;
  return SPH_OK;
}

int sph_build_cells(sph_ctx *ctx, sph_particles *p, void *stream) {
  if (!ctx) return SPH_ERR_ARG;
  return build_cells(ctx, p, S(stream));
}

const int32_t *sph_perm(const sph_ctx *ctx) { return ctx && ctx->built ? ctx->b.perm : nullptr; }

int sph_grid_info(const sph_ctx *ctx, int *nc, int *n_leaves) {
  if (!ctx) return SPH_ERR_ARG;
  if (!ctx->built) return SPH_ERR_NOT_BUILT;
  if (nc) *nc = ctx->nc;
  if (n_leaves) *n_leaves = ctx->n_leaves;
  return SPH_OK;
}

int sph_mark_active(sph_ctx *ctx, sph_particles *p, int64_t ti_current, void *stream) {
  if (!ctx || !valid_particles(ctx, p)) return SPH_ERR_ARG;
  if (!ctx->built) return SPH_ERR_NOT_BUILT;
  SPH_CUDA(launch_mark(make_view(ctx, p), ti_current < 0 ? -1 : ti_current, S(stream)));
  return SPH_OK;
}

int sph_kick_drift(sph_ctx *ctx, sph_particles *p, int phase, void *stream) {
  if (!ctx || !valid_particles(ctx, p)) return SPH_ERR_ARG;
  if (!ctx->built) return SPH_ERR_NOT_BUILT;
  View v = make_view(ctx, p);
  switch (phase) {
    case SPH_DRIFT: SPH_CUDA(launch_drift(v, S(stream))); break;
    case SPH_KICK_CLOSE:
    case SPH_KICK_OPEN: SPH_CUDA(launch_kick(v, phase, S(stream))); break;
    default: return SPH_ERR_ARG;
  }
  return SPH_OK;
}

int sph_density_active(sph_ctx *ctx, sph_particles *p, int flags, void *stream) {
  if (!ctx || !valid_particles(ctx, p)) return SPH_ERR_ARG;
  if (!ctx->built) return SPH_ERR_NOT_BUILT;
  View v = make_view(ctx, p);
  SPH_CUDA(launch_density(v, flags, -1, true, ctx->grid_dens, S(stream)));
  if (flags & SPH_DENSITY_INIT_ENTROPY) SPH_CUDA(launch_entropy_from_u(v, S(stream)));
  if (v.balsara || v.predict) SPH_CUDA(launch_gradient(v, ctx->grid_force, S(stream)));
  return SPH_OK;
}

int sph_force_active(sph_ctx *ctx, sph_particles *p, void *stream) {
  if (!ctx || !valid_particles(ctx, p)) return SPH_ERR_ARG;
  if (!ctx->built) return SPH_ERR_NOT_BUILT;
  SPH_CUDA(launch_force(make_view(ctx, p), -1, true, ctx->grid_force, S(stream)));
  return SPH_OK;
}

int sph_timestep_bins(sph_ctx *ctx, sph_particles *p, int64_t *ti_next_dev, void *stream) {
  if (!ctx || !valid_particles(ctx, p)) return SPH_ERR_ARG;
  if (!ctx->built) return SPH_ERR_NOT_BUILT;
  SPH_CUDA(launch_bins(make_view(ctx, p), reinterpret_cast<long long *>(ti_next_dev), 0, S(stream)));
  return SPH_OK;
}

int sph_begin_run(sph_ctx *ctx, void *stream) {
  if (!ctx) return SPH_ERR_ARG;
  cudaStream_t st = S(stream);
  long long zero = 0;
  SPH_CUDA(cudaMemcpyAsync(SPH_DS_FIELD(ctx->b.ds, ti), &zero, sizeof(zero), cudaMemcpyHostToDevice, st));
  SPH_CUDA(cudaMemcpyAsync(SPH_DS_FIELD(ctx->b.ds, ti_next), &zero, sizeof(zero), cudaMemcpyHostToDevice, st));
  SPH_TRY(sph_clear_status(ctx, stream));
  SPH_TRY(sph_reset_counters(ctx, stream));
  SPH_CUDA(cudaStreamSynchronize(st));
  ctx->entropy_ready = false;
  ctx->pending = 0;
  ctx->init_pending = false;
  return SPH_OK;
}

int sph_step_async(sph_ctx *ctx, sph_particles *p, int form, void *stream) {
  if (!ctx || !valid_particles(ctx, p) ||
      (form != SPH_FORM_PLAIN && form != SPH_FORM_BATCHED && form != SPH_FORM_BATCHED_NOGRAPH))
    return SPH_ERR_ARG;
  cudaStream_t st = S(stream);
  if (!ctx->built) SPH_TRY(build_cells(ctx, p, st));
  View v = make_view(ctx, p);
  if (!ctx->entropy_ready) {
    // the first step of a run sets the entropy from u (outside any graph)
    if (form == SPH_FORM_PLAIN) SPH_TRY(plain_body(ctx, v, SPH_DENSITY_INIT_ENTROPY, st));
    else SPH_TRY(batched_body(ctx, v, SPH_DENSITY_INIT_ENTROPY, st));
    ctx->entropy_ready = true;
    ctx->init_pending = true;
  } else if (form == SPH_FORM_BATCHED) {
    if (!ctx->graph || ctx->graph_version != ctx->alloc_version ||
        ctx->graph_profiled != ctx->prof_on || ctx->graph_uniform != ctx->uniform_mass ||
        std::memcmp(&ctx->graph_p, p, sizeof(*p)) != 0) {
      prof_collect(ctx);
      SPH_TRY(capture_graph(ctx, p));
    }
    SPH_CUDA(cudaGraphLaunch(ctx->graph, st));
    note_launches(ctx->graph_kernels);
    if (ctx->prof_on) ctx->prof_n[0] = ctx->prof_n[1] = 1;  // slot 0, recorded by the graph
  } else if (form == SPH_FORM_BATCHED_NOGRAPH) {
    SPH_TRY(batched_body(ctx, v, 0, st));
  } else {
    SPH_TRY(plain_body(ctx, v, 0, st));
  }
  ctx->pending++;
  return SPH_OK;
}

int sph_step_sync(sph_ctx *ctx, sph_particles *p, int *completed, void *stream) {
  if (!ctx || !valid_particles(ctx, p)) return SPH_ERR_ARG;
  cudaStream_t st = S(stream);
  SPH_TRY(read_state(ctx, st));
  prof_collect(ctx);
  const long long steps = (long long)ctx->b.h_ds->steps;
  const long long done = steps - ctx->steps_seen;
  ctx->steps_seen = steps;
  if (completed) *completed = (int)done;
  if (ctx->init_pending && done == 0) ctx->entropy_ready = false;  // the first step must rerun
  if (done > 0) ctx->init_pending = false;
  ctx->pending = 0;
  bool redo = false;
  SPH_TRY(recover(ctx, p, st, &redo));
  return SPH_OK;
}

int sph_step(sph_ctx *ctx, sph_particles *p, int form, void *stream) {
  for (int attempt = 0; attempt < 64; attempt++) {
    SPH_TRY(sph_step_async(ctx, p, form, stream));
    int done = 0;
    SPH_TRY(sph_step_sync(ctx, p, &done, stream));
    if (done == 1) return SPH_OK;
  }
  return SPH_ERR_CELL_OVERFLOW;
}

int sph_step_graph(sph_ctx *ctx, sph_particles *p, int n_steps, void *stream) {
  if (!ctx || !valid_particles(ctx, p) || n_steps < 0) return SPH_ERR_ARG;
  int done = 0, guard = 0;
  while (done < n_steps) {
    for (int k = done; k < n_steps; k++) SPH_TRY(sph_step_async(ctx, p, SPH_FORM_BATCHED, stream));
    int c = 0;
    SPH_TRY(sph_step_sync(ctx, p, &c, stream));
    done += c;
    if (++guard > 64) return SPH_ERR_CELL_OVERFLOW;
  }
  return SPH_OK;
}

int sph_get_time(sph_ctx *ctx, int64_t *ti_current, int64_t *ti_next) {
  if (!ctx) return SPH_ERR_ARG;
  SPH_CUDA(cudaMemcpy(ctx->b.h_ds, ctx->b.ds, sizeof(DevState), cudaMemcpyDeviceToHost));
  if (ti_current) *ti_current = ctx->b.h_ds->ti;
  if (ti_next) *ti_next = ctx->b.h_ds->ti_next;
  return SPH_OK;
}

int sph_set_time(sph_ctx *ctx, int64_t ti_current, void *stream) {
  if (!ctx || ti_current < 0) return SPH_ERR_ARG;
  long long t = ti_current;
  SPH_CUDA(cudaMemcpyAsync(SPH_DS_FIELD(ctx->b.ds, ti), &t, sizeof(t), cudaMemcpyHostToDevice, S(stream)));
  SPH_CUDA(cudaMemcpyAsync(SPH_DS_FIELD(ctx->b.ds, ti_next), &t, sizeof(t), cudaMemcpyHostToDevice, S(stream)));
  SPH_CUDA(cudaStreamSynchronize(S(stream)));
  return SPH_OK;
}

int sph_get_status(sph_ctx *ctx, int *status, int64_t *detail) {
  if (!ctx) return SPH_ERR_ARG;
  SPH_CUDA(cudaDeviceSynchronize());
  SPH_CUDA(cudaMemcpy(ctx->b.h_ds, ctx->b.ds, sizeof(DevState), cudaMemcpyDeviceToHost));
  const DevState &h = *ctx->b.h_ds;
  if (status) *status = h.first_error;
  if (detail) *detail = h.first_error ? (int64_t)h.err_count[h.first_error & 15] : 0;
  return SPH_OK;
}

int sph_built_with_checks(void) {
#ifdef SPH_CHECKS
  return 1;
#else
  return 0;
#endif
}

int sph_get_check_report(sph_ctx *ctx, int *site, int64_t *index, int64_t *bound) {
  if (!ctx) return SPH_ERR_ARG;
  SPH_CUDA(cudaDeviceSynchronize());
  SPH_CUDA(cudaMemcpy(ctx->b.h_ds, ctx->b.ds, sizeof(DevState), cudaMemcpyDeviceToHost));
  const DevState &h = *ctx->b.h_ds;
  if (site) *site = h.check_site;
  if (index) *index = h.check_site ? (int64_t)h.check_index : 0;
  if (bound) *bound = h.check_site ? (int64_t)h.check_bound : 0;
  return SPH_OK;
}

int sph_clear_status(sph_ctx *ctx, void *stream) {
  if (!ctx) return SPH_ERR_ARG;
  cudaStream_t st = S(stream);
  SPH_CUDA(cudaMemsetAsync(SPH_DS_FIELD(ctx->b.ds, halt), 0, sizeof(unsigned int), st));
  SPH_CUDA(cudaMemsetAsync(SPH_DS_FIELD(ctx->b.ds, first_error), 0, sizeof(int), st));
  SPH_CUDA(cudaMemsetAsync(SPH_DS_FIELD(ctx->b.ds, err_count), 0, sizeof(((DevState *)0)->err_count), st));
  SPH_CUDA(cudaMemsetAsync(SPH_DS_FIELD(ctx->b.ds, check_site), 0, sizeof(int), st));
  // (a halted step may have left wake requests that its close never applied)
  if (ctx->n_max > 0)
    SPH_CUDA(cudaMemsetAsync(ctx->b.wake_bin, 0x7f, sizeof(int32_t) * (size_t)ctx->n_max, st));
  return SPH_OK;
}

int sph_get_counters(sph_ctx *ctx, sph_counters *out) {
  if (!ctx || !out) return SPH_ERR_ARG;
  SPH_CUDA(cudaDeviceSynchronize());
  SPH_CUDA(cudaMemcpy(ctx->b.h_ds, ctx->b.ds, sizeof(DevState), cudaMemcpyDeviceToHost));
  const DevState &h = *ctx->b.h_ds;
  // totals of completed steps plus the calls made outside a step since
  out->pairs_density = (int64_t)(h.pairs_density + h.s_pairs_density);
  out->pairs_force = (int64_t)(h.pairs_force + h.s_pairs_force);
  out->cand_density = (int64_t)(h.cand_density + h.s_cand_density);
  out->cand_force = (int64_t)(h.cand_force + h.s_cand_force);
  out->iters_density = (int64_t)(h.iters_density + h.s_iters_density);
  out->active_particles = (int64_t)(h.active_particles + h.s_active_particles);
  out->steps = (int64_t)h.steps;
  out->rebuilds = ctx->rebuilds;
  out->redone_steps = ctx->redone;
  out->kernel_launches = (int64_t)g_launches.load();
  out->gathers_density = (int64_t)(h.gathers_density + h.s_gathers_density);
  out->list_overflows = (int64_t)(h.list_overflows + h.s_list_overflows);
  out->evals_density = (int64_t)(h.evals_density + h.s_evals_density);
  out->wakes = (int64_t)h.wakes;
  return SPH_OK;
}

int sph_get_bin_counts(sph_ctx *ctx, int64_t *counts, int n_bins, void *stream) {
  if (!ctx || !counts || n_bins < 1 || n_bins > MAX_BINS) return SPH_ERR_ARG;
  SPH_TRY(read_state(ctx, S(stream)));
  for (int b = 0; b < n_bins; b++) counts[b] = (int64_t)ctx->b.h_ds->bin_count[b];
  return SPH_OK;
}

int sph_reset_counters(sph_ctx *ctx, void *stream) {
  if (!ctx) return SPH_ERR_ARG;
  cudaStream_t st = S(stream);
  const size_t off = offsetof(DevState, s_pairs_density);
  const size_t len = offsetof(DevState, bin_count) - off;
  SPH_CUDA(cudaMemsetAsync(reinterpret_cast<char *>(ctx->b.ds) + off, 0, len, st));
  ctx->rebuilds = 0;
  ctx->redone = 0;
  ctx->steps_seen = 0;
  return SPH_OK;
}

int sph_set_profiling(sph_ctx *ctx, int enable) {
  if (!ctx) return SPH_ERR_ARG;
  if (enable && !ctx->prof_ev[0][0][0]) {
    for (auto &kind : ctx->prof_ev)
      for (auto &pair : kind)
        for (auto &ev : pair) SPH_CUDA(cudaEventCreate(&ev));
  }
  ctx->prof_on = enable != 0;
  ctx->prof_n[0] = ctx->prof_n[1] = 0;
  return SPH_OK;
}

int sph_get_kernel_times(sph_ctx *ctx, sph_kernel_times *out) {
  if (!ctx || !out) return SPH_ERR_ARG;
  SPH_CUDA(cudaDeviceSynchronize());
  prof_collect(ctx);
  out->density_ms = ctx->prof_ms[0];
  out->force_ms = ctx->prof_ms[1];
  out->density_launches = ctx->prof_launches[0];
  out->force_launches = ctx->prof_launches[1];
  return SPH_OK;
}

int sph_reset_kernel_times(sph_ctx *ctx) {
  if (!ctx) return SPH_ERR_ARG;
  SPH_CUDA(cudaDeviceSynchronize());
  ctx->prof_n[0] = ctx->prof_n[1] = 0;
  ctx->prof_ms[0] = ctx->prof_ms[1] = 0.0;
  ctx->prof_launches[0] = ctx->prof_launches[1] = 0;
  return SPH_OK;
}

int sph_state_copy(const sph_ctx *ctx, const sph_particles *src, sph_particles *dst,
                   int to_input_order, void *stream) {
  if (!ctx || !valid_particles(ctx, src) || !valid_particles(ctx, dst) || src->n != dst->n)
    return SPH_ERR_ARG;
  const int32_t *perm = (to_input_order && ctx->built) ? ctx->b.perm : nullptr;
  SPH_CUDA(launch_state_copy(*src, *dst, perm, S(stream)));
  return SPH_OK;
}

int sph_resume(sph_ctx *ctx, sph_particles *p, int64_t ti_current, int first, void *stream) {
  if (!ctx || !valid_particles(ctx, p) || ti_current < 0) return SPH_ERR_ARG;
  SPH_TRY(sph_set_time(ctx, ti_current, stream));
  SPH_TRY(sph_clear_status(ctx, stream));
  SPH_CUDA(cudaStreamSynchronize(S(stream)));
  ctx->built = false;  // a new input order: the next step rebuilds, the permutation restarts
  ctx->entropy_ready = !first;
  ctx->pending = 0;
  ctx->init_pending = false;
  return SPH_OK;
}

int sph_diagnostics(sph_ctx *ctx, const sph_particles *p, int64_t ti, double *out,
                    void *stream) {
  if (!ctx || !valid_particles(ctx, p) || !out) return SPH_ERR_ARG;
  cudaStream_t st = S(stream);
  long long t = ti;
  if (t < 0) {
    SPH_TRY(read_state(ctx, st));
    t = ctx->b.h_ds->ti;
  }
  double *dout = ctx->b.diag + (size_t)DIAG_BLOCKS * DIAG_FIELDS;
  SPH_CUDA(launch_diagnostics(*p, t, ctx->prm.dt_min, ctx->prm.gamma, ctx->b.diag, dout, st));
  SPH_CUDA(cudaMemcpyAsync(out, dout, sizeof(double) * DIAG_FIELDS, cudaMemcpyDeviceToHost, st));
  SPH_CUDA(cudaStreamSynchronize(st));
  return SPH_OK;
}

int sph_grid_density(sph_ctx *ctx, const sph_particles *p, int n_grid, int64_t ti,
                     double *rho_grid, void *stream) {
  if (!ctx || !valid_particles(ctx, p) || n_grid < 1 || n_grid > 1024 || !rho_grid || ti < 0)
    return SPH_ERR_ARG;
  const size_t ng3 = (size_t)n_grid * n_grid * n_grid;
  SPH_CUDA(cudaMemsetAsync(rho_grid, 0, ng3 * sizeof(double), S(stream)));
  SPH_CUDA(launch_grid_density(*p, n_grid, ti, ctx->prm.dt_min, ctx->prm.box, rho_grid, nullptr,
                               nullptr, S(stream)));
  return SPH_OK;
}

int sph_grid_density_bwd(sph_ctx *ctx, const sph_particles *p, int n_grid, int64_t ti,
                         const double *rho_grid_bar, sph_adjoint *adj, void *stream) {
  if (!ctx || !valid_particles(ctx, p) || n_grid < 1 || n_grid > 1024 || !rho_grid_bar ||
      ti < 0 || !valid_adjoint(adj, p->n))
    return SPH_ERR_ARG;
  SPH_CUDA(launch_grid_density(*p, n_grid, ti, ctx->prm.dt_min, ctx->prm.box, nullptr,
                               rho_grid_bar, adj, S(stream)));
  return SPH_OK;
}

int sph_step_bwd(sph_ctx *ctx, const sph_particles *pre, const sph_particles *post, int64_t ti,
                 int first, sph_adjoint *adj, void *stream) {
  if (!ctx || !valid_particles(ctx, pre) || !valid_particles(ctx, post) || post->n != pre->n ||
      !valid_adjoint(adj, pre->n) || ti < 0)
    return SPH_ERR_ARG;
  // the reverse pass covers the base scheme only
  if (ctx->prm.balsara || ctx->prm.predict_inactive || ctx->prm.limiter) return SPH_ERR_ARG;
  const long long n = pre->n;
  if (n == 0) return SPH_OK;
  SPH_TRY(ensure_adj(ctx));
  AdjBuffers &a = *ctx->adj;
  cudaStream_t st = S(stream);
  sph_particles W = adj_particles(a, ctx->n_max, n);
  SPH_CUDA(launch_adj_prepare(*pre, *post, W, *adj, ti, first, ctx->prm.dt_min, ctx->prm.box,
                              ctx->prm.gamma, st));
  sph_ctx *sub = a.sub;
  sub->built = false;  // the permutation of this build starts from the caller's order
  SPH_TRY(build_cells(sub, &W, st));
  View v = make_view(sub, &W);
  SPH_CUDA(launch_mark(v, 1, st));  // bin 0 (the step's active particles) is active at tick 1
  const AdjWork w = adj_work(a, ctx->n_max, sub->b.perm);
  SPH_CUDA(launch_adj_step(v, w, *pre, *post, *adj, ti, first, a.grid_pairs, st));
  SPH_TRY(read_state(sub, st));
  const DevState &h = *sub->b.h_ds;
  if (h.halt || h.first_error) {
    const int e = h.first_error ? h.first_error : SPH_ERR_CUDA;
    SPH_TRY(sph_clear_status(sub, stream));
    return e;
  }
  return SPH_OK;
}

}  // extern "C"
