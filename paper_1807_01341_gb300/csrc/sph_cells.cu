// Top-level cells and leaves (Sec. III-A of arXiv 1807.01341).
//
// Particles are binned into an n_c^3 grid whose width is at least the largest
// kernel support, so a particle only interacts with the 27 cells around its
// own.  Inside a cell the particles are ordered by the Morton code of their
// cell-relative position; the Morton order is the cell's octree, and the
// leaves are octree nodes holding at most leaf_max particles -- the GPU form
// of the paper's refinement of top-level cells into small sub-cells.  The
// (cell, Morton) keys are sorted by a stable LSD radix sort, so ties keep the
// previous particle order and the result is deterministic.
#include <algorithm>
#include <cstddef>
#include <utility>

#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// ---------------------------------------------------------------------------
// maximum smoothing length
// ---------------------------------------------------------------------------
__global__ void k_reduce_hmax(const float *__restrict__ h, long long n, unsigned int *out) {
  float m = 0.0f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, h[i]);
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomic_max_float_pos(out, m);
}

// Smallest and largest particle mass, as float bits (atomic min and max on
// the bit patterns: masses are positive, and any other value only makes the
// two differ, which selects the general density loop).
__global__ void k_mass_range(const float *__restrict__ m, long long n, unsigned int *lo_bits,
                             unsigned int *hi_bits) {
  unsigned int lo = 0xffffffffu, hi = 0u;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned int b = __float_as_uint(m[i]);
    lo = min(lo, b);
    hi = max(hi, b);
  }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(lo_bits, lo);
    atomicMax(hi_bits, hi);
  }
}

// ---------------------------------------------------------------------------
// cell keys: exact FP64 arithmetic (no contraction) so the cell of every
// particle is a function of its FP64 position alone
// ---------------------------------------------------------------------------
__device__ __forceinline__ double wrap_box(double x, double box) {
  if (x < 0.0) x = __dadd_rn(x, box);
  if (x >= box) x = __dsub_rn(x, box);
  return x;
}

__device__ __forceinline__ int axis_cell(double x, double w, int nc) {
  int c = (int)floor(__ddiv_rn(x, w));
  return c < 0 ? 0 : (c > nc - 1 ? nc - 1 : c);
}

__device__ __forceinline__ unsigned long long axis_morton(double x, int c, double w) {
  double t = __ddiv_rn(__dsub_rn(x, __dmul_rn((double)c, w)), w);
  t = __dmul_rn(t, (double)(1 << MORTON_BITS));
  double ft = floor(t);
  long long q = (long long)ft;
  if (ft < 0.0) q = 0;
  if (q > (1 << MORTON_BITS) - 1) q = (1 << MORTON_BITS) - 1;
  return (unsigned long long)q;
}

__device__ __forceinline__ unsigned long long spread3(unsigned long long v) {
  unsigned long long r = 0;
#pragma unroll
  for (int b = 0; b < MORTON_BITS; b++) r |= ((v >> b) & 1ull) << (3 * b);
  return r;
}

// (also counts in *bad the particles whose position is not finite or whose h
// is not a positive finite number: the caller rejects such input)
__global__ void k_cell_keys(View v, int nc, double w, unsigned long long *__restrict__ keys,
                            unsigned int *__restrict__ vals, unsigned int *__restrict__ bad) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const float hi = v.h[i];
  if (!(isfinite(v.x[i]) && isfinite(v.y[i]) && isfinite(v.z[i]) && hi > 0.0f && isfinite(hi)))
    atomicAdd(bad, 1u);
  double x = wrap_box(v.x[i], v.box), y = wrap_box(v.y[i], v.box), z = wrap_box(v.z[i], v.box);
  v.x[i] = x;
  v.y[i] = y;
  v.z[i] = z;
  int cx = axis_cell(x, w, nc), cy = axis_cell(y, w, nc), cz = axis_cell(z, w, nc);
  unsigned long long cid = ((unsigned long long)cx * nc + cy) * nc + cz;
  unsigned long long mort = (spread3(axis_morton(x, cx, w)) << 2) |
                            (spread3(axis_morton(y, cy, w)) << 1) | spread3(axis_morton(z, cz, w));
  keys[i] = (cid << KEY_MORTON_BITS) | mort;
  vals[i] = (unsigned int)i;
}

// ---------------------------------------------------------------------------
// block-wide exclusive scan of one value per thread (blockDim.x = SCAN_THREADS)
// ---------------------------------------------------------------------------
__device__ unsigned int block_exclusive_scan(unsigned int x, unsigned int *total) {
  __shared__ unsigned int warp_sums[32];
  __shared__ unsigned int grand_total;
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned int inc = x;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_sums[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    unsigned int s = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0u;
    unsigned int si = s;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned int y = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += y;
    }
    warp_sums[lane] = si - s;  // exclusive prefix of warp totals
    if (lane == 31) grand_total = si;
  }
  __syncthreads();
  unsigned int res = warp_sums[wid] + inc - x;
  if (total) *total = grand_total;
  __syncthreads();
  return res;
}

__global__ void k_scan_reduce(const unsigned int *in, int n,
                              unsigned int *__restrict__ block_sums) {
  long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
  unsigned int s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++)
    if (base + k < n) s += in[base + k];
  unsigned int tot;
  block_exclusive_scan(s, &tot);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void k_scan_tops(unsigned int *__restrict__ sums, int nb) {
  // one block: exclusive scan of nb <= SCAN_TILE block sums in place
  int base = threadIdx.x * SCAN_ITEMS;
  unsigned int v[SCAN_ITEMS];
  unsigned int s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    v[k] = (base + k < nb) ? sums[base + k] : 0u;
    s += v[k];
  }
  unsigned int pre = block_exclusive_scan(s, nullptr);
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    if (base + k < nb) sums[base + k] = pre;
    pre += v[k];
  }
}

// `in` and `out` may be the same array: each thread reads its items before
// the block-wide barrier and writes the same items after it.
__global__ void k_scan_down(const unsigned int *in, unsigned int *out, int n,
                            const unsigned int *__restrict__ block_sums) {
  long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
  unsigned int v[SCAN_ITEMS];
  unsigned int s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    v[k] = (base + k < n) ? in[base + k] : 0u;
    s += v[k];
  }
  unsigned int pre = block_exclusive_scan(s, nullptr) + block_sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    if (base + k < n) out[base + k] = pre;
    pre += v[k];
  }
}

// one block: exclusive scan of n <= SCAN_TILE values (in and out may coincide)
__global__ void k_scan_one(const unsigned int *in, unsigned int *out, int n) {
  const int base = threadIdx.x * SCAN_ITEMS;
  unsigned int v[SCAN_ITEMS];
  unsigned int s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    v[k] = (base + k < n) ? in[base + k] : 0u;
    s += v[k];
  }
  unsigned int pre = block_exclusive_scan(s, nullptr);
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    if (base + k < n) out[base + k] = pre;
    pre += v[k];
  }
}

// ---------------------------------------------------------------------------
// stable LSD radix sort, 8-bit digits
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(RS_THREADS)
    k_rs_hist(const unsigned long long *__restrict__ keys, int n, int shift,
              unsigned int *__restrict__ hist, int n_tiles) {
  __shared__ unsigned int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  long long base = (long long)blockIdx.x * RS_TILE;
#pragma unroll 4
  for (int r = 0; r < RS_ITEMS; r++) {
    long long idx = base + r * RS_THREADS + threadIdx.x;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(long long)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_THREADS)
    k_rs_scatter(const unsigned long long *__restrict__ keys, const unsigned int *__restrict__ vals,
                 unsigned long long *__restrict__ okeys, unsigned int *__restrict__ ovals, int n,
                 int shift, const unsigned int *__restrict__ offs, int n_tiles, DevState *ds) {
  __shared__ unsigned int base[256];
  __shared__ unsigned int goff[256];
  __shared__ unsigned int wcnt[RS_THREADS / 32][256];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  base[t] = 0;
  goff[t] = offs[(long long)t * n_tiles + blockIdx.x];
  const unsigned int lt_mask = (1u << lane) - 1u;
  long long tile = (long long)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ITEMS; r++) {
#pragma unroll
    for (int k = 0; k < RS_THREADS / 32; k++) wcnt[k][t] = 0;
    __syncthreads();
    long long idx = tile + r * RS_THREADS + t;
    bool valid = idx < n;
    unsigned long long key = valid ? keys[idx] : 0ull;
    unsigned int d = valid ? (unsigned int)((key >> shift) & 255u) : 256u + lane;
    unsigned int peers = __match_any_sync(0xffffffffu, d);
    unsigned int rank = __popc(peers & lt_mask);
    if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      unsigned int pre = base[d];
      for (int k = 0; k < warp; k++) pre += wcnt[k][d];
      unsigned int pos = goff[d] + pre + rank;
      if (SPH_IN(ds, pos, n, SPH_CHECK_SCATTER)) {
        okeys[pos] = key;
        ovals[pos] = vals[idx];
      }
    }
    __syncthreads();
    unsigned int s = 0;
#pragma unroll
    for (int k = 0; k < RS_THREADS / 32; k++) s += wcnt[k][t];
    base[t] += s;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// gather
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_gather(T *__restrict__ dst, const T *__restrict__ src,
                         const unsigned int *__restrict__ idx, long long n, DevState *ds) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k < n) {
    const unsigned int s = idx[k];
    if (SPH_IN(ds, s, n, SPH_CHECK_SCATTER)) dst[k] = src[s];
  }
}

// ---------------------------------------------------------------------------
// cell boundaries and leaves
// ---------------------------------------------------------------------------
__global__ void k_cell_start(const unsigned long long *__restrict__ keys, long long n, int n_cells,
                             int32_t *__restrict__ cell_start, int32_t *__restrict__ pcell) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= n) return;
  int c = (int)(keys[k] >> KEY_MORTON_BITS);
  pcell[k] = c;
  int cp = (k > 0) ? (int)(keys[k - 1] >> KEY_MORTON_BITS) : -1;
  for (int cc = cp + 1; cc <= c; cc++) cell_start[cc] = (int32_t)k;
  if (k == n - 1)
    for (int cc = c + 1; cc <= n_cells; cc++) cell_start[cc] = (int32_t)n;
}

__device__ __forceinline__ unsigned int child_of(unsigned long long key, int shift) {
  return (unsigned int)((key >> shift) & 7ull);
}

__device__ __forceinline__ uint32_t compact3(unsigned long long m) {
  uint32_t r = 0;
#pragma unroll
  for (int b = 0; b < MORTON_BITS; b++) r |= (uint32_t)((m >> (3 * b)) & 1ull) << b;
  return r;
}

// Morton-grid corner (packed kx | ky << 10 | kz << 20) of a particle's code,
// truncated to the octree level of its node
__device__ __forceinline__ uint32_t corner_of(unsigned long long key, int level) {
  const unsigned long long m = key & ((1ull << KEY_MORTON_BITS) - 1ull);
  const int drop = 3 * (MORTON_BITS - level);
  const unsigned long long t = drop >= KEY_MORTON_BITS ? 0ull : (m >> drop) << drop;
  return compact3(t >> 2) | (compact3(t >> 1) << 10) | (compact3(t) << 20);
}

// Leaves: the octree of each cell's Morton-ordered particles, split level by
// level.  A node holding more than leaf_max particles is split into its 8
// children; consecutive children that hold at most leaf_max particles between
// them are merged into one leaf (siblings, so the leaf stays inside the parent
// node), and larger children are split at the next level.  At the deepest
// level a node is cut into runs of leaf_max.  Every leaf is marked at its
// first particle by lead[s] = 1 + the level of the node it lies in; the marks,
// compacted in particle order, give the leaves cell by cell in the order of a
// depth-first walk.  All particles of a leaf share the Morton prefix of that
// level, so its corner follows from the first particle's code.

// Level 0: each cell is one node; a cell of at most leaf_max particles is a leaf.
__global__ void k_leaf_cells(const int32_t *__restrict__ cell_start, int n_cells, int leaf_max,
                             uint8_t *__restrict__ lead, int2 *__restrict__ nodes,
                             unsigned int *__restrict__ n_nodes, unsigned int cap) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  const int a = cell_start[c], b = cell_start[c + 1];
  if (b <= a) return;
  if (b - a <= leaf_max) {
    lead[a] = 1;
    return;
  }
  const unsigned int slot = atomicAdd(n_nodes, 1u);
  if (slot < cap) nodes[slot] = make_int2(a, b);  // nodes of >= 2 particles: cap = n/2 suffices
}

// One level: 8 lanes per node.  Lane k (1..7) finds the first particle of
// child k by binary search; lane 0 merges runs of small siblings, marks their
// leaves and queues the large children for the next level.
__global__ void __launch_bounds__(256)
k_leaf_level(const unsigned long long *__restrict__ keys, int level, int leaf_max,
             const int2 *__restrict__ nodes, const unsigned int *__restrict__ n_nodes,
             int2 *__restrict__ next, unsigned int *__restrict__ n_next, unsigned int cap,
             uint8_t *__restrict__ lead) {
  const unsigned int cnt = *n_nodes;
  const int lane = threadIdx.x & 31, k = lane & 7;
  const unsigned int gmask = 0xFFu << (lane & 24);
  const int shift = 3 * (MORTON_BITS - 1 - level);
  const unsigned int stride = (gridDim.x * blockDim.x) >> 3;
  for (unsigned int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 3; i < min(cnt, cap);
       i += stride) {
    const int2 nd = nodes[i];
    int lo = nd.x, hi = nd.y;
    if (k > 0) {
      // first index in [a, b) whose child digit is >= k
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (child_of(keys[mid], shift) < (unsigned int)k) lo = mid + 1;
        else hi = mid;
      }
    }
    int bnd[9];
#pragma unroll
    for (int j = 0; j < 8; j++) bnd[j] = __shfl_sync(gmask, lo, j, 8);
    bnd[0] = nd.x;
    bnd[8] = nd.y;
    if (k != 0) continue;
    for (int j = 0; j < 8;) {
      const int c = bnd[j + 1] - bnd[j];
      if (c == 0) {
        j++;
        continue;
      }
      if (c > leaf_max) {
        if (level + 1 == MORTON_BITS) {
          for (int s = bnd[j]; s < bnd[j + 1]; s += leaf_max) lead[s] = (uint8_t)(MORTON_BITS + 1);
        } else {
          const unsigned int slot = atomicAdd(n_next, 1u);
          if (slot < cap) next[slot] = make_int2(bnd[j], bnd[j + 1]);
        }
        j++;
        continue;
      }
      int j2 = j + 1, sum = c;
      while (j2 < 8 && sum + (bnd[j2 + 1] - bnd[j2]) <= leaf_max) {
        sum += bnd[j2 + 1] - bnd[j2];
        j2++;
      }
      lead[bnd[j]] = (uint8_t)(level + 1);
      j = j2;
    }
  }
}

__device__ __forceinline__ void load_lead(const uint8_t *__restrict__ lead, long long base,
                                          long long n, uint8_t l[SCAN_ITEMS]) {
  if (base + SCAN_ITEMS <= n) {
    const uchar4 q = *reinterpret_cast<const uchar4 *>(lead + base);
    l[0] = q.x; l[1] = q.y; l[2] = q.z; l[3] = q.w;
  } else {
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) l[k] = base + k < n ? lead[base + k] : (uint8_t)0;
  }
}

// leaves per tile of SCAN_TILE particles; tile_cnt[n_tiles] = 0 closes the scan
__global__ void __launch_bounds__(SCAN_THREADS)
k_leaf_tiles(const uint8_t *__restrict__ lead, long long n, unsigned int *__restrict__ tile_cnt,
             int n_tiles) {
  static_assert(SCAN_ITEMS == 4, "lead bytes are read as uchar4");
  uint8_t l[SCAN_ITEMS];
  load_lead(lead, (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS, n, l);
  unsigned int s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) s += l[k] != 0;
  unsigned int tot;
  block_exclusive_scan(s, &tot);
  if (threadIdx.x == 0) {
    tile_cnt[blockIdx.x] = tot;
    if (blockIdx.x == 0) tile_cnt[n_tiles] = 0u;
  }
}

// compaction of the marks: leaf records, first leaf of every cell, closing entry
__global__ void __launch_bounds__(SCAN_THREADS)
k_leaf_emit(const unsigned long long *__restrict__ keys, const uint8_t *__restrict__ lead,
            long long n, int n_cells, const unsigned int *__restrict__ tile_off,
            int32_t *__restrict__ leaf_start, int32_t *__restrict__ leaf_cell,
            uint32_t *__restrict__ leaf_k, int32_t *__restrict__ cell_leaf_start) {
  const long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
  uint8_t l[SCAN_ITEMS];
  load_lead(lead, base, n, l);
  unsigned int s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) s += l[k] != 0;
  unsigned int off = block_exclusive_scan(s, nullptr) + tile_off[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    const long long i = base + k;
    if (i >= n) break;
    if (l[k]) {
      const unsigned long long key = keys[i];
      const int c = (int)(key >> KEY_MORTON_BITS);
      leaf_start[off] = (int32_t)i;
      leaf_cell[off] = c;
      leaf_k[off] = corner_of(key, l[k] - 1);
      // the first particle of a cell always starts a leaf
      const int cp = i > 0 ? (int)(keys[i - 1] >> KEY_MORTON_BITS) : -1;
      for (int cc = cp + 1; cc <= c; cc++) cell_leaf_start[cc] = (int32_t)off;
      off++;
    }
    if (i == n - 1) {
      for (int cc = (int)(keys[i] >> KEY_MORTON_BITS) + 1; cc <= n_cells; cc++)
        cell_leaf_start[cc] = (int32_t)off;
      leaf_start[off] = (int32_t)n;
    }
  }
}

__global__ void k_bin_hist(const int8_t *__restrict__ bin, long long n, int *__restrict__ out) {
  __shared__ int h[MAX_BINS];
  if (threadIdx.x < MAX_BINS) h[threadIdx.x] = 0;
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    atomicAdd(&h[bin[i] & (MAX_BINS - 1)], 1);
  __syncthreads();
  if (threadIdx.x < MAX_BINS && h[threadIdx.x]) atomicAdd(&out[threadIdx.x], h[threadIdx.x]);
}

// Chunks: the leaves of a cell placed in the cell's octree by the Morton code
// of their first particles and split as the particles are split into leaves
// (k_leaf_cells, k_leaf_level), with CHUNK leaves in place of leaf_max
// particles.  A chunk is then an octree node (or a run of consecutive sibling
// nodes) holding at most CHUNK leaves, so its box stays compact; runs of CHUNK
// consecutive leaves in Morton order can straddle the boundary of a large
// node and span a box far wider than their leaves.
__global__ void k_leaf_keys(const unsigned long long *__restrict__ keys,
                            const int32_t *__restrict__ leaf_start, int n_leaves,
                            unsigned long long *__restrict__ leaf_keys) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < n_leaves) leaf_keys[l] = keys[leaf_start[l]];
}

// leaf -> chunk, one thread per chunk (at most n_leaves of them)
__global__ void k_leaf_chunk(const int32_t *__restrict__ chunk_leaf_start,
                             const unsigned int *__restrict__ n_chunks, int n_leaves,
                             int32_t *__restrict__ leaf_chunk) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (int)*n_chunks) return;
  const int a = chunk_leaf_start[g], b = min(chunk_leaf_start[g + 1], n_leaves);
  for (int l = a; l < b; l++) leaf_chunk[l] = g;
}

// Work groups: the leaves of a cell taken in order, a new group whenever the
// next leaf would bring the group above WG_MAX particles.
__global__ void k_group_count(const int32_t *__restrict__ cell_leaf_start,
                              const int32_t *__restrict__ leaf_start, int n_cells,
                              unsigned int *__restrict__ counts) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c > n_cells) return;
  if (c == n_cells) {
    counts[c] = 0;
    return;
  }
  unsigned int ng = 0;
  int cur = 0;
  for (int l = cell_leaf_start[c]; l < cell_leaf_start[c + 1]; l++) {
    const int cl = leaf_start[l + 1] - leaf_start[l];
    if (ng == 0 || cur + cl > WG_MAX) {
      ng++;
      cur = 0;
    }
    cur += cl;
  }
  counts[c] = ng;
}

__global__ void k_group_write(const int32_t *__restrict__ cell_leaf_start,
                              const int32_t *__restrict__ leaf_start, int n_cells,
                              const unsigned int *__restrict__ offsets,
                              int32_t *__restrict__ group_leaf0, int32_t *__restrict__ group_cell,
                              int n_leaves) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c > n_cells) return;
  if (c == n_cells) {
    group_leaf0[offsets[c]] = n_leaves;
    return;
  }
  unsigned int g = offsets[c];
  int cur = 0;
  bool first = true;
  for (int l = cell_leaf_start[c]; l < cell_leaf_start[c + 1]; l++) {
    const int cl = leaf_start[l + 1] - leaf_start[l];
    if (first || cur + cl > WG_MAX) {
      if (!first) g++;
      group_leaf0[g] = l;
      group_cell[g] = c;
      cur = 0;
      first = false;
    }
    cur += cl;
  }
}

__global__ void k_leaf_pleaf(const int32_t *__restrict__ leaf_start, int n_leaves,
                             int32_t *__restrict__ pleaf) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n_leaves) return;
  for (int i = leaf_start[l]; i < leaf_start[l + 1]; i++) pleaf[i] = l;
}

inline int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_reduce_hmax(const View &v, float *out_max, cudaStream_t st) {
  note_launches(1);
  cudaError_t e = cudaMemsetAsync(out_max, 0, sizeof(float), st);
  if (e != cudaSuccess) return e;
  int blocks = (int)std::min<long long>(1024, std::max<long long>(1, (v.n + 255) / 256));
  k_reduce_hmax<<<blocks, 256, 0, st>>>(v.h, v.n, reinterpret_cast<unsigned int *>(out_max));
  return cudaGetLastError();
}

cudaError_t launch_mass_range(const View &v, cudaStream_t st) {
  note_launches(1);
  cudaError_t e = cudaMemsetAsync(SPH_DS_FIELD(v.ds, m_lo_bits), 0xff, sizeof(unsigned int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(SPH_DS_FIELD(v.ds, m_hi_bits), 0, sizeof(unsigned int), st);
  if (e != cudaSuccess || v.n == 0) return e;
  const int blocks = (int)std::min<long long>(v.grid_util, (v.n + 255) / 256);
  k_mass_range<<<blocks, 256, 0, st>>>(v.m, v.n, SPH_DS_FIELD(v.ds, m_lo_bits),
                                       SPH_DS_FIELD(v.ds, m_hi_bits));
  return cudaGetLastError();
}

cudaError_t launch_cell_keys(const View &v, int nc, double w, unsigned long long *keys,
                             unsigned int *vals, unsigned int *bad, cudaStream_t st) {
  note_launches(1);
  if (v.n == 0) return cudaSuccess;
  k_cell_keys<<<blocks_for(v.n, 256), 256, 0, st>>>(v, nc, w, keys, vals, bad);
  return cudaGetLastError();
}

cudaError_t exclusive_scan_u32(const unsigned int *in, unsigned int *out, int n,
                               unsigned int *tmp, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nb > SCAN_TILE) return cudaErrorInvalidValue;
  if (nb == 1) {  // one tile: a single launch
    note_launches(1);
    k_scan_one<<<1, SCAN_THREADS, 0, st>>>(in, out, n);
    return cudaGetLastError();
  }
  note_launches(3);
  k_scan_reduce<<<nb, SCAN_THREADS, 0, st>>>(in, n, tmp);
  k_scan_tops<<<1, SCAN_THREADS, 0, st>>>(tmp, nb);
  k_scan_down<<<nb, SCAN_THREADS, 0, st>>>(in, out, n, tmp);
  return cudaGetLastError();
}

cudaError_t radix_sort_pairs(unsigned long long *keys, unsigned int *vals,
                             unsigned long long *keys_alt, unsigned int *vals_alt, int n,
                             int nbits, unsigned int *hist, unsigned int *scan_tmp,
                             int n_hist_max, bool *result_in_alt, cudaStream_t st, DevState *ds) {
  *result_in_alt = false;
  if (n <= 1) return cudaSuccess;
  int n_tiles = (n + RS_TILE - 1) / RS_TILE;
  if (256LL * n_tiles > n_hist_max) return cudaErrorInvalidValue;
  unsigned long long *ka = keys, *kb = keys_alt;
  unsigned int *va = vals, *vb = vals_alt;
  for (int shift = 0; shift < nbits; shift += 8) {
    note_launches(2);
    k_rs_hist<<<n_tiles, RS_THREADS, 0, st>>>(ka, n, shift, hist, n_tiles);
    cudaError_t e = exclusive_scan_u32(hist, hist, 256 * n_tiles, scan_tmp, st);
    if (e != cudaSuccess) return e;
    k_rs_scatter<<<n_tiles, RS_THREADS, 0, st>>>(ka, va, kb, vb, n, shift, hist, n_tiles, ds);
    std::swap(ka, kb);
    std::swap(va, vb);
    *result_in_alt = !*result_in_alt;
  }
  return cudaGetLastError();
}

cudaError_t launch_gather(void *dst, const void *src, const unsigned int *idx, long long n,
                          int elem_bytes, cudaStream_t st, DevState *ds) {
  note_launches(1);
  if (n == 0) return cudaSuccess;
  int b = blocks_for(n, 256);
  switch (elem_bytes) {
    case 1: k_gather<uint8_t><<<b, 256, 0, st>>>((uint8_t *)dst, (const uint8_t *)src, idx, n, ds); break;
    case 4: k_gather<uint32_t><<<b, 256, 0, st>>>((uint32_t *)dst, (const uint32_t *)src, idx, n, ds); break;
    case 8: k_gather<unsigned long long><<<b, 256, 0, st>>>((unsigned long long *)dst,
                                                          (const unsigned long long *)src, idx, n, ds); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_cell_start(const unsigned long long *sorted_keys, long long n, int n_cells,
                              int32_t *cell_start, int32_t *pcell, cudaStream_t st) {
  note_launches(1);
  if (n == 0) return cudaMemsetAsync(cell_start, 0, sizeof(int32_t) * (n_cells + 1), st);
  k_cell_start<<<blocks_for(n, 256), 256, 0, st>>>(sorted_keys, n, n_cells, cell_start, pcell);
  return cudaGetLastError();
}

cudaError_t launch_leaves(const unsigned long long *sorted_keys, const int32_t *cell_start,
                          int n_cells, long long n, int leaf_max, uint8_t *lead, int2 *nodes,
                          unsigned int *work, unsigned int *scan_tmp, int32_t *leaf_start,
                          int32_t *leaf_cell, uint32_t *leaf_k, int32_t *cell_leaf_start,
                          int grid, const unsigned int **n_leaves, cudaStream_t st) {
  const long long n_tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  unsigned int *tile_cnt = work, *n_nodes = work + n_tiles + 1;
  *n_leaves = tile_cnt + n_tiles;
  if (n == 0) {
    cudaError_t e = cudaMemsetAsync(cell_leaf_start, 0, sizeof(int32_t) * (n_cells + 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(leaf_start, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(tile_cnt, 0, sizeof(unsigned int), st);
    return e;
  }
  if (n_tiles > SCAN_TILE) return cudaErrorInvalidValue;
  const unsigned int cap = (unsigned int)(n / 2);
  int2 *list[2] = {nodes, nodes + cap};
  cudaError_t e = cudaMemsetAsync(lead, 0, (size_t)n, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(n_nodes, 0, sizeof(unsigned int) * MORTON_BITS, st);
  if (e != cudaSuccess) return e;
  note_launches(1 + MORTON_BITS + 2);
  k_leaf_cells<<<blocks_for(n_cells, 128), 128, 0, st>>>(cell_start, n_cells, leaf_max, lead,
                                                          list[0], n_nodes, cap);
  for (int L = 0; L < MORTON_BITS; L++) {
    unsigned int *n_next = L + 1 < MORTON_BITS ? n_nodes + L + 1 : n_nodes;  // unused at the last level
    k_leaf_level<<<grid, 256, 0, st>>>(sorted_keys, L, leaf_max, list[L & 1], n_nodes + L,
                                        list[(L + 1) & 1], n_next, cap, lead);
  }
  k_leaf_tiles<<<(int)n_tiles, SCAN_THREADS, 0, st>>>(lead, n, tile_cnt, (int)n_tiles);
  e = exclusive_scan_u32(tile_cnt, tile_cnt, (int)n_tiles + 1, scan_tmp, st);
  if (e != cudaSuccess) return e;
  k_leaf_emit<<<(int)n_tiles, SCAN_THREADS, 0, st>>>(sorted_keys, lead, n, n_cells, tile_cnt,
                                                     leaf_start, leaf_cell, leaf_k,
                                                     cell_leaf_start);
  return cudaGetLastError();
}

// Chunks: octree nodes of at most CHUNK leaves (k_leaf_keys), numbered cell by
// cell; the leaf build's kernels run over the leaves' first keys.  `nodes`
// holds n_leaves int2, `lead` n_leaves bytes, `corner_tmp` n_leaves words
// (written, unused), `work` the counters of launch_leaves.
cudaError_t launch_chunks(const unsigned long long *sorted_keys, const int32_t *leaf_start,
                          const int32_t *cell_leaf_start, int n_cells, int n_leaves,
                          unsigned long long *leaf_keys, uint8_t *lead, int2 *nodes,
                          unsigned int *work, unsigned int *scan_tmp, uint32_t *corner_tmp,
                          int32_t *chunk_leaf_start, int32_t *chunk_cell,
                          int32_t *cell_chunk_start, int32_t *leaf_chunk, int grid,
                          const unsigned int **n_chunks, cudaStream_t st) {
  if (n_leaves > 0) {
    note_launches(1);
    k_leaf_keys<<<blocks_for(n_leaves, 256), 256, 0, st>>>(sorted_keys, leaf_start, n_leaves,
                                                            leaf_keys);
  }
  cudaError_t e = launch_leaves(leaf_keys, cell_leaf_start, n_cells, n_leaves, CHUNK, lead, nodes,
                                work, scan_tmp, chunk_leaf_start, chunk_cell, corner_tmp,
                                cell_chunk_start, grid, n_chunks, st);
  if (e != cudaSuccess || n_leaves == 0) return e;
  note_launches(1);
  k_leaf_chunk<<<blocks_for(n_leaves, 256), 256, 0, st>>>(chunk_leaf_start, *n_chunks, n_leaves,
                                                           leaf_chunk);
  return cudaGetLastError();
}

cudaError_t launch_groups(const int32_t *cell_leaf_start, const int32_t *leaf_start, int n_cells,
                          int n_leaves_max, unsigned int *counts, unsigned int *offsets,
                          unsigned int *scan_tmp, int32_t *group_leaf0, int32_t *group_cell,
                          int32_t *pleaf, int n_leaves_host, cudaStream_t st) {
  (void)n_leaves_max;
  note_launches(3);
  k_group_count<<<blocks_for(n_cells + 1, 128), 128, 0, st>>>(cell_leaf_start, leaf_start, n_cells,
                                                               counts);
  cudaError_t e = exclusive_scan_u32(counts, offsets, n_cells + 1, scan_tmp, st);
  if (e != cudaSuccess) return e;
  k_group_write<<<blocks_for(n_cells + 1, 128), 128, 0, st>>>(cell_leaf_start, leaf_start, n_cells,
                                                               offsets, group_leaf0, group_cell,
                                                               n_leaves_host);
  if (n_leaves_host > 0)
    k_leaf_pleaf<<<blocks_for(n_leaves_host, 256), 256, 0, st>>>(leaf_start, n_leaves_host, pleaf);
  return cudaGetLastError();
}

cudaError_t launch_bin_histogram(const View &v, cudaStream_t st) {
  note_launches(1);
  int *counts = reinterpret_cast<int *>(reinterpret_cast<char *>(v.ds) +
                                         offsetof(DevState, bin_count));
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int) * MAX_BINS, st);
  if (e != cudaSuccess || v.n == 0) return e;
  int blocks = (int)std::min<long long>(1024, (v.n + 255) / 256);
  k_bin_hist<<<blocks, 256, 0, st>>>(v.bin, v.n, counts);
  return cudaGetLastError();
}

}  // namespace sph
