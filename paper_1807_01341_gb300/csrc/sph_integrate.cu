// Time integration around the pair loops (Sec. II-A and Sec. III-D of
// arXiv 1807.01341): the active set of the current tick, the cells that must
// be drifted (active cells and their neighbours), the drift with prediction of
// v and A, the two half-kicks, the CFL time step (Eq. 1) and the power-of-two
// time bins (Eq. 2) with the synchronisation of bin increases.
//
// All kernels read their sizes and the current tick from the device-resident
// DevState and loop grid-stride, so the same launches serve every step and a
// captured CUDA graph stays valid.
#include <climits>
#include <cstddef>

#include <cfloat>

#include "sph_internal.cuh"
#include "sph_diag.cuh"

namespace sph {

namespace {

constexpr int UT = 256;  // threads per block of the utility kernels

__device__ __forceinline__ int gwarp() { return (blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ int nwarps() { return (gridDim.x * blockDim.x) >> 5; }
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// ---------------------------------------------------------------------------
// active set
// ---------------------------------------------------------------------------

// Clears `active` for the previous step's active leaves (their queue is still
// in place), then starts the step: current tick, largest active bin, epoch,
// empty queues.
// (one thread per leaf: a leaf holds at most 32 particles)
__global__ void k_mark_clear(View v) {
  DevState *ds = v.ds;
  const int nq = ds->n_active_leaves;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nq; k += gridDim.x * blockDim.x) {
    const int leaf = v.q_active[k];
    if (!SPH_IN(ds, leaf, ds->n_leaves, SPH_CHECK_ACTIVE_LEAF)) continue;
    const int a = v.leaf_start[leaf], b = v.leaf_start[leaf + 1];
    for (int i = a; i < b; i++) v.active[i] = 0;
  }
}

__global__ void k_begin_step(View v, long long ti_arg) {
  DevState *ds = v.ds;
  long long ti = ti_arg >= 0 ? ti_arg : ds->ti_next;
  ds->ti = ti;
  ds->m_act = max_active_bin(ti);
  ds->epoch += 1u;
  ds->n_active_leaves = 0;
  ds->n_active_cells = 0;
  ds->n_drift_chunks = 0;
  ds->n_bin_groups = 0;
  ds->n_active_groups = 0;
  ds->n_heavy_groups = 0;
  ds->head_density = ds->head_force = ds->head_drift = ds->head_kick = 0;
  ds->head_open = ds->head_bins = ds->head_misc = 0;
  ds->head_coop_force = ds->head_grad = 0;
  ds->n_wake = 0;
  ds->s_pairs_density = ds->s_pairs_force = 0ull;
  ds->s_cand_density = ds->s_cand_force = 0ull;
  ds->s_iters_density = ds->s_active_particles = 0ull;
  ds->s_gathers_density = ds->s_list_overflows = ds->s_evals_density = 0ull;
}

// One thread per leaf: a leaf holds active particles when its smallest bin is
// active.  Queues the leaf, and the first leaf of each cell queues the cell.
__global__ void k_mark_leaves(View v) {
  DevState *ds = v.ds;
  const int nl = ds->n_leaves, m_act = ds->m_act;
  const unsigned int epoch = ds->epoch;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += gridDim.x * blockDim.x) {
    if ((int)v.leaf_min_bin[l] > m_act) continue;
    v.q_active[atomicAdd(&ds->n_active_leaves, 1)] = l;
    int c = v.leaf_cell[l];
    if (atomicExch(&v.cell_stamp[c], epoch) != epoch)
      v.q_act_cells[atomicAdd(&ds->n_active_cells, 1)] = c;
  }
}

// One thread per work group: queues the groups whose smallest bin is active,
// the heavy ones (estimated cost above heavy_factor times the mean) apart so
// that the pair loops start them first.
// (blocks [b0, b0 + nb) of the launch take this task)
__device__ void mark_groups_part(View &v, int b0, int nb) {
  DevState *ds = v.ds;
  const int ng = ds->n_groups, m_act = ds->m_act;
  const unsigned long long csum = ds->group_cost_sum;
  const int t0 = ((int)blockIdx.x - b0) * blockDim.x + threadIdx.x, nt = nb * blockDim.x;
  const int lane = lane_id();
  const unsigned below = (1u << lane) - 1u;
  // (the same trip count in every lane of a warp: one queue atomic per warp)
  for (int gb = t0 - lane; gb < ng; gb += nt) {
    const int g = gb + lane;
    bool act = false, heavy = false;
    if (g < ng) {
      int mb = 127;
      for (int l = v.group_leaf0[g]; l < v.group_leaf0[g + 1]; l++)
        mb = min(mb, (int)v.leaf_min_bin[l]);
      act = mb <= m_act;
      heavy = act && v.heavy_factor > 0.0 &&
              (double)v.group_cost[g] * (double)ng > v.heavy_factor * (double)csum;
    }
    const unsigned mh = __ballot_sync(0xffffffffu, heavy);
    const unsigned mw = __ballot_sync(0xffffffffu, act && !heavy);
    int bh = 0, bw = 0;
    if (lane == 0) {
      if (mh) bh = atomicAdd(&ds->n_heavy_groups, __popc(mh));
      if (mw) bw = atomicAdd(&ds->n_active_groups, __popc(mw));
    }
    bh = __shfl_sync(0xffffffffu, bh, 0);
    bw = __shfl_sync(0xffffffffu, bw, 0);
    if (heavy) v.q_group[ng - 1 - (bh + __popc(mh & below))] = g;
    else if (act) v.q_group[bw + __popc(mw & below)] = g;
  }
}

// One thread per active leaf (at most 32 particles): writes `active` for its
// particles; the active count goes to the device state once per warp.
__device__ void mark_particles_part(View &v, int b0, int nb) {
  DevState *ds = v.ds;
  const int nq = ds->n_active_leaves, m_act = ds->m_act;
  const int t0 = ((int)blockIdx.x - b0) * blockDim.x + threadIdx.x, nt = nb * blockDim.x;
  unsigned long long cnt = 0;
  for (int k = t0; k < nq; k += nt) {
    const int leaf = v.q_active[k];
    if (!SPH_IN(ds, leaf, ds->n_leaves, SPH_CHECK_ACTIVE_LEAF)) continue;
    const int a = v.leaf_start[leaf], b = v.leaf_start[leaf + 1];
    for (int i = a; i < b; i++) {
      const bool act = (int)v.bin[i] <= m_act;
      v.active[i] = act ? 1 : 0;
      cnt += act ? 1ull : 0ull;
    }
  }
  for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane_id() == 0 && cnt) atomicAdd(&ds->s_active_particles, cnt);
}

// One thread per (active cell, neighbour offset): queues the leaf chunks of
// every cell next to an active cell that is not queued yet (Sec. III-D: only
// these particles can be neighbours of an active particle and need drifting).
__device__ void relevant_part(View &v, int b0, int nb) {
  DevState *ds = v.ds;
  const int nq = ds->n_active_cells * 27, nc = ds->nc;
  const unsigned int epoch = ds->epoch;
  const int t0 = ((int)blockIdx.x - b0) * blockDim.x + threadIdx.x, nt = nb * blockDim.x;
  for (int k = t0; k < nq; k += nt) {
    const int c = v.q_act_cells[k / 27], o = k % 27;
    const int dx = o / 9 - 1, dy = (o / 3) % 3 - 1, dz = o % 3 - 1;
    const int cx = c / (nc * nc), cy = (c / nc) % nc, cz = c % nc;
    const int cc = (wrap_cell(cx + dx, nc) * nc + wrap_cell(cy + dy, nc)) * nc + wrap_cell(cz + dz, nc);
    if (atomicExch(&v.cell_rel_stamp[cc], epoch) == epoch) continue;
    const int g0 = v.cell_chunk_start[cc], g1 = v.cell_chunk_start[cc + 1];
    if (g1 <= g0) continue;
    const int pos = atomicAdd(&ds->n_drift_chunks, g1 - g0);
    for (int t = 0; t < g1 - g0; t++) v.q_drift[pos + t] = g0 + t;
  }
}

// ---------------------------------------------------------------------------
// drift / refresh of one leaf (one warp)
// ---------------------------------------------------------------------------
// x - g wq (g: a corner's index on the box-wide grid of step wq) rounded
// once, then to FP32, as the periodic image nearest the corner
__device__ __forceinline__ float leaf_rel(double x, int g, double wq, double box, float hbox) {
  double d = fma(-(double)g, wq, x);
  float f = (float)d;
  if (fabsf(f) > hbox) {  // (only across the periodic boundary)
    d -= copysign(box, d);
    f = (float)d;
  }
  return f;
}

__device__ __forceinline__ double wrap_pos(double x, double box) {
  if (x < 0.0) x += box;
  if (x >= box) x -= box;
  return x;
}

// wrap_pos with the test done on the bit patterns (no FP64 instruction in the
// common case): x is outside [0, box) exactly when its sign bit is set or,
// for positive x, its bits order at or above box's
__device__ __forceinline__ double wrap_pos_fast(double x, double box) {
  const long long xb = __double_as_longlong(x);
  return (xb < 0 || xb >= __double_as_longlong(box)) ? wrap_pos(x, box) : x;
}

// One block per chunk (up to CHUNK leaves of one cell, contiguous particles):
// its threads drift (when do_drift) the chunk's particles to the current tick,
// predict v and A at that tick, refresh the FP32 records the pair loops read
// (positions relative to each particle's leaf corner) and give inactive
// particles P and c from their frozen density and predicted entropy -- a
// chunk of a dense clump holds up to CHUNK * leaf_max particles, a few rounds
// of the block -- keeping each particle's position record and bin in shared
// memory; then each warp reduces whole leaves (one particle per lane) to the
// leaf's bounding box and largest support (and, when do_bins, its smallest
// bin and bin mask), and the first warp combines the leaves into the chunk's
// box in the cell frame.  Min and max are exact, so the boxes do not depend
// on the order of the reduction.  Called by every thread of the block.
constexpr int CHUNK_PARTICLES = CHUNK * WG_MAX;  // leaf_max <= WG_MAX
static_assert(WG_MAX == 32, "one lane per particle of a leaf");

__device__ void chunk_update(const View &v, int g, bool do_drift, bool do_bins) {
  __shared__ float s_exc[UT / 32];
  __shared__ float4 s_rec[CHUNK_PARTICLES];  // leaf-frame position and support
  __shared__ uint8_t s_bin[CHUNK_PARTICLES];
  __shared__ float4 s_lo[CHUNK], s_hi[CHUNK];  // leaf boxes in the cell frame (w: largest H)
  const DevState *ds = v.ds;
  const int lane = lane_id(), warp = threadIdx.x >> 5;
  const int cell = v.chunk_cell[g];
  const int l0 = v.chunk_leaf_start[g];
  const int l1 = min(v.chunk_leaf_start[g + 1], l0 + CHUNK);  // (at most CHUNK by construction)
  const int pa = v.leaf_start[l0], pb = v.leaf_start[l1];
  const int nc = ds->nc;
  const double w = ds->w;
  const long long ti = ds->ti;
  const int cx = cell / (nc * nc), cy = (cell / nc) % nc, cz = cell % nc;
  const double wq = w / (double)(1 << MORTON_BITS);
  const float wf = (float)w, wqf = (float)wq, hbox = (float)(0.5 * v.box);
  const int gcx = cx << MORTON_BITS, gcy = cy << MORTON_BITS, gcz = cz << MORTON_BITS;
  const float g_ = (float)v.gamma;
  float exc = 0.0f;
  // phase 1: particles, coalesced
  for (int i = pa + (int)threadIdx.x; i < pb; i += (int)blockDim.x) {
    double x = v.x[i], y = v.y[i], z = v.z[i];
    if (do_drift) {
      const long long td = v.ti_drift[i];
      if (td != ti) {
        const double dt = (double)(ti - td) * v.dt_min;
        x = wrap_pos_fast(x + (double)v.vx[i] * dt, v.box);
        y = wrap_pos_fast(y + (double)v.vy[i] * dt, v.box);
        z = wrap_pos_fast(z + (double)v.vz[i] * dt, v.box);
        v.x[i] = x;
        v.y[i] = y;
        v.z[i] = z;
        v.ti_drift[i] = ti;
      }
    }
    // position relative to the leaf corner (the periodic image nearest it).
    // FP64 runs at 1/64 of the FP32 rate on this GPU and bounds this pass,
    // so the only FP64 step is one fused multiply-add from the corner's
    // index on the box-wide Morton grid (one rounding).
    const uint32_t lk = v.leaf_k[v.pleaf[i]];
    const int kx = leaf_kx(lk), ky = leaf_ky(lk), kz = leaf_kz(lk);
    const float fx = leaf_rel(x, gcx + kx, wq, v.box, hbox);
    const float fy = leaf_rel(y, gcy + ky, wq, v.box, hbox);
    const float fz = leaf_rel(z, gcz + kz, wq, v.box, hbox);
    // distance outside the particle's cell (the rebuild criterion), in FP32
    // (the bound is padded by 1e-6 of the cell width below)
    const float ex = fx + (float)kx * wqf, ey = fy + (float)ky * wqf, ez = fz + (float)kz * wqf;
    exc = fmaxf(exc, fmaxf(fmaxf(fmaxf(-ex, ex - wf), fmaxf(-ey, ey - wf)), fmaxf(-ez, ez - wf)));
    const int bi = v.bin[i] & (MAX_BINS - 1);
    // (the middle of the particle's step: its length is 2^bin, or shorter once
    // the limiter woke it)
    const double dtp =
        ((double)(ti - v.ti_begin[i]) - 0.5 * (double)(v.ti_end[i] - v.ti_begin[i])) * v.dt_min;
    const float fdtp = (float)dtp;
    const float vpx = v.vx[i] + v.ax[i] * fdtp;
    const float vpy = v.vy[i] + v.ay[i] * fdtp;
    const float vpz = v.vz[i] + v.az[i] * fdtp;
    const float Ap = v.A[i] + v.Adot[i] * fdtp;  // (as the density loop predicts it)
    float hh = v.h[i], rho = v.rho[i];
    if (v.predict) {
      // Gadget-2 prediction from the last density (at the start of the step):
      // rho exp(-div v dt), h exp(div v dt / 3)
      const float x = v.div_v[i] * (float)((double)(ti - v.ti_begin[i]) * v.dt_min);
      rho *= expf(-x);
      hh *= expf(x * (1.0f / 3.0f));
    }
    const float H = GAMMA_K * hh, m = v.m[i];
    v.rec_xm[i] = make_float4(fx, fy, fz, m);
    v.rec_xH[i] = make_float4(fx, fy, fz, H);
    v.rec_v[i] = make_float4(vpx, vpy, vpz, m);
    s_rec[i - pa] = make_float4(fx, fy, fz, H);
    s_bin[i - pa] = (uint8_t)bi;
    float fP = 0.0f, c = 0.0f;
    if (rho > 0.0f) {
      const float P = Ap * powf(rho, g_);
      c = sqrtf(g_ * P / rho);
      fP = v.f[i] * P / (rho * rho);
      v.P[i] = P;
      v.c[i] = c;
    }
    v.rec_h[i] = make_float4(rho, fP, c, 1.0f / H);
  }
  for (int o = 16; o; o >>= 1) exc = fmaxf(exc, __shfl_xor_sync(0xffffffffu, exc, o));
  if (lane == 0) s_exc[warp] = exc;
  __syncthreads();  // the chunk's records are in shared memory
  // phase 2: one leaf per warp, one particle per lane
  for (int q = warp; q < l1 - l0; q += (int)(blockDim.x >> 5)) {
    const int leaf = l0 + q;
    const int a = v.leaf_start[leaf], cnt = v.leaf_start[leaf + 1] - a;
    float bx = INFINITY, by = INFINITY, bz = INFINITY, tx = -INFINITY, ty = -INFINITY, tz = -INFINITY;
    float Hm = 0.0f;
    int minb = 127;
    unsigned long long mask = 0ull;
    if (lane < cnt) {
      const float4 r = s_rec[a - pa + lane];
      bx = tx = r.x;
      by = ty = r.y;
      bz = tz = r.z;
      Hm = r.w;
      if (do_bins) {
        minb = s_bin[a - pa + lane];
        mask = 1ull << minb;
      }
    }
    for (int o = 16; o; o >>= 1) {
      bx = fminf(bx, __shfl_xor_sync(0xffffffffu, bx, o));
      by = fminf(by, __shfl_xor_sync(0xffffffffu, by, o));
      bz = fminf(bz, __shfl_xor_sync(0xffffffffu, bz, o));
      tx = fmaxf(tx, __shfl_xor_sync(0xffffffffu, tx, o));
      ty = fmaxf(ty, __shfl_xor_sync(0xffffffffu, ty, o));
      tz = fmaxf(tz, __shfl_xor_sync(0xffffffffu, tz, o));
      Hm = fmaxf(Hm, __shfl_xor_sync(0xffffffffu, Hm, o));
      if (do_bins) {
        minb = min(minb, __shfl_xor_sync(0xffffffffu, minb, o));
        mask |= __shfl_xor_sync(0xffffffffu, mask, o);
      }
    }
    if (lane == 0) {
      v.leaf_lo[leaf] = make_float4(bx, by, bz, Hm);
      v.leaf_hi[leaf] = make_float4(tx, ty, tz, 0.0f);
      if (do_bins) {
        v.leaf_min_bin[leaf] = (uint8_t)minb;
        v.leaf_bin_mask[leaf] = mask;
      }
      const uint32_t k = v.leaf_k[leaf];
      const float sx = leaf_kx(k) * wqf, sy = leaf_ky(k) * wqf, sz = leaf_kz(k) * wqf;
      s_lo[q] = make_float4(bx + sx, by + sy, bz + sz, Hm);
      s_hi[q] = make_float4(tx + sx, ty + sy, tz + sz, 0.0f);
    }
  }
  __syncthreads();
  // phase 3: the chunk's box from its leaves (first warp)
  if (warp == 0) {
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) exc = fmaxf(exc, s_exc[k]);
    float lx = INFINITY, ly = INFINITY, lz = INFINITY;
    float hx = -INFINITY, hy = -INFINITY, hz = -INFINITY, Hm = 0.0f;
    if (lane < l1 - l0) {
      const float4 lo = s_lo[lane], hi = s_hi[lane];
      lx = lo.x; ly = lo.y; lz = lo.z; Hm = lo.w;
      hx = hi.x; hy = hi.y; hz = hi.z;
    }
    for (int o = 16; o; o >>= 1) {
      lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
      ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
      lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, o));
      hx = fmaxf(hx, __shfl_xor_sync(0xffffffffu, hx, o));
      hy = fmaxf(hy, __shfl_xor_sync(0xffffffffu, hy, o));
      hz = fmaxf(hz, __shfl_xor_sync(0xffffffffu, hz, o));
      Hm = fmaxf(Hm, __shfl_xor_sync(0xffffffffu, Hm, o));
    }
    if (lane == 0) {
      v.chunk_lo[g] = make_float4(lx, ly, lz, Hm);
      v.chunk_hi[g] = make_float4(hx, hy, hz, 0.0f);
      atomic_max_float_pos(&v.ds->excursion_bits, exc + 1e-6f * wf);
      atomic_max_float_pos(&v.ds->Hmax_bits, Hm);
    }
  }
  __syncthreads();  // the shared arrays are reused by the block's next chunk
}

__global__ void __launch_bounds__(UT) k_refresh(View v) {
  const int ng = v.ds->n_chunks;
  for (int g = blockIdx.x; g < ng; g += gridDim.x) chunk_update(v, g, false, true);
}

__global__ void __launch_bounds__(UT) k_drift(View v) {
  const DevState *ds = v.ds;
  const int nq = v.drift_all ? ds->n_chunks : ds->n_drift_chunks;
  for (int k = blockIdx.x; k < nq; k += gridDim.x) {
    const int g = v.drift_all ? k : v.q_drift[k];
    if (!SPH_IN(v.ds, g, ds->n_chunks, SPH_CHECK_DRIFT_CHUNK)) continue;  // (block-uniform)
    chunk_update(v, g, true, false);
  }
}

// ---------------------------------------------------------------------------
// kicks and time bins (one warp per active leaf)
// ---------------------------------------------------------------------------
// Eq. 1 and Eq. 2: the bin of a particle, the largest n with
// dt >= 2^n dt_min for dt = C h / v_sig, i.e. the binary exponent of the FP64
// quotient q = (C h / v_sig) / dt_min (capped at bin_cap); q < 1 sets *small
// and gives bin 0.  An FP32 estimate of q (five roundings: relative error below
// 4e-7) decides whenever it lies more than 2e-6 (relative) away from a power of
// two, where the FP64 quotient necessarily has the same exponent; near a power
// of two, below 2 or when not finite, q is computed in FP64 as defined.
__device__ __forceinline__ int bin_of(const View &v, float h, float vsig, bool &small) {
  // (every intermediate normal, so each rounding is relative)
  const float t1 = (float)v.cfl * h, t2 = t1 / vsig, q32 = t2 / (float)v.dt_min;
  int e32;
  const float m32 = frexpf(q32, &e32);  // q32 = m32 2^e32, m32 in [0.5, 1)
  int nb;
  small = false;
  if (t1 >= FLT_MIN && t2 >= FLT_MIN && isfinite(q32) && q32 >= 2.0f && m32 > 0.500001f &&
      m32 < 0.999998f) {
    nb = e32 - 1;
  } else {
    const double dt = __ddiv_rn(__dmul_rn(v.cfl, (double)h), (double)vsig);
    const double q = __ddiv_rn(dt, v.dt_min);
    if (!(q >= 1.0)) {
      small = true;
      return 0;
    }
    int e;
    frexp(q, &e);
    nb = e - 1;
  }
  return nb > v.bin_cap ? v.bin_cap : nb;
}

// Bin-occupancy change of the lanes in `changed` (old -> nb), one shared
// atomic per distinct bin of the warp instead of one per particle.
__device__ __forceinline__ void count_bin_change(int *delta, bool changed, int old, int nb) {
  const unsigned cm = __ballot_sync(0xffffffffu, changed);
  if (!changed) return;
  const int lane = lane_id();
  const unsigned same_old = __match_any_sync(cm, old);
  if (lane == __ffs(same_old) - 1) atomicSub(&delta[old], __popc(same_old));
  const unsigned same_new = __match_any_sync(cm, nb);
  if (lane == __ffs(same_new) - 1) atomicAdd(&delta[nb], __popc(same_new));
}

__global__ void k_kick(View v, int phase) {
  DevState *ds = v.ds;
  if (ds->halt) return;
  const int nq = ds->n_active_leaves, m_act = ds->m_act;
  for (int k = gwarp(); k < nq; k += nwarps()) {
    int leaf = v.q_active[k];
    if (!SPH_IN(ds, leaf, ds->n_leaves, SPH_CHECK_ACTIVE_LEAF)) continue;  // (warp-uniform)
    int a = v.leaf_start[leaf], b = v.leaf_start[leaf + 1];
    for (int i = a + lane_id(); i < b; i += 32) {
      if ((int)v.bin[i] > m_act) continue;
      // half of the step that closes (its end is now) or opens (its start is now)
      double half = 0.5 * (double)(v.ti_end[i] - v.ti_begin[i]) * v.dt_min;
      float hf = (float)half;
      v.vx[i] += v.ax[i] * hf;
      v.vy[i] += v.ay[i] * hf;
      v.vz[i] += v.az[i] * hf;
      v.A[i] = (float)((double)v.A[i] + (double)v.Adot[i] * half);
    }
  }
  (void)phase;
}

__global__ void k_bins(View v) {
  DevState *ds = v.ds;
  __shared__ int delta[MAX_BINS];
  __shared__ unsigned int too_small;
  for (int t = threadIdx.x; t < MAX_BINS; t += blockDim.x) delta[t] = 0;
  if (threadIdx.x == 0) too_small = 0u;
  __syncthreads();
  const bool halted = ds->halt != 0u;
  const int nq = ds->n_active_leaves, m_act = ds->m_act;
  const long long ti = ds->ti;
  for (int k = gwarp(); k < nq && !halted; k += nwarps()) {
    int leaf = v.q_active[k];
    if (!SPH_IN(ds, leaf, ds->n_leaves, SPH_CHECK_ACTIVE_LEAF)) continue;  // (warp-uniform)
    int a = v.leaf_start[leaf], b = v.leaf_start[leaf + 1];
    int minb = 127;
    unsigned long long mask = 0ull;
    for (int base = a; base < b; base += 32) {  // (the same trip count in every lane)
      const int i = base + lane_id();
      int old = 0, nb = 0;
      if (i < b) {
        old = v.bin[i];
        nb = old;
      }
      if (i < b && old <= m_act) {
        // Eq. 1: dt = C h / v_sig; Eq. 2: largest n with dt >= 2^n dt_min
        bool small;
        nb = bin_of(v, v.h[i], v.vsig[i], small);
        if (small) atomicAdd(&too_small, 1u);
        // limiter: at most 2 bins above the smallest neighbour's
        if (v.limiter) nb = min(nb, (int)v.ngb_bin[i] + 2);
        // a longer step only when the current tick is a multiple of it
        while (nb > old && (ti & ((1ll << nb) - 1)) != 0) nb--;
        v.bin[i] = (int8_t)nb;
        v.ti_begin[i] = ti;
        v.ti_end[i] = ti + (1ll << nb);
      }
      count_bin_change(delta, i < b && nb != old, old, nb);
      if (i < b) {
        minb = min(minb, nb);
        mask |= 1ull << nb;
      }
    }
    for (int o = 16; o; o >>= 1) {
      minb = min(minb, __shfl_xor_sync(0xffffffffu, minb, o));
      mask |= __shfl_xor_sync(0xffffffffu, mask, o);
    }
    if (lane_id() == 0) {
      v.leaf_min_bin[leaf] = (uint8_t)minb;
      v.leaf_bin_mask[leaf] = mask;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < MAX_BINS; t += blockDim.x)
    if (delta[t]) atomicAdd(&ds->bin_count[t], delta[t]);
  if (threadIdx.x == 0 && too_small) record_error(ds, SPH_ERR_DT_TOO_SMALL, too_small, false);
}

// Next tick: a particle on bin b ends its step at the next multiple of 2^b
// after the current tick, so the earliest end over all particles is the
// smallest such multiple over the occupied bins.
__device__ void next_time(View &v, long long *out, int count_step) {
  DevState *ds = v.ds;
  const long long ti = ds->ti;
  long long tn = LLONG_MAX;
  for (int b = 0; b < MAX_BINS; b++)
    if (ds->bin_count[b] > 0) {
      long long t = ((ti >> b) + 1) << b;
      if (t < tn) tn = t;
    }
  ds->ti_next = tn;
  if (out) *out = tn;
  // the step completed: its counters join the totals
  ds->pairs_density += ds->s_pairs_density;
  ds->pairs_force += ds->s_pairs_force;
  ds->cand_density += ds->s_cand_density;
  ds->cand_force += ds->s_cand_force;
  ds->iters_density += ds->s_iters_density;
  ds->active_particles += ds->s_active_particles;
  ds->gathers_density += ds->s_gathers_density;
  ds->list_overflows += ds->s_list_overflows;
  ds->evals_density += ds->s_evals_density;
  ds->s_pairs_density = ds->s_pairs_force = 0ull;
  ds->s_cand_density = ds->s_cand_force = 0ull;
  ds->s_iters_density = ds->s_active_particles = 0ull;
  ds->s_gathers_density = ds->s_list_overflows = ds->s_evals_density = 0ull;
  if (count_step) ds->steps += 1ull;
}

__global__ void k_next_time(View v, long long *out, int count_step) {
  if (v.ds->halt) return;
  next_time(v, out, count_step);
}

// The end of a step in one launch: for every active particle (one warp per
// active leaf) the closing half-kick of its old step, its new bin (as
// k_bins), the opening half-kick of the new step -- the same arithmetic as
// k_kick and k_bins in the same order -- then, in the last block to finish,
// the next tick and the step's counters (as k_next_time).
__global__ void __launch_bounds__(UT) k_close_step(View v) {
  DevState *ds = v.ds;
  __shared__ int delta[MAX_BINS];
  __shared__ unsigned int too_small;
  __shared__ int s_go, s_last;
  if (threadIdx.x == 0) {
    s_go = ds->halt ? 0 : 1;
    too_small = 0u;
  }
  for (int t = threadIdx.x; t < MAX_BINS; t += blockDim.x) delta[t] = 0;
  __syncthreads();
  if (!s_go) return;  // the whole block (a halted step changes nothing)
  const int nq = ds->n_active_leaves, m_act = ds->m_act;
  const long long ti = ds->ti;
  for (int k = gwarp(); k < nq; k += nwarps()) {
    const int leaf = v.q_active[k];
    if (!SPH_IN(ds, leaf, ds->n_leaves, SPH_CHECK_ACTIVE_LEAF)) continue;  // (warp-uniform)
    const int a = v.leaf_start[leaf], b = v.leaf_start[leaf + 1];
    int minb = 127;
    unsigned long long mask = 0ull;
    for (int base = a; base < b; base += 32) {  // (the same trip count in every lane)
      const int i = base + lane_id();
      const int old = i < b ? (int)v.bin[i] : 0;
      int nb = old;
      if (i < b && old <= m_act) {
        // closing half-kick of the old step
        double half = 0.5 * (double)(v.ti_end[i] - v.ti_begin[i]) * v.dt_min;
        float hf = (float)half;
        v.vx[i] += v.ax[i] * hf;
        v.vy[i] += v.ay[i] * hf;
        v.vz[i] += v.az[i] * hf;
        v.A[i] = (float)((double)v.A[i] + (double)v.Adot[i] * half);
        // Eq. 1 and Eq. 2, increases only on a multiple of the new step
        bool small;
        nb = bin_of(v, v.h[i], v.vsig[i], small);
        if (small) atomicAdd(&too_small, 1u);
        // limiter: at most 2 bins above the smallest neighbour's
        if (v.limiter) nb = min(nb, (int)v.ngb_bin[i] + 2);
        while (nb > old && (ti & ((1ll << nb) - 1)) != 0) nb--;
        v.bin[i] = (int8_t)nb;
        v.ti_begin[i] = ti;
        v.ti_end[i] = ti + (1ll << nb);
        // opening half-kick of the new step
        half = 0.5 * (double)(v.ti_end[i] - v.ti_begin[i]) * v.dt_min;
        hf = (float)half;
        v.vx[i] += v.ax[i] * hf;
        v.vy[i] += v.ay[i] * hf;
        v.vz[i] += v.az[i] * hf;
        v.A[i] = (float)((double)v.A[i] + (double)v.Adot[i] * half);
      }
      count_bin_change(delta, i < b && nb != old, old, nb);
      if (i < b) {
        minb = min(minb, nb);
        mask |= 1ull << nb;
      }
    }
    for (int o = 16; o; o >>= 1) {
      minb = min(minb, __shfl_xor_sync(0xffffffffu, minb, o));
      mask |= __shfl_xor_sync(0xffffffffu, mask, o);
    }
    if (lane_id() == 0) {
      v.leaf_min_bin[leaf] = (uint8_t)minb;
      v.leaf_bin_mask[leaf] = mask;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < MAX_BINS; t += blockDim.x)
    if (delta[t]) atomicAdd(&ds->bin_count[t], delta[t]);
  if (threadIdx.x == 0 && too_small) record_error(ds, SPH_ERR_DT_TOO_SMALL, too_small, false);
  // the last block to finish sees every block's bin counts
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&ds->blocks_done, 1u) == gridDim.x - 1u;
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    ds->blocks_done = 0u;
    next_time(v, nullptr, 1);
  }
}

// smallest bin of a leaf lowered to b (a byte of a 4-byte word: compare-and-swap
// on the word)
__device__ __forceinline__ void atomic_min_u8(uint8_t *p, int b) {
  unsigned int *w = reinterpret_cast<unsigned int *>(reinterpret_cast<uintptr_t>(p) & ~(uintptr_t)3);
  const int sh = (int)(reinterpret_cast<uintptr_t>(p) & 3) * 8;
  unsigned int old = *w, assumed;
  do {
    assumed = old;
    if ((int)((assumed >> sh) & 0xffu) <= b) return;
    old = atomicCAS(w, assumed, (assumed & ~(0xffu << sh)) | ((unsigned int)b << sh));
  } while (old != assumed);
}

// The limiter's waking of inactive neighbours (Saitoh & Makino 2009, as
// Durier & Dalla Vecchia 2012 describe it): the force loop asked each
// inactive particle j with an active neighbour i of bin_j > bin_i + 2 down to
// the smallest such bin_i + 2 (wake_bin).  After the step's close, j's step
// is cut to end at the first multiple of 2^b after the current tick, when
// that comes before its old end: its bin becomes b (it is active then), and
// the opening half-kick of its step is cut to the shortened step,
// v -= a (D_old - D_new) / 2, A -= Adot (D_old - D_new) / 2 (D in ticks).
// The particle's leaf learns the new bin (its smallest bin and bin mask;
// the leaf's next close recomputes both exactly); with adjust_next, the
// step's next tick (already computed) is lowered to the woken ends.  Every
// request is reset, applied or not.
__global__ void k_wake(View v, int adjust_next) {
  DevState *ds = v.ds;
  if (ds->halt) return;
  const int nw = ds->n_wake;
  const long long ti = ds->ti;
  unsigned long long woken = 0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nw; k += gridDim.x * blockDim.x) {
    const int j = v.q_wake[k];
    if (!SPH_IN(ds, j, v.n, SPH_CHECK_WAKE)) continue;
    const int b = v.wake_bin[j];
    v.wake_bin[j] = WAKE_NONE;
    const int old = v.bin[j];
    if (b >= old || b < 0) continue;
    const long long tw = ((ti >> b) + 1) << b;
    if (tw >= v.ti_end[j]) continue;
    const double corr = 0.5 * (double)(v.ti_end[j] - tw) * v.dt_min;  // (D_old - D_new) / 2
    const float cf = (float)corr;
    v.vx[j] -= v.ax[j] * cf;
    v.vy[j] -= v.ay[j] * cf;
    v.vz[j] -= v.az[j] * cf;
    v.A[j] = (float)((double)v.A[j] - (double)v.Adot[j] * corr);
    v.ti_end[j] = tw;
    v.bin[j] = (int8_t)b;
    atomicSub(&ds->bin_count[old], 1);
    atomicAdd(&ds->bin_count[b], 1);
    const int leaf = v.pleaf[j];
    atomic_min_u8(&v.leaf_min_bin[leaf], b);
    atomicOr(&v.leaf_bin_mask[leaf], 1ull << b);
    if (adjust_next) atomicMin(&ds->ti_next, tw);
    woken++;
  }
  for (int o = 16; o; o >>= 1) woken += __shfl_xor_sync(0xffffffffu, woken, o);
  if (lane_id() == 0 && woken) atomicAdd(&ds->wakes, woken);
}

// Active work groups, active particles and the cells to drift, in one launch
// (the three read only what k_mark_leaves wrote): the blocks of the grid are
// split into three ranges, one per task.
__global__ void __launch_bounds__(UT) k_mark_rest(View v) {
  const int third = gridDim.x / 3;
  if ((int)blockIdx.x < third) mark_groups_part(v, 0, third);
  else if ((int)blockIdx.x < 2 * third) mark_particles_part(v, third, third);
  else if (!v.drift_all) relevant_part(v, 2 * third, gridDim.x - 2 * third);
}

// One thread per active work group: queues the groups holding particles of
// one bin; with one lane per particle, in a step with few active groups, they
// go to the back of the queue (the force loop's blocks process them
// cooperatively, as in the batched form).
__global__ void k_mark_bin(View v, int bin) {
  DevState *ds = v.ds;
  const int nh = ds->n_heavy_groups, ng = ds->n_groups;
  const int nq = ds->n_active_groups + nh;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nq; k += gridDim.x * blockDim.x) {
    const int g = active_group(v, ds, k);
    unsigned long long mask = 0ull;
    for (int l = v.group_leaf0[g]; l < v.group_leaf0[g + 1]; l++) mask |= v.leaf_bin_mask[l];
    if (!((mask >> bin) & 1ull)) continue;
    if (v.G == 1 && all_coop(v, ds)) v.q_bin[ng - 1 - atomicAdd(&ds->n_bin_coop, 1)] = g;
    else v.q_bin[atomicAdd(&ds->n_bin_groups, 1)] = g;
  }
}

// ---------------------------------------------------------------------------
// diagnostics: total energy and momentum in FP64
// ---------------------------------------------------------------------------
// Per particle, the velocity and entropy at tick ti predicted from the
// half-step state (v_half + a (t - t_mid), A + Adot (t - t_mid), Sec. II-A),
// u = A rho^(gamma-1) / (gamma-1) from the last density; summed per block in
// a fixed order (each thread a fixed stride of particles, then a tree in
// shared memory), so the result does not depend on scheduling.
__global__ void __launch_bounds__(DIAG_THREADS)
k_diag(const sph_particles p, long long ti, double dt_min, double gamma, double *partials) {
  __shared__ double s[DIAG_FIELDS][DIAG_THREADS];
  double acc[DIAG_FIELDS];
#pragma unroll
  for (int k = 0; k < DIAG_FIELDS; k++) acc[k] = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += stride) {
    const double dtp =
        ((double)(ti - p.ti_begin[i]) - 0.5 * (double)(p.ti_end[i] - p.ti_begin[i])) * dt_min;
    const double m = (double)p.m[i];
    const double vx = (double)p.vx[i] + (double)p.ax[i] * dtp;
    const double vy = (double)p.vy[i] + (double)p.ay[i] * dtp;
    const double vz = (double)p.vz[i] + (double)p.az[i] * dtp;
    const double A = (double)p.A[i] + (double)p.Adot[i] * dtp;
    const double rho = (double)p.rho[i];
    acc[0] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
    if (rho > 0.0) acc[1] += m * A * pow(rho, gamma - 1.0) / (gamma - 1.0);
    else acc[6] += 1.0;
    acc[2] += m * vx;
    acc[3] += m * vy;
    acc[4] += m * vz;
    acc[5] += m;
  }
#pragma unroll
  for (int k = 0; k < DIAG_FIELDS; k++) s[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = DIAG_THREADS / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int k = 0; k < DIAG_FIELDS; k++) s[k][threadIdx.x] += s[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < DIAG_FIELDS) partials[blockIdx.x * DIAG_FIELDS + threadIdx.x] = s[threadIdx.x][0];
}

// the block partials summed in block order
__global__ void k_diag_final(const double *partials, int nblocks, double *out) {
  if (threadIdx.x >= DIAG_FIELDS) return;
  double t = 0.0;
  for (int b = 0; b < nblocks; b++) t += partials[b * DIAG_FIELDS + threadIdx.x];
  out[threadIdx.x] = t;
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_refresh_all(const View &v, cudaStream_t st) {
  note_launches(1);
  k_refresh<<<2 * v.grid_util, UT, 0, st>>>(v);
  return cudaGetLastError();
}

cudaError_t launch_mark(const View &v, long long ti_or_neg, cudaStream_t st) {
  note_launches(4);
  k_mark_clear<<<v.grid_util, UT, 0, st>>>(v);
  k_begin_step<<<1, 1, 0, st>>>(v, ti_or_neg);
  k_mark_leaves<<<v.grid_util, UT, 0, st>>>(v);
  k_mark_rest<<<3 * (v.grid_util / 3 > 0 ? v.grid_util / 3 : 1), UT, 0, st>>>(v);
  return cudaGetLastError();
}

cudaError_t launch_close_step(const View &v, cudaStream_t st) {
  note_launches(v.limiter ? 2 : 1);
  k_close_step<<<v.grid_util, UT, 0, st>>>(v);
  if (v.limiter) k_wake<<<v.grid_util, UT, 0, st>>>(v, 1);
  return cudaGetLastError();
}

cudaError_t launch_drift(const View &v, cudaStream_t st) {
  note_launches(1);
  // (blocks of 128 threads: twice the chunks in flight per SM of 256-thread
  // blocks, which the registers limit to five per SM; a sparse step's drift
  // is bound by the latency of its chunks' dependent phases)
  k_drift<<<4 * v.grid_util, 128, 0, st>>>(v);
  return cudaGetLastError();
}

cudaError_t launch_kick(const View &v, int phase, cudaStream_t st) {
  note_launches(1);
  k_kick<<<v.grid_util, UT, 0, st>>>(v, phase);
  return cudaGetLastError();
}

cudaError_t launch_bins(const View &v, long long *ti_next_out, int count_step, cudaStream_t st) {
  note_launches(v.limiter ? 3 : 2);
  k_bins<<<v.grid_util, UT, 0, st>>>(v);
  if (v.limiter) k_wake<<<v.grid_util, UT, 0, st>>>(v, 0);
  k_next_time<<<1, 1, 0, st>>>(v, ti_next_out, count_step);
  return cudaGetLastError();
}

cudaError_t launch_diagnostics(const sph_particles &p, long long ti, double dt_min, double gamma,
                               double *partials, double *out, cudaStream_t st) {
  note_launches(2);
  k_diag<<<DIAG_BLOCKS, DIAG_THREADS, 0, st>>>(p, ti, dt_min, gamma, partials);
  k_diag_final<<<1, 32, 0, st>>>(partials, DIAG_BLOCKS, out);
  return cudaGetLastError();
}

cudaError_t launch_mark_bin(const View &v, int bin, cudaStream_t st) {
  note_launches(1);
  cudaError_t e = cudaMemsetAsync(SPH_DS_FIELD(v.ds, n_bin_groups), 0, 2 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  // the head of the force loop's blocks that take the shared groups
  e = cudaMemsetAsync(SPH_DS_FIELD(v.ds, head_coop_force), 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  // (the per-bin density launch pulls its groups from head_density)
  e = cudaMemsetAsync(SPH_DS_FIELD(v.ds, head_density), 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_mark_bin<<<v.grid_util, UT, 0, st>>>(v, bin);
  return cudaGetLastError();
}

}  // namespace sph
