// Shared machinery of the neighbour loops (the forward density and force
// loops and their adjoints): the per-warp shared-memory staging area, the TMA
// bulk copies with their mbarrier, the neighbour-leaf search over the 27
// cells around a work group, and small warp helpers.  Included by the
// translation units that hold pair kernels; everything has internal linkage.
#pragma once

#include <cstddef>

#include "sph_internal.cuh"

namespace sph {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int PT = WARPS_PER_BLOCK * 32;
constexpr int S_DENS = 256;   // staged candidate records per warp, density loop
constexpr int S_FORCE = 128;  // staged candidates per warp, force loop (3 records each)
constexpr long long WAIT_LIMIT = 1ll << 22;  // bounded mbarrier wait (iterations)

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// ---------------------------------------------------------------------------
// mbarrier + bulk copy (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\tmbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}

// bounded wait for the completion of the barrier phase with this parity
// (limit: polls; after the first 16 each poll sleeps ~64 ns)
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit) {
  for (long long k = 0; k < limit; k++) {
    if (mbar_try_wait(bar, parity)) return true;
    if (k > 16) __nanosleep(64);
  }
  return false;
}

// global -> shared bulk copy (TMA), bytes a multiple of 16, both ends 16-byte aligned
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// orders this thread's earlier shared-memory reads before later bulk writes
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
// compensated accumulation: hi + lo holds the sum of the parts
__device__ __forceinline__ void fold(float &hi, float &lo, float part) {
  float s = hi + part;
  float bp = s - hi;
  float err = (hi - (s - bp)) + (part - bp);
  hi = s;
  lo += err;
}

template <int G>
__device__ __forceinline__ double group_sum(double x) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
  return x;
}

template <int G>
__device__ __forceinline__ int group_sum_i(int x) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
  return x;
}

template <int G>
__device__ __forceinline__ float group_max(float x) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(FULL, x, o));
  return x;
}

// Squared distances of two pairs at once, a - b per component, with packed
// FP32 instructions; each component is rounded exactly as the scalar
// fmaf(dx, dx, fmaf(dy, dy, dz * dz)) with dx = a.x - b.x.
__device__ __forceinline__ float2 dist2_x2(float2 ax, float2 ay, float2 az, float2 bx, float2 by,
                                           float2 bz) {
  const float2 dx = __fadd2_rn(ax, make_float2(-bx.x, -bx.y));
  const float2 dy = __fadd2_rn(ay, make_float2(-by.x, -by.y));
  const float2 dz = __fadd2_rn(az, make_float2(-bz.x, -bz.y));
  return __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
}

__device__ __forceinline__ float warp_max(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(FULL, x, o));
  return x;
}

__device__ __forceinline__ int warp_incl_scan(int x) {
  const int lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Active particles of leaf [a, b) (bin <= m_act, and == bin_filter when that
// is >= 0) written to s_act in particle order; returns their number.
__device__ __forceinline__ int leaf_actives(const View &v, int a, int b, int m_act,
                                            int bin_filter, int *s_act) {
  const int lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  int n = 0;
  for (int base = a; base < b; base += 32) {
    int i = base + lane;
    bool ok = false;
    if (i < b) {
      int bi = v.bin[i];
      ok = bi <= m_act && (bin_filter < 0 || bi == bin_filter);
    }
    unsigned mk = __ballot_sync(FULL, ok);
    if (ok) s_act[n + __popc(mk & lt)] = i;
    n += __popc(mk);
  }
  __syncwarp();
  return n;
}

// squared gap between box i and box j shifted by s
__device__ __forceinline__ float box_gap2(float lix, float liy, float liz, float hix, float hiy,
                                          float hiz, const float4 &loj, const float4 &hij, float sx,
                                          float sy, float sz) {
  float gx = fmaxf(0.0f, fmaxf(loj.x + sx - hix, lix - (hij.x + sx)));
  float gy = fmaxf(0.0f, fmaxf(loj.y + sy - hiy, liy - (hij.y + sy)));
  float gz = fmaxf(0.0f, fmaxf(loj.z + sz - hiz, liz - (hij.z + sz)));
  return gx * gx + gy * gy + gz * gz;
}

// Candidate test of a staged block of 32 records with the records across the
// lanes: one ballot per live particle (tst[0..ntst), lane order) gives that
// particle's accept mask, which lands on the lane whose rank among the live
// lanes is the particle's.  Each (particle, record) test is the very
// expression of the per-lane test, so the masks are the same bits; for few
// live particles it costs ntst votes instead of 32 serial tests per lane.
constexpr int TRANSPOSE_MAX = 24;

// Writes the spheres (centre, radius) of the lanes with `has` set to
// sph[0..n) in lane order and returns n (all lanes of the warp call it).
__device__ __forceinline__ int compact_spheres(float4 *sph, bool has, float4 s) {
  const unsigned mk = __ballot_sync(FULL, has);
  if (has) sph[__popc(mk & ((1u << lane_id()) - 1u))] = s;
  __syncwarp();
  return __popc(mk);
}

// Whether sphere c (centre, radius in w; a radius <= 0 never reaches) comes
// within max(radius, grow) of the box [l, h]; `grow` is the leaf's own
// support, a lower bound of every radius when > 0.
__device__ __forceinline__ bool sphere_reaches(const float4 &c, float grow, float lx, float ly,
                                               float lz, float hx, float hy, float hz) {
  const float R = fmaxf(c.w, grow);
  const float gx = fmaxf(0.0f, fmaxf(lx - c.x, c.x - hx));
  const float gy = fmaxf(0.0f, fmaxf(ly - c.y, c.y - hy));
  const float gz = fmaxf(0.0f, fmaxf(lz - c.z, c.z - hz));
  return c.w > 0.0f && gx * gx + gy * gy + gz * gz < R * R * 1.0002f;
}

// A leaf that passed a search's box test, for the support-sphere test after
// it: its box shifted into the group's frame and its own support.
struct LeafBox {
  float lx, ly, lz, hx, hy, hz, grow;
};

__device__ __forceinline__ LeafBox leaf_box(const float4 &lo, const float4 &hi, float sx, float sy,
                                            float sz, float grow) {
  return LeafBox{lo.x + sx, lo.y + sy, lo.z + sz, hi.x + sx, hi.y + sy, hi.z + sz, grow};
}

// For the lanes with `ok` set, whether any of the n spheres sph[0..n)
// reaches the lane's leaf box (all lanes of the warp call it).  With many
// boxes (or lanes_only) each lane loops over the spheres; with few, the
// spheres go across the lanes (lane p holds sphere p) and each box is
// broadcast and tested by one vote -- the same expression either way.
__device__ __forceinline__ bool spheres_reach_any(const float4 *sph, int n, bool ok,
                                                  const LeafBox &b, bool lanes_only) {
  const unsigned pend0 = __ballot_sync(FULL, ok);
  const int nb = __popc(pend0);
  if (lanes_only || nb * 4 >= n * 3) {
    if (!ok) return false;
    for (int p = 0; p < n; p++)
      if (sphere_reaches(sph[p], b.grow, b.lx, b.ly, b.lz, b.hx, b.hy, b.hz)) return true;
    return false;
  }
  const int lane = lane_id();
  const float4 c = sph[min(lane, n - 1)];  // n > 0 here
  unsigned hit = 0u, pend = pend0;
  while (pend) {
    const int s = __ffs(pend) - 1;
    pend &= pend - 1;
    const float lx = __shfl_sync(FULL, b.lx, s), ly = __shfl_sync(FULL, b.ly, s),
                lz = __shfl_sync(FULL, b.lz, s);
    const float hx = __shfl_sync(FULL, b.hx, s), hy = __shfl_sync(FULL, b.hy, s),
                hz = __shfl_sync(FULL, b.hz, s);
    const float g = __shfl_sync(FULL, b.grow, s);
    const bool r = lane < n && sphere_reaches(c, g, lx, ly, lz, hx, hy, hz);
    if (__any_sync(FULL, r)) hit |= 1u << s;
  }
  return (hit >> lane) & 1u;
}

// Cubic spline: w(q) / (8/pi) and w'(q) / (8/pi), q in [0, 1)
__device__ __forceinline__ void kernel_wd(float q, float &wq, float &dwq) {
  const float s = 1.0f - q;
  const float s2 = s * s;
  const float q2 = q * q;
  const float wa = fmaf(q2, fmaf(6.0f, q, -6.0f), 1.0f);  // 1 - 6q^2 + 6q^3
  const float da = q * fmaf(18.0f, q, -12.0f);           // -12q + 18q^2
  const float wb = 2.0f * s2 * s;                        // 2 (1-q)^3
  const float db = -6.0f * s2;                           // -6 (1-q)^2
  const bool inner = q < 0.5f;
  wq = inner ? wa : wb;
  dwq = inner ? da : db;
}

// w''(q) / (8/pi): -12 + 36 q (q < 1/2), 12 (1 - q) (q < 1)
__device__ __forceinline__ float kernel_d2w(float q) {
  return q < 0.5f ? fmaf(36.0f, q, -12.0f) : 12.0f * (1.0f - q);
}

__device__ __forceinline__ float kernel_dw(float q) {
  const float s = 1.0f - q;
  const float da = q * fmaf(18.0f, q, -12.0f);
  const float db = -6.0f * s * s;
  return q < 0.5f ? da : db;
}

struct CellFrame {
  int cx, cy, cz, nc;
  float wq;        // Morton grid step w / 1024
  float wf;        // cell width
  int kx, ky, kz;  // the work leaf's corner on its cell's Morton grid
};

__device__ __forceinline__ CellFrame frame_of(const View &v, const DevState *ds, int grp) {
  CellFrame F;
  const int cell = v.group_cell[grp];
  const uint32_t k = v.leaf_k[v.group_leaf0[grp]];
  F.nc = ds->nc;
  F.cx = cell / (F.nc * F.nc);
  F.cy = (cell / F.nc) % F.nc;
  F.cz = cell % F.nc;
  F.wq = (float)(ds->w / (double)(1 << MORTON_BITS));
  F.wf = (float)ds->w;
  F.kx = leaf_kx(k);
  F.ky = leaf_ky(k);
  F.kz = leaf_kz(k);
  return F;
}

struct WarpCounters {
  unsigned long long pairs, cand, iters, noconv, overflow, timeout;
  unsigned long long gathers, list_overflows;  // density loop: particle gathers, full lists
  unsigned long long evals;                    // density loop: list entries evaluated
};

// A work group: particles [a, b) in leaves [L0, L1) of one cell, and the
// group's bounding box in the frame of its first leaf's corner (all lanes).
struct Group {
  int a, b, L0, L1;
  float lx, ly, lz, hx, hy, hz;
};

__device__ __forceinline__ Group group_of(const View &v, int g, const CellFrame &F) {
  Group G;
  G.L0 = v.group_leaf0[g];
  G.L1 = v.group_leaf0[g + 1];
  // (checks build: at most WG_MAX leaves in range, then at most WG_MAX
  // particles in range; otherwise an empty group)
  if (!(SPH_IN(v.ds, G.L0, G.L1, SPH_CHECK_GROUP_LEAVES) &&
        SPH_IN(v.ds, G.L1 - 1, v.ds->n_leaves, SPH_CHECK_GROUP_LEAVES) &&
        SPH_IN(v.ds, G.L1 - G.L0 - 1, WG_MAX, SPH_CHECK_GROUP_LEAVES)))
    G.L0 = G.L1 = 0;
  G.a = v.leaf_start[G.L0];
  G.b = v.leaf_start[G.L1];
  if (!(SPH_IN(v.ds, G.a, G.b + 1, SPH_CHECK_LEAF) && SPH_IN(v.ds, G.b, v.n + 1, SPH_CHECK_LEAF) &&
        SPH_IN(v.ds, G.b - G.a, WG_MAX + 1, SPH_CHECK_GROUP_SIZE))) {
    G.L0 = G.L1 = 0;
    G.a = G.b = 0;
  }
  const int lane = lane_id();
  float lx = INFINITY, ly = INFINITY, lz = INFINITY, hx = -INFINITY, hy = -INFINITY, hz = -INFINITY;
  if (G.L0 + lane < G.L1) {
    const int l = G.L0 + lane;
    const uint32_t k = v.leaf_k[l];
    const float ox = (float)(leaf_kx(k) - F.kx) * F.wq;
    const float oy = (float)(leaf_ky(k) - F.ky) * F.wq;
    const float oz = (float)(leaf_kz(k) - F.kz) * F.wq;
    const float4 lo = v.leaf_lo[l], hi = v.leaf_hi[l];
    lx = lo.x + ox; ly = lo.y + oy; lz = lo.z + oz;
    hx = hi.x + ox; hy = hi.y + oy; hz = hi.z + oz;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lx = fminf(lx, __shfl_xor_sync(FULL, lx, o));
    ly = fminf(ly, __shfl_xor_sync(FULL, ly, o));
    lz = fminf(lz, __shfl_xor_sync(FULL, lz, o));
    hx = fmaxf(hx, __shfl_xor_sync(FULL, hx, o));
    hy = fmaxf(hy, __shfl_xor_sync(FULL, hy, o));
    hz = fmaxf(hz, __shfl_xor_sync(FULL, hz, o));
  }
  G.lx = lx; G.ly = ly; G.lz = lz; G.hx = hx; G.hy = hy; G.hz = hz;
  return G;
}

// offset of particle i's leaf corner from the group frame's corner
__device__ __forceinline__ float3 leaf_offset(const View &v, int i, const CellFrame &F) {
  const int l = v.pleaf[i];
  if (!SPH_IN(v.ds, l, v.ds->n_leaves, SPH_CHECK_PARTICLE_LEAF)) return make_float3(0.f, 0.f, 0.f);
  const uint32_t k = v.leaf_k[l];
  return make_float3((float)(leaf_kx(k) - F.kx) * F.wq, (float)(leaf_ky(k) - F.ky) * F.wq,
                     (float)(leaf_kz(k) - F.kz) * F.wq);
}

// ---------------------------------------------------------------------------
// per-warp staging area in dynamic shared memory
// ---------------------------------------------------------------------------
constexpr int STAGE_DEPTH_MAX = 3;  // staging buffers per warp (copies in flight)

template <int S, int NREC, int LC>
struct Stage {
  static constexpr int LCAP = LC;  // accepted neighbour leaves listed per search pass
  static constexpr int CCAP = 128; // accepted chunks gathered per search segment
  float4 *rec;     // NREC arrays of S staged records, back to back (first: positions);
                   // with depth d, buffer b holds slots [b S/d, (b+1) S/d) of each
  float4 *lshift;  // per listed leaf: offset of its corner (x, y, z), first particle (w bits)
  int *lpack;      // per listed leaf: count | cell index << 16
  int *act;        // active particles of the work group
  int *recj;       // per staged record: particle index
  uint8_t *recc;   // per staged record: neighbour-cell index (0..26)
  float4 *sph;     // the round's particles: position (group frame), search radius
  float4 *tst;     // the round's live particles: position (group frame), squared test radius
  int2 *chk;       // accepted chunks of a search segment: first leaf, count | cell << 16
  uint64_t *bar;   // one mbarrier per staging buffer
  int *meta;       // per staging buffer: first listed leaf, leaves, records
  uint32_t phase;  // parity of the next phase of each buffer's barrier (bit b)
  int depth;       // staging buffers in use (1..STAGE_DEPTH_MAX)
  long long wait_limit;  // polls of a bounded barrier wait
  int *stall_ctr;  // testing: stalls still to make (a launch's first staging claims one)
  bool stall;      // testing: this staging issues no copy and never arrives
  bool failed;
  static constexpr size_t bytes() {
    return sizeof(float4) * ((size_t)S * NREC + LC + 64) + sizeof(int2) * CCAP +
           sizeof(int) * (LC + LEAF_MAX_LIMIT + S) + (size_t)S + 64;
  }
  // sph, tst and chk back to back: free between one round's last consume and
  // the next search, they serve a block's cross-warp reductions (the staged
  // records and the leaf list stay in place)
  static constexpr size_t red_offset() { return sizeof(float4) * ((size_t)S * NREC + LC); }
  static constexpr size_t red_bytes() { return sizeof(float4) * 64 + sizeof(int2) * CCAP; }
  __device__ void carve(char *base) {
    rec = reinterpret_cast<float4 *>(base);
    lshift = rec + (size_t)S * NREC;
    sph = lshift + LC;
    tst = sph + 32;
    chk = reinterpret_cast<int2 *>(tst + 32);
    lpack = reinterpret_cast<int *>(chk + CCAP);
    act = lpack + LC;
    recj = act + LEAF_MAX_LIMIT;
    recc = reinterpret_cast<uint8_t *>(recj + S);
    bar = reinterpret_cast<uint64_t *>(recc + S);  // 8-byte aligned: every part above is
    meta = reinterpret_cast<int *>(bar + STAGE_DEPTH_MAX);
  }
};

// Lane `lane` holds v_lane (lanes 0..n-1, ascending); returns, for this lane's
// key t, the largest index c < n with v_c <= t (the segment holding t).
__device__ __forceinline__ int seg_of(int v_lane, int n, int t) {
  int lo = 0, hi = n - 1;
#pragma unroll
  for (int step = 0; step < 5; step++) {
    const int mid = (lo + hi + 1) >> 1;
    const int vm = __shfl_sync(FULL, v_lane, mid);
    if (lo < hi) {
      if (vm <= t) lo = mid;
      else hi = mid - 1;
    }
  }
  return lo;
}

// What a search may reach: the work group's box in its cell's frame and the
// largest distance at which a leaf can still pass the caller's tests (every
// leaf test implies box distance < R).  Neighbour cells farther than R from
// the box -- their particles may lie up to `exc` outside the cell -- are
// skipped without reading anything.
struct Reach {
  float lx, ly, lz, hx, hy, hz;  // group box, cell frame
  float R;                       // reach
  float exc;                     // largest excursion of a particle out of its cell
  const float4 *sph;             // support spheres a leaf must also meet (or nullptr)
  int nsph;
  bool lanes_only = false;       // sphere test per lane only (fewer registers)
  bool chunk_spheres = false;    // test the spheres on the chunks' boxes too (before
                                 // their leaves), in the group frame:
  float fx = 0.f, fy = 0.f, fz = 0.f;  // the group frame's corner in its cell's frame
  bool grow_own = false;         // a box is also reached within its own largest support
};

// Lists, in cell-then-leaf order, the leaves of the 27 cells around the work
// group that pass `leaf_ok` (a box test; then, with reach.sph set, one of the
// support spheres must reach the leaf box leaf_ok returned) (in cells of more than CHUNK leaves, only those of
// chunks passing `chunk_ok`; cells out of `reach` entirely skipped; with
// part >= 0 only chunks with index = part modulo WARPS_PER_BLOCK): accepted
// leaves skip, skip + 1, ... up to LCAP of them.  Returns how many were
// listed; `more` tells whether the list stopped because it was full.  With
// reach.chunk_spheres, a chunk whose box (padded by 1e-5 of the cell width)
// no sphere reaches is dropped before its leaves are read: every leaf box
// lies inside its chunk's box and has at most its chunk's largest support, so
// no leaf that the sphere test would accept is lost.  The
// cells' chunks, then the accepted chunks' leaves, are tested 32 at a time
// across all 27 cells, so the number of dependent global-memory rounds does
// not grow with the cell count.
template <class St, class LeafOk, class ChunkOk>
__device__ __forceinline__ int search(const View &v, const CellFrame &F, const Reach &reach,
                                      St &st, LeafOk leaf_ok,
                                      ChunkOk chunk_ok, int skip, bool &more, int part = -1) {
  constexpr int LCAP = St::LCAP;
  constexpr int CCAP = St::CCAP;
  const int lane = lane_id();
  more = false;
  const int limit = skip + LCAP;
  // phase 1: the 27 neighbour cells, one per lane
  int g0 = 0, nch = 0, l0 = 0, l1 = 0;
  if (lane < 27) {
    const int dxc = lane / 9 - 1, dyc = (lane / 3) % 3 - 1, dzc = lane % 3 - 1;
    // gap between the group's box and the neighbour cell (grown by exc)
    const float e = reach.exc;
    const float gx = fmaxf(0.0f, fmaxf(dxc * F.wf - e - reach.hx, reach.lx - ((dxc + 1) * F.wf + e)));
    const float gy = fmaxf(0.0f, fmaxf(dyc * F.wf - e - reach.hy, reach.ly - ((dyc + 1) * F.wf + e)));
    const float gz = fmaxf(0.0f, fmaxf(dzc * F.wf - e - reach.hz, reach.lz - ((dzc + 1) * F.wf + e)));
    if (gx * gx + gy * gy + gz * gz < reach.R * reach.R * 1.0002f) {
      const int cj = (wrap_cell(F.cx + dxc, F.nc) * F.nc + wrap_cell(F.cy + dyc, F.nc)) * F.nc +
                     wrap_cell(F.cz + dzc, F.nc);
      g0 = v.cell_chunk_start[cj];
      nch = v.cell_chunk_start[cj + 1] - g0;
      l0 = v.cell_leaf_start[cj];
      l1 = v.cell_leaf_start[cj + 1];
      // (checks build: a cell whose leaf or chunk range is out of bounds is skipped)
      if (!(SPH_IN(v.ds, l0, l1 + 1, SPH_CHECK_CELL_LEAVES) &&
            SPH_IN(v.ds, l1, v.ds->n_leaves + 1, SPH_CHECK_CELL_LEAVES) &&
            SPH_IN(v.ds, g0, v.ds->n_chunks + 1, SPH_CHECK_CELL_LEAVES) &&
            SPH_IN(v.ds, g0 + nch, v.ds->n_chunks + 1, SPH_CHECK_CELL_LEAVES)))
        nch = 0;
    }
  }
  const int cstart = warp_incl_scan(nch) - nch;  // first flat chunk index of this lane's cell
  const int T = __shfl_sync(FULL, cstart + nch, 26);
  int seen = 0;  // accepted leaves so far
  // phase 2: all chunks of the 27 cells, 32 per round; accepted chunks are
  // gathered (in order) into st.chk, then phase 3 runs over their leaves
  for (int tb = 0; tb < T; tb += 32 * 32) {
    int nacc = 0;  // accepted chunks gathered in this segment
    int tnext = T;
    for (int t0 = tb; t0 < T; t0 += 32) {
      const int t = t0 + lane;
      const int ci = seg_of(cstart, 27, min(t, T - 1));
      const int cg0 = __shfl_sync(FULL, g0, ci), cnch = __shfl_sync(FULL, nch, ci);
      const int cl0 = __shfl_sync(FULL, l0, ci), cl1 = __shfl_sync(FULL, l1, ci);
      const int cs = __shfl_sync(FULL, cstart, ci);
      bool okc = false, tbox = false;
      int la = 0, lb = 0;
      LeafBox cbx = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (t < T) {
        const int k = t - cs;  // chunk number inside cell ci
        la = v.chunk_leaf_start[cg0 + k];
        lb = v.chunk_leaf_start[cg0 + k + 1];
        // (checks build: a chunk whose leaves leave its cell's range is empty)
        if (!(SPH_IN(v.ds, la - cl0, cl1 - cl0 + 1, SPH_CHECK_CELL_LEAVES) &&
              SPH_IN(v.ds, lb - la, CHUNK + 1, SPH_CHECK_CELL_LEAVES) &&
              SPH_IN(v.ds, lb - cl0, cl1 - cl0 + 1, SPH_CHECK_CELL_LEAVES)))
          lb = la;
        // part >= 0: a warp of a cooperating block takes only the chunks
        // whose index is its warp number modulo WARPS_PER_BLOCK
        okc = part < 0 || ((cg0 + k) & (WARPS_PER_BLOCK - 1)) == part;
        if (okc && cl1 - cl0 > CHUNK) {
          const int dxc = ci / 9 - 1, dyc = (ci / 3) % 3 - 1, dzc = ci % 3 - 1;
          okc = chunk_ok(cg0 + k, dxc * F.wf, dyc * F.wf, dzc * F.wf);
          if (okc && reach.chunk_spheres) {
            // (the boxes chunk_ok just read: L1 hits)
            const float4 lo = v.chunk_lo[cg0 + k], hi = v.chunk_hi[cg0 + k];
            const float pad = 1e-5f * F.wf;
            const float sx = dxc * F.wf - reach.fx, sy = dyc * F.wf - reach.fy,
                        sz = dzc * F.wf - reach.fz;
            cbx = LeafBox{lo.x + sx - pad, lo.y + sy - pad, lo.z + sz - pad,
                          hi.x + sx + pad, hi.y + sy + pad, hi.z + sz + pad,
                          reach.grow_own ? lo.w : 0.0f};
            tbox = true;
          }
        }
        (void)cnch;
      }
      if (reach.chunk_spheres && reach.sph) {
        const bool hit = spheres_reach_any(reach.sph, reach.nsph, tbox, cbx, reach.lanes_only);
        if (tbox) okc = hit;
      }
      const unsigned mk = __ballot_sync(FULL, okc);
      const int room = CCAP - nacc;
      if (__popc(mk) > room) {  // this round does not fit: resume from it next segment
        tnext = t0;
        break;
      }
      if (okc) {
        const int pos = nacc + __popc(mk & ((1u << lane) - 1u));
        st.chk[pos] = make_int2(la, (lb - la) | (ci << 16));
      }
      nacc += __popc(mk);
    }
    __syncwarp();
    // phase 3: leaves of the accepted chunks, 32 per round, in order
    int lcount = 0;
    if (lane < nacc) lcount = st.chk[lane].y & 0xffff;
    // (at most 32 chunks per sub-round so that one lane holds each chunk)
    for (int cb = 0; cb < nacc; cb += 32) {
      const int cn = min(32, nacc - cb);
      int2 ch = make_int2(0, 0);
      if (lane < cn) ch = st.chk[cb + lane];
      const int cnt_l = lane < cn ? (ch.y & 0xffff) : 0;
      const int lst = warp_incl_scan(cnt_l) - cnt_l;
      const int L = __shfl_sync(FULL, lst + cnt_l, 31);
      for (int u0 = 0; u0 < L; u0 += 32) {
        const int u = u0 + lane;
        const int cc = seg_of(lst, cn, min(u, L - 1));
        const int cla = __shfl_sync(FULL, ch.x, cc);
        const int cy = __shfl_sync(FULL, ch.y, cc);
        const int cls = __shfl_sync(FULL, lst, cc);
        const int ci = cy >> 16;
        bool ok = false;
        int ja = 0, cnt = 0;
        float sx = 0.f, sy = 0.f, sz = 0.f;
        LeafBox lbox = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (u < L) {
          const int l = cla + (u - cls);
          const int dxc = ci / 9 - 1, dyc = (ci / 3) % 3 - 1, dzc = ci % 3 - 1;
          // every load of the round depends only on l: one memory round trip
          const uint32_t kl = v.leaf_k[l];
          int la = v.leaf_start[l], lb = v.leaf_start[l + 1];
          // (checks build: a leaf whose particle range is out of bounds is empty)
          if (!(SPH_IN(v.ds, la, lb + 1, SPH_CHECK_LEAF) && SPH_IN(v.ds, lb, v.n + 1, SPH_CHECK_LEAF) &&
                SPH_IN(v.ds, lb - la, LEAF_MAX_LIMIT + 1, SPH_CHECK_LEAF)))
            la = lb = 0;
          sx = (float)(dxc * (1 << MORTON_BITS) - F.kx + leaf_kx(kl)) * F.wq;
          sy = (float)(dyc * (1 << MORTON_BITS) - F.ky + leaf_ky(kl)) * F.wq;
          sz = (float)(dzc * (1 << MORTON_BITS) - F.kz + leaf_kz(kl)) * F.wq;
          ok = leaf_ok(l, sx, sy, sz, lbox);
          if (ok) {
            ja = la;
            cnt = lb - la;
          }
        }
        if (reach.sph) ok = spheres_reach_any(reach.sph, reach.nsph, ok, lbox, reach.lanes_only);
        const unsigned mk = __ballot_sync(FULL, ok);
        const int idx = seen + __popc(mk & ((1u << lane) - 1u));
        if (ok && idx >= skip && idx < limit) {
          st.lshift[idx - skip] = make_float4(sx, sy, sz, __int_as_float(ja));
          st.lpack[idx - skip] = cnt | (ci << 16);
        }
        seen += __popc(mk);
        if (seen > limit) {
          more = true;
          __syncwarp();
          return LCAP;
        }
      }
    }
    (void)lcount;
    __syncwarp();
    tb = tnext - 32 * 32;  // continue after the last gathered round
    if (tnext >= T) break;
  }
  __syncwarp();
  return max(0, min(seen - skip, LCAP));
}

// Stages the records of listed leaves [0, nlist) into shared memory by bulk
// copies (TMA), through `depth` buffers of S / depth records (rounded down to
// a multiple of 32) each: the copies
// of the next depth - 1 batches are in flight while a batch is consumed.  A
// batch is as many consecutive listed leaves as fit one buffer.  When a batch
// has landed, each position record is moved into the work group's frame (its
// leaf's corner offset added) and tagged with its particle index and
// neighbour-cell index (TAG; a loop that reads only the positions skips the
// tags); then consume(base, total) sees records base .. base + total - 1.
// Batches are consumed in list order whatever the depth.
// A barrier wait that gives up sets st.failed and counts a timeout; the warp
// then waits (bounded again) for every copy it still has in flight before it
// returns, so that no copy lands in shared memory the warp has left.
template <bool TAG = true, int S, int NREC, int LC, class Consume>
__device__ __forceinline__ void stage_list(const float4 *const *srcs, Stage<S, NREC, LC> &st,
                                           int nlist, Consume consume, WarpCounters &wc) {
  const int lane = lane_id();
  const int depth = st.depth;
  // (a multiple of 32 records per buffer: the tests read whole blocks of 32)
  const int Sb = (S / depth) & ~31;
  int e_next = 0, issued = 0, done = 0;
  // the next listed leaves that fit Sb records, into buffer b
  auto issue = [&](int b) {
    const int e = e_next;
    const bool in = e + lane < nlist;
    const int c = in ? (st.lpack[e + lane] & 0xffff) : 0;
    const int incl = warp_incl_scan(c);
    // a prefix of the list; never empty (a leaf holds at most 32 <= Sb records)
    const unsigned take = __ballot_sync(FULL, in && incl <= Sb);
    const int k = __popc(take);
    const int total = __shfl_sync(FULL, incl, k - 1);
    if (st.stall_ctr) {
      // testing: the first warp of the launch to stage claims the stall
      int claim = 0;
      if (lane == 0) {
        claim = atomicSub(st.stall_ctr, 1) > 0 ? 1 : 0;
        if (!claim) atomicAdd(st.stall_ctr, 1);
      }
      st.stall = __shfl_sync(FULL, claim, 0) != 0;
      st.stall_ctr = nullptr;
    }
    const bool stall = st.stall;
    if (lane == 0) {
      st.meta[3 * b] = e;
      st.meta[3 * b + 1] = k;
      st.meta[3 * b + 2] = total;
      if (!stall) mbar_expect_tx(&st.bar[b], (uint32_t)(total * NREC * (int)sizeof(float4)));
    }
    __syncwarp();
    if (!stall && ((take >> lane) & 1u)) {
      const int ja = __float_as_int(st.lshift[e + lane].w);
      const int slot = b * Sb + incl - c;
      for (int r = 0; r < NREC; r++)
        bulk_g2s(st.rec + (size_t)r * S + slot, srcs[r] + ja, (uint32_t)(c * sizeof(float4)),
                 &st.bar[b]);
    }
    __syncwarp();
    if (lane == 0 && !stall) mbar_arrive(&st.bar[b]);
    e_next = e + k;
    issued++;
  };
  int b = 0, bi = 0;  // next buffer to consume, next buffer to fill
  for (;;) {
    // keep every free buffer filling while listed leaves remain
    while (issued - done < depth && e_next < nlist) {
      issue(bi);
      bi = bi + 1 == depth ? 0 : bi + 1;
    }
    if (done == issued || st.failed) break;
    if (!mbar_wait(&st.bar[b], (st.phase >> b) & 1u, st.wait_limit)) {
      st.failed = true;
      wc.timeout++;
      break;
    }
    st.phase ^= 1u << b;
    const int e = st.meta[3 * b], k = st.meta[3 * b + 1], total = st.meta[3 * b + 2];
    const int base0 = b * Sb;
    int base = base0;
    for (int q = 0; q < k; q++) {
      const float4 sh = st.lshift[e + q];
      const int pk = st.lpack[e + q];
      const int cq = pk & 0xffff;
      const int ja = __float_as_int(sh.w);
      (void)ja;
      for (int t = lane; t < cq; t += 32) {
        float4 rr = st.rec[base + t];
        rr.x += sh.x;
        rr.y += sh.y;
        rr.z += sh.z;
        st.rec[base + t] = rr;
        if constexpr (TAG) {
          st.recj[base + t] = ja + t;
          st.recc[base + t] = (uint8_t)(pk >> 16);
        }
      }
      base += cq;
    }
    __syncwarp();
    consume(base0, total);
    __syncwarp();
    fence_proxy_async();  // this warp's reads of the buffer before the next bulk writes
    done++;
    b = b + 1 == depth ? 0 : b + 1;
  }
  if (st.failed) {
    // copies still in flight: wait for them (bounded) before leaving
    for (; done < issued; done++) {
      if (!st.stall && mbar_wait(&st.bar[b], (st.phase >> b) & 1u, st.wait_limit))
        st.phase ^= 1u << b;
      b = b + 1 == depth ? 0 : b + 1;
    }
    st.stall = false;
  }
  __syncwarp();
}

using StageD = Stage<S_DENS, 1, 320>;
using StageF = Stage<S_FORCE, 3, 256>;

// depth: staging buffers (1..STAGE_DEPTH_MAX, and S / depth >= 32);
// wait_limit: polls of each bounded barrier wait (<= 0: WAIT_LIMIT);
// stall_ctr (testing, normally null): a counter of stalls still to make; the
// first staging of the warp claims one if any is left and then never completes.
template <class St>
__device__ __forceinline__ void stage_init(St &st, int depth = 1, long long wait_limit = 0,
                                           int *stall_ctr = nullptr) {
  extern __shared__ __align__(16) char smem_dyn[];
  const int warp = threadIdx.x >> 5;
  st.carve(smem_dyn + (size_t)warp * St::bytes());
  st.phase = 0u;
  st.failed = false;
  st.depth = depth < 1 ? 1 : (depth > STAGE_DEPTH_MAX ? STAGE_DEPTH_MAX : depth);
  st.wait_limit = wait_limit > 0 ? wait_limit : WAIT_LIMIT;
  st.stall_ctr = stall_ctr;
  st.stall = false;
  if (lane_id() == 0) {
    for (int b = 0; b < STAGE_DEPTH_MAX; b++) mbar_init(&st.bar[b], 1);
    fence_mbar_init();
  }
  __syncwarp();
}

}  // namespace
}  // namespace sph
