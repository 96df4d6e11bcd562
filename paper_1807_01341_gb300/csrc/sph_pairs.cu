// The two neighbour loops of the SPH hot path (Sec. III-A/III-B of
// arXiv 1807.01341): the density loop with the smoothing-length iteration
// (the "ghost" task) and the hydro force loop, for the active particles only.
//
// Work item: one work group -- a run of consecutive leaves (octree sub-cells)
// of one cell holding at most 32 particles, some of them active -- processed
// by one warp.  The warp splits into groups of G lanes;
// each group owns one active particle i, and its lanes stride over the
// candidate particles j.  Candidates come from the 27 top-level cells around
// the leaf's cell: cells holding more than CHUNK leaves are first pruned by
// chunk (CHUNK consecutive leaves) bounding boxes, then leaves by their own
// boxes, 32 boxes per warp ballot.  The records of the accepted leaves
// (contiguous in memory) are staged into shared memory by cp.async.bulk
// (TMA bulk copies) completing on a per-warp mbarrier, a batch at a time, and
// every group of the warp reads the staged batch.
//
// Record positions are relative to each leaf's corner on its cell's 1024^3
// Morton grid; the offset between two leaves is an exact integer number of
// grid steps times w / 1024, so FP32 keeps a relative precision set by the
// leaf size even deep inside clumps.  Both loops add every term to a
// compensated (hi, lo) FP32 pair by Fast2Sum; the G lanes of a group are
// combined in FP64, and the Halley update of h is done in FP64.  The order of every sum
// depends only on the particle, so the plain and batched forms agree bit for
// bit.
//
// The work queue is read either one item per warp (grid sized on the host) or
// by persistent warps pulling items from a device counter (batched form).
#include <cstddef>

#include "sph_pairloop.cuh"

namespace sph {

namespace {

// Cooperative processing of a heavy work group: the 8 warps of a block share
// it, each taking the neighbour chunks with its warp number modulo 8 (so the
// partial sums of a particle depend only on the particle), and combine their
// per-lane partial sums through shared memory in warp order.  The reduction
// area of a warp is the part of its staging buffer that is free between a
// round's last consume and the next search (Stage::red_offset), so the leaf
// list of the group's last search stays valid for its next gather.
template <class St>
__device__ __forceinline__ float *red_area(int warp) {
  extern __shared__ __align__(16) char smem_dyn[];
  static_assert(St::red_bytes() >= 12 * 32 * sizeof(float), "the reduction area holds 12 words");
  return reinterpret_cast<float *>(smem_dyn + (size_t)warp * St::bytes() + St::red_offset());
}

// The largest support of each leaf [L0, L1) of a work group after its
// particles' h changed; the chunk's and the global largest support keep upper
// bounds.  One lane per particle of the group (at most 32), then one warp-wide
// max per leaf (every lane of the warp calls it).
__device__ __forceinline__ void leaf_hmax_update(const View &v, int L0, int L1) {
  const int lane = lane_id();
  const int a = v.leaf_start[L0], b = v.leaf_start[L1];
  const int i = a + lane;
  unsigned hb = 0u;  // support (positive float bits: ordered as unsigned), 0 past the group
  int leaf = -1;
  if (i < b && lane < WG_MAX) {
    hb = __float_as_uint(v.rec_xH[i].w);
    leaf = v.pleaf[i];
  }
  for (int l = L0; l < L1; l++) {
    const float Hm = __uint_as_float(__reduce_max_sync(FULL, leaf == l ? hb : 0u));
    if (lane == 0) {
      reinterpret_cast<float *>(&v.leaf_lo[l])[3] = Hm;
      atomic_max_float_pos(reinterpret_cast<unsigned int *>(&v.chunk_lo[v.leaf_chunk[l]]) + 3, Hm);
      atomic_max_float_pos(&v.ds->Hmax_bits, Hm);
    }
  }
}

// ---------------------------------------------------------------------------
// density loop + smoothing-length iteration for the active particles of a group
// ---------------------------------------------------------------------------
// Sums of one particle: S_w = sum w(q), S_t = sum (3 w + q w'), the
// mass-weighted pair, sum q^2 w'' and the neighbour count.  The first four
// are compensated (hi, lo) pairs: each term goes in by Dekker's Fast2Sum
// (t = hi + x; lo += x - (t - hi); hi = t), whose lo collects the rounding
// error of every addition exactly while |hi| >= |x| (the running sum of a
// particle's terms is, after its first terms, much larger than one term), at
// three adds per term and no branch.  The order and the rounding of every sum
// depend only on the particle's accepted candidates in record order -- not on
// the list entries beyond its support nor on the particles sharing its warp.
// (Partial sums of 8 terms folded into (hi, lo) by a six-add two-sum, the
// form this replaced, cost 8 % more step-0 density time: the fold branch of
// the lane that reached 8 terms was taken by almost every warp at almost
// every entry.)
__device__ __forceinline__ void fast2sum(float &hi, float &lo, float x) {
  const float t = hi + x;
  lo += x - (t - hi);
  hi = t;
}

struct DSum {
  float n_hi, n_lo, t_hi, t_lo, r_hi, r_lo, rt_hi, rt_lo;
  float p2;
  int cnt;
  __device__ __forceinline__ void zero() {
    n_hi = n_lo = t_hi = t_lo = r_hi = r_lo = rt_hi = rt_lo = 0.0f;
    p2 = 0.0f;
    cnt = 0;
  }
};

// A candidate at squared distance r2 (FP32, group frame) with mass mj, at the
// support H (H2 = H^2, Hinv = 1/H): a neighbour when r2 < H2 (strict).  With
// equal masses (UM) the mass-weighted sums are not formed: they are the common
// mass times S_w and S_t.
template <bool UM>
__device__ __forceinline__ void dens_pair(DSum &s, float r2, float mj, float H2, float Hinv) {
  if (!(r2 < H2)) return;
  const float rr = r2 * rsqrtf(fmaxf(r2, 1e-30f));
  const float qq = rr * Hinv;
  float wq, dwq;
  kernel_wd(qq, wq, dwq);
  const float tt = fmaf(qq, dwq, 3.0f * wq);
  s.p2 = fmaf(qq * qq, kernel_d2w(qq), s.p2);
  fast2sum(s.n_hi, s.n_lo, wq);
  fast2sum(s.t_hi, s.t_lo, tt);
  if constexpr (!UM) {
    fast2sum(s.r_hi, s.r_lo, mj * wq);
    fast2sum(s.rt_hi, s.rt_lo, mj * tt);
  }
  s.cnt++;
}

// Entries [0, nl) of a neighbour list (entry k at lst[k * ls]), in order, in
// blocks of LQ: the loads of the next block are issued before the current
// block is evaluated, so a warp running alone (a sparse step) waits for one
// L2 round trip per LQ entries rather than per entry.  The loads may be
// served by L1 (every later h iteration reads the list again): each lane
// reads only entries it wrote itself, and a list area is used by one warp of
// one launch (L1 lines are invalidated between dependent launches).
constexpr int LQ = 4;
constexpr float FIRST_MARGIN = 1.05f;  // search margin of a run's first density pass (at least)
template <bool UM>
__device__ __forceinline__ void dens_list(DSum &s, const float2 *lst, int ls, int nl, float H2,
                                          float Hinv) {
  if (nl <= 0) return;
  float2 e[LQ];
#pragma unroll
  for (int j = 0; j < LQ; j++) e[j] = j < nl ? lst[(size_t)j * ls] : make_float2(INFINITY, 0.0f);
#pragma unroll 1
  for (int k = 0; k < nl; k += LQ) {
    float2 cur[LQ];
#pragma unroll
    for (int j = 0; j < LQ; j++) {
      cur[j] = e[j];
      const int kn = k + LQ + j;
      e[j] = kn < nl ? lst[(size_t)kn * ls] : make_float2(INFINITY, 0.0f);
    }
#pragma unroll
    for (int j = 0; j < LQ; j++) dens_pair<UM>(s, cur[j].x, cur[j].y, H2, Hinv);
  }
}

// The same for a list of squared distances alone (equal masses).
__device__ __forceinline__ void dens_list_r(DSum &s, const float *lst, int ls, int nl, float H2,
                                            float Hinv) {
  if (nl <= 0) return;
  float e[LQ];
#pragma unroll
  for (int j = 0; j < LQ; j++) e[j] = j < nl ? lst[(size_t)j * ls] : INFINITY;
#pragma unroll 1
  for (int k = 0; k < nl; k += LQ) {
    float cur[LQ];
#pragma unroll
    for (int j = 0; j < LQ; j++) {
      cur[j] = e[j];
      const int kn = k + LQ + j;
      e[j] = kn < nl ? lst[(size_t)kn * ls] : INFINITY;
    }
#pragma unroll
    for (int j = 0; j < LQ; j++) dens_pair<true>(s, cur[j], 0.0f, H2, Hinv);
  }
}

// Newton step on F(h) = h^3 n(h) - eta^3 in dimensionless form: with H = GAMMA_K h,
// h^3 n = (8/pi) S_w / GAMMA_K^3 and h dF/dh = 3 h^3 n + h^4 dn/dh, so
// dh / h = -(S_w - C) / (3 S_w - S_t), C = eta^3 GAMMA_K^3 / (8/pi),
// S_w = sum w(q), S_t = sum (3 w + q w').
//
// Gathers and neighbour lists.  A particle's candidates are found by a
// "gather": the search lists the leaves that the particle's sphere of radius
// R_i = search_margin x H reaches, their records are staged, and every record
// with r^2 < R_i^2 goes into the particle's neighbour list (squared distance
// and mass).  Each h iteration evaluates its sums at its H from the list
// alone, in record order, as long as H <= R_i; a particle whose h outgrows
// R_i gathers again.  A list holds list_cap entries per particle (list_cap / G
// per lane): a gather that accepts more runs in passes over the same leaves,
// each pass listing (and summing) the next list_cap accepted records, and the
// particle's list is then not kept (later iterations gather at R_i = H).
// Whatever the capacity, margin or staging depth, a particle's sums visit the
// same pairs in the same order with the same arithmetic.  A work group is
// handled by one warp (sharing it between the warps of a block, as the force
// loop does in sparse steps, was measured slower here: every warp pays the
// search's latency, then waits at the barriers of each h iteration), or, in
// steps with few active groups, split by its active particles into `nslices`
// consecutive slices, each a warp's own work item (slice `slice`): no warp
// waits for another, and a slice's sums are those the whole group would give
// (a particle's candidates and their order do not depend on the particles it
// shares a warp with).  A split group's leaves get their largest support from
// k_leaf_hmax, after every slice is done.
template <int G, bool UM>
__device__ void density_group(const View &v, int wg, int slice, int nslices, int flags,
                              int bin_filter, int m_act, const CellFrame &F, float hcap, float exc,
                              long long ti, StageD &st, WarpCounters &wc) {
  const int lane = lane_id();
  const int warp = threadIdx.x >> 5;
  constexpr int part = -1;       // (every chunk of the neighbour cells)
  constexpr bool writer = true;  // the warp writes its particles' results
  const Group W = group_of(v, wg, F);
  const int a = W.a, b = W.b;
  const int nact = leaf_actives(v, a, b, m_act, bin_filter, st.act);
  if (nact == 0) return;
  // this warp's slice [s0, s1) of the group's active particles
  int s0 = 0, s1 = nact;
  if (nslices > 1) {
    const int per = (nact + nslices - 1) / nslices;
    s0 = min(nact, slice * per);
    s1 = min(nact, s0 + per);
    if (s0 == s1) return;
  }
  constexpr int P = 32 / G;
  const int grp = lane / G, sub = lane % G;
  const unsigned gmask = G == 32 ? FULL : ((1u << G) - 1u) << (grp * G);  // this lane's group
  // the group's box in its cell's frame (for the chunk tests)
  const float qox = F.kx * F.wq, qoy = F.ky * F.wq, qoz = F.kz * F.wq;
  const float clx = W.lx + qox, cly = W.ly + qoy, clz = W.lz + qoz;
  const float chx = W.hx + qox, chy = W.hy + qoy, chz = W.hz + qoz;
  const float ceps = 1e-5f * F.wf;
  const double Cw = v.eta * v.eta * v.eta * GAMMA_K_D * GAMMA_K_D * GAMMA_K_D / (double)KERNEL_NORM;
  const bool init_entropy = (flags & SPH_DENSITY_INIT_ENTROPY) != 0;
  const float4 *srcs[1] = {v.rec_xm};
  // this lane's neighbour list: entry k at lst[k * 32], in the warp's own
  // area (the launch has at most list_blocks blocks)
  const int cap = v.list_cap;
  constexpr int ls = 32;
  float2 *const lst = v.nbr + ((size_t)blockIdx.x * WARPS_PER_BLOCK + warp) * 32 * v.list_cap + lane;
  // (equal masses: the entries are the squared distances alone, in the first
  // half of the warp's area)
  float *const lstr = reinterpret_cast<float *>(v.nbr + ((size_t)blockIdx.x * WARPS_PER_BLOCK + warp) *
                                                             32 * v.list_cap) + lane;

  for (int r = s0; r < s1 && !st.failed; r += P) {
    const int slot = r + grp;
    const bool valid = slot < s1;
    const int i = valid ? st.act[slot] : a;
    const float4 xl = v.rec_xm[i];  // position in its own leaf's frame
    const float3 lo3 = leaf_offset(v, i, F);
    const float4 xi = make_float4(xl.x + lo3.x, xl.y + lo3.y, xl.z + lo3.z, xl.w);
    // the initial guess: the last h, or (prediction) the h the drift predicted
    float h = v.predict ? v.rec_xH[i].w * (1.0f / GAMMA_K) : v.h[i];
    double lo = 0.0, hi = INFINITY;
    bool done = !valid;
    float Ri = 0.0f;         // radius of this lane's neighbour list
    int nl = -1;             // entries of its list (-1: no list valid)
    bool keep = true;        // the list may be kept across iterations (not after it filled up)
    bool have_list = false;  // the shared-memory leaf list is complete for the last search
    int nlist = 0;           // leaves in the shared-memory leaf list
    for (int it = 0; it < v.h_max_iter && !st.failed; it++) {
      const float H = GAMMA_K * h;
      const float Hs = warp_max(done ? 0.0f : H);
      if (Hs == 0.0f) break;  // every particle of the round has converged
      const float H2 = H * H, Hinv = 1.0f / H;
      DSum s;
      s.zero();
      // lanes without a list valid at this H gather (a whole particle's G lanes together)
      const bool need = !done && (nl < 0 || H > Ri);
      if (need) {
        // (the first pass of a run, whose h comes from the initial
        // conditions, gathers a little wider: fewer second gathers, the same
        // sums; 20 steps of the 2.1M clustered set: density -1.3 %)
        const float margin = init_entropy && it == 0 ? fmaxf(v.search_margin, FIRST_MARGIN)
                                                     : v.search_margin;
        Ri = keep ? H * margin : H;
        nl = 0;
      }
      bool gath = need;   // this lane gathers in the current pass
      int skipc = 0;      // accepted records this lane has listed in earlier passes
      bool first = true;
      int nsph = 0;
      float R = 0.0f;
      bool overflowed = false;
      for (;;) {
        int acc = 0;  // records this lane accepted in the pass
        if (__any_sync(FULL, gath)) {
          // every pass of a gather uses the spheres and reach of its first
          // pass, so that all passes stage the same records in the same order
          // (later passes reuse its leaf list when that list was complete)
          const bool search_now = first || !have_list;
          if (first) {
            R = warp_max(gath ? Ri : 0.0f);
            const unsigned gb = __ballot_sync(FULL, gath);
            nsph = compact_spheres(st.sph, sub == 0 && (gb & gmask) != 0u,
                                   make_float4(xi.x, xi.y, xi.z, Ri));
          }
          const float T2 = Ri * Ri;
          int ntst = 32 + 1, my_rank = 0;
          if constexpr (G == 1) {
            const unsigned vm = __ballot_sync(FULL, gath);
            ntst = __popc(vm);
            my_rank = __popc(vm & ((1u << lane) - 1u));
            if (gath) st.tst[my_rank] = make_float4(xi.x, xi.y, xi.z, T2);
            __syncwarp();
          }
          const unsigned nlive = __popc(__ballot_sync(FULL, gath && sub == 0));
          // accept mask of the staged records base+kb .. base+kb+31 for this lane
          // (a staging buffer holds a multiple of 32 records, so the block
          // is read whole and the records past the batch are masked off)
          auto test_block = [&](int base, int total, int kb) -> unsigned {
            unsigned mask = 0u;
            const unsigned bvalid = total - kb >= 32 ? FULL : (1u << (total - kb)) - 1u;
            if (G == 1 && ntst <= TRANSPOSE_MAX) {
              const float4 pj = st.rec[base + kb + lane];
              const float2 px = make_float2(pj.x, pj.x), py = make_float2(pj.y, pj.y),
                           pz = make_float2(pj.z, pj.z);
              int q = 0;
#pragma unroll 2
              for (; q + 1 < ntst; q += 2) {  // two live particles per packed test
                const float4 t0 = st.tst[q], t1 = st.tst[q + 1];
                const float2 r2 = dist2_x2(make_float2(t0.x, t1.x), make_float2(t0.y, t1.y),
                                           make_float2(t0.z, t1.z), px, py, pz);
                const unsigned m0 = __ballot_sync(FULL, r2.x < t0.w);
                const unsigned m1 = __ballot_sync(FULL, r2.y < t1.w);
                if (q == my_rank) mask = m0;
                if (q + 1 == my_rank) mask = m1;
              }
              if (q < ntst) {
                const float4 t = st.tst[q];
                const float dx = t.x - pj.x, dy = t.y - pj.y, dz = t.z - pj.z;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                const unsigned m = __ballot_sync(FULL, r2 < t.w);
                if (q == my_rank) mask = m;
              }
            } else if (G == 1) {
              const float2 xx = make_float2(xi.x, xi.x), yy = make_float2(xi.y, xi.y),
                           zz = make_float2(xi.z, xi.z);
#pragma unroll 4
              for (int u = 0; u < 32; u += 2) {  // two records per packed test
                const float4 p0 = st.rec[base + kb + u];
                const float4 p1 = st.rec[base + kb + u + 1];
                const float2 r2 = dist2_x2(xx, yy, zz, make_float2(p0.x, p1.x),
                                           make_float2(p0.y, p1.y), make_float2(p0.z, p1.z));
                mask |= r2.x < T2 ? (1u << u) : 0u;
                mask |= r2.y < T2 ? (2u << u) : 0u;
              }
            } else {
#pragma unroll
              for (int u = sub; u < 32; u += G) {
                const float4 pj = st.rec[base + kb + u];
                const float dx = xi.x - pj.x, dy = xi.y - pj.y, dz = xi.z - pj.z;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                mask |= r2 < T2 ? (1u << u) : 0u;
              }
            }
            return mask & bvalid;
          };
          // accepted records go into the list (those past the earlier passes' share)
          auto consume = [&](int base, int total) {
            wc.cand += (unsigned long long)total * nlive;
            for (int k0 = 0; k0 < total; k0 += 32) {
              unsigned mask = test_block(base, total, k0);  // (every lane: the test votes)
              if (!gath) mask = 0u;
              // two accepted records per round (independent load-compute-store
              // chains), listed in record order
              while (mask) {
                const int ka = base + k0 + __ffs(mask) - 1;
                mask &= mask - 1;
                const bool two = mask != 0u;
                const int kb = two ? base + k0 + __ffs(mask) - 1 : ka;
                mask &= mask - 1;
                const float4 pa = st.rec[ka], pb = st.rec[kb];
                const int e = acc - skipc;
                if ((unsigned)e < (unsigned)cap) {
                  const float dx = xi.x - pa.x, dy = xi.y - pa.y, dz = xi.z - pa.z;
                  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                  if constexpr (UM) __stcg(lstr + (size_t)e * ls, r2);
                  else __stcg(lst + (size_t)e * ls, make_float2(r2, pa.w));
                }
                if (two && (unsigned)(e + 1) < (unsigned)cap) {
                  const float dx = xi.x - pb.x, dy = xi.y - pb.y, dz = xi.z - pb.z;
                  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                  if constexpr (UM) __stcg(lstr + (size_t)(e + 1) * ls, r2);
                  else __stcg(lst + (size_t)(e + 1) * ls, make_float2(r2, pb.w));
                }
                acc += two ? 2 : 1;
              }
            }
          };
          const float R2 = R * R * 1.0002f, Rc = R + ceps;
          auto leaf_ok = [&](int l, float sx, float sy, float sz, LeafBox &lb) {
            const float4 lo4 = v.leaf_lo[l], hi4 = v.leaf_hi[l];
            lb = leaf_box(lo4, hi4, sx, sy, sz, 0.0f);
            return box_gap2(W.lx, W.ly, W.lz, W.hx, W.hy, W.hz, lo4, hi4, sx, sy, sz) < R2;
          };
          auto chunk_ok = [&](int g, float sx, float sy, float sz) {
            return box_gap2(clx, cly, clz, chx, chy, chz, v.chunk_lo[g], v.chunk_hi[g], sx, sy,
                            sz) < Rc * Rc;
          };
          // (the density loop keeps the per-lane sphere test: at its register
          // limit the transposed form costs more in spills than it saves)
          const Reach reach = {clx, cly, clz, chx, chy, chz, Rc, exc, st.sph, nsph, true,
                               true, qox, qoy, qoz, false};
          int skip = 0;
          bool more = false, complete = true;
          do {
            if (search_now) {
              nlist = search(v, F, reach, st, leaf_ok, chunk_ok, skip, more, part);
              complete = complete && !more;
            }
            stage_list<false>(srcs, st, nlist, consume, wc);  // (positions only: no tags)
            skip += nlist;
          } while (search_now && more && !st.failed);
          if (search_now) have_list = complete;
          if (writer) wc.gathers += nlive;
          if (gath) nl = min(acc - skipc, cap);
        }
        // the list this pass built (or, in the first pass, the one kept from
        // an earlier iteration), in order
        if (!done && (gath || first) && nl > 0) {
          if constexpr (UM) dens_list_r(s, lstr, ls, nl, H2, Hinv);
          else dens_list<false>(s, lst, ls, nl, H2, Hinv);
          if (writer) wc.evals += (unsigned long long)nl;
        }
        // a list that filled up: the next pass lists the records after it (for
        // several lanes per particle, every lane of the particle goes on)
        const unsigned ob = __ballot_sync(FULL, gath && acc > skipc + cap);
        const bool over = gath && (ob & gmask) != 0u;
        if (over) {
          skipc += cap;
          overflowed = true;
          if (sub == 0 && writer) wc.list_overflows++;
        }
        gath = over;
        first = false;
        if (ob == 0u || st.failed) break;
      }
      if (overflowed) {
        keep = false;
        nl = -1;  // the list holds only the last pass's share
      }
      if (st.failed) break;
      const double sn = group_sum<G>((double)s.n_hi + (double)s.n_lo);
      const double stt = group_sum<G>((double)s.t_hi + (double)s.t_lo);
      // (the mass-weighted sums are needed only once h has converged: with
      // one lane per particle they are formed there, in the same arithmetic)
      float sr = 0.0f, srt = 0.0f;
      if constexpr (G > 1) {
        sr = (float)group_sum<G>((double)s.r_hi + (double)s.r_lo);
        srt = (float)group_sum<G>((double)s.rt_hi + (double)s.rt_lo);
      }
      const double s2 = group_sum<G>((double)s.p2);
      const int cnt = group_sum_i<G>(s.cnt) - 1;  // (the particle itself is among its candidates)
      if (!done) {
        // Halley step in FP64 (Newton where its denominator is not positive),
        // kept inside the bracket [lo, hi] (F grows with h).  With
        // g = S_w - C: a = h g' = 3 S_w - S_t, b = h^2 g'' = sum q^2 w'' - 2 a,
        // dh / h = -2 g a / (2 a^2 - g b)
        const double hd = (double)h;
        const double Fr = sn - Cw;              // g, the sign of F(h)
        const double dFr = 3.0 * sn - stt;      // a
        if (Fr < 0.0) lo = hd;
        else hi = hd;
        double hn;
        if (Fr == 0.0) {
          hn = hd;
        } else if (dFr > 0.0) {
          const double den = 2.0 * dFr * dFr - Fr * (s2 - 2.0 * dFr);
          // (Halley, or Newton where its denominator is not positive: one division)
          // (the quotient in FP32: the conversions and the 2-ulp division move
          // the new h by about 4e-7 of the step, far inside the FP64
          // convergence test's tolerance)
          const bool hal = den > 0.0;
          hn = hd - hd * (double)__fdividef((float)(hal ? 2.0 * Fr * dFr : Fr),
                                            (float)(hal ? den : dFr));
        } else {
          hn = NAN;
        }
        if (!(hn >= lo && hn <= hi)) hn = isinf(hi) ? 2.0 * hd : 0.5 * (lo + hi);
        hn = fmin(fmax(hn, 0.5 * hd), 2.0 * hd);
        const bool conv = fabs(hn - hd) <= v.h_tol * hd;
        const bool over = !conv && hn > (double)hcap;
        const bool last = it == v.h_max_iter - 1;
        if (conv || over || last) {
          done = true;
          if constexpr (UM) {
            const double mu = (double)v.ds->m_uniform;
            sr = (float)(mu * sn);
            srt = (float)(mu * stt);
          } else if constexpr (G == 1) {
            sr = (float)((double)s.r_hi + (double)s.r_lo);
            srt = (float)((double)s.rt_hi + (double)s.rt_lo);
          }
          if (sub == 0 && writer) {
            wc.pairs += (unsigned long long)cnt;
            wc.iters += (unsigned long long)(it + 1);
            if (over) {
              wc.overflow++;
              atomic_max_float_pos(&v.ds->want_h_bits, (float)hn);
            } else if (!conv) {
              wc.noconv++;
            }
            // density, grad-h factor f = [1 + h/(3 rho) drho/dh]^-1, equation of state
            const float Hinv3 = Hinv * Hinv * Hinv;
            const float rho = KERNEL_NORM * sr * Hinv3;
            const float f = 3.0f * sr / (3.0f * sr - srt);
            const double dtp =
                ((double)(ti - v.ti_begin[i]) - 0.5 * (double)(v.ti_end[i] - v.ti_begin[i])) *
                v.dt_min;
            float Ap = v.A[i] + v.Adot[i] * (float)dtp;
            const float g = (float)v.gamma;
            if (init_entropy) Ap = (g - 1.0f) * v.A[i] / powf(rho, g - 1.0f);  // A holds u
            const float P = Ap * powf(rho, g);
            const float c = sqrtf(g * P / rho);
            v.h[i] = h;
            v.rho[i] = rho;
            v.f[i] = f;
            v.P[i] = P;
            v.c[i] = c;
            v.rec_xH[i] = make_float4(xl.x, xl.y, xl.z, H);
            v.rec_h[i] = make_float4(rho, f * P / (rho * rho), c, Hinv);
            if (v.ngb_density) v.ngb_density[i] = cnt;
          }
        } else {
          h = (float)hn;
        }
      }
    }
  }
  // largest support of each leaf after the update (a split group's: k_leaf_hmax)
  __syncwarp();
  if (writer && nslices == 1) leaf_hmax_update(v, W.L0, W.L1);
  __syncwarp();
}

// ---------------------------------------------------------------------------
// force loop for the active particles of a group
// ---------------------------------------------------------------------------
// The limiter's request that inactive particle j wake down to bin b (the
// smallest request stands; the first one queues j for the step's close).
__device__ __forceinline__ void request_wake(const View &v, int j, int b) {
  if (atomicMin(&v.wake_bin[j], b) == WAKE_NONE) v.q_wake[atomicAdd(&v.ds->n_wake, 1)] = j;
}

// VAR: the code of the scheme's variants (Balsara switch, neighbour limiter)
// is compiled in; the base scheme runs the instance without it.
template <int G, bool COOP, bool VAR>
__device__ void force_group(const View &v, int wg, int slice, int nslices, int bin_filter, int m_act,
                            const CellFrame &F, float Hmax, float exc, StageF &st,
                            WarpCounters &wc) {
  static_assert(!COOP || G == 1, "cooperative groups use one lane per particle");
  const int lane = lane_id();
  const int warp = threadIdx.x >> 5;
  const int part = COOP ? warp : -1;
  const bool writer = !COOP || warp == 0;
  const Group W = group_of(v, wg, F);
  const int a = W.a, b = W.b;
  const int nact = leaf_actives(v, a, b, m_act, bin_filter, st.act);
  if (nact == 0) return;
  // this warp's slice [s0, s1) of the group's active particles (a split group)
  int s0 = 0, s1 = nact;
  if (nslices > 1) {
    const int per = (nact + nslices - 1) / nslices;
    s0 = min(nact, slice * per);
    s1 = min(nact, s0 + per);
    if (s0 == s1) return;
  }
  constexpr int P = 32 / G;
  const int grp = lane / G, sub = lane % G;
  const float qox = F.kx * F.wq, qoy = F.ky * F.wq, qoz = F.kz * F.wq;
  const float clx = W.lx + qox, cly = W.ly + qoy, clz = W.lz + qoz;
  const float chx = W.hx + qox, chy = W.hy + qoy, chz = W.hz + qoz;
  const float ceps = 1e-5f * F.wf;
  const float alpha = (float)v.alpha;
  const float g = (float)v.gamma;
  const float4 *srcs[3] = {v.rec_xH, v.rec_v, v.rec_h};
  const float4 *sx_rec = st.rec, *sv_rec = st.rec + S_FORCE, *sh_rec = st.rec + 2 * S_FORCE;

  for (int r = s0; r < s1 && !st.failed; r += P) {
    const int slot = r + grp;
    const bool valid = slot < s1;
    const int i = valid ? st.act[slot] : a;
    const float4 xl = v.rec_xH[i];
    const float3 lo3 = leaf_offset(v, i, F);
    const float4 xi = make_float4(xl.x + lo3.x, xl.y + lo3.y, xl.z + lo3.z, xl.w);
    const float4 vi = v.rec_v[i];
    const float4 hi4 = v.rec_h[i];
    const float Hi2 = xi.w * xi.w;
    const float Hinv2 = hi4.w * hi4.w;
    const float nHi4 = KERNEL_NORM * Hinv2 * Hinv2;
    const float Hs = warp_max(valid ? xi.w : 0.0f);
    const int nsph = compact_spheres(st.sph, sub == 0 && valid, make_float4(xi.x, xi.y, xi.z, xi.w));
    float ax_hi = 0.f, ax_lo = 0.f, ay_hi = 0.f, ay_lo = 0.f, az_hi = 0.f, az_lo = 0.f;
    float ad_hi = 0.f, ad_lo = 0.f;
    float vs = 2.0f * hi4.z;
    int cnt = 0;
    int bmin = 127;  // limiter: smallest bin among the neighbours
    const int bi = ((VAR && v.limiter) && valid) ? (int)v.bin[i] : 0;  // limiter: i's bin
    // Balsara factor of i: |div v| / (|div v| + |curl v| + 1e-4 c / h), h = 1 / (GAMMA_K / H)
    float Bi = 1.0f;
    if ((VAR && v.balsara) && valid) {
      const float dv = fabsf(v.div_v[i]);
      Bi = dv / (dv + fabsf(v.curl_v[i]) + 1e-4f * hi4.z * GAMMA_K * hi4.w);
    }
    auto leaf_ok = [&](int l, float sx, float sy, float sz, LeafBox &lb) {
      const float4 loj = v.leaf_lo[l], hij = v.leaf_hi[l];
      const float R = fmaxf(Hs, loj.w);
      lb = leaf_box(loj, hij, sx, sy, sz, loj.w);
      return box_gap2(W.lx, W.ly, W.lz, W.hx, W.hy, W.hz, loj, hij, sx, sy, sz) < R * R * 1.0002f;
    };
    auto chunk_ok = [&](int gg, float sx, float sy, float sz) {
      const float4 loc = v.chunk_lo[gg];
      const float R = fmaxf(Hs, loc.w) + ceps;
      return box_gap2(clx, cly, clz, chx, chy, chz, loc, v.chunk_hi[gg], sx, sy, sz) < R * R;
    };
    // the valid particles of the round, for the transposed candidate test
    int ntst = 32 + 1, my_rank = 0;
    if constexpr (G == 1) {
      const unsigned vm = __ballot_sync(FULL, valid);
      ntst = __popc(vm);
      my_rank = __popc(vm & ((1u << lane) - 1u));
      if (valid) st.tst[my_rank] = make_float4(xi.x, xi.y, xi.z, Hi2);
      __syncwarp();
    }
    const unsigned nlive = __popc(__ballot_sync(FULL, valid && sub == 0));
    // accept mask of the staged records kb .. kb+31 for this lane's particle
    // (each record tested against the batch's end: reading the block whole
    // and masking the tail, as the density loop does, measured slower here)
    auto test_block = [&](int base, int total, int kb) -> unsigned {
      unsigned mask = 0u;
      // (one lane per particle: always the transposed form here -- with its
      // test on the record's support as well, it measured faster than the
      // per-lane form for every count of live particles)
      if (G == 1) {
        const bool in = kb + lane < total;
        const float4 pj = sx_rec[min(base + kb + lane, S_FORCE - 1)];
        const float Hj2 = pj.w * pj.w;
        const float2 px = make_float2(pj.x, pj.x), py = make_float2(pj.y, pj.y),
                     pz = make_float2(pj.z, pj.z);
        int q = 0;
        for (; q + 1 < ntst; q += 2) {  // two valid particles per packed test
          const float4 t0 = st.tst[q], t1 = st.tst[q + 1];
          const float2 r2 = dist2_x2(make_float2(t0.x, t1.x), make_float2(t0.y, t1.y),
                                     make_float2(t0.z, t1.z), px, py, pz);
          const unsigned m0 = __ballot_sync(FULL, in && (r2.x < t0.w || r2.x < Hj2));
          const unsigned m1 = __ballot_sync(FULL, in && (r2.y < t1.w || r2.y < Hj2));
          if (q == my_rank) mask = m0;
          if (q + 1 == my_rank) mask = m1;
        }
        if (q < ntst) {
          const float4 t = st.tst[q];
          const float dx = t.x - pj.x, dy = t.y - pj.y, dz = t.z - pj.z;
          const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          const unsigned m = __ballot_sync(FULL, in && (r2 < t.w || r2 < Hj2));
          if (q == my_rank) mask = m;
        }
      } else {
#pragma unroll
        for (int u = sub; u < 32; u += G) {
          const float4 pj = sx_rec[min(base + kb + u, S_FORCE - 1)];
          const float dx = xi.x - pj.x, dy = xi.y - pj.y, dz = xi.z - pj.z;
          const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          mask |= (kb + u < total && (r2 < Hi2 || r2 < pj.w * pj.w)) ? (1u << u) : 0u;
        }
      }
      return mask;
    };
    auto consume = [&](int base, int total) {
      wc.cand += (unsigned long long)total * nlive;
      // two blocks of 32 records per evaluation round: the lanes' accepted
      // counts even out over 64 records (records still in index order; the
      // density loop, at its register limit, keeps rounds of 32)
      for (int k0 = 0; k0 < total; k0 += 64) {
        // (every lane calls the test, which votes; the second call's
        // condition is the same in all lanes)
        const unsigned m0 = test_block(base, total, k0);
        const unsigned m1 = k0 + 32 < total ? test_block(base, total, k0 + 32) : 0u;
        unsigned long long mask = valid ? ((unsigned long long)m1 << 32) | m0 : 0ull;
        while (mask) {
          // (the particle itself is accepted too: r = 0, it adds nothing but
          // the signal velocity 2 c_i, the start value; one count subtracted below)
          const int k = base + k0 + __ffsll(mask) - 1;
          mask &= mask - 1;
          const float4 pj = sx_rec[k];
          const float4 vj = sv_rec[k];
          const float4 hj = sh_rec[k];
          const float dx = xi.x - pj.x, dy = xi.y - pj.y, dz = xi.z - pj.z;
          const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          cnt++;
          if ((VAR && v.limiter)) {
            const int j = st.recj[k];
            if (j != i) {
              const int bj = v.bin[j];
              bmin = min(bmin, bj);
              // waking: an inactive neighbour on a step more than 4x longer
              if (bj > m_act && bj > bi + 2) request_wake(v, j, bi + 2);
            }
          }
          if (r2 > 0.0f) {
            const float rinv = rsqrtf(r2);
            const float rr = r2 * rinv;
            const float qi = rr * hi4.w, qj = rr * hj.w;
            const float dwi = qi < 1.0f ? kernel_dw(qi) * nHi4 : 0.0f;
            const float hj2 = hj.w * hj.w;
            const float dwj = qj < 1.0f ? kernel_dw(qj) * (KERNEL_NORM * hj2 * hj2) : 0.0f;
            const float dvdr = fmaf(vi.x - vj.x, dx, fmaf(vi.y - vj.y, dy, (vi.z - vj.z) * dz));
            // Monaghan signal-velocity viscosity, beta = 3 (as in Eq. 1)
            const float wij = fminf(0.0f, dvdr * rinv);
            const float vsij = hi4.z + hj.z - 3.0f * wij;
            // (fast division: 2 ulp, the pair term's only divide)
            float Pi = __fdividef(-alpha * vsij * wij, hi4.x + hj.x);
            if ((VAR && v.balsara)) {
              // mean of the pair's Balsara factors (j's from its last density)
              const int j = st.recj[k];
              const float dv = fabsf(v.div_v[j]);
              const float Bj = dv / (dv + fabsf(v.curl_v[j]) + 1e-4f * hj.z * GAMMA_K * hj.w);
              Pi *= 0.5f * (Bi + Bj);
            }
            const float dWb = 0.5f * (dwi + dwj);
            const float sc = vj.w * fmaf(hi4.y, dwi, fmaf(hj.y, dwj, Pi * dWb)) * rinv;
            // (the terms of a cancel in part, so a term can exceed the running
            // sum; that addition then keeps an error of about one unit in the
            // last place of the sum, as a plain FP32 partial sum would)
            fast2sum(ax_hi, ax_lo, -sc * dx);
            fast2sum(ay_hi, ay_lo, -sc * dy);
            fast2sum(az_hi, az_lo, -sc * dz);
            fast2sum(ad_hi, ad_lo, vj.w * Pi * dWb * (dvdr * rinv));
            vs = fmaxf(vs, vsij);
          } else {
            vs = fmaxf(vs, hi4.z + hj.z);
          }
        }
      }
    };
    // a leaf passes only within max(Hs, its own largest H) <= max(Hs, Hmax)
    // (no sphere test on the chunk boxes here: with the neighbours' own supports
    // in the reach it rejects few chunks, and measured slower)
    const Reach reach = {clx, cly, clz, chx, chy, chz, fmaxf(Hs, Hmax) + ceps, exc, st.sph, nsph};
    int skip = 0, nlist = 0;
    bool more = false;
    do {
      nlist = search(v, F, reach, st, leaf_ok, chunk_ok, skip, more, part);
      stage_list<VAR>(srcs, st, nlist, consume, wc);  // (particle tags for the variants only)
      skip += nlist;
    } while (more && !st.failed);
    if (!COOP && st.failed) break;
    double sax, say, saz, sad;
    if constexpr (COOP) {
      // combine the 8 warps' partial sums, in warp order
      float *mine = red_area<StageF>(warp);
      mine[0 * 32 + lane] = ax_hi; mine[1 * 32 + lane] = ax_lo;
      mine[2 * 32 + lane] = ay_hi; mine[3 * 32 + lane] = ay_lo;
      mine[4 * 32 + lane] = az_hi; mine[5 * 32 + lane] = az_lo;
      mine[6 * 32 + lane] = ad_hi; mine[7 * 32 + lane] = ad_lo;
      mine[8 * 32 + lane] = vs;
      reinterpret_cast<int *>(mine)[9 * 32 + lane] = cnt;
      reinterpret_cast<int *>(mine)[10 * 32 + lane] = st.failed ? 1 : 0;
      reinterpret_cast<int *>(mine)[11 * 32 + lane] = bmin;
      __syncthreads();
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      float vm = 0.0f;
      int c = 0, fl = 0, bm = 127;
      for (int w = 0; w < WARPS_PER_BLOCK; w++) {
        const float *rw = red_area<StageF>(w);
        a0 += (double)rw[0 * 32 + lane] + (double)rw[1 * 32 + lane];
        a1 += (double)rw[2 * 32 + lane] + (double)rw[3 * 32 + lane];
        a2 += (double)rw[4 * 32 + lane] + (double)rw[5 * 32 + lane];
        a3 += (double)rw[6 * 32 + lane] + (double)rw[7 * 32 + lane];
        vm = fmaxf(vm, rw[8 * 32 + lane]);
        c += reinterpret_cast<const int *>(rw)[9 * 32 + lane];
        fl |= reinterpret_cast<const int *>(rw)[10 * 32 + lane];
        bm = min(bm, reinterpret_cast<const int *>(rw)[11 * 32 + lane]);
      }
      fl = __any_sync(FULL, fl != 0) ? 1 : 0;
      __syncthreads();
      fence_proxy_async();
      if (fl) st.failed = true;
      if (st.failed) break;  // the same decision in every warp
      sax = a0;
      say = a1;
      saz = a2;
      sad = a3;
      vs = vm;
      cnt = c - 1;
      bmin = bm;
    } else {
      sax = group_sum<G>((double)ax_hi + (double)ax_lo);
      say = group_sum<G>((double)ay_hi + (double)ay_lo);
      saz = group_sum<G>((double)az_hi + (double)az_lo);
      sad = group_sum<G>((double)ad_hi + (double)ad_lo);
      cnt = group_sum_i<G>(cnt) - 1;
      vs = group_max<G>(vs);
      if ((VAR && v.limiter)) {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) bmin = min(bmin, __shfl_xor_sync(FULL, bmin, o));
      }
    }
    if (valid && sub == 0 && writer) {
      wc.pairs += (unsigned long long)cnt;
      v.ax[i] = (float)sax;
      v.ay[i] = (float)say;
      v.az[i] = (float)saz;
      v.Adot[i] = 0.5f * (g - 1.0f) * powf(hi4.x, 1.0f - g) * (float)sad;
      v.vsig[i] = vs;
      if (v.ngb_force) v.ngb_force[i] = cnt;
      if ((VAR && v.limiter)) v.ngb_bin[i] = (int8_t)bmin;
    }
  }
}

// ---------------------------------------------------------------------------
// velocity divergence and curl of the active particles of a group (for the
// variants that use them; after the density loop, at the new h):
//   div v_i  = -(1 / rho_i) sum_j m_j v_ij . grad_i W(r_ij, h_i)
//   curl v_i =  (1 / rho_i) sum_j m_j v_ij x grad_i W(r_ij, h_i)
// with grad_i W = (r_ij / r) dW/dr, over j != i with r_ij < H_i, the step's
// predicted velocities; one lane per particle, the sums folded (compensated)
// at neighbour-cell boundaries in record order.
// ---------------------------------------------------------------------------
__device__ void gradient_group(const View &v, int wg, int m_act, const CellFrame &F, float exc,
                               StageF &st, WarpCounters &wc) {
  const int lane = lane_id();
  const Group W = group_of(v, wg, F);
  const int a = W.a, b = W.b;
  const int nact = leaf_actives(v, a, b, m_act, -1, st.act);
  if (nact == 0) return;
  const float qox = F.kx * F.wq, qoy = F.ky * F.wq, qoz = F.kz * F.wq;
  const float clx = W.lx + qox, cly = W.ly + qoy, clz = W.lz + qoz;
  const float chx = W.hx + qox, chy = W.hy + qoy, chz = W.hz + qoz;
  const float ceps = 1e-5f * F.wf;
  const float4 *srcs[3] = {v.rec_xH, v.rec_v, v.rec_h};
  const float4 *sx_rec = st.rec, *sv_rec = st.rec + S_FORCE;
  const bool valid = lane < nact;  // (a group holds at most 32 particles)
  const int i = valid ? st.act[lane] : a;
  const float4 xl = v.rec_xH[i];
  const float3 lo3 = leaf_offset(v, i, F);
  const float4 xi = make_float4(xl.x + lo3.x, xl.y + lo3.y, xl.z + lo3.z, xl.w);
  const float4 vi = v.rec_v[i];
  const float Hi2 = xi.w * xi.w, Hinv = 1.0f / xi.w;
  const float nHi4 = KERNEL_NORM * Hinv * Hinv * Hinv * Hinv;
  const float Hs = warp_max(valid ? xi.w : 0.0f);
  const int nsph = compact_spheres(st.sph, valid, make_float4(xi.x, xi.y, xi.z, xi.w));
  float d_hi = 0.f, d_lo = 0.f, x_hi = 0.f, x_lo = 0.f, y_hi = 0.f, y_lo = 0.f, z_hi = 0.f,
        z_lo = 0.f;
  float pd = 0.f, px = 0.f, py = 0.f, pz = 0.f;
  int cur = -1;
  auto consume = [&](int base, int total) {
    wc.cand += (unsigned long long)total * (unsigned long long)nact;
    for (int k0 = 0; k0 < total; k0 += 32) {
      unsigned mask = 0u;
      for (int u = 0; u < 32; u++) {
        const float4 pj = sx_rec[min(base + k0 + u, S_FORCE - 1)];
        const float dx = xi.x - pj.x, dy = xi.y - pj.y, dz = xi.z - pj.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        mask |= (k0 + u < total && r2 < Hi2) ? (1u << u) : 0u;
      }
      if (!valid) mask = 0u;
      while (mask) {
        const int k = base + k0 + __ffs(mask) - 1;
        mask &= mask - 1;
        const int ci = st.recc[k];
        if (ci != cur) {
          fold(d_hi, d_lo, pd);
          fold(x_hi, x_lo, px);
          fold(y_hi, y_lo, py);
          fold(z_hi, z_lo, pz);
          pd = px = py = pz = 0.f;
          cur = ci;
        }
        const float4 pj = sx_rec[k];
        const float4 vj = sv_rec[k];
        const float dx = xi.x - pj.x, dy = xi.y - pj.y, dz = xi.z - pj.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (r2 > 0.0f) {  // (the particle itself and coincident ones add nothing)
          const float rinv = rsqrtf(r2);
          const float g1 = vj.w * kernel_dw(r2 * rinv * Hinv) * nHi4 * rinv;
          const float wx = vi.x - vj.x, wy = vi.y - vj.y, wz = vi.z - vj.z;
          pd = fmaf(fmaf(wx, dx, fmaf(wy, dy, wz * dz)), g1, pd);
          px = fmaf(fmaf(wy, dz, -wz * dy), g1, px);
          py = fmaf(fmaf(wz, dx, -wx * dz), g1, py);
          pz = fmaf(fmaf(wx, dy, -wy * dx), g1, pz);
        }
      }
    }
  };
  const float R2 = Hs * Hs * 1.0002f, Rc = Hs + ceps;
  auto leaf_ok = [&](int l, float sx, float sy, float sz, LeafBox &lb) {
    const float4 lo4 = v.leaf_lo[l], hi4 = v.leaf_hi[l];
    lb = leaf_box(lo4, hi4, sx, sy, sz, 0.0f);
    return box_gap2(W.lx, W.ly, W.lz, W.hx, W.hy, W.hz, lo4, hi4, sx, sy, sz) < R2;
  };
  auto chunk_ok = [&](int g, float sx, float sy, float sz) {
    return box_gap2(clx, cly, clz, chx, chy, chz, v.chunk_lo[g], v.chunk_hi[g], sx, sy, sz) <
           Rc * Rc;
  };
  const Reach reach = {clx, cly, clz, chx, chy, chz, Rc, exc, st.sph, nsph, true};
  int skip = 0;
  bool more = false;
  do {
    const int nlist = search(v, F, reach, st, leaf_ok, chunk_ok, skip, more);
    stage_list(srcs, st, nlist, consume, wc);
    skip += nlist;
  } while (more && !st.failed);
  if (st.failed) return;
  fold(d_hi, d_lo, pd);
  fold(x_hi, x_lo, px);
  fold(y_hi, y_lo, py);
  fold(z_hi, z_lo, pz);
  if (valid) {
    const float rho = v.rec_h[i].x;  // this step's density
    const float cx = x_hi + x_lo, cy = y_hi + y_lo, cz = z_hi + z_lo;
    v.div_v[i] = -(d_hi + d_lo) / rho;
    v.curl_v[i] = sqrtf(fmaf(cx, cx, fmaf(cy, cy, cz * cz))) / rho;
  }
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// The work of a force launch: `ncoop` work groups processed by whole blocks
// (one lane per particle, in steps with few active groups: all of them), or
// `nwarp` groups one warp each (heavy ones first).  Batched form: the step's
// active groups; plain form: the groups of one bin (q_bin: those of the
// shared form at its back).
struct Queues {
  int ncoop, nwarp;
};

template <int G>
__device__ __forceinline__ Queues queues(const View &v, const DevState *ds, int bin_filter) {
  if (bin_filter >= 0) return {ds->n_bin_coop, ds->n_bin_groups};
  if (G == 1 && all_coop(v, ds)) return {ds->n_active_groups + ds->n_heavy_groups, 0};
  return {0, ds->n_active_groups + ds->n_heavy_groups};
}

// Plain (per-bin) launches: blocks that take the shared groups (each with its
// own neighbour-list slot), the rest of the grid one group per warp.
template <int G>
__device__ __forceinline__ int coop_blocks(const View &v, const Queues &qs) {
  return G == 1 ? min(qs.ncoop, v.list_blocks) : 0;
}

__device__ __forceinline__ int coop_group(const View &v, const DevState *ds, int bin_filter, int k) {
  if (bin_filter >= 0) return v.q_bin[ds->n_groups - 1 - k];
  return active_group(v, ds, k);
}

template <int G>
__device__ __forceinline__ int warp_group(const View &v, const DevState *ds, int bin_filter, int k) {
  if (bin_filter >= 0) return v.q_bin[k];
  return active_group(v, ds, k);
}
__device__ __forceinline__ void flush_counters(DevState *ds, WarpCounters &wc, bool density) {
  // pairs and iterations are held by group leaders; sum over the warp
  unsigned long long p = wc.pairs, it = wc.iters, nc = wc.noconv, ov = wc.overflow;
  unsigned long long lo = wc.list_overflows, ev = wc.evals;
  for (int o = 16; o; o >>= 1) {
    p += __shfl_xor_sync(FULL, p, o);
    it += __shfl_xor_sync(FULL, it, o);
    nc += __shfl_xor_sync(FULL, nc, o);
    ov += __shfl_xor_sync(FULL, ov, o);
    lo += __shfl_xor_sync(FULL, lo, o);
    ev += __shfl_xor_sync(FULL, ev, o);
  }
  // candidates, gathers and timeouts are warp-uniform (every lane counted the same)
  if (lane_id() == 0) {
    if (density) {
      if (p) atomicAdd(&ds->s_pairs_density, p);
      if (wc.cand) atomicAdd(&ds->s_cand_density, wc.cand);
      if (it) atomicAdd(&ds->s_iters_density, it);
      if (wc.gathers) atomicAdd(&ds->s_gathers_density, wc.gathers);
      if (lo) atomicAdd(&ds->s_list_overflows, lo);
      if (ev) atomicAdd(&ds->s_evals_density, ev);
      if (nc) record_error(ds, SPH_ERR_H_NOCONV, nc, false);
      if (ov) record_error(ds, SPH_ERR_CELL_OVERFLOW, ov, true);
    } else {
      if (p) atomicAdd(&ds->s_pairs_force, p);
      if (wc.cand) atomicAdd(&ds->s_cand_force, wc.cand);
    }
    if (wc.timeout) record_error(ds, SPH_ERR_TIMEOUT, wc.timeout, true);
  }
}


// The work of a density launch: every work group, one per warp.  Per-bin
// launches take the bin's groups (q_bin: those at the front, then those kept
// at the back for the force loop's shared groups); whole-step launches take
// the active queue (heavy groups first).
__device__ __forceinline__ int density_count(const DevState *ds, int bin_filter) {
  return bin_filter >= 0 ? ds->n_bin_groups + ds->n_bin_coop
                         : ds->n_active_groups + ds->n_heavy_groups;
}
__device__ __forceinline__ int density_item(const View &v, const DevState *ds, int bin_filter,
                                            int k) {
  if (bin_filter >= 0) {
    const int nl = ds->n_bin_groups;
    return k < nl ? v.q_bin[k] : v.q_bin[ds->n_groups - 1 - (k - nl)];
  }
  return active_group(v, ds, k);
}

// Work groups are split into at most SPLIT_MAX slices of their active
// particles, each taken by its own warp, when a whole-step launch (one lane
// per particle) has at least twice as many warps as active groups: the
// slices fill the warps that would otherwise idle, and a step's time is that
// of its slowest work item.
constexpr int SPLIT_MAX = 16;
__device__ __forceinline__ int split_parts(int nq, int nwarps) {
  return nq > 0 ? max(1, min(SPLIT_MAX, nwarps / nq)) : 1;
}

// Testing (a library built with SPH_CHECKS; sph_params.test_bad_group): the
// first test_bad_group claims replace the work group taken from the queue by
// an index past the last group, which the SPH_CHECK_GROUP check catches.
__device__ __forceinline__ int planted_group(DevState *ds, int wg) {
#ifdef SPH_CHECKS
  if (ds->test_bad_group > 0 && atomicSub(&ds->test_bad_group, 1) > 0) return ds->n_groups + 7;
#else
  (void)ds;
#endif
  return wg;
}

template <int G, bool UM>
__global__ void __launch_bounds__(PT, 2) k_density(View v, int flags, int bin_filter, int persistent) {
  DevState *ds = v.ds;
  const int warp = threadIdx.x >> 5, lane = lane_id();
  // every support must stay inside the 27 cells around its particle's cell:
  // H + 2 (largest excursion of a particle out of its cell) <= cell width.
  // Thread 0 reads the device state once for the block, so that every warp
  // of a block takes the same decisions (its warps meet at block barriers).
  __shared__ int s_go, s_stall;
  __shared__ float s_exc;
  const double w = ds->w;
  if (threadIdx.x == 0) {
    const float exc0 = __uint_as_float(ds->excursion_bits);
    const float Hmax0 = __uint_as_float(ds->Hmax_bits);
    int go = ds->halt ? 0 : 1;
    if (go && (double)Hmax0 + 2.0 * (double)exc0 > w) {
      record_error(ds, SPH_ERR_CELL_OVERFLOW, 1, true);
      go = 0;
    }
    s_go = go;
    s_exc = exc0;
    // testing (sph_params.test_stall): while stalls are left, the launch's
    // first warp to stage claims one
    s_stall = go && ds->test_stall > 0 ? 1 : 0;
  }
  __syncthreads();
  if (!s_go) return;
  const float exc = s_exc;
  StageD st;
  stage_init(st, v.stage_depth, v.wait_limit, s_stall ? &ds->test_stall : nullptr);
  const float hcap = (float)((w - 2.0 * (double)exc) / GAMMA_K_D * (1.0 - 1e-6));
  const int m_act = ds->m_act;
  const long long ti = ds->ti;
  const int nq = density_count(ds, bin_filter);
  // whole-step persistent launches split the groups of sparse steps (their
  // leaves' largest supports then come from k_leaf_hmax, which reads nparts)
  const int nparts = (G == 1 && bin_filter < 0 && persistent)
                         ? split_parts(nq, (int)gridDim.x * WARPS_PER_BLOCK) : 1;
  if (bin_filter < 0 && blockIdx.x == 0 && threadIdx.x == 0) ds->dens_split = nparts;
  const int nitems = nq * nparts;
  WarpCounters wc = {0, 0, 0, 0, 0, 0};
  // every work item one per warp: pulled from a head (persistent) or by index
  // (one call site of the loop keeps the kernel's code small)
  for (int k = 0;; k++) {
    int item;
    if (persistent) {
      item = 0;
      if (lane == 0) item = atomicAdd(&ds->head_density, 1);
      item = __shfl_sync(FULL, item, 0);
    } else {
      item = k == 0 ? (int)blockIdx.x * WARPS_PER_BLOCK + warp : nitems;
    }
    if (item >= nitems || st.failed) break;
    const int q = item / nparts;
    int wg = density_item(v, ds, bin_filter, q);
    if (lane == 0) wg = planted_group(ds, wg);
    wg = __shfl_sync(FULL, wg, 0);
    if (!SPH_IN(ds, wg, ds->n_groups, SPH_CHECK_GROUP)) break;
    density_group<G, UM>(v, wg, item - q * nparts, nparts, flags, bin_filter, m_act,
                         frame_of(v, ds, wg), hcap, exc, ti, st, wc);
  }
  flush_counters(ds, wc, true);
}

template <int G, bool VAR>
__global__ void __launch_bounds__(PT, 2) k_force(View v, int bin_filter, int persistent) {
  DevState *ds = v.ds;
  const int warp = threadIdx.x >> 5, lane = lane_id();
  // one read of the device state per block (its warps meet at block barriers)
  __shared__ int s_go;
  __shared__ float s_Hmax, s_exc;
  if (threadIdx.x == 0) {
    s_go = ds->halt ? 0 : 1;
    s_Hmax = __uint_as_float(ds->Hmax_bits);
    s_exc = __uint_as_float(ds->excursion_bits);
  }
  __syncthreads();
  if (!s_go) return;
  StageF st;
  stage_init(st, v.stage_depth, v.wait_limit);
  const int m_act = ds->m_act;
  const float Hmax = s_Hmax;
  const float exc = s_exc;
  const Queues qs = queues<G>(v, ds, bin_filter);
  WarpCounters wc = {0, 0, 0, 0, 0, 0};
  const int cb = coop_blocks<G>(v, qs);
  if constexpr (G == 1) {
    if (persistent || (int)blockIdx.x < cb) {
      // (whole-step persistent launches split the shared groups too when
      // blocks outnumber them: each slice is one block's work item)
      const int nparts = (bin_filter < 0 && persistent) ? split_parts(qs.ncoop, (int)gridDim.x) : 1;
      const int nitems = qs.ncoop * nparts;
      __shared__ int s_item;
      for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&ds->head_coop_force, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= nitems || st.failed) break;
        const int q = item / nparts;
        const int wg = coop_group(v, ds, bin_filter, q);
        if (!SPH_IN(ds, wg, ds->n_groups, SPH_CHECK_GROUP)) break;
        force_group<1, true, VAR>(v, wg, item - q * nparts, nparts, bin_filter, m_act,
                                  frame_of(v, ds, wg), Hmax, exc, st, wc);
      }
    }
  }
  if (persistent || (int)blockIdx.x >= cb) {
    // (whole-step persistent launches split the groups when warps outnumber
    // them, as the density loop does)
    const int nparts = (G == 1 && bin_filter < 0 && persistent)
                           ? split_parts(qs.nwarp, (int)gridDim.x * WARPS_PER_BLOCK) : 1;
    const int nitems = qs.nwarp * nparts;
    for (int k = 0;; k++) {
      int item;
      if (persistent) {
        item = 0;
        if (lane == 0) item = atomicAdd(&ds->head_force, 1);
        item = __shfl_sync(FULL, item, 0);
      } else {
        item = k == 0 ? ((int)blockIdx.x - cb) * WARPS_PER_BLOCK + warp : nitems;
      }
      if (item >= nitems || st.failed) break;
      const int q = item / nparts;
      const int wg = warp_group<G>(v, ds, bin_filter, q);
      if (!SPH_IN(ds, wg, ds->n_groups, SPH_CHECK_GROUP)) break;
      force_group<G, false, VAR>(v, wg, item - q * nparts, nparts, bin_filter, m_act,
                                 frame_of(v, ds, wg), Hmax, exc, st, wc);
    }
  }
  flush_counters(ds, wc, false);
}

// The largest support of the leaves of every work group that the last
// whole-step density launch split (one warp per group; nothing when it split
// none).
__global__ void __launch_bounds__(PT) k_leaf_hmax(View v) {
  DevState *ds = v.ds;
  if (ds->halt || ds->dens_split <= 1) return;
  const int nq = ds->n_active_groups + ds->n_heavy_groups;
  const int nw = (int)(gridDim.x * blockDim.x) >> 5;
  for (int k = (int)(blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < nq; k += nw) {
    const int wg = active_group(v, ds, k);
    if (!SPH_IN(ds, wg, ds->n_groups, SPH_CHECK_GROUP)) break;
    const int L0 = v.group_leaf0[wg], L1 = v.group_leaf0[wg + 1];
    // (checks build: a leaf range out of bounds is skipped, as group_of does)
    if (!(SPH_IN(ds, L0, L1, SPH_CHECK_GROUP_LEAVES) &&
          SPH_IN(ds, L1 - 1, ds->n_leaves, SPH_CHECK_GROUP_LEAVES) &&
          SPH_IN(ds, L1 - L0 - 1, WG_MAX, SPH_CHECK_GROUP_LEAVES)))
      continue;
    leaf_hmax_update(v, L0, L1);
  }
}

// Velocity divergence and curl of the step's active particles: persistent
// warps, one work group each, pulled from head_grad.
__global__ void __launch_bounds__(PT, 2) k_gradient(View v) {
  DevState *ds = v.ds;
  __shared__ int s_go;
  __shared__ float s_exc;
  if (threadIdx.x == 0) {
    s_go = ds->halt ? 0 : 1;
    s_exc = __uint_as_float(ds->excursion_bits);
  }
  __syncthreads();
  if (!s_go) return;
  StageF st;
  stage_init(st, v.stage_depth, v.wait_limit);
  const int lane = lane_id();
  const int m_act = ds->m_act;
  const int nq = ds->n_active_groups + ds->n_heavy_groups;
  WarpCounters wc = {0, 0, 0, 0, 0, 0};
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(&ds->head_grad, 1);
    item = __shfl_sync(FULL, item, 0);
    if (item >= nq || st.failed) break;
    const int wg = active_group(v, ds, item);
    if (!SPH_IN(ds, wg, ds->n_groups, SPH_CHECK_GROUP)) break;
    gradient_group(v, wg, m_act, frame_of(v, ds, wg), s_exc, st, wc);
  }
  if (lane == 0 && wc.timeout) record_error(ds, SPH_ERR_TIMEOUT, wc.timeout, true);
}

// Estimated cost of each work group: the particles in the leaves (in cells of
// more than CHUNK leaves: in the leaf chunks) that a box around the group,
// grown by the largest support among its particles, reaches.  One warp per
// group; the search lists nothing, its tests only count.  The sum over all
// groups goes to group_cost_sum (the mark kernel compares each group with the
// mean).
__global__ void __launch_bounds__(PT, 2) k_group_cost(View v) {
  DevState *ds = v.ds;
  StageD st;
  stage_init(st);
  const int lane = lane_id();
  const int ng = ds->n_groups;
  const int nwarps = gridDim.x * WARPS_PER_BLOCK;
  for (int g = blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5); g < ng; g += nwarps) {
    const CellFrame F = frame_of(v, ds, g);
    const Group W = group_of(v, g, F);
    const int i = W.a + lane;  // a work group holds at most 32 particles
    const float Hl = i < W.b ? GAMMA_K * v.h[i] : 0.0f;
    const float R = warp_max(Hl);
    const float qox = F.kx * F.wq, qoy = F.ky * F.wq, qoz = F.kz * F.wq;
    const float clx = W.lx + qox, cly = W.ly + qoy, clz = W.lz + qoz;
    const float chx = W.hx + qox, chy = W.hy + qoy, chz = W.hz + qoz;
    const float Rc = R + 1e-5f * F.wf;
    long long count = 0;
    auto leaf_ok = [&](int l, float sx, float sy, float sz, LeafBox &) {
      if (box_gap2(W.lx, W.ly, W.lz, W.hx, W.hy, W.hz, v.leaf_lo[l], v.leaf_hi[l], sx, sy, sz) <
          R * R * 1.0002f)
        count += v.leaf_start[l + 1] - v.leaf_start[l];
      return false;
    };
    auto chunk_ok = [&](int c, float sx, float sy, float sz) {
      if (box_gap2(clx, cly, clz, chx, chy, chz, v.chunk_lo[c], v.chunk_hi[c], sx, sy, sz) < Rc * Rc) {
        count += v.leaf_start[v.chunk_leaf_start[c + 1]] - v.leaf_start[v.chunk_leaf_start[c]];
      }
      return false;
    };
    bool more = false;
    const Reach reach = {clx, cly, clz, chx, chy, chz, Rc, __uint_as_float(ds->excursion_bits),
                         nullptr, 0};
    search(v, F, reach, st, leaf_ok, chunk_ok, 0, more);
    for (int o = 16; o; o >>= 1) count += __shfl_xor_sync(FULL, count, o);
    if (lane == 0) {
      const int c = (int)min(count, (long long)0x7fffffff);
      v.group_cost[g] = c;
      atomicAdd(&ds->group_cost_sum, (unsigned long long)c);
    }
    __syncwarp();
  }
}

// Entropy from the initial internal energy (A holds u before the first
// density pass): A = (gamma - 1) u / rho^(gamma - 1), for the active particles.
__global__ void k_entropy_from_u(View v) {
  DevState *ds = v.ds;
  if (ds->halt) return;
  const int nq = ds->n_active_leaves, m_act = ds->m_act;
  const float g = (float)v.gamma;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < nq; k += nw) {
    const int leaf = v.q_active[k];
    if (!SPH_IN(ds, leaf, ds->n_leaves, SPH_CHECK_ACTIVE_LEAF)) continue;
    const int a = v.leaf_start[leaf], b = v.leaf_start[leaf + 1];
    for (int i = a + lane_id(); i < b; i += 32)
      if ((int)v.bin[i] <= m_act) v.A[i] = (g - 1.0f) * v.A[i] / powf(v.rho[i], g - 1.0f);
  }
}

constexpr size_t DENS_SMEM = StageD::bytes() * WARPS_PER_BLOCK;
constexpr size_t FORCE_SMEM = StageF::bytes() * WARPS_PER_BLOCK;

template <int G>
cudaError_t density_g(const View &v, int flags, int bin_filter, bool persistent, int grid,
                      cudaStream_t st) {
  if constexpr (G == 1) {
    if (v.uniform_mass)
      k_density<1, true><<<grid, PT, DENS_SMEM, st>>>(v, flags, bin_filter, persistent ? 1 : 0);
    else
      k_density<1, false><<<grid, PT, DENS_SMEM, st>>>(v, flags, bin_filter, persistent ? 1 : 0);
  } else {
    k_density<G, false><<<grid, PT, DENS_SMEM, st>>>(v, flags, bin_filter, persistent ? 1 : 0);
  }
  cudaError_t e = cudaGetLastError();
  // after a whole-step launch: the leaves of the groups it split
  if (e == cudaSuccess && G == 1 && bin_filter < 0 && persistent) {
    note_launches(1);
    k_leaf_hmax<<<v.grid_util / 2 > 0 ? v.grid_util / 2 : 1, PT, 0, st>>>(v);
    e = cudaGetLastError();
  }
  return e;
}

template <int G>
cudaError_t force_g(const View &v, int bin_filter, bool persistent, int grid, cudaStream_t st) {
  if (G == 1 && (v.balsara || v.limiter))
    k_force<1, true><<<grid, PT, FORCE_SMEM, st>>>(v, bin_filter, persistent ? 1 : 0);
  else
    k_force<G, false><<<grid, PT, FORCE_SMEM, st>>>(v, bin_filter, persistent ? 1 : 0);
  return cudaGetLastError();
}

template <int G>
int blocks_per_sm_g(bool density) {
  const void *fn = density ? (const void *)k_density<G, false> : (const void *)k_force<G, false>;
  const size_t smem = density ? DENS_SMEM : FORCE_SMEM;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (density && G == 1) {
    // the equal-mass instance uses the same staging area
    if (cudaFuncSetAttribute((const void *)k_density<1, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
  }
  if (!density && G == 1) {
    // the force kernel with the variants' code and the gradient kernel use the
    // same staging area (set here, at context creation, outside any capture)
    if (cudaFuncSetAttribute((const void *)k_force<1, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute((const void *)k_gradient, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, PT, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

}  // namespace

// grid: number of blocks (persistent: a multiple of the SM count; otherwise
// ceil(queue length / WARPS_PER_BLOCK))
cudaError_t launch_density(const View &v, int flags, int bin_filter, bool persistent, int grid,
                           cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  note_launches(1);
  switch (v.G) {
    case 1: return density_g<1>(v, flags, bin_filter, persistent, grid, st);
    case 2: return density_g<2>(v, flags, bin_filter, persistent, grid, st);
    case 4: return density_g<4>(v, flags, bin_filter, persistent, grid, st);
    case 8: return density_g<8>(v, flags, bin_filter, persistent, grid, st);
    case 16: return density_g<16>(v, flags, bin_filter, persistent, grid, st);
    case 32: return density_g<32>(v, flags, bin_filter, persistent, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_force(const View &v, int bin_filter, bool persistent, int grid,
                         cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  note_launches(1);
  switch (v.G) {
    case 1: return force_g<1>(v, bin_filter, persistent, grid, st);
    case 2: return force_g<2>(v, bin_filter, persistent, grid, st);
    case 4: return force_g<4>(v, bin_filter, persistent, grid, st);
    case 8: return force_g<8>(v, bin_filter, persistent, grid, st);
    case 16: return force_g<16>(v, bin_filter, persistent, grid, st);
    case 32: return force_g<32>(v, bin_filter, persistent, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

// Sets the dynamic shared-memory limit of the pair kernels for this G and
// returns the resident blocks per SM (0 when the configuration cannot run).
int persistent_blocks_per_sm(int G, bool density) {
  switch (G) {
    case 1: return blocks_per_sm_g<1>(density);
    case 2: return blocks_per_sm_g<2>(density);
    case 4: return blocks_per_sm_g<4>(density);
    case 8: return blocks_per_sm_g<8>(density);
    case 16: return blocks_per_sm_g<16>(density);
    case 32: return blocks_per_sm_g<32>(density);
    default: return 0;
  }
}

cudaError_t launch_group_cost(const View &v, int grid, cudaStream_t st) {
  note_launches(1);
  cudaError_t e = cudaFuncSetAttribute(k_group_cost, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)DENS_SMEM);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(SPH_DS_FIELD(v.ds, group_cost_sum), 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  k_group_cost<<<grid, PT, DENS_SMEM, st>>>(v);
  return cudaGetLastError();
}

cudaError_t launch_gradient(const View &v, int grid, cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  note_launches(1);
  k_gradient<<<grid, PT, FORCE_SMEM, st>>>(v);
  return cudaGetLastError();
}

cudaError_t launch_entropy_from_u(const View &v, cudaStream_t st) {
  note_launches(1);
  k_entropy_from_u<<<v.grid_util, 256, 0, st>>>(v);
  return cudaGetLastError();
}

}  // namespace sph
