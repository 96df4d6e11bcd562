// The two neighbour loops of the SPH hot path (Sec. III-A/III-B of
// arXiv 1807.01341): the density loop with the smoothing-length iteration
// (the "ghost" task) and the hydro force loop, for the active particles only.
//
// Work item: one leaf (octree sub-cell of <= 64 particles) that holds active
// particles, processed by one warp.  The warp splits into groups of G lanes;
// each group owns one active particle i and its lanes stride over the
// candidate particles j of every neighbour leaf whose bounding box comes
// within the search radius of the leaf's bounding box.  Neighbour leaves are
// found in the 27 top-level cells around the leaf's cell; their bounding boxes
// are tested 32 at a time with a warp ballot.  Pair arithmetic is FP32 on
// cell-relative coordinates (the periodic shift of a neighbour cell is a
// multiple of the cell width applied once per cell); per-cell partial sums are
// folded into compensated (hi, lo) accumulators, the G lanes of a group are
// combined in FP64, and the Newton update of h is done in FP64.
//
// The work queue is read either one item per warp (grid sized on the host) or
// by persistent warps pulling items from a device counter (batched form).
#include <cstddef>

#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int PT = WARPS_PER_BLOCK * 32;

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

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

__device__ __forceinline__ float warp_max(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(FULL, x, o));
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

// squared gap between leaf i's box and leaf j's box shifted by s
__device__ __forceinline__ float box_gap2(const float4 &loi, const float4 &hii, const float4 &loj,
                                          const float4 &hij, float sx, float sy, float sz) {
  float gx = fmaxf(0.0f, fmaxf(loj.x + sx - hii.x, loi.x - (hij.x + sx)));
  float gy = fmaxf(0.0f, fmaxf(loj.y + sy - hii.y, loi.y - (hij.y + sy)));
  float gz = fmaxf(0.0f, fmaxf(loj.z + sz - hii.z, loi.z - (hij.z + sz)));
  return gx * gx + gy * gy + gz * gz;
}

// Cubic spline: w(q) / (8/pi) and q w'(q) / (8/pi)-weighted derivative, q in [0, 1)
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

__device__ __forceinline__ float kernel_dw(float q) {
  const float s = 1.0f - q;
  const float da = q * fmaf(18.0f, q, -12.0f);
  const float db = -6.0f * s * s;
  return q < 0.5f ? da : db;
}

struct CellFrame {
  int cx, cy, cz, nc;
  float wf;
};

__device__ __forceinline__ int neighbour_cell(const CellFrame &F, int dx, int dy, int dz) {
  return (wrap_cell(F.cx + dx, F.nc) * F.nc + wrap_cell(F.cy + dy, F.nc)) * F.nc +
         wrap_cell(F.cz + dz, F.nc);
}

// ---------------------------------------------------------------------------
// density loop + smoothing-length iteration for the active particles of a leaf
// ---------------------------------------------------------------------------
struct WarpCounters {
  unsigned long long pairs, cand, iters, noconv, overflow;
};

template <int G>
__device__ void density_leaf(const View &v, int leaf, int flags, int bin_filter, int m_act,
                             const CellFrame &F, float hcap, long long ti, int *s_act,
                             WarpCounters &wc) {
  const int lane = lane_id();
  const int a = v.leaf_start[leaf], b = v.leaf_start[leaf + 1];
  const int nact = leaf_actives(v, a, b, m_act, bin_filter, s_act);
  if (nact == 0) return;
  constexpr int P = 32 / G;
  const int grp = lane / G, sub = lane % G;
  const float4 blo = v.leaf_lo[leaf], bhi = v.leaf_hi[leaf];
  const double eta3 = v.eta * v.eta * v.eta;
  const bool init_entropy = (flags & SPH_DENSITY_INIT_ENTROPY) != 0;

  for (int r = 0; r < nact; r += P) {
    const int slot = r + grp;
    const bool valid = slot < nact;
    const int i = valid ? s_act[slot] : a;
    const float4 xi = v.rec_xm[i];
    float h = v.h[i];
    double lo = 0.0, hi = INFINITY;
    bool done = !valid;
    for (int it = 0; it < v.h_max_iter; it++) {
      const float H = GAMMA_K * h;
      const float Hs = warp_max(done ? 0.0f : H);
      if (Hs == 0.0f) break;  // every particle of the round has converged
      const float H2 = H * H, Hinv = 1.0f / H;
      const float Hs2 = Hs * Hs * 1.0002f;
      float n_hi = 0.f, n_lo = 0.f, t_hi = 0.f, t_lo = 0.f;
      float r_hi = 0.f, r_lo = 0.f, rt_hi = 0.f, rt_lo = 0.f;
      int cnt = 0;
      for (int dxc = -1; dxc <= 1; dxc++)
        for (int dyc = -1; dyc <= 1; dyc++)
          for (int dzc = -1; dzc <= 1; dzc++) {
            const int cj = neighbour_cell(F, dxc, dyc, dzc);
            const float sx = dxc * F.wf, sy = dyc * F.wf, sz = dzc * F.wf;
            const float xx = xi.x - sx, xy = xi.y - sy, xz = xi.z - sz;
            const int l0 = v.cell_leaf_start[cj], l1 = v.cell_leaf_start[cj + 1];
            float pn = 0.f, pt = 0.f, pr = 0.f, prt = 0.f;
            for (int lb = l0; lb < l1; lb += 32) {
              const int l = lb + lane;
              bool ok = false;
              if (l < l1) ok = box_gap2(blo, bhi, v.leaf_lo[l], v.leaf_hi[l], sx, sy, sz) < Hs2;
              unsigned mk = __ballot_sync(FULL, ok);
              while (mk) {
                const int jl = lb + __ffs(mk) - 1;
                mk &= mk - 1;
                const int ja = v.leaf_start[jl], jb = v.leaf_start[jl + 1];
                wc.cand += (unsigned long long)(jb - ja);
                for (int j = ja + sub; j < jb; j += G) {
                  const float4 pj = __ldg(&v.rec_xm[j]);
                  const float dx = xx - pj.x, dy = xy - pj.y, dz = xz - pj.z;
                  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                  if (!done && r2 < H2) {
                    const float rr = r2 * rsqrtf(fmaxf(r2, 1e-30f));
                    const float q = rr * Hinv;
                    float wq, dwq;
                    kernel_wd(q, wq, dwq);
                    const float t = fmaf(q, dwq, 3.0f * wq);
                    pn += wq;
                    pt += t;
                    pr = fmaf(pj.w, wq, pr);
                    prt = fmaf(pj.w, t, prt);
                    cnt += (j != i);
                  }
                }
              }
            }
            fold(n_hi, n_lo, pn);
            fold(t_hi, t_lo, pt);
            fold(r_hi, r_lo, pr);
            fold(rt_hi, rt_lo, prt);
          }
      const double sn = group_sum<G>((double)n_hi + (double)n_lo);
      const double st = group_sum<G>((double)t_hi + (double)t_lo);
      const double sr = group_sum<G>((double)r_hi + (double)r_lo);
      const double srt = group_sum<G>((double)rt_hi + (double)rt_lo);
      cnt = group_sum_i<G>(cnt);
      if (!done) {
        // Newton step on F(h) = h^3 n(h) - eta^3, kept inside a bracket
        const double Hd = (double)H, Hi = 1.0 / Hd;
        const double Hi3 = Hi * Hi * Hi, Hi4 = Hi3 * Hi;
        const double nn = (double)KERNEL_NORM * sn * Hi3;
        const double dndh = -GAMMA_K_D * (double)KERNEL_NORM * st * Hi4;
        const double hd = (double)h;
        const double F3 = hd * hd * hd * nn - eta3;
        const double dF = 3.0 * hd * hd * nn + hd * hd * hd * dndh;
        if (F3 < 0.0) lo = hd;
        else hi = hd;
        double hn;
        if (F3 == 0.0) hn = hd;
        else if (dF > 0.0) hn = hd - F3 / dF;
        else hn = NAN;
        if (!(hn >= lo && hn <= hi)) hn = isinf(hi) ? 2.0 * hd : 0.5 * (lo + hi);
        hn = fmin(fmax(hn, 0.5 * hd), 2.0 * hd);
        bool conv = fabs(hn - hd) <= v.h_tol * hd;
        const bool over = !conv && hn > (double)hcap;
        const bool last = it == v.h_max_iter - 1;
        if (conv || over || last) {
          done = true;
          if (sub == 0) {
            wc.pairs += (unsigned long long)cnt;
            wc.iters += (unsigned long long)(it + 1);
            if (over) {
              wc.overflow++;
              atomic_max_float_pos(&v.ds->want_h_bits, (float)hn);
            }
            else if (!conv) wc.noconv++;
            // density, grad-h factor, equation of state at the final h
            const double rho_d = (double)KERNEL_NORM * sr * Hi3;
            const double drho = -GAMMA_K_D * (double)KERNEL_NORM * srt * Hi4;
            const float rho = (float)rho_d;
            const float f = (float)(1.0 / (1.0 + hd / (3.0 * rho_d) * drho));
            const int bi = v.bin[i];
            const double dtp =
                ((double)(ti - v.ti_begin[i]) - 0.5 * (double)(1ll << bi)) * v.dt_min;
            float Ap = (float)((double)v.A[i] + (double)v.Adot[i] * dtp);
            const float g = (float)v.gamma;
            if (init_entropy) Ap = (g - 1.0f) * v.A[i] / powf(rho, g - 1.0f);  // A holds u
            const float P = Ap * powf(rho, g);
            const float c = sqrtf(g * P / rho);
            v.h[i] = h;
            v.rho[i] = rho;
            v.f[i] = f;
            v.P[i] = P;
            v.c[i] = c;
            v.rec_xH[i] = make_float4(xi.x, xi.y, xi.z, H);
            v.rec_h[i] = make_float4(rho, f * P / (rho * rho), c, Hinv);
            if (v.ngb_density) v.ngb_density[i] = cnt;
          }
        } else {
          h = (float)hn;
        }
      }
    }
  }
  // largest support in the leaf after the update
  __syncwarp();
  float Hm = 0.0f;
  for (int k = a + lane; k < b; k += 32) Hm = fmaxf(Hm, v.rec_xH[k].w);
  Hm = warp_max(Hm);
  if (lane == 0) {
    reinterpret_cast<float *>(&v.leaf_lo[leaf])[3] = Hm;
    atomic_max_float_pos(&v.ds->Hmax_bits, Hm);
  }
}

// ---------------------------------------------------------------------------
// force loop for the active particles of a leaf
// ---------------------------------------------------------------------------
template <int G>
__device__ void force_leaf(const View &v, int leaf, int bin_filter, int m_act, const CellFrame &F,
                           int *s_act, WarpCounters &wc) {
  const int lane = lane_id();
  const int a = v.leaf_start[leaf], b = v.leaf_start[leaf + 1];
  const int nact = leaf_actives(v, a, b, m_act, bin_filter, s_act);
  if (nact == 0) return;
  constexpr int P = 32 / G;
  const int grp = lane / G, sub = lane % G;
  const float4 blo = v.leaf_lo[leaf], bhi = v.leaf_hi[leaf];
  const float alpha = (float)v.alpha;
  const float g = (float)v.gamma;

  for (int r = 0; r < nact; r += P) {
    const int slot = r + grp;
    const bool valid = slot < nact;
    const int i = valid ? s_act[slot] : a;
    const float4 xi = v.rec_xH[i];
    const float4 vi = v.rec_v[i];
    const float4 hi4 = v.rec_h[i];
    const float Hi2 = xi.w * xi.w;
    const float Hinv2 = hi4.w * hi4.w;
    const float nHi4 = KERNEL_NORM * Hinv2 * Hinv2;
    const float Hs = warp_max(valid ? xi.w : 0.0f);
    float ax_hi = 0.f, ax_lo = 0.f, ay_hi = 0.f, ay_lo = 0.f, az_hi = 0.f, az_lo = 0.f;
    float ad_hi = 0.f, ad_lo = 0.f;
    float vs = 2.0f * hi4.z;
    int cnt = 0;
    for (int dxc = -1; dxc <= 1; dxc++)
      for (int dyc = -1; dyc <= 1; dyc++)
        for (int dzc = -1; dzc <= 1; dzc++) {
          const int cj = neighbour_cell(F, dxc, dyc, dzc);
          const float sx = dxc * F.wf, sy = dyc * F.wf, sz = dzc * F.wf;
          const float xx = xi.x - sx, xy = xi.y - sy, xz = xi.z - sz;
          const int l0 = v.cell_leaf_start[cj], l1 = v.cell_leaf_start[cj + 1];
          float pax = 0.f, pay = 0.f, paz = 0.f, pad = 0.f;
          for (int lb = l0; lb < l1; lb += 32) {
            const int l = lb + lane;
            bool ok = false;
            if (l < l1) {
              const float4 loj = v.leaf_lo[l];
              const float R = fmaxf(Hs, loj.w);
              ok = box_gap2(blo, bhi, loj, v.leaf_hi[l], sx, sy, sz) < R * R * 1.0002f;
            }
            unsigned mk = __ballot_sync(FULL, ok);
            while (mk) {
              const int jl = lb + __ffs(mk) - 1;
              mk &= mk - 1;
              const int ja = v.leaf_start[jl], jb = v.leaf_start[jl + 1];
              wc.cand += (unsigned long long)(jb - ja);
              for (int j = ja + sub; j < jb; j += G) {
                const float4 pj = __ldg(&v.rec_xH[j]);
                const float dx = xx - pj.x, dy = xy - pj.y, dz = xz - pj.z;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                if (valid && j != i && (r2 < Hi2 || r2 < pj.w * pj.w)) {
                  const float4 vj = __ldg(&v.rec_v[j]);
                  const float4 hj = __ldg(&v.rec_h[j]);
                  cnt++;
                  if (r2 > 0.0f) {
                    const float rinv = rsqrtf(r2);
                    const float rr = r2 * rinv;
                    const float qi = rr * hi4.w, qj = rr * hj.w;
                    const float dwi = qi < 1.0f ? kernel_dw(qi) * nHi4 : 0.0f;
                    const float hj2 = hj.w * hj.w;
                    const float dwj = qj < 1.0f ? kernel_dw(qj) * (KERNEL_NORM * hj2 * hj2) : 0.0f;
                    const float dvdr =
                        fmaf(vi.x - vj.x, dx, fmaf(vi.y - vj.y, dy, (vi.z - vj.z) * dz));
                    // Monaghan signal-velocity viscosity, beta = 3 (as in Eq. 1)
                    const float wij = fminf(0.0f, dvdr * rinv);
                    const float vsij = hi4.z + hj.z - 3.0f * wij;
                    const float Pi = -alpha * vsij * wij / (hi4.x + hj.x);
                    const float dWb = 0.5f * (dwi + dwj);
                    const float sc = vj.w * fmaf(hi4.y, dwi, fmaf(hj.y, dwj, Pi * dWb)) * rinv;
                    pax = fmaf(-sc, dx, pax);
                    pay = fmaf(-sc, dy, pay);
                    paz = fmaf(-sc, dz, paz);
                    pad = fmaf(vj.w * Pi * dWb, dvdr * rinv, pad);
                    vs = fmaxf(vs, vsij);
                  } else {
                    vs = fmaxf(vs, hi4.z + hj.z);
                  }
                }
              }
            }
          }
          fold(ax_hi, ax_lo, pax);
          fold(ay_hi, ay_lo, pay);
          fold(az_hi, az_lo, paz);
          fold(ad_hi, ad_lo, pad);
        }
    const double sax = group_sum<G>((double)ax_hi + (double)ax_lo);
    const double say = group_sum<G>((double)ay_hi + (double)ay_lo);
    const double saz = group_sum<G>((double)az_hi + (double)az_lo);
    const double sad = group_sum<G>((double)ad_hi + (double)ad_lo);
    cnt = group_sum_i<G>(cnt);
    vs = group_max<G>(vs);
    if (valid && sub == 0) {
      wc.pairs += (unsigned long long)cnt;
      v.ax[i] = (float)sax;
      v.ay[i] = (float)say;
      v.az[i] = (float)saz;
      v.Adot[i] = (float)(0.5 * ((double)g - 1.0) * (double)powf(hi4.x, 1.0f - g) * sad);
      v.vsig[i] = vs;
      if (v.ngb_force) v.ngb_force[i] = cnt;
    }
  }
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ void flush_counters(DevState *ds, WarpCounters &wc, bool density) {
  // every lane holds its own share; sum over the warp, one atomic per counter
  unsigned long long p = wc.pairs, c = wc.cand, it = wc.iters, nc = wc.noconv, ov = wc.overflow;
  for (int o = 16; o; o >>= 1) {
    p += __shfl_xor_sync(FULL, p, o);
    it += __shfl_xor_sync(FULL, it, o);
    nc += __shfl_xor_sync(FULL, nc, o);
    ov += __shfl_xor_sync(FULL, ov, o);
  }
  // the candidate count is warp-uniform (every lane counted the same leaves)
  if (lane_id() == 0) {
    if (density) {
      if (p) atomicAdd(&ds->s_pairs_density, p);
      if (c) atomicAdd(&ds->s_cand_density, c);
      if (it) atomicAdd(&ds->s_iters_density, it);
      if (nc) record_error(ds, SPH_ERR_H_NOCONV, nc, false);
      if (ov) record_error(ds, SPH_ERR_CELL_OVERFLOW, ov, true);
    } else {
      if (p) atomicAdd(&ds->s_pairs_force, p);
      if (c) atomicAdd(&ds->s_cand_force, c);
    }
  }
}

__device__ __forceinline__ CellFrame frame_of(const DevState *ds, int cell) {
  CellFrame F;
  F.nc = ds->nc;
  F.cx = cell / (F.nc * F.nc);
  F.cy = (cell / F.nc) % F.nc;
  F.cz = cell % F.nc;
  F.wf = (float)ds->w;
  return F;
}

template <int G>
__global__ void __launch_bounds__(PT) k_density(View v, int flags, int bin_filter, int persistent) {
  __shared__ int s_act[WARPS_PER_BLOCK][LEAF_MAX_LIMIT];
  DevState *ds = v.ds;
  if (ds->halt) return;
  const int warp = threadIdx.x >> 5, lane = lane_id();
  // every support must stay inside the 27 cells around its particle's cell:
  // H + 2 (largest excursion of a particle out of its cell) <= cell width
  const double w = ds->w;
  const float exc = __uint_as_float(ds->excursion_bits);
  const float Hmax = __uint_as_float(ds->Hmax_bits);
  if ((double)Hmax + 2.0 * (double)exc > w) {
    if (blockIdx.x == 0 && threadIdx.x == 0) record_error(ds, SPH_ERR_CELL_OVERFLOW, 1, true);
    return;
  }
  const float hcap = (float)((w - 2.0 * (double)exc) / GAMMA_K_D * (1.0 - 1e-6));
  const int m_act = ds->m_act;
  const long long ti = ds->ti;
  const int *q = bin_filter >= 0 ? v.q_bin : v.q_active;
  const int nq = bin_filter >= 0 ? ds->n_bin_leaves : ds->n_active_leaves;
  WarpCounters wc = {0, 0, 0, 0, 0};
  if (persistent) {
    for (;;) {
      int item = 0;
      if (lane == 0) item = atomicAdd(&ds->head_density, 1);
      item = __shfl_sync(FULL, item, 0);
      if (item >= nq) break;
      const int leaf = q[item];
      density_leaf<G>(v, leaf, flags, bin_filter, m_act, frame_of(ds, v.leaf_cell[leaf]), hcap, ti,
                      s_act[warp], wc);
    }
  } else {
    const int item = blockIdx.x * WARPS_PER_BLOCK + warp;
    if (item < nq) {
      const int leaf = q[item];
      density_leaf<G>(v, leaf, flags, bin_filter, m_act, frame_of(ds, v.leaf_cell[leaf]), hcap, ti,
                      s_act[warp], wc);
    }
  }
  flush_counters(ds, wc, true);
}

template <int G>
__global__ void __launch_bounds__(PT) k_force(View v, int bin_filter, int persistent) {
  __shared__ int s_act[WARPS_PER_BLOCK][LEAF_MAX_LIMIT];
  DevState *ds = v.ds;
  if (ds->halt) return;
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const int m_act = ds->m_act;
  const int *q = bin_filter >= 0 ? v.q_bin : v.q_active;
  const int nq = bin_filter >= 0 ? ds->n_bin_leaves : ds->n_active_leaves;
  WarpCounters wc = {0, 0, 0, 0, 0};
  if (persistent) {
    for (;;) {
      int item = 0;
      if (lane == 0) item = atomicAdd(&ds->head_force, 1);
      item = __shfl_sync(FULL, item, 0);
      if (item >= nq) break;
      const int leaf = q[item];
      force_leaf<G>(v, leaf, bin_filter, m_act, frame_of(ds, v.leaf_cell[leaf]), s_act[warp], wc);
    }
  } else {
    const int item = blockIdx.x * WARPS_PER_BLOCK + warp;
    if (item < nq) {
      const int leaf = q[item];
      force_leaf<G>(v, leaf, bin_filter, m_act, frame_of(ds, v.leaf_cell[leaf]), s_act[warp], wc);
    }
  }
  flush_counters(ds, wc, false);
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
    const int a = v.leaf_start[leaf], b = v.leaf_start[leaf + 1];
    for (int i = a + lane_id(); i < b; i += 32)
      if ((int)v.bin[i] <= m_act) v.A[i] = (g - 1.0f) * v.A[i] / powf(v.rho[i], g - 1.0f);
  }
}

template <int G>
cudaError_t density_g(const View &v, int flags, int bin_filter, bool persistent, int grid,
                      cudaStream_t st) {
  k_density<G><<<grid, PT, 0, st>>>(v, flags, bin_filter, persistent ? 1 : 0);
  return cudaGetLastError();
}

template <int G>
cudaError_t force_g(const View &v, int bin_filter, bool persistent, int grid, cudaStream_t st) {
  k_force<G><<<grid, PT, 0, st>>>(v, bin_filter, persistent ? 1 : 0);
  return cudaGetLastError();
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

int persistent_blocks_per_sm(int G, bool density) {
  int nb = 0;
  const void *fn = nullptr;
  switch (G) {
    case 1: fn = density ? (const void *)k_density<1> : (const void *)k_force<1>; break;
    case 2: fn = density ? (const void *)k_density<2> : (const void *)k_force<2>; break;
    case 4: fn = density ? (const void *)k_density<4> : (const void *)k_force<4>; break;
    case 8: fn = density ? (const void *)k_density<8> : (const void *)k_force<8>; break;
    case 16: fn = density ? (const void *)k_density<16> : (const void *)k_force<16>; break;
    case 32: fn = density ? (const void *)k_density<32> : (const void *)k_force<32>; break;
    default: return 1;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, PT, 0) != cudaSuccess || nb < 1) nb = 1;
  return nb;
}

cudaError_t launch_entropy_from_u(const View &v, cudaStream_t st) {
  note_launches(1);
  k_entropy_from_u<<<v.grid_util, 256, 0, st>>>(v);
  return cudaGetLastError();
}

}  // namespace sph
