// Reverse mode of one kick-drift-kick step and of the grid-density loss.
//
// The paper has no adjoint; these kernels differentiate the forward path of
// this library (Sec. II-A time integration with the density loop, the
// smoothing-length solve and the force loop of Sec. III) with respect to the
// state before the step, for a loss on a later state.  The discrete parts
// (active set, time bins, integer times, which pairs are neighbours) are
// piecewise constant and are taken from the forward run.
//
// One step backwards (sph_step_bwd): the caller hands in the state before
// and after the step (in the caller's particle order) and the adjoint of the
// state after it; the adjoint is replaced by the adjoint of the state before.
//   1. prepare (caller order): positions at the step's tick, predicted v and
//      A, P and c inputs, h / rho / f as the force loop saw them; the adjoint
//      of both half-kicks of the active particles;
//   2. a cell build of these internal copies (its own sort) and the active
//      work groups;
//   3. force adjoint: for every active i and neighbour j, the derivative of
//      a_i and Adot_i with respect to positions, predicted velocities, H,
//      f P / rho^2, c and rho of both particles (j's share by FP64 atomics);
//   4. equation-of-state adjoint: f P / rho^2 and c back to f, P, rho, then
//      P = A_pred rho^gamma back to A_pred and rho (on the first step
//      A = (gamma - 1) u / rho^(gamma - 1) back to u and rho);
//   5. density adjoint in two passes over the same pairs: the sums that fix
//      the derivatives of rho, f and of the smoothing-length equation
//      F(h, x) = h^3 n(h) - eta^3 (implicit h: dh/dx = -F_x / F_h), then the
//      position derivatives of every pair;
//   6. scatter back to caller order with the prediction (v_pred = v + a dtp,
//      A_pred = A + Adot dtp) and drift (x += v dt) adjoints.
// Pair arithmetic is FP32 as in the forward loops; every adjoint accumulator
// is FP64.
#include <cstddef>
#include <cstring>

#include "sph_pairloop.cuh"

namespace sph {
namespace {

constexpr double KN_D = 2.5464790894703255;  // 8 / pi

__device__ __forceinline__ double wrap_box(double x, double box) {
  if (x < 0.0) x += box;
  if (x >= box) x -= box;
  return x;
}

__device__ __forceinline__ double min_img(double d, double box) {
  if (d > 0.5 * box) d -= box;
  else if (d < -0.5 * box) d += box;
  return d;
}

// ---------------------------------------------------------------------------
// 1. prepare, in caller order
// ---------------------------------------------------------------------------
__global__ void k_adj_prepare(sph_particles pre, sph_particles post, sph_particles W,
                              sph_adjoint adj, long long ti, int first, double dt_min, double box,
                              double gamma) {
  const long long n = pre.n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const bool act = pre.ti_end[i] == ti;
    // positions at the step's tick (the forward drift, applied to every particle)
    const double dtd = (double)(ti - pre.ti_drift[i]) * dt_min;
    double x = pre.x[i], y = pre.y[i], z = pre.z[i];
    if (dtd != 0.0) {
      x = wrap_box(x + (double)pre.vx[i] * dtd, box);
      y = wrap_box(y + (double)pre.vy[i] * dtd, box);
      z = wrap_box(z + (double)pre.vz[i] * dtd, box);
    }
    W.x[i] = x;
    W.y[i] = y;
    W.z[i] = z;
    // prediction at the tick
    const int bi = pre.bin[i] & (MAX_BINS - 1);
    const double dtp = ((double)(ti - pre.ti_begin[i]) - 0.5 * (double)(1ll << bi)) * dt_min;
    const float fdtp = (float)dtp;
    W.vx[i] = pre.vx[i] + pre.ax[i] * fdtp;
    W.vy[i] = pre.vy[i] + pre.ay[i] * fdtp;
    W.vz[i] = pre.vz[i] + pre.az[i] * fdtp;
    const float h = act ? post.h[i] : pre.h[i];
    const float rho = act ? post.rho[i] : pre.rho[i];
    const float f = act ? post.f[i] : pre.f[i];
    float Ap;
    if (first) Ap = (float)(gamma - 1.0) * pre.A[i] / powf(rho, (float)gamma - 1.0f);  // A holds u
    else Ap = (float)((double)pre.A[i] + (double)pre.Adot[i] * dtp);
    W.A[i] = Ap;
    W.h[i] = h;
    W.rho[i] = rho;
    W.f[i] = f;
    W.m[i] = pre.m[i];
    // the cell build's refresh predicts with a and Adot: zero, so the records
    // carry exactly v_pred and A_pred; vsig carries the forward Adot of the
    // active particles (the force adjoint needs it)
    W.ax[i] = 0.0f;
    W.ay[i] = 0.0f;
    W.az[i] = 0.0f;
    W.Adot[i] = 0.0f;
    W.vsig[i] = act ? post.Adot[i] : 0.0f;
    W.P[i] = 0.0f;
    W.c[i] = 0.0f;
    W.bin[i] = act ? 0 : 1;  // the backward marks bin 0 active
    W.ti_begin[i] = ti;
    W.ti_end[i] = ti + 1;
    W.ti_drift[i] = ti;
    W.active[i] = 0;
    // adjoint of the two half-kicks of an active particle:
    // v += a dt_old / 2 and v += a dt_new / 2 (likewise A with Adot)
    if (act) {
      const double half = 0.5 * (double)(pre.ti_end[i] - pre.ti_begin[i]) * dt_min +
                          0.5 * (double)(post.ti_end[i] - post.ti_begin[i]) * dt_min;
      adj.ax[i] += adj.vx[i] * half;
      adj.ay[i] += adj.vy[i] * half;
      adj.az[i] += adj.vz[i] * half;
      adj.Adot[i] += adj.A[i] * half;
    }
  }
}

// ---------------------------------------------------------------------------
// 2b. gather the adjoint state into the backward build's order
// ---------------------------------------------------------------------------
__global__ void k_adj_gather(View v, AdjWork w, sph_adjoint adj, double gamma) {
  const long long n = v.n;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const int o = w.perm[k];
    w.xb[k] = adj.x[o];
    w.yb[k] = adj.y[o];
    w.zb[k] = adj.z[o];
    w.hb[k] = adj.h[o];
    w.rhob[k] = adj.rho[o];
    w.fb[k] = adj.f[o];
    w.vpxb[k] = 0.0;
    w.vpyb[k] = 0.0;
    w.vpzb[k] = 0.0;
    w.Qb[k] = 0.0;
    w.cb[k] = 0.0;
    if (v.bin[k] == 0) {
      // this step computed a and Adot of the active particles: their adjoints
      // are consumed here (what remains for the old values comes from the
      // prediction, added in the scatter)
      w.axb[k] = adj.ax[o];
      w.ayb[k] = adj.ay[o];
      w.azb[k] = adj.az[o];
      const double Adb = adj.Adot[o];
      w.Adotb[k] = Adb;
      adj.ax[o] = 0.0;
      adj.ay[o] = 0.0;
      adj.az[o] = 0.0;
      adj.Adot[o] = 0.0;
      // Adot = (gamma - 1)/2 rho^(1 - gamma) sum(...): its rho-dependence
      w.rhob[k] += Adb * (double)v.vsig[k] * (1.0 - gamma) / (double)v.rho[k];
    } else {
      w.axb[k] = w.ayb[k] = w.azb[k] = w.Adotb[k] = 0.0;
    }
  }
}

// ---------------------------------------------------------------------------
// 3. force adjoint: one warp per active work group, one lane per particle;
//    with COOP the 8 warps of a block share a group (each takes the neighbour
//    chunks with its index modulo 8) and combine the particle's own sums in
//    warp order through the start of their staging buffers
// ---------------------------------------------------------------------------
template <class St = StageF>
__device__ __forceinline__ double *adj_red_area(int warp) {
  extern __shared__ __align__(16) char smem_dyn[];
  static_assert(StageF::bytes() % 16 == 0 && S_FORCE * 3 * 16 >= 11 * 32 * 8 &&
                    StageD::bytes() % 16 == 0 && S_DENS * 16 >= 5 * 32 * 8,
                "the reduction areas fit the start of a staging buffer");
  return reinterpret_cast<double *>(smem_dyn + (size_t)warp * St::bytes());
}

// The COOP reduction: the 8 warps' per-lane partial sums part[0..N) added in
// warp order, the result in every warp; a failure in any warp becomes every
// warp's (so that all take the same branches).
template <class St, int N>
__device__ __forceinline__ void coop_reduce(double (&part)[N], bool &failed) {
  const int lane = lane_id(), warp = threadIdx.x >> 5;
  double *mine = adj_red_area<St>(warp);
#pragma unroll
  for (int k = 0; k < N; k++) mine[k * 32 + lane] = part[k];
  mine[N * 32 + lane] = failed ? 1.0 : 0.0;
  __syncthreads();
  bool any = false;
#pragma unroll
  for (int k = 0; k < N; k++) part[k] = 0.0;
  for (int q = 0; q < WARPS_PER_BLOCK; q++) {
    const double *rw = adj_red_area<St>(q);
#pragma unroll
    for (int k = 0; k < N; k++) part[k] += rw[k * 32 + lane];
    any = any || rw[N * 32 + lane] != 0.0;
  }
  __syncthreads();
  fence_proxy_async();  // the staging buffers take bulk copies again
  failed = __any_sync(FULL, any);
}

template <bool COOP>
__device__ void force_adj_group(const View &v, const AdjWork &w, int wg, const CellFrame &F,
                                StageF &st, WarpCounters &wc) {
  const int lane = lane_id();
  const int warp = threadIdx.x >> 5;
  const Group Wg = group_of(v, wg, F);
  const int a = Wg.a, b = Wg.b;
  const int nact = leaf_actives(v, a, b, 0, -1, st.act);
  if (nact == 0) return;
  const float qox = F.kx * F.wq, qoy = F.ky * F.wq, qoz = F.kz * F.wq;
  const float clx = Wg.lx + qox, cly = Wg.ly + qoy, clz = Wg.lz + qoz;
  const float chx = Wg.hx + qox, chy = Wg.hy + qoy, chz = Wg.hz + qoz;
  const float ceps = 1e-5f * F.wf;
  const float alpha = (float)v.alpha;
  const float4 *srcs[3] = {v.rec_xH, v.rec_v, v.rec_h};
  const float4 *sx_rec = st.rec, *sv_rec = st.rec + S_FORCE, *sh_rec = st.rec + 2 * S_FORCE;
  // one round: a work group holds at most 32 particles
  const bool valid = lane < nact;
  const int i = valid ? st.act[lane] : a;
  const float4 xl = v.rec_xH[i];
  const float3 lo3 = leaf_offset(v, i, F);
  const float4 xi = make_float4(xl.x + lo3.x, xl.y + lo3.y, xl.z + lo3.z, xl.w);
  const float4 vi = v.rec_v[i];
  const float4 hi4 = v.rec_h[i];  // rho, Q = f P / rho^2, c, 1 / H
  const float Hi2 = xi.w * xi.w;
  const float Hinv2 = hi4.w * hi4.w;
  const float nHi4 = KERNEL_NORM * Hinv2 * Hinv2;
  const float Hs = warp_max(valid ? xi.w : 0.0f);
  // adjoints of the outputs a_i and Adot_i
  const float abx = valid ? (float)w.axb[i] : 0.0f, aby = valid ? (float)w.ayb[i] : 0.0f,
              abz = valid ? (float)w.azb[i] : 0.0f;
  const float Bi = valid ? (float)(0.5 * (v.gamma - 1.0) * pow((double)hi4.x, 1.0 - v.gamma) *
                                   w.Adotb[i])
                         : 0.0f;
  const bool live = valid && (abx != 0.0f || aby != 0.0f || abz != 0.0f || Bi != 0.0f);
  const int nsph = compact_spheres(st.sph, live, make_float4(xi.x, xi.y, xi.z, xi.w));
  // the particle's own adjoint sums: FP32 partial sums per neighbour cell,
  // folded into FP64 where the cell changes (FP64 arithmetic is scarce)
  double dxi = 0.0, dyi = 0.0, dzi = 0.0, dvxi = 0.0, dvyi = 0.0, dvzi = 0.0;
  double Hbi = 0.0, Qbi = 0.0, cbi = 0.0, rbi = 0.0;
  float pdx = 0.f, pdy = 0.f, pdz = 0.f, pvx = 0.f, pvy = 0.f, pvz = 0.f;
  float pH = 0.f, pQ = 0.f, pc = 0.f, pr = 0.f;
  int cur = -1;
  auto fold_cell = [&]() {
    dxi += (double)pdx; dyi += (double)pdy; dzi += (double)pdz;
    dvxi += (double)pvx; dvyi += (double)pvy; dvzi += (double)pvz;
    Hbi += (double)pH; Qbi += (double)pQ; cbi += (double)pc; rbi += (double)pr;
    pdx = pdy = pdz = pvx = pvy = pvz = pH = pQ = pc = pr = 0.f;
  };
  auto leaf_ok = [&](int l, float sx, float sy, float sz, LeafBox &lb) {
    const float4 loj = v.leaf_lo[l], hij = v.leaf_hi[l];
    const float R = fmaxf(Hs, loj.w);
    lb = leaf_box(loj, hij, sx, sy, sz, loj.w);
    return box_gap2(Wg.lx, Wg.ly, Wg.lz, Wg.hx, Wg.hy, Wg.hz, loj, hij, sx, sy, sz) <
           R * R * 1.0002f;
  };
  auto chunk_ok = [&](int gg, float sx, float sy, float sz) {
    const float4 loc = v.chunk_lo[gg];
    const float R = fmaxf(Hs, loc.w) + ceps;
    return box_gap2(clx, cly, clz, chx, chy, chz, loc, v.chunk_hi[gg], sx, sy, sz) < R * R;
  };
  auto consume = [&](int base, int total) {
    const int end = base + total;
    for (int k0 = base; k0 < end; k0 += 32) {
      unsigned mask = 0u;
#pragma unroll
      for (int u = 0; u < 32; u++) {
        const float4 pj = sx_rec[min(k0 + u, S_FORCE - 1)];
        const float dx = xi.x - pj.x, dy = xi.y - pj.y, dz = xi.z - pj.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        mask |= (k0 + u < end && (r2 < Hi2 || r2 < pj.w * pj.w)) ? (1u << u) : 0u;
      }
      if (!live) mask = 0u;
      while (mask) {
        const int k = k0 + __ffs(mask) - 1;
        mask &= mask - 1;
        const int j = st.recj[k];
        if (j == i) continue;
        const int ci = st.recc[k];
        if (ci != cur) {
          fold_cell();
          cur = ci;
        }
        const float4 pj = sx_rec[k];
        const float4 vj = sv_rec[k];
        const float4 hj = sh_rec[k];
        const float dx = xi.x - pj.x, dy = xi.y - pj.y, dz = xi.z - pj.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (!(r2 > 0.0f)) continue;  // coincident: no direction, no gradient
        const float rinv = rsqrtf(r2);
        const float r = r2 * rinv;
        const float qi = r * hi4.w, qj = r * hj.w;
        const float hj2 = hj.w * hj.w;
        const float nHj4 = KERNEL_NORM * hj2 * hj2;
        const float wpi = qi < 1.0f ? kernel_dw(qi) : 0.0f;
        const float wpj = qj < 1.0f ? kernel_dw(qj) : 0.0f;
        const float wppi = qi < 1.0f ? kernel_d2w(qi) : 0.0f;
        const float wppj = qj < 1.0f ? kernel_d2w(qj) : 0.0f;
        const float dWi = wpi * nHi4, dWj = wpj * nHj4;
        const float dvx = vi.x - vj.x, dvy = vi.y - vj.y, dvz = vi.z - vj.z;
        const float dvdr = fmaf(dvx, dx, fmaf(dvy, dy, dvz * dz));
        const float uu = dvdr * rinv;
        const float wij = fminf(0.0f, uu);
        const float vsij = hi4.z + hj.z - 3.0f * wij;
        const float rs = hi4.x + hj.x;
        const float Pi = -alpha * vsij * wij / rs;
        const float Wb = 0.5f * (dWi + dWj);
        const float K = fmaf(hi4.y, dWi, fmaf(hj.y, dWj, Pi * Wb));
        const float mj = vj.w;
        const float gdot = fmaf(abx, dx, fmaf(aby, dy, abz * dz));
        // the pair's share of the loss: -m_j K / r (abar . d) + B m_j Pi Wb u
        const float Kb = -mj * rinv * gdot;
        const float Pib = fmaf(Kb, Wb, Bi * mj * Wb * uu);
        const float Wbb = fmaf(Kb, Pi, Bi * mj * Pi * uu);
        float ub = Bi * mj * Pi * Wb;
        const float dWib = fmaf(Kb, hi4.y, 0.5f * Wbb);
        const float dWjb = fmaf(Kb, hj.y, 0.5f * Wbb);
        const float cpart = Pib * (-alpha * wij / rs);
        const float rpart = Pib * (-Pi / rs);
        if (uu < 0.0f) ub = fmaf(Pib, -alpha * (vsij - 3.0f * wij) / rs, ub);
        const float rinvb = fmaf(-mj * K, gdot, ub * dvdr);
        // dW/dr and dW/dH of each smoothing length (q w'' + 4 w' over H^5)
        const float rb = fmaf(dWib, wppi * nHi4 * hi4.w,
                              fmaf(dWjb, wppj * nHj4 * hj.w, -rinvb * rinv * rinv));
        const float Hib = -dWib * fmaf(qi, wppi, 4.0f * wpi) * nHi4 * hi4.w;
        const float Hjb = -dWjb * fmaf(qj, wppj, 4.0f * wpj) * nHj4 * hj.w;
        const float gK = -mj * K * rinv;
        const float ex = dx * rinv, ey = dy * rinv, ez = dz * rinv;
        const float bx = fmaf(gK, abx, fmaf(ub * rinv, dvx, rb * ex));
        const float by = fmaf(gK, aby, fmaf(ub * rinv, dvy, rb * ey));
        const float bz = fmaf(gK, abz, fmaf(ub * rinv, dvz, rb * ez));
        const float vbx = ub * ex, vby = ub * ey, vbz = ub * ez;
        pdx += bx; pdy += by; pdz += bz;
        pvx += vbx; pvy += vby; pvz += vbz;
        pH += Hib;
        pQ += Kb * dWi;
        pc += cpart;
        pr += rpart;
        atomicAdd(&w.xb[j], -(double)bx);
        atomicAdd(&w.yb[j], -(double)by);
        atomicAdd(&w.zb[j], -(double)bz);
        atomicAdd(&w.vpxb[j], -(double)vbx);
        atomicAdd(&w.vpyb[j], -(double)vby);
        atomicAdd(&w.vpzb[j], -(double)vbz);
        atomicAdd(&w.hb[j], (double)GAMMA_K * (double)Hjb);
        atomicAdd(&w.Qb[j], (double)(Kb * dWj));
        atomicAdd(&w.cb[j], (double)cpart);
        atomicAdd(&w.rhob[j], (double)rpart);
      }
    }
  };
  const Reach reach = {clx, cly, clz, chx, chy, chz,
                       fmaxf(Hs, __uint_as_float(v.ds->Hmax_bits)) + ceps,
                       __uint_as_float(v.ds->excursion_bits), st.sph, nsph};
  int skip = 0, nlist = 0;
  bool more = false;
  do {
    nlist = search(v, F, reach, st, leaf_ok, chunk_ok, skip, more, COOP ? warp : -1);
    stage_list(srcs, st, nlist, consume, wc);
    skip += nlist;
  } while (more && !st.failed);
  fold_cell();
  if constexpr (COOP) {
    double sum[10] = {dxi, dyi, dzi, dvxi, dvyi, dvzi, Hbi, Qbi, cbi, rbi};
    bool failed = st.failed;
    coop_reduce<StageF, 10>(sum, failed);
    st.failed = failed;  // the same in every warp
    dxi = sum[0]; dyi = sum[1]; dzi = sum[2];
    dvxi = sum[3]; dvyi = sum[4]; dvzi = sum[5];
    Hbi = sum[6]; Qbi = sum[7]; cbi = sum[8]; rbi = sum[9];
  }
  if (live && (!COOP || warp == 0)) {
    atomicAdd(&w.xb[i], dxi);
    atomicAdd(&w.yb[i], dyi);
    atomicAdd(&w.zb[i], dzi);
    atomicAdd(&w.vpxb[i], dvxi);
    atomicAdd(&w.vpyb[i], dvyi);
    atomicAdd(&w.vpzb[i], dvzi);
    atomicAdd(&w.hb[i], (double)GAMMA_K * Hbi);
    atomicAdd(&w.Qb[i], Qbi);
    atomicAdd(&w.cb[i], cbi);
    atomicAdd(&w.rhob[i], rbi);
  }
  __syncwarp();
}

// A step with at most two groups per block gives each group a whole block
// (its time is otherwise the latency of single warps on the largest groups).
__global__ void __launch_bounds__(PT, 1) k_adj_force(View v, AdjWork w) {
  DevState *ds = v.ds;
  __shared__ int s_go, s_nq, s_item;
  if (threadIdx.x == 0) {
    s_go = ds->halt ? 0 : 1;
    s_nq = ds->n_active_groups + ds->n_heavy_groups;
  }
  __syncthreads();
  if (!s_go) return;  // the whole block
  StageF st;
  stage_init(st);
  const int lane = lane_id();
  const int nq = s_nq;
  WarpCounters wc = {0, 0, 0, 0, 0, 0};
  if (nq <= 2 * (int)gridDim.x) {
    for (;;) {
      if (threadIdx.x == 0) s_item = atomicAdd(&ds->head_force, 1);
      __syncthreads();
      const int item = s_item;
      __syncthreads();
      if (item >= nq || st.failed) break;  // (st.failed is the same in every warp)
      const int wg = active_group(v, ds, item);
      if (!SPH_IN(ds, wg, ds->n_groups, SPH_CHECK_GROUP)) break;
      force_adj_group<true>(v, w, wg, frame_of(v, ds, wg), st, wc);
    }
  } else {
    for (;;) {
      int item = 0;
      if (lane == 0) item = atomicAdd(&ds->head_force, 1);
      item = __shfl_sync(FULL, item, 0);
      if (item >= nq || st.failed) break;
      const int wg = active_group(v, ds, item);
      if (!SPH_IN(ds, wg, ds->n_groups, SPH_CHECK_GROUP)) break;
      force_adj_group<false>(v, w, wg, frame_of(v, ds, wg), st, wc);
    }
  }
  if (lane == 0 && wc.timeout) record_error(ds, SPH_ERR_TIMEOUT, wc.timeout, true);
}

// ---------------------------------------------------------------------------
// 4. equation-of-state adjoint (backward-build order)
// ---------------------------------------------------------------------------
// Q = f P / rho^2, c = sqrt(gamma P / rho), P = A_pred rho^gamma.  Leaves
// d loss / d A_pred in Qb and, on the first step (A_pred = (gamma - 1) u /
// rho^(gamma - 1)), d loss / d u in cb.
__global__ void k_adj_eos(View v, AdjWork w, sph_adjoint adj, int first) {
  const long long n = v.n;
  const double g = v.gamma;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const double rho = v.rho[k];
    if (!(rho > 0.0)) {
      w.Qb[k] = 0.0;
      w.cb[k] = 0.0;
      continue;
    }
    const double f = v.f[k], P = v.P[k], c = v.c[k], Ap = v.A[k];
    const double Qb = w.Qb[k], cbar = w.cb[k];
    double rb = w.rhob[k];
    w.fb[k] += Qb * P / (rho * rho);
    double Pb = Qb * f / (rho * rho);
    rb += -2.0 * Qb * (f * P / (rho * rho)) / rho;
    if (P > 0.0) Pb += cbar * c / (2.0 * P);
    rb += -cbar * c / (2.0 * rho);
    const double Apb = Pb * pow(rho, g);
    rb += Pb * g * P / rho;
    if (first) {
      // the entropy of the first step: A = (gamma - 1) u / rho^(gamma - 1);
      // the state's A adjoint (after the kicks) and A_pred's both land on it
      const double Ab = adj.A[w.perm[k]] + Apb;
      w.cb[k] = Ab * (g - 1.0) / pow(rho, g - 1.0);  // d loss / d u
      rb += Ab * Ap * (1.0 - g) / rho;
    } else {
      w.cb[k] = 0.0;
    }
    w.Qb[k] = Apb;
    w.rhob[k] = rb;
  }
}

// ---------------------------------------------------------------------------
// 5. density adjoint (two passes over the pairs r < H_i of the active i)
// ---------------------------------------------------------------------------
// Pass 1 sums, per active i (q = r / H, w and derivatives over 8/pi, self
// included where it contributes):
//   sr = sum m w,  srt = sum m (3 w + q w'),  s1 = sum q w',
//   s2 = sum m q (4 w' + q w'')
// rho = (8/pi) sr / H^3, f = 3 sr / (3 sr - srt), F = (8/pi)/GAMMA_K^3 sum w - eta^3.
// With h_bar the adjoint of h as an output, the total h adjoint is
//   hbt = h_bar + rho_bar d rho/dh + f_bar d f/dh   (explicit h-dependence)
// and the implicit solve turns it into lambda = -hbt / F_h, F_h = -(8/pi)/GAMMA_K^3 s1 / h.
// Pass 2: every pair's r-derivative r_bar = (ka m_j w' + kb m_j (4 w' + q w'') + km w') / H.
template <int PASS, bool COOP>
__device__ void density_adj_group(const View &v, const AdjWork &w, int wg, const CellFrame &F,
                                  StageD &st, WarpCounters &wc) {
  const int lane = lane_id();
  const int warp = threadIdx.x >> 5;
  const Group Wg = group_of(v, wg, F);
  const int a = Wg.a, b = Wg.b;
  const int nact = leaf_actives(v, a, b, 0, -1, st.act);
  if (nact == 0) return;
  const float qox = F.kx * F.wq, qoy = F.ky * F.wq, qoz = F.kz * F.wq;
  const float clx = Wg.lx + qox, cly = Wg.ly + qoy, clz = Wg.lz + qoz;
  const float chx = Wg.hx + qox, chy = Wg.hy + qoy, chz = Wg.hz + qoz;
  const float ceps = 1e-5f * F.wf;
  const float4 *srcs[1] = {v.rec_xm};
  const bool valid = lane < nact;
  const int i = valid ? st.act[lane] : a;
  const float4 xl = v.rec_xm[i];
  const float3 lo3 = leaf_offset(v, i, F);
  const float4 xi = make_float4(xl.x + lo3.x, xl.y + lo3.y, xl.z + lo3.z, xl.w);
  const float H = GAMMA_K * v.h[i];
  const float Hinv = 1.0f / H;
  const float H2 = H * H;
  float ka = 0.0f, kb = 0.0f, km = 0.0f;
  bool live;
  if (PASS == 1) {
    live = valid && (w.hb[i] != 0.0 || w.rhob[i] != 0.0 || w.fb[i] != 0.0);
  } else {
    if (valid) {
      ka = (float)w.ka[i];
      kb = (float)w.kb[i];
      km = (float)w.km[i];
    }
    live = valid && (ka != 0.0f || kb != 0.0f || km != 0.0f);
  }
  const float Hs = warp_max(live ? H : 0.0f);
  const int nsph = compact_spheres(st.sph, live, make_float4(xi.x, xi.y, xi.z, H));
  // FP32 partial sums per neighbour cell, folded into FP64 where the cell changes
  double sr = 0.0, srt = 0.0, s1 = 0.0, s2 = 0.0;
  double dxi = 0.0, dyi = 0.0, dzi = 0.0;
  float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
  int cur = -1;
  auto fold_cell = [&]() {
    if (PASS == 1) {
      sr += (double)p0; srt += (double)p1; s1 += (double)p2; s2 += (double)p3;
    } else {
      dxi += (double)p0; dyi += (double)p1; dzi += (double)p2;
    }
    p0 = p1 = p2 = p3 = 0.f;
  };
  const float R2 = Hs * Hs * 1.0002f, Rc = Hs + ceps;
  auto leaf_ok = [&](int l, float sx, float sy, float sz, LeafBox &lb) {
    const float4 lo = v.leaf_lo[l], hi = v.leaf_hi[l];
    lb = leaf_box(lo, hi, sx, sy, sz, 0.0f);
    return box_gap2(Wg.lx, Wg.ly, Wg.lz, Wg.hx, Wg.hy, Wg.hz, lo, hi, sx, sy, sz) < R2;
  };
  auto chunk_ok = [&](int gg, float sx, float sy, float sz) {
    return box_gap2(clx, cly, clz, chx, chy, chz, v.chunk_lo[gg], v.chunk_hi[gg], sx, sy, sz) <
           Rc * Rc;
  };
  auto consume = [&](int base, int total) {
    const int end = base + total;
    for (int k0 = base; k0 < end; k0 += 32) {
      unsigned mask = 0u;
#pragma unroll
      for (int u = 0; u < 32; u++) {
        const float4 pj = st.rec[min(k0 + u, S_DENS - 1)];
        const float dx = xi.x - pj.x, dy = xi.y - pj.y, dz = xi.z - pj.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        mask |= (k0 + u < end && r2 < H2) ? (1u << u) : 0u;
      }
      if (!live) mask = 0u;
      while (mask) {
        const int k = k0 + __ffs(mask) - 1;
        mask &= mask - 1;
        const int j = st.recj[k];
        const int ci = st.recc[k];
        if (ci != cur) {
          fold_cell();
          cur = ci;
        }
        const float4 pj = st.rec[k];
        const float dx = xi.x - pj.x, dy = xi.y - pj.y, dz = xi.z - pj.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float rr = r2 * rsqrtf(fmaxf(r2, 1e-30f));
        const float q = rr * Hinv;
        float wq, dwq;
        kernel_wd(q, wq, dwq);
        const float d2 = kernel_d2w(q);
        if (PASS == 1) {
          p0 += pj.w * wq;
          p1 += pj.w * fmaf(q, dwq, 3.0f * wq);
          p2 += q * dwq;
          p3 += pj.w * q * fmaf(q, d2, 4.0f * dwq);
        } else {
          if (j == i || !(r2 > 0.0f)) continue;
          const float rbar = (ka * pj.w * dwq + kb * pj.w * fmaf(q, d2, 4.0f * dwq) + km * dwq) * Hinv;
          const float rinv = rsqrtf(r2);
          const float bx = rbar * dx * rinv, by = rbar * dy * rinv, bz = rbar * dz * rinv;
          p0 += bx; p1 += by; p2 += bz;
          atomicAdd(&w.xb[j], -(double)bx);
          atomicAdd(&w.yb[j], -(double)by);
          atomicAdd(&w.zb[j], -(double)bz);
        }
      }
    }
  };
  int skip = 0, nlist = 0;
  bool more = false;
  const Reach reach = {clx, cly, clz, chx, chy, chz, Rc, __uint_as_float(v.ds->excursion_bits),
                       st.sph, nsph};
  if (Hs > 0.0f) {
    do {
      nlist = search(v, F, reach, st, leaf_ok, chunk_ok, skip, more, COOP ? warp : -1);
      stage_list(srcs, st, nlist, consume, wc);
      skip += nlist;
    } while (more && !st.failed);
  }
  fold_cell();
  if constexpr (COOP) {
    double sum[4] = {PASS == 1 ? sr : dxi, PASS == 1 ? srt : dyi, PASS == 1 ? s1 : dzi, s2};
    bool failed = st.failed;
    coop_reduce<StageD, 4>(sum, failed);
    st.failed = failed;  // the same in every warp
    if (PASS == 1) {
      sr = sum[0]; srt = sum[1]; s1 = sum[2]; s2 = sum[3];
    } else {
      dxi = sum[0]; dyi = sum[1]; dzi = sum[2];
    }
    if (warp != 0) return;  // the first warp writes the results
  }
  if (PASS == 1 && valid && !live) {
    // nothing flows back through this particle's density
    w.ka[i] = 0.0;
    w.kb[i] = 0.0;
    w.km[i] = 0.0;
  } else if (PASS == 1 && live) {
    // (the self pair r = 0 was among the records: w(0) = 1, w'(0) = 0)
    const double h = (double)v.h[i];
    const double Hd = (double)GAMMA_K * h;
    const double H3 = Hd * Hd * Hd;
    const double D = 3.0 * sr - srt;
    const double dfdsr = -3.0 * srt / (D * D), dfdsrt = 3.0 * sr / (D * D);
    const double drho_dh = -KN_D * srt / (H3 * h);
    const double S1 = srt - 3.0 * sr;  // sum m q w'
    const double df_dh = dfdsr * (-S1 / h) + dfdsrt * (-s2 / h);
    const double g3 = (double)GAMMA_K * (double)GAMMA_K * (double)GAMMA_K;
    const double Fh = -(KN_D / g3) * s1 / h;
    const double rb = w.rhob[i], fbar = w.fb[i];
    const double hbt = w.hb[i] + rb * drho_dh + fbar * df_dh;
    const double lam = Fh != 0.0 ? -hbt / Fh : 0.0;
    w.ka[i] = rb * KN_D / H3 + fbar * dfdsr;
    w.kb[i] = fbar * dfdsrt;
    w.km[i] = lam * KN_D / g3;
    // consumed: this step computed h, rho and f of i
    w.hb[i] = 0.0;
    w.rhob[i] = 0.0;
    w.fb[i] = 0.0;
  } else if (PASS == 2 && live) {
    atomicAdd(&w.xb[i], dxi);
    atomicAdd(&w.yb[i], dyi);
    atomicAdd(&w.zb[i], dzi);
  }
  __syncwarp();
}

// (as k_adj_force: a whole block per group in steps with few groups)
template <int PASS>
__global__ void __launch_bounds__(PT, 1) k_adj_density(View v, AdjWork w) {
  DevState *ds = v.ds;
  __shared__ int s_go, s_nq, s_item;
  if (threadIdx.x == 0) {
    s_go = ds->halt ? 0 : 1;
    s_nq = ds->n_active_groups + ds->n_heavy_groups;
  }
  __syncthreads();
  if (!s_go) return;  // the whole block
  StageD st;
  stage_init(st);
  const int lane = lane_id();
  const int nq = s_nq;
  int *head = PASS == 1 ? &ds->head_density : &ds->head_misc;
  WarpCounters wc = {0, 0, 0, 0, 0, 0};
  if (nq <= 2 * (int)gridDim.x) {
    for (;;) {
      if (threadIdx.x == 0) s_item = atomicAdd(head, 1);
      __syncthreads();
      const int item = s_item;
      __syncthreads();
      if (item >= nq || st.failed) break;  // (st.failed is the same in every warp)
      const int wg = active_group(v, ds, item);
      if (!SPH_IN(ds, wg, ds->n_groups, SPH_CHECK_GROUP)) break;
      density_adj_group<PASS, true>(v, w, wg, frame_of(v, ds, wg), st, wc);
    }
  } else {
    for (;;) {
      int item = 0;
      if (lane == 0) item = atomicAdd(head, 1);
      item = __shfl_sync(FULL, item, 0);
      if (item >= nq || st.failed) break;
      const int wg = active_group(v, ds, item);
      if (!SPH_IN(ds, wg, ds->n_groups, SPH_CHECK_GROUP)) break;
      density_adj_group<PASS, false>(v, w, wg, frame_of(v, ds, wg), st, wc);
    }
  }
  if (lane == 0 && wc.timeout) record_error(ds, SPH_ERR_TIMEOUT, wc.timeout, true);
}

// ---------------------------------------------------------------------------
// 6. back to caller order: prediction and drift adjoints
// ---------------------------------------------------------------------------
__global__ void k_adj_scatter(View v, AdjWork w, sph_particles pre, sph_particles post,
                              sph_adjoint adj, long long ti, int first, double dt_min) {
  const long long n = v.n;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const int o = w.perm[k];
    const double xb = w.xb[k], yb = w.yb[k], zb = w.zb[k];
    adj.x[o] = xb;
    adj.y[o] = yb;
    adj.z[o] = zb;
    // drift of this step: x(ti) = x + v (ti - ti_drift) dt_min, for the
    // particles the forward drifted (those whose ti_drift moved)
    const double dtd = (double)(post.ti_drift[o] - pre.ti_drift[o]) * dt_min;
    // prediction: v_pred = v + a dtp, A_pred = A + Adot dtp
    const int bi = pre.bin[o] & (MAX_BINS - 1);
    const double dtp = ((double)(ti - pre.ti_begin[o]) - 0.5 * (double)(1ll << bi)) * dt_min;
    const double vpx = w.vpxb[k], vpy = w.vpyb[k], vpz = w.vpzb[k];
    adj.vx[o] += vpx + xb * dtd;
    adj.vy[o] += vpy + yb * dtd;
    adj.vz[o] += vpz + zb * dtd;
    adj.ax[o] += vpx * dtp;
    adj.ay[o] += vpy * dtp;
    adj.az[o] += vpz * dtp;
    if (first) {
      adj.A[o] = w.cb[k];  // A held u before the first step
    } else {
      adj.A[o] += w.Qb[k];
      adj.Adot[o] += w.Qb[k] * dtp;
    }
    adj.h[o] = w.hb[k];
    adj.rho[o] = w.rhob[k];
    adj.f[o] = w.fb[k];
  }
}

// ---------------------------------------------------------------------------
// grid-density loss
// ---------------------------------------------------------------------------
// Range of grid indices (unwrapped) whose point centres (a + 1/2) s lie within
// H of x along one axis; at most n_grid of them.
__device__ __forceinline__ void grid_range(double x, double H, double s, int ng, int &a0, int &cnt) {
  a0 = (int)ceil((x - H) / s - 0.5);
  const int a1 = (int)floor((x + H) / s - 0.5);
  cnt = min(a1 - a0 + 1, ng);
}

__device__ __forceinline__ double kernel_w_d(double q) {
  if (q < 0.5) return 1.0 - 6.0 * q * q + 6.0 * q * q * q;
  if (q < 1.0) {
    const double s = 1.0 - q;
    return 2.0 * s * s * s;
  }
  return 0.0;
}

__device__ __forceinline__ double kernel_dw_d(double q) {
  if (q < 0.5) return -12.0 * q + 18.0 * q * q;
  if (q < 1.0) {
    const double s = 1.0 - q;
    return -6.0 * s * s;
  }
  return 0.0;
}

// One thread per particle: adds m W(|x_g - x|, h) to every grid point within
// its support (FP64 atomics); with BWD, reads d loss / d rho_g instead and
// accumulates d loss / d x, d h (and d v through the drift to the tick).
template <bool BWD>
__global__ void k_grid_density(sph_particles p, int ng, long long ti, double dt_min, double box,
                               double *rho_g, const double *rho_bar, sph_adjoint adj) {
  const long long n = p.n;
  const double s = box / ng;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    const double dtd = (double)(ti - p.ti_drift[j]) * dt_min;
    const double x = wrap_box(p.x[j] + (double)p.vx[j] * dtd, box);
    const double y = wrap_box(p.y[j] + (double)p.vy[j] * dtd, box);
    const double z = wrap_box(p.z[j] + (double)p.vz[j] * dtd, box);
    const double h = p.h[j], m = p.m[j];
    const double H = GAMMA_K_D * h;
    const double Hinv = 1.0 / H;
    const double H3inv = Hinv * Hinv * Hinv;
    int ax, cx, ay, cy, az, cz;
    grid_range(x, H, s, ng, ax, cx);
    grid_range(y, H, s, ng, ay, cy);
    grid_range(z, H, s, ng, az, cz);
    double gx = 0.0, gy = 0.0, gz = 0.0, gh = 0.0;
    for (int c = 0; c < cz; c++) {
      const int iz = ((az + c) % ng + ng) % ng;
      const double dz = min_img(z - (iz + 0.5) * s, box);
      for (int b = 0; b < cy; b++) {
        const int iy = ((ay + b) % ng + ng) % ng;
        const double dy = min_img(y - (iy + 0.5) * s, box);
        for (int a = 0; a < cx; a++) {
          const int ix = ((ax + a) % ng + ng) % ng;
          const double dx = min_img(x - (ix + 0.5) * s, box);
          const double r2 = dx * dx + dy * dy + dz * dz;
          if (!(r2 < H * H)) continue;
          const long long gidx = ix + (long long)ng * (iy + (long long)ng * iz);
          const double r = sqrt(r2);
          const double q = r * Hinv;
          if (!BWD) {
            atomicAdd(&rho_g[gidx], m * KN_D * kernel_w_d(q) * H3inv);
          } else {
            const double gb = rho_bar[gidx];
            const double wp = kernel_dw_d(q);
            if (r > 0.0) {
              const double t = gb * m * KN_D * wp * H3inv * Hinv / r;  // dW/dr / r
              gx += t * dx;
              gy += t * dy;
              gz += t * dz;
            }
            // dW/dh = -GAMMA_K (8/pi) H^-4 (3 w + q w')
            gh += gb * m * (-GAMMA_K_D * KN_D * H3inv * Hinv *
                            (3.0 * kernel_w_d(q) + q * wp));
          }
        }
      }
    }
    if (BWD) {
      adj.x[j] += gx;
      adj.y[j] += gy;
      adj.z[j] += gz;
      adj.vx[j] += gx * dtd;
      adj.vy[j] += gy * dtd;
      adj.vz[j] += gz * dtd;
      adj.h[j] += gh;
    }
  }
}

// ---------------------------------------------------------------------------
// state copy (optionally into the caller's order)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void cp(T *dst, const T *src, long long d, long long s) {
  if (dst && src) dst[d] = src[s];
}

__global__ void k_state_copy(sph_particles src, sph_particles dst, const int32_t *perm) {
  const long long n = src.n;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const long long d = perm ? (long long)perm[k] : k;
    cp(dst.x, src.x, d, k); cp(dst.y, src.y, d, k); cp(dst.z, src.z, d, k);
    cp(dst.vx, src.vx, d, k); cp(dst.vy, src.vy, d, k); cp(dst.vz, src.vz, d, k);
    cp(dst.ax, src.ax, d, k); cp(dst.ay, src.ay, d, k); cp(dst.az, src.az, d, k);
    cp(dst.A, src.A, d, k); cp(dst.Adot, src.Adot, d, k); cp(dst.h, src.h, d, k);
    cp(dst.rho, src.rho, d, k); cp(dst.f, src.f, d, k); cp(dst.P, src.P, d, k);
    cp(dst.c, src.c, d, k); cp(dst.vsig, src.vsig, d, k); cp(dst.m, src.m, d, k);
    cp(dst.bin, src.bin, d, k); cp(dst.ti_begin, src.ti_begin, d, k);
    cp(dst.ti_end, src.ti_end, d, k); cp(dst.ti_drift, src.ti_drift, d, k);
    cp(dst.active, src.active, d, k);
    cp(dst.ngb_density, src.ngb_density, d, k); cp(dst.ngb_force, src.ngb_force, d, k);
    cp(dst.div_v, src.div_v, d, k); cp(dst.curl_v, src.curl_v, d, k);
  }
}

constexpr size_t ADJ_DENS_SMEM = StageD::bytes() * WARPS_PER_BLOCK;
constexpr size_t ADJ_FORCE_SMEM = StageF::bytes() * WARPS_PER_BLOCK;

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  if (g < 1) g = 1;
  if (g > 4096) g = 4096;
  return (int)g;
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_adj_prepare(const sph_particles &pre, const sph_particles &post,
                               const sph_particles &W, const sph_adjoint &adj, long long ti,
                               int first, double dt_min, double box, double gamma,
                               cudaStream_t st) {
  if (pre.n == 0) return cudaSuccess;
  note_launches(1);
  k_adj_prepare<<<grid_for(pre.n), 256, 0, st>>>(pre, post, W, adj, ti, first, dt_min, box, gamma);
  return cudaGetLastError();
}

cudaError_t launch_adj_step(const View &v, const AdjWork &w, const sph_particles &pre,
                            const sph_particles &post, const sph_adjoint &adj, long long ti,
                            int first, int grid_pairs, cudaStream_t st) {
  if (v.n == 0) return cudaSuccess;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_adj_force, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ADJ_FORCE_SMEM)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_adj_density<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ADJ_DENS_SMEM)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_adj_density<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ADJ_DENS_SMEM)) != cudaSuccess)
    return e;
  const int g = grid_for(v.n);
  note_launches(6);
  k_adj_gather<<<g, 256, 0, st>>>(v, w, adj, v.gamma);
  k_adj_force<<<grid_pairs, PT, ADJ_FORCE_SMEM, st>>>(v, w);
  k_adj_eos<<<g, 256, 0, st>>>(v, w, adj, first);
  k_adj_density<1><<<grid_pairs, PT, ADJ_DENS_SMEM, st>>>(v, w);
  k_adj_density<2><<<grid_pairs, PT, ADJ_DENS_SMEM, st>>>(v, w);
  k_adj_scatter<<<g, 256, 0, st>>>(v, w, pre, post, adj, ti, first, v.dt_min);
  return cudaGetLastError();
}

cudaError_t launch_grid_density(const sph_particles &p, int n_grid, long long ti, double dt_min,
                                double box, double *rho_g, const double *rho_bar,
                                const sph_adjoint *adj, cudaStream_t st) {
  if (p.n == 0) return cudaSuccess;
  note_launches(1);
  if (adj) {
    k_grid_density<true><<<grid_for(p.n), 256, 0, st>>>(p, n_grid, ti, dt_min, box, nullptr,
                                                        rho_bar, *adj);
  } else {
    sph_adjoint none;
    memset(&none, 0, sizeof(none));
    k_grid_density<false><<<grid_for(p.n), 256, 0, st>>>(p, n_grid, ti, dt_min, box, rho_g,
                                                         nullptr, none);
  }
  return cudaGetLastError();
}

// Resident blocks per SM of the adjoint pair kernels (the smallest over the
// three; 0 when they cannot run).
int adj_blocks_per_sm() {
  struct K {
    const void *fn;
    size_t smem;
  } ks[3] = {{(const void *)k_adj_force, ADJ_FORCE_SMEM},
             {(const void *)k_adj_density<1>, ADJ_DENS_SMEM},
             {(const void *)k_adj_density<2>, ADJ_DENS_SMEM}};
  int best = 1 << 30;
  for (const K &k : ks) {
    if (cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem) !=
        cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k.fn, PT, k.smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    best = nb < best ? nb : best;
  }
  return best;
}

cudaError_t launch_state_copy(const sph_particles &src, const sph_particles &dst,
                              const int32_t *perm, cudaStream_t st) {
  if (src.n == 0) return cudaSuccess;
  note_launches(1);
  k_state_copy<<<grid_for(src.n), 256, 0, st>>>(src, dst, perm);
  return cudaGetLastError();
}

}  // namespace sph
