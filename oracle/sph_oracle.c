/*
 * sph_oracle.c -- plain, slow FP64 CPU oracle of the SWIFT SPH hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this file; it shares no code, header, table or constant with the CUDA
 * path.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load it.
 *
 * What it computes (arXiv 1807.01341; the paper defers the SPH equations to
 * "a standard SPH scheme" in Sec. II, so the readings below are ours and are
 * listed, with their sources, in the design notes):
 *   - cubic-spline (M4) kernel with compact support H = GAMMA_K * h;
 *   - density rho_i = sum_j m_j W(r_ij, h_i) over r_ij < H_i (self included);
 *   - smoothing length: root of h^3 n(h) = eta^3 (n = sum_j W), solved with a
 *     bracket-safeguarded Newton iteration (the "ghost" task of Sec. III-B,
 *     which corrects h between the density and force loops);
 *   - grad-h factor f_i, density-entropy equation of state;
 *   - hydro force with Monaghan signal-velocity viscosity (its beta = 3 form is
 *     the one inside the CFL condition, Eq. 1);
 *   - the CFL time-step of Eq. 1 and the power-of-two time bins of Eq. 2 with
 *     the synchronisation rule for bin increases (Sec. II-A);
 *   - top-level cell index and the stable (cell, Morton) particle order used by
 *     the cell structure of Sec. III-A.
 *
 * Neighbour search: brute force over all j (mode 0), or the uniform cell grid
 * of Sec. III-A (mode 1): the 27 cells around i in a grid whose width is at
 * least the search radius.  Both visit exactly the same neighbour set; only the
 * order of the FP64 sums differs.
 *
 * Parity of every function here is pinned by tests against closed forms,
 * invariants and independent computations (kernel normalisation, lattice sums,
 * numerical derivatives, energy gradients, conservation laws, hand-computed
 * bins).  Build with -ffp-contract=off so no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846
/* Ratio of the kernel's compact support H to the smoothing length h for the
 * cubic spline in three dimensions (Dehnen & Aly 2012). */
#define ORC_GAMMA_K 1.825742

/* ------------------------------------------------------------------------- */
/* Kernel: w(q) on q = r / H in [0, 1), W(r, h) = H^-3 w(r / H).              */
/* ------------------------------------------------------------------------- */

double orc_kernel_w(double q) {
  if (q < 0.5) return (8.0 / ORC_PI) * (1.0 - 6.0 * q * q + 6.0 * q * q * q);
  if (q < 1.0) {
    double s = 1.0 - q;
    return (8.0 / ORC_PI) * 2.0 * s * s * s;
  }
  return 0.0;
}

double orc_kernel_dw(double q) {
  if (q < 0.5) return (8.0 / ORC_PI) * (-12.0 * q + 18.0 * q * q);
  if (q < 1.0) {
    double s = 1.0 - q;
    return (8.0 / ORC_PI) * (-6.0 * s * s);
  }
  return 0.0;
}

double orc_gamma_k(void) { return ORC_GAMMA_K; }

/* ------------------------------------------------------------------------- */
/* Periodic geometry                                                          */
/* ------------------------------------------------------------------------- */

static double min_image(double d, double box) {
  if (d > 0.5 * box) d -= box;
  else if (d < -0.5 * box) d += box;
  return d;
}

static double wrap(double x, double box) {
  if (x < 0.0) x += box;
  if (x >= box) x -= box;
  return x;
}

/* ------------------------------------------------------------------------- */
/* Neighbour search (Sec. III-A): a uniform grid of n_g^3 cells of width      */
/* >= the largest radius searched; a radius above the width falls back to     */
/* brute force for that particle.                                             */
/* ------------------------------------------------------------------------- */

typedef struct {
  int64_t n;
  const double *x, *y, *z;
  double box;
  int ng;            /* 0: brute force */
  double width;
  int64_t *start;    /* [ng^3 + 1] */
  int64_t *index;    /* [n] particles by cell, ascending index inside a cell */
} orc_grid;

static int cell_coord(double x, double width, int ng) {
  int c = (int)floor(wrap(x, width * ng) / width);
  if (c < 0) c = 0;
  if (c >= ng) c = ng - 1;
  return c;
}

static void grid_build(orc_grid *g, int64_t n, const double *x, const double *y,
                       const double *z, double box, double rmax, int use_cells) {
  g->n = n; g->x = x; g->y = y; g->z = z; g->box = box;
  g->ng = 0; g->start = NULL; g->index = NULL; g->width = box;
  if (!use_cells || !(rmax > 0.0)) return;
  int ng = (int)floor(box / rmax);
  if (ng > 256) ng = 256;
  if (ng < 3) return;
  g->ng = ng;
  g->width = box / ng;
  int64_t nc = (int64_t)ng * ng * ng;
  g->start = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
  g->index = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  int64_t *cid = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  for (int64_t i = 0; i < n; i++) {
    int cx = cell_coord(x[i], g->width, ng), cy = cell_coord(y[i], g->width, ng),
        cz = cell_coord(z[i], g->width, ng);
    cid[i] = ((int64_t)cx * ng + cy) * ng + cz;
    g->start[cid[i] + 1]++;
  }
  for (int64_t c = 0; c < nc; c++) g->start[c + 1] += g->start[c];
  int64_t *fill = (int64_t *)malloc((size_t)nc * sizeof(int64_t));
  memcpy(fill, g->start, (size_t)nc * sizeof(int64_t));
  for (int64_t i = 0; i < n; i++) g->index[fill[cid[i]]++] = i;
  free(fill);
  free(cid);
}

static void grid_free(orc_grid *g) {
  free(g->start);
  free(g->index);
  g->start = NULL;
  g->index = NULL;
}

/* Candidates for particle i at search radius r: every j when brute force (or
 * r above the grid width), else the particles of the 27 surrounding cells. */
static int64_t grid_candidates(const orc_grid *g, int64_t i, double r, int64_t *out) {
  if (g->ng == 0 || r > g->width) {
    for (int64_t j = 0; j < g->n; j++) out[j] = j;
    return g->n;
  }
  int ng = g->ng;
  int cx = cell_coord(g->x[i], g->width, ng), cy = cell_coord(g->y[i], g->width, ng),
      cz = cell_coord(g->z[i], g->width, ng);
  int64_t k = 0;
  for (int dx = -1; dx <= 1; dx++)
    for (int dy = -1; dy <= 1; dy++)
      for (int dz = -1; dz <= 1; dz++) {
        int ax = (cx + dx + ng) % ng, ay = (cy + dy + ng) % ng, az = (cz + dz + ng) % ng;
        int64_t c = ((int64_t)ax * ng + ay) * ng + az;
        for (int64_t s = g->start[c]; s < g->start[c + 1]; s++) out[k++] = g->index[s];
      }
  return k;
}

/* ------------------------------------------------------------------------- */
/* Density sums at fixed h                                                    */
/* ------------------------------------------------------------------------- */

typedef struct {
  double n, dn_dh, rho, drho_dh;
  int64_t count; /* neighbours j != i with r_ij < H_i */
} dens_sums;

static dens_sums density_sums(const orc_grid *g, const double *m, int64_t i, double h,
                              int64_t *cand) {
  dens_sums s = {0.0, 0.0, 0.0, 0.0, 0};
  double H = ORC_GAMMA_K * h;
  int64_t nc = grid_candidates(g, i, H, cand);
  for (int64_t k = 0; k < nc; k++) {
    int64_t j = cand[k];
    double dx = min_image(g->x[i] - g->x[j], g->box);
    double dy = min_image(g->y[i] - g->y[j], g->box);
    double dz = min_image(g->z[i] - g->z[j], g->box);
    double r2 = dx * dx + dy * dy + dz * dz;
    if (!(r2 < H * H)) continue;
    double q = sqrt(r2) / H;
    double w = orc_kernel_w(q);
    double dwq = orc_kernel_dw(q);
    /* dW/dh = -GAMMA_K H^-4 (3 w + q w') */
    double wh = -(3.0 * w + q * dwq);
    s.n += w;
    s.dn_dh += wh;
    s.rho += m[j] * w;
    s.drho_dh += m[j] * wh;
    if (j != i) s.count++;
  }
  double Hi = 1.0 / H;
  double Hi3 = Hi * Hi * Hi;
  double Hi4 = Hi3 * Hi;
  s.n *= Hi3;
  s.rho *= Hi3;
  s.dn_dh *= ORC_GAMMA_K * Hi4;
  s.drho_dh *= ORC_GAMMA_K * Hi4;
  return s;
}

/* Density at the given h (no iteration): rho, d rho / dh, n, dn / dh, count. */
void orc_density_fixed_h(int64_t n, const double *x, const double *y, const double *z,
                         const double *m, const double *h, const uint8_t *active,
                         double box, int use_cells, double *rho, double *drho_dh,
                         double *wn, double *dwn_dh, int64_t *count) {
  double hmax = 0.0;
  for (int64_t i = 0; i < n; i++)
    if (h[i] > hmax) hmax = h[i];
  orc_grid g;
  grid_build(&g, n, x, y, z, box, ORC_GAMMA_K * hmax, use_cells);
#pragma omp parallel
  {
    int64_t *cand = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; i++) {
      if (active && !active[i]) continue;
      dens_sums s = density_sums(&g, m, i, h[i], cand);
      rho[i] = s.rho;
      drho_dh[i] = s.drho_dh;
      wn[i] = s.n;
      dwn_dh[i] = s.dn_dh;
      count[i] = s.count;
    }
    free(cand);
  }
  grid_free(&g);
}

/* ------------------------------------------------------------------------- */
/* Smoothing-length solve: F(h) = h^3 n(h) - eta^3 = 0.  F is non-decreasing  */
/* in h, so a bracket [lo, hi] with F(lo) < 0 <= F(hi) is kept; a Newton step */
/* that leaves the bracket is replaced by bisection (or doubling while no     */
/* upper end is known), and every step is limited to [h/2, 2h].               */
/* ------------------------------------------------------------------------- */

typedef struct {
  double h;
  dens_sums s;
  int iters;
  int converged;
} h_solve;

static h_solve solve_h(const orc_grid *g, const double *m, int64_t i, double h0,
                       double eta, double tol, int max_iter, int64_t *cand) {
  h_solve r;
  double h = h0, lo = 0.0, hi = INFINITY;
  double eta3 = eta * eta * eta;
  r.converged = 0;
  r.iters = 0;
  for (int it = 0; it < max_iter; it++) {
    dens_sums s = density_sums(g, m, i, h, cand);
    r.iters = it + 1;
    double F = h * h * h * s.n - eta3;
    double dF = 3.0 * h * h * s.n + h * h * h * s.dn_dh;
    if (F < 0.0) lo = h;
    else hi = h;
    double hn;
    if (F == 0.0) hn = h;
    else if (dF > 0.0) hn = h - F / dF;
    else hn = NAN;
    if (!(hn >= lo && hn <= hi)) hn = isinf(hi) ? 2.0 * h : 0.5 * (lo + hi);
    if (hn < 0.5 * h) hn = 0.5 * h;
    if (hn > 2.0 * h) hn = 2.0 * h;
    if (fabs(hn - h) <= tol * h) {
      h = hn;
      r.converged = 1;
      break;
    }
    h = hn;
  }
  r.h = h;
  r.s = density_sums(g, m, i, h, cand);
  return r;
}

/* Density loop with smoothing-length iteration for the active particles.
 * h is read as the initial guess and overwritten with the solution.  Returns
 * the number of active particles that did not converge. */
int64_t orc_density(int64_t n, const double *x, const double *y, const double *z,
                    const double *m, double *h, const uint8_t *active, double box,
                    double eta, double tol, int max_iter, int use_cells, double *rho,
                    double *drho_dh, double *wn, double *dwn_dh, int64_t *count,
                    int32_t *iters) {
  double hmax = 0.0;
  for (int64_t i = 0; i < n; i++)
    if (h[i] > hmax) hmax = h[i];
  orc_grid g;
  /* the grid covers twice the largest initial support; any larger search
   * falls back to brute force for that particle */
  grid_build(&g, n, x, y, z, box, 2.0 * ORC_GAMMA_K * hmax, use_cells);
  int64_t bad = 0;
#pragma omp parallel reduction(+ : bad)
  {
    int64_t *cand = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; i++) {
      if (active && !active[i]) continue;
      h_solve r = solve_h(&g, m, i, h[i], eta, tol, max_iter, cand);
      h[i] = r.h;
      rho[i] = r.s.rho;
      drho_dh[i] = r.s.drho_dh;
      wn[i] = r.s.n;
      dwn_dh[i] = r.s.dn_dh;
      count[i] = r.s.count;
      if (iters) iters[i] = r.iters;
      if (!r.converged) bad++;
    }
    free(cand);
  }
  grid_free(&g);
  return bad;
}

/* ------------------------------------------------------------------------- */
/* Velocity divergence and curl at the particle's own h (the standard SPH     */
/* estimates used by Gadget-2; the paper names Gadget-2 as its reference      */
/* scheme, Sec. II): with v_ij = v_i - v_j and grad_i W = (r_ij / r) dW/dr,    */
/*   div v_i  = -(1 / rho_i) sum_j m_j v_ij . grad_i W(r_ij, h_i)              */
/*   curl v_i =  (1 / rho_i) sum_j m_j v_ij x grad_i W(r_ij, h_i)              */
/* over j with r_ij < H_i.                                                    */
/* ------------------------------------------------------------------------- */

void orc_gradient(int64_t n, const double *x, const double *y, const double *z,
                  const double *vx, const double *vy, const double *vz, const double *m,
                  const double *h, const double *rho, const uint8_t *active, double box,
                  int use_cells, double *divv, double *curlx, double *curly, double *curlz) {
  double hmax = 0.0;
  for (int64_t i = 0; i < n; i++)
    if (h[i] > hmax) hmax = h[i];
  orc_grid g;
  grid_build(&g, n, x, y, z, box, ORC_GAMMA_K * hmax, use_cells);
#pragma omp parallel
  {
    int64_t *cand = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; i++) {
      if (active && !active[i]) continue;
      double Hi = ORC_GAMMA_K * h[i];
      double sd = 0.0, cx = 0.0, cy = 0.0, cz = 0.0;
      int64_t nc = grid_candidates(&g, i, Hi, cand);
      for (int64_t k = 0; k < nc; k++) {
        int64_t j = cand[k];
        if (j == i) continue;
        double dx = min_image(x[i] - x[j], box);
        double dy = min_image(y[i] - y[j], box);
        double dz = min_image(z[i] - z[j], box);
        double r2 = dx * dx + dy * dy + dz * dz;
        if (!(r2 < Hi * Hi) || r2 == 0.0) continue;
        double r = sqrt(r2);
        /* grad_i W = (r_ij / r) dW/dr, dW/dr = H^-4 w'(r / H) */
        double g1 = m[j] * orc_kernel_dw(r / Hi) / (Hi * Hi * Hi * Hi) / r;
        double gx = g1 * dx, gy = g1 * dy, gz = g1 * dz;
        double wx = vx[i] - vx[j], wy = vy[i] - vy[j], wz = vz[i] - vz[j];
        sd += wx * gx + wy * gy + wz * gz;
        cx += wy * gz - wz * gy;
        cy += wz * gx - wx * gz;
        cz += wx * gy - wy * gx;
      }
      divv[i] = -sd / rho[i];
      curlx[i] = cx / rho[i];
      curly[i] = cy / rho[i];
      curlz[i] = cz / rho[i];
    }
    free(cand);
  }
  grid_free(&g);
}

/* Balsara (1995) switch in the form Gadget-2 uses:
 * B = |div v| / (|div v| + |curl v| + 1e-4 c / h). */
double orc_balsara(double divv, double curl, double c, double h) {
  double a = fabs(divv);
  return a / (a + fabs(curl) + 1e-4 * c / h);
}

/* ------------------------------------------------------------------------- */
/* Hydro force loop (pressure with grad-h terms plus artificial viscosity)    */
/* for the active particles; j runs over r_ij < max(H_i, H_j), j != i.        */
/* ------------------------------------------------------------------------- */

void orc_force(int64_t n, const double *x, const double *y, const double *z,
               const double *vx, const double *vy, const double *vz, const double *m,
               const double *h, const double *rho, const double *f, const double *P,
               const double *c, const uint8_t *active, double box, double alpha,
               double gamma, int use_cells, const double *balsara, const int8_t *bin,
               double *ax, double *ay, double *az, double *Adot, double *vsig,
               int64_t *count, int8_t *bin_ngb_min) {
  double hmax = 0.0;
  for (int64_t i = 0; i < n; i++)
    if (h[i] > hmax) hmax = h[i];
  double Hmax = ORC_GAMMA_K * hmax;
  orc_grid g;
  grid_build(&g, n, x, y, z, box, Hmax, use_cells);
#pragma omp parallel
  {
    int64_t *cand = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; i++) {
      if (active && !active[i]) continue;
      double Hi = ORC_GAMMA_K * h[i];
      double PoRho2i = f[i] * P[i] / (rho[i] * rho[i]);
      double sax = 0.0, say = 0.0, saz = 0.0, sA = 0.0;
      double vs = 2.0 * c[i];
      int64_t cnt = 0;
      int bmin = 127; /* smallest time bin among the neighbours */
      int64_t nc = grid_candidates(&g, i, Hmax, cand);
      for (int64_t k = 0; k < nc; k++) {
        int64_t j = cand[k];
        if (j == i) continue;
        double Hj = ORC_GAMMA_K * h[j];
        double dx = min_image(x[i] - x[j], box);
        double dy = min_image(y[i] - y[j], box);
        double dz = min_image(z[i] - z[j], box);
        double r2 = dx * dx + dy * dy + dz * dz;
        if (!(r2 < Hi * Hi || r2 < Hj * Hj)) continue;
        cnt++;
        if (bin && bin[j] < bmin) bmin = bin[j];
        double r = sqrt(r2);
        double dvx = vx[i] - vx[j], dvy = vy[i] - vy[j], dvz = vz[i] - vz[j];
        double dvdr = dvx * dx + dvy * dy + dvz * dz;
        if (r == 0.0) {
          /* coincident particles: no direction, no gradient; only the signal
           * velocity sees the pair */
          double v = c[i] + c[j];
          if (v > vs) vs = v;
          continue;
        }
        /* dW/dr for each smoothing length (zero outside its own support) */
        double dWi = orc_kernel_dw(r / Hi) / (Hi * Hi * Hi * Hi);
        double dWj = orc_kernel_dw(r / Hj) / (Hj * Hj * Hj * Hj);
        double PoRho2j = f[j] * P[j] / (rho[j] * rho[j]);
        /* Monaghan (1997) signal-velocity viscosity, beta = 3 (Eq. 1) */
        double wij = dvdr / r;
        if (wij > 0.0) wij = 0.0;
        double vsig_ij = c[i] + c[j] - 3.0 * wij;
        double Pi = -0.5 * alpha * vsig_ij * wij / (0.5 * (rho[i] + rho[j]));
        /* Balsara switch: the mean of the two particles' factors */
        if (balsara) Pi *= 0.5 * (balsara[i] + balsara[j]);
        double dWbar = 0.5 * (dWi + dWj);
        /* grad_i W = (r_ij / r) dW/dr */
        double s = m[j] * (PoRho2i * dWi + PoRho2j * dWj + Pi * dWbar) / r;
        sax -= s * dx;
        say -= s * dy;
        saz -= s * dz;
        sA += m[j] * Pi * (dvdr / r) * dWbar;
        if (vsig_ij > vs) vs = vsig_ij;
      }
      ax[i] = sax;
      ay[i] = say;
      az[i] = saz;
      Adot[i] = 0.5 * (gamma - 1.0) * pow(rho[i], 1.0 - gamma) * sA;
      vsig[i] = vs;
      if (count) count[i] = cnt;
      if (bin_ngb_min) bin_ngb_min[i] = (int8_t)bmin;
    }
    free(cand);
  }
  grid_free(&g);
}

/* ------------------------------------------------------------------------- */
/* Waking of inactive neighbours (Saitoh & Makino 2009, second half; the     */
/* reading of Durier & Dalla Vecchia 2012 with the bins of the step): for    */
/* every active i and every inactive j != i with r_ij < max(H_i, H_j) (the   */
/* force loop's pairs) whose bin exceeds bin_i + 2, req[j] = the smallest    */
/* such bin_i + 2; req[j] = 127 where no active neighbour asks.  A plain     */
/* serial double loop over the force loop's candidate grid.                  */
/* ------------------------------------------------------------------------- */

void orc_wake_bins(int64_t n, const double *x, const double *y, const double *z,
                   const double *h, const uint8_t *active, const int8_t *bin, double box,
                   int use_cells, int8_t *req) {
  double hmax = 0.0;
  for (int64_t i = 0; i < n; i++) {
    req[i] = 127;
    if (h[i] > hmax) hmax = h[i];
  }
  double Hmax = ORC_GAMMA_K * hmax;
  orc_grid g;
  grid_build(&g, n, x, y, z, box, Hmax, use_cells);
  int64_t *cand = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  for (int64_t i = 0; i < n; i++) {
    if (!active[i]) continue;
    double Hi = ORC_GAMMA_K * h[i];
    int64_t nc = grid_candidates(&g, i, Hmax, cand);
    for (int64_t k = 0; k < nc; k++) {
      int64_t j = cand[k];
      if (j == i || active[j]) continue;
      double Hj = ORC_GAMMA_K * h[j];
      double dx = min_image(x[i] - x[j], box);
      double dy = min_image(y[i] - y[j], box);
      double dz = min_image(z[i] - z[j], box);
      double r2 = dx * dx + dy * dy + dz * dz;
      if (!(r2 < Hi * Hi || r2 < Hj * Hj)) continue;
      int want = bin[i] + 2;
      if (bin[j] > want && want < req[j]) req[j] = (int8_t)want;
    }
  }
  free(cand);
  grid_free(&g);
}

/* ------------------------------------------------------------------------- */
/* Time-step (Eq. 1) and time bins (Eq. 2) on the integer timeline           */
/* ------------------------------------------------------------------------- */

/* Bin of a time-step: the largest n with dt >= 2^n dt_min, capped at bin_cap.
 * Returns -1 when dt < dt_min (or is not a number). */
int orc_bin_of_dt(double dt, double dt_min, int bin_cap) {
  double q = dt / dt_min;
  if (!(q >= 1.0)) return -1;
  int e;
  frexp(q, &e); /* q = mant * 2^e, mant in [0.5, 1) => floor(log2 q) = e - 1 */
  int b = e - 1;
  if (b > bin_cap) b = bin_cap;
  return b;
}

/* New bins for the active particles at ti_current.  Increases of the bin are
 * accepted only while ti_current is a multiple of the new step (Gadget-2
 * synchronisation); decreases are always accepted.  Returns the number of
 * particles whose dt fell below dt_min (they are put on bin 0). */
/* With bin_ngb_min (may be NULL): the Saitoh & Makino (2009) time-step
 * limiter on the neighbours, dt_i <= 4 min_j dt_j, i.e. a new bin at most
 * 2 above the smallest bin among the particle's force neighbours; applied
 * before the synchronisation rule. */
int64_t orc_timestep_bins(int64_t n, const double *h, const double *vsig,
                          const uint8_t *active, double cfl, double dt_min, int bin_cap,
                          int64_t ti_current, const int8_t *bin_ngb_min, int8_t *bin,
                          int64_t *ti_begin, int64_t *ti_end, double *dt_out) {
  int64_t bad = 0;
  for (int64_t i = 0; i < n; i++) {
    if (active && !active[i]) continue;
    double dt = cfl * h[i] / vsig[i];
    if (dt_out) dt_out[i] = dt;
    int b = orc_bin_of_dt(dt, dt_min, bin_cap);
    if (b < 0) {
      bad++;
      b = 0;
    }
    if (bin_ngb_min && b > bin_ngb_min[i] + 2) b = bin_ngb_min[i] + 2;
    int old = bin[i];
    while (b > old && (ti_current % ((int64_t)1 << b)) != 0) b--;
    bin[i] = (int8_t)b;
    ti_begin[i] = ti_current;
    ti_end[i] = ti_current + ((int64_t)1 << b);
  }
  return bad;
}

/* ------------------------------------------------------------------------- */
/* Top-level cells (Sec. III-A): cell index of the wrapped position in an     */
/* n_c^3 grid and the stable order by (cell, Morton code inside the cell).    */
/* ------------------------------------------------------------------------- */

#define ORC_MORTON_BITS 10

static uint64_t spread3(uint64_t v) {
  uint64_t r = 0;
  for (int b = 0; b < ORC_MORTON_BITS; b++) r |= ((v >> b) & 1u) << (3 * b);
  return r;
}

typedef struct {
  uint64_t key;
  int64_t idx;
} key_idx;

static int cmp_key_idx(const void *a, const void *b) {
  const key_idx *p = (const key_idx *)a, *q = (const key_idx *)b;
  if (p->key < q->key) return -1;
  if (p->key > q->key) return 1;
  return (p->idx < q->idx) ? -1 : (p->idx > q->idx);
}

static int axis_cell(double x, double w, int nc) {
  int c = (int)floor(x / w);
  if (c < 0) c = 0;
  if (c > nc - 1) c = nc - 1;
  return c;
}

static uint64_t axis_morton(double x, int c, double w) {
  double t = (x - (double)c * w) / w;
  t = t * (double)(1 << ORC_MORTON_BITS);
  double ft = floor(t);
  int64_t q = (int64_t)ft;
  if (ft < 0.0) q = 0;
  if (q > (1 << ORC_MORTON_BITS) - 1) q = (1 << ORC_MORTON_BITS) - 1;
  return (uint64_t)q;
}

/* x, y, z are wrapped into [0, box) in place.  Outputs: cell[i] (flattened
 * (cx * nc + cy) * nc + cz), key[i] = cell << 30 | morton, and perm[k] = the
 * original index of the particle at sorted position k. */
void orc_cells(int64_t n, double *x, double *y, double *z, double box, int nc,
               int64_t *cell, uint64_t *key, int64_t *perm) {
  double w = box / (double)nc;
  key_idx *ki = (key_idx *)malloc((size_t)(n > 0 ? n : 1) * sizeof(key_idx));
  for (int64_t i = 0; i < n; i++) {
    x[i] = wrap(x[i], box);
    y[i] = wrap(y[i], box);
    z[i] = wrap(z[i], box);
    int cx = axis_cell(x[i], w, nc), cy = axis_cell(y[i], w, nc), cz = axis_cell(z[i], w, nc);
    int64_t cid = ((int64_t)cx * nc + cy) * nc + cz;
    uint64_t mort = (spread3(axis_morton(x[i], cx, w)) << 2) |
                    (spread3(axis_morton(y[i], cy, w)) << 1) |
                    spread3(axis_morton(z[i], cz, w));
    cell[i] = cid;
    key[i] = ((uint64_t)cid << (3 * ORC_MORTON_BITS)) | mort;
    ki[i].key = key[i];
    ki[i].idx = i;
  }
  qsort(ki, (size_t)n, sizeof(key_idx), cmp_key_idx);
  for (int64_t k = 0; k < n; k++) perm[k] = ki[k].idx;
  free(ki);
}

/* Threads the oracle runs with (OpenMP), for the CPU-baseline record. */
int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_num_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}
