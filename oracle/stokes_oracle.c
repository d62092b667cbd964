/*
 * stokes_oracle.c -- plain FP64 CPU definition of the Stokes layer-potential
 * sums.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
 * benchmark's CPU-baseline leg call it to check and time the GPU library; the
 * GPU library never links, loads or calls it, and the two share no code.
 *
 * Every sum is the plain O(Ns * Nt) double loop of the discrete quadrature
 * (Sec. 3.1, Eq. "smooth_double_layer_int_eq_patches_disc"): the integral of
 * a kernel against a density becomes sum_j K(x, y_j) w_j density_j.
 *
 *   single layer (Eq. "sl_stokes"):  S(x, y) = (1 / (8 pi mu)) (I / |r| + r r^T / |r|^3)
 *   double layer (Sec. 2.1):         D(x, y) = (6 / (8 pi)) r r^T (r . n(y)) / |r|^5
 *   with r = x - y and n(y) the outward unit normal at the source.
 *
 * Readings where the paper is garbled or silent:
 *   - the single-layer "1/r" is the identity divided by |r| (Oseen tensor);
 *   - the double-layer kernel carries no viscosity and its sign is as printed;
 *   - a pair at exactly zero distance (the self pair when targets are the
 *     sources) contributes nothing;
 *   - the quadrature weight multiplies the density.
 *
 * Accumulation: per target and component, Neumaier-compensated FP64 sums
 * in source order.  OpenMP parallelises over independent outputs only, so
 * results do not depend on the thread count.
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared.
 */
#include "stokes_oracle.h"

#include <math.h>
#include <stddef.h>

#define ORC_PI 3.14159265358979323846

typedef struct { double s, c; } neum;

static inline void neum_add(neum *a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
  else a->c += (v - t) + a->s;
  a->s = t;
}
static inline double neum_val(const neum *a) { return a->s + a->c; }

/* Single-layer contribution of source j at target x (unscaled by 1/(8 pi mu)). */
static inline int sl_pair(const double *x, const double *y, const double *q, double u[3]) {
  double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
  double r2 = d0 * d0 + d1 * d1 + d2 * d2;
  if (r2 == 0.0) return 0;
  double r = sqrt(r2);
  double ir = 1.0 / r;
  double ir3 = ir / r2;
  double dq = d0 * q[0] + d1 * q[1] + d2 * q[2];
  u[0] = q[0] * ir + d0 * dq * ir3;
  u[1] = q[1] * ir + d1 * dq * ir3;
  u[2] = q[2] * ir + d2 * dq * ir3;
  return 1;
}

/* Double-layer contribution of source j at target x (unscaled by 6/(8 pi)). */
static inline int dl_pair(const double *x, const double *y, const double *n, const double *psi,
                          double u[3]) {
  double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
  double r2 = d0 * d0 + d1 * d1 + d2 * d2;
  if (r2 == 0.0) return 0;
  double r = sqrt(r2);
  double r5 = r2 * r2 * r;
  double dpsi = d0 * psi[0] + d1 * psi[1] + d2 * psi[2];
  double dn = d0 * n[0] + d1 * n[1] + d2 * n[2];
  double c = dpsi * dn / r5;
  u[0] = d0 * c;
  u[1] = d1 * c;
  u[2] = d2 * c;
  return 1;
}

static void eval_target(const double *x, int64_t j0, int64_t j1, const double *y,
                        const double *f, const double *nrm, const double *phi, const double *w,
                        double csl, double cdl, neum acc[3]) {
  for (int64_t j = j0; j < j1; ++j) {
    double u[3];
    if (f) {
      double q[3] = {w[j] * f[3 * j], w[j] * f[3 * j + 1], w[j] * f[3 * j + 2]};
      if (sl_pair(x, y + 3 * j, q, u))
        for (int k = 0; k < 3; ++k) neum_add(&acc[k], csl * u[k]);
    }
    if (phi) {
      double psi[3] = {w[j] * phi[3 * j], w[j] * phi[3 * j + 1], w[j] * phi[3 * j + 2]};
      if (dl_pair(x, y + 3 * j, nrm + 3 * j, psi, u))
        for (int k = 0; k < 3; ++k) neum_add(&acc[k], cdl * u[k]);
    }
  }
}

double oracle_sl_scale(double mu) { return 1.0 / (8.0 * ORC_PI * mu); }
double oracle_dl_scale(void) { return 6.0 / (8.0 * ORC_PI); }

void oracle_sl(int64_t ns, const double *y, const double *f, const double *w, int64_t nt,
               const double *x, double mu, double *out) {
  const double csl = oracle_sl_scale(mu);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < nt; ++i) {
    neum acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    eval_target(x + 3 * i, 0, ns, y, f, NULL, NULL, w, csl, 0.0, acc);
    for (int k = 0; k < 3; ++k) out[3 * i + k] = neum_val(&acc[k]);
  }
}

void oracle_dl(int64_t ns, const double *y, const double *nrm, const double *phi,
               const double *w, int64_t nt, const double *x, double *out) {
  const double cdl = oracle_dl_scale();
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < nt; ++i) {
    neum acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    eval_target(x + 3 * i, 0, ns, y, NULL, nrm, phi, w, 0.0, cdl, acc);
    for (int k = 0; k < 3; ++k) out[3 * i + k] = neum_val(&acc[k]);
  }
}

void oracle_sldl(int64_t ns, const double *y, const double *f, const double *nrm,
                 const double *phi, const double *w, int64_t nt, const double *x, double mu,
                 double *out) {
  const double csl = oracle_sl_scale(mu), cdl = oracle_dl_scale();
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < nt; ++i) {
    neum acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    eval_target(x + 3 * i, 0, ns, y, f, nrm, phi, w, csl, cdl, acc);
    for (int k = 0; k < 3; ++k) out[3 * i + k] = neum_val(&acc[k]);
  }
}

/* Leaf containing sorted point i: the last l with leaf_ptr[l] <= i. */
static int32_t leaf_of(int32_t nleaf, const int32_t *leaf_ptr, int64_t i) {
  int32_t lo = 0, hi = nleaf - 1;
  while (lo < hi) {
    int32_t mid = lo + (hi - lo + 1) / 2;
    if (leaf_ptr[mid] <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

void oracle_p2p(int64_t npts, const double *pts, const double *f, const double *phi,
                const double *nrm, const double *w, int32_t nleaf, const int32_t *leaf_ptr,
                const int32_t *ulist_ptr, const int32_t *ulist_idx, int32_t kernels, double mu,
                int64_t ntarget, const int64_t *targets, double *out) {
  const double csl = oracle_sl_scale(mu), cdl = oracle_dl_scale();
  const double *fs = (kernels & 1) ? f : NULL;
  const double *ps = (kernels & 2) ? phi : NULL;
  (void)npts;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t t = 0; t < ntarget; ++t) {
    int64_t i = targets ? targets[t] : t;
    int32_t b = leaf_of(nleaf, leaf_ptr, i);
    neum acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int32_t e = ulist_ptr[b]; e < ulist_ptr[b + 1]; ++e) {
      int32_t a = ulist_idx[e];
      eval_target(pts + 3 * i, leaf_ptr[a], leaf_ptr[a + 1], pts, fs, nrm, ps, w, csl, cdl, acc);
    }
    for (int k = 0; k < 3; ++k) out[3 * t + k] = neum_val(&acc[k]);
  }
}

void oracle_batched(int64_t npts, const double *pts, const double *f, const double *phi,
                    const double *nrm, const double *w, int32_t nsusp, const int64_t *susp_ptr,
                    const int64_t *n_cell, double mu, int64_t ntarget, const int64_t *targets,
                    double *out) {
  const double csl = oracle_sl_scale(mu), cdl = oracle_dl_scale();
  (void)npts;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t t = 0; t < ntarget; ++t) {
    int64_t i = targets ? targets[t] : t;
    int32_t lo = 0, hi = nsusp - 1;
    while (lo < hi) {
      int32_t mid = lo + (hi - lo + 1) / 2;
      if (susp_ptr[mid] <= i) lo = mid;
      else hi = mid - 1;
    }
    int64_t s0 = susp_ptr[lo], sc = s0 + n_cell[lo], s1 = susp_ptr[lo + 1];
    neum acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    eval_target(pts + 3 * i, s0, sc, pts, f, NULL, NULL, w, csl, 0.0, acc);
    eval_target(pts + 3 * i, sc, s1, pts, NULL, nrm, phi, w, 0.0, cdl, acc);
    for (int k = 0; k < 3; ++k) out[3 * t + k] = neum_val(&acc[k]);
  }
}

/*
 * Adjoint of L = sum_i g_i . u_i with u = SL[f] + DL[phi] over the same sources.
 * Analytic derivatives of the two pair terms (derived from the kernels above,
 * d = x - y, q = w f, psi = w phi):
 *   s = g.q/r + (d.g)(d.q)/r^3
 *     ds/dq = g/r + d (d.g)/r^3
 *     ds/dd = [g (d.q) + q (d.g) - (g.q) d]/r^3 - 3 (d.g)(d.q) d/r^5
 *   t = (d.g)(d.psi)(d.n)/r^5
 *     dt/dpsi = (d.g)(d.n) d/r^5,  dt/dn = (d.g)(d.psi) d/r^5
 *     dt/dd = [g (d.psi)(d.n) + psi (d.g)(d.n) + n (d.g)(d.psi)]/r^5 - 5 t d/r^2
 * dL/dx_i sums dd over sources; dL/dy_j is minus the sum over targets.  Weights
 * are constants; the normal is differentiated as given (not renormalised).
 * Any output pointer may be NULL to skip it.
 */
static void pair_grad(const double *x, const double *y, const double *g, const double *q,
                      const double *n, const double *psi, double csl, double cdl,
                      double gq[3], double gpsi[3], double gn[3], double gd[3]) {
  double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
  double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  for (int k = 0; k < 3; ++k) gq[k] = gpsi[k] = gn[k] = gd[k] = 0.0;
  if (r2 == 0.0) return;
  double r = sqrt(r2), ir = 1.0 / r, ir3 = ir / r2, ir5 = ir3 / r2;
  double dg = d[0] * g[0] + d[1] * g[1] + d[2] * g[2];
  if (q) {
    double dq = d[0] * q[0] + d[1] * q[1] + d[2] * q[2];
    double gdotq = g[0] * q[0] + g[1] * q[1] + g[2] * q[2];
    for (int k = 0; k < 3; ++k) {
      gq[k] = csl * (g[k] * ir + d[k] * dg * ir3);
      gd[k] += csl * ((g[k] * dq + q[k] * dg - gdotq * d[k]) * ir3 - 3.0 * dg * dq * d[k] * ir5);
    }
  }
  if (psi) {
    double dp = d[0] * psi[0] + d[1] * psi[1] + d[2] * psi[2];
    double dn = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
    double t = dg * dp * dn * ir5;
    for (int k = 0; k < 3; ++k) {
      gpsi[k] = cdl * dg * dn * d[k] * ir5;
      gn[k] = cdl * dg * dp * d[k] * ir5;
      gd[k] += cdl * ((g[k] * dp * dn + psi[k] * dg * dn + n[k] * dg * dp) * ir5 - 5.0 * t * d[k] / r2);
    }
  }
}

void oracle_sldl_grad(int64_t ns, const double *y, const double *f, const double *nrm,
                      const double *phi, const double *w, int64_t nt, const double *x,
                      const double *g, double mu, double *grad_f, double *grad_phi,
                      double *grad_y, double *grad_n, double *grad_x) {
  const double csl = f ? oracle_sl_scale(mu) : 0.0, cdl = phi ? oracle_dl_scale() : 0.0;
  /* source-major pass: gradients that belong to source j are sums over targets */
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t j = 0; j < ns; ++j) {
    neum af[3] = {{0, 0}, {0, 0}, {0, 0}}, ap[3] = {{0, 0}, {0, 0}, {0, 0}};
    neum ay[3] = {{0, 0}, {0, 0}, {0, 0}}, an[3] = {{0, 0}, {0, 0}, {0, 0}};
    double q[3], psi[3];
    const double *qp = NULL, *pp = NULL;
    if (f) { for (int k = 0; k < 3; ++k) q[k] = w[j] * f[3 * j + k]; qp = q; }
    if (phi) { for (int k = 0; k < 3; ++k) psi[k] = w[j] * phi[3 * j + k]; pp = psi; }
    for (int64_t i = 0; i < nt; ++i) {
      double gq[3], gpsi[3], gn[3], gd[3];
      pair_grad(x + 3 * i, y + 3 * j, g + 3 * i, qp, nrm ? nrm + 3 * j : NULL, pp, csl, cdl,
                gq, gpsi, gn, gd);
      for (int k = 0; k < 3; ++k) {
        neum_add(&af[k], gq[k]);
        neum_add(&ap[k], gpsi[k]);
        neum_add(&an[k], gn[k]);
        neum_add(&ay[k], -gd[k]);
      }
    }
    for (int k = 0; k < 3; ++k) {
      if (grad_f) grad_f[3 * j + k] = w[j] * neum_val(&af[k]);
      if (grad_phi) grad_phi[3 * j + k] = w[j] * neum_val(&ap[k]);
      if (grad_n) grad_n[3 * j + k] = neum_val(&an[k]);
      if (grad_y) grad_y[3 * j + k] = neum_val(&ay[k]);
    }
  }
  if (!grad_x) return;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < nt; ++i) {
    neum ax[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int64_t j = 0; j < ns; ++j) {
      double q[3], psi[3], gq[3], gpsi[3], gn[3], gd[3];
      const double *qp = NULL, *pp = NULL;
      if (f) { for (int k = 0; k < 3; ++k) q[k] = w[j] * f[3 * j + k]; qp = q; }
      if (phi) { for (int k = 0; k < 3; ++k) psi[k] = w[j] * phi[3 * j + k]; pp = psi; }
      pair_grad(x + 3 * i, y + 3 * j, g + 3 * i, qp, nrm ? nrm + 3 * j : NULL, pp, csl, cdl,
                gq, gpsi, gn, gd);
      for (int k = 0; k < 3; ++k) neum_add(&ax[k], gd[k]);
    }
    for (int k = 0; k < 3; ++k) grad_x[3 * i + k] = neum_val(&ax[k]);
  }
}
