/*
 * stokes_oracle.h -- FP64 CPU oracle for the Stokes layer-potential sums.
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).
 * All arrays are host FP64, vectors AoS [n][3] row-major.  Outputs are
 * overwritten.  Pairs at exactly zero distance contribute nothing.
 */
#ifndef STOKES_ORACLE_H
#define STOKES_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

double oracle_sl_scale(double mu); /* 1 / (8 pi mu) */
double oracle_dl_scale(void);      /* 6 / (8 pi) */

/* Single layer, Eq. "sl_stokes": out_i = 1/(8 pi mu) sum_j (I/r + d d^T/r^3) w_j f_j */
void oracle_sl(int64_t ns, const double *y, const double *f, const double *w, int64_t nt,
               const double *x, double mu, double *out);
/* Double layer (Sec. 2.1): out_i = 6/(8 pi) sum_j d d^T (d . n_j)/r^5 w_j phi_j */
void oracle_dl(int64_t ns, const double *y, const double *nrm, const double *phi,
               const double *w, int64_t nt, const double *x, double *out);
/* Superposition SL[f] + DL[phi] over one source set (Eq. "velocity_combined"). */
void oracle_sldl(int64_t ns, const double *y, const double *f, const double *nrm,
                 const double *phi, const double *w, int64_t nt, const double *x, double mu,
                 double *out);
/* Near field of the FMM: target i in leaf B sums over sources in the leaves of U(B).
 * kernels: 1 = SL, 2 = DL, 3 = both.  targets == NULL means all ntarget = npts points. */
void oracle_p2p(int64_t npts, const double *pts, const double *f, const double *phi,
                const double *nrm, const double *w, int32_t nleaf, const int32_t *leaf_ptr,
                const int32_t *ulist_ptr, const int32_t *ulist_idx, int32_t kernels, double mu,
                int64_t ntarget, const int64_t *targets, double *out);
/* Batched suspensions: target i of suspension s sums SL over the cell points of s
 * (the first n_cell[s] points) and DL over its wall points (the rest). */
void oracle_batched(int64_t npts, const double *pts, const double *f, const double *phi,
                    const double *nrm, const double *w, int32_t nsusp, const int64_t *susp_ptr,
                    const int64_t *n_cell, double mu, int64_t ntarget, const int64_t *targets,
                    double *out);
/* Adjoint of L = sum_i g_i . (SL[f] + DL[phi])(x_i); f or phi may be NULL. */
void oracle_sldl_grad(int64_t ns, const double *y, const double *f, const double *nrm,
                      const double *phi, const double *w, int64_t nt, const double *x,
                      const double *g, double mu, double *grad_f, double *grad_phi,
                      double *grad_y, double *grad_n, double *grad_x);

#ifdef __cplusplus
}
#endif
#endif
