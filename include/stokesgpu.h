/*
 * stokesgpu.h -- C ABI of the GB300 (sm_103a) Stokes layer-potential library.
 *
 * The library evaluates the smooth-quadrature sums of the two Stokes layer
 * potentials used by the boundary-integral red-blood-cell method of Lu,
 * Morse, Rahimian, Stadler and Zorin (SC'19):
 *
 *   single layer, Eq. "sl_stokes" (Sec. 2.1):
 *     u(x_i) = 1/(8 pi mu) sum_j [ I/|r| + r r^T/|r|^3 ] w_j f_j
 *   double layer, kernel of Eq. "double_layer_int_eq" (Sec. 2.1):
 *     u(x_i) = 6/(8 pi)    sum_j [ r r^T (r . n_j)/|r|^5 ] w_j phi_j
 *   with r = x_i - y_j, n_j the outward unit normal at source y_j and w_j its
 *   quadrature weight; the sum over quadrature nodes is the discretisation of
 *   Sec. 3.1, Eq. "smooth_double_layer_int_eq_patches_disc", and their
 *   superposition is Eq. "velocity_combined".
 *
 * Conventions shared by every entry point:
 *   - All array arguments are DEVICE pointers owned by the caller, FP64,
 *     vectors as AoS [n][3] row-major; index arrays are int32 or int64 as
 *     declared.  Nothing is retained after the call returns.
 *   - A pair at exactly zero distance (in particular target i == source i
 *     when the targets are the sources) contributes nothing.
 *   - `out` is [nt][3] FP64.  With opts->accumulate == 0 it is overwritten,
 *     otherwise the result is added to it.
 *   - `workspace` is caller-allocated device memory of at least the size the
 *     matching *_workspace_size query returns for the same sizes and options,
 *     aligned to 256 bytes.  The library allocates nothing itself.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call
 *     only enqueues work on it and never synchronises it.
 *   - Errors are returned as stk_status; stokes_last_error() gives a message
 *     for the calling thread.  Arguments are validated before anything is
 *     enqueued; an invalid call enqueues nothing.
 *   - Device-side failures (a bounded wait that ran out) are recorded in the
 *     workspace and reported by stokes_device_status() after the caller has
 *     synchronised the stream.
 */
#ifndef STOKESGPU_H
#define STOKESGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  STK_OK = 0,
  STK_EINVAL = 1,       /* bad argument (NULL pointer, negative size, bad option) */
  STK_ENOMEM = 2,       /* workspace smaller than required */
  STK_ECUDA = 3,        /* a CUDA runtime call failed */
  STK_ETIMEOUT = 4,     /* a device wait ran out (see stokes_device_status) */
  STK_EUNSUPPORTED = 5  /* size or option outside what the library supports */
} stk_status;

typedef enum {
  /* FP64 throughout: pair differences, 1/r and products in double. */
  STK_FP64 = 0,
  /* FP32 pair arithmetic in per-work-item local frames with compensated
   * (two-sum) accumulation; pairs closer than near_ratio * h_j get their
   * difference x - y and 1/|r| in FP64. */
  STK_MIXED = 1
} stk_precision;

typedef struct {
  int32_t precision;    /* stk_precision */
  double near_ratio;    /* alpha: a pair is "near" when |r| < alpha * h_j (MIXED only); >= 0 */
  int32_t accumulate;   /* 0: out = u; 1: out += u */
  int32_t source_splits;/* direct sums: split the sources into this many parts (0 = automatic) */
  int32_t tile_config;  /* -1 = default work-item shape; else an id < stokes_tile_config_count() */
} stk_opts;

/* Defaults: MIXED, alpha = 1, overwrite, automatic splits, tuned config. */
void stokes_default_opts(stk_opts *opts);

/* ---------------------------------------------------------------- direct sums
 * src [ns][3], trg [nt][3]; f, phi, nrm [ns][3]; w [ns]; h [ns] local spacing
 * (may be NULL: then only exactly coincident pairs take the FP64 path).
 * Targets may alias the sources.  ns, nt in [0, 2^31 - 1].
 * In the mixed form with the default options (source_splits = 0,
 * tile_config = -1), a sum of at most 2^26 target-source pairs runs as one
 * launch over blocks of 256 targets x source splits (no sort, no work items,
 * near pairs queued per warp and evaluated in FP64 in the same launch, the
 * last split of a target block adding the splits in order; it has no device
 * waits, so its workspace's status word stays 0); larger sums and any other
 * options take the work-item engine.  Both meet the same accuracy.
 */
stk_status stokes_sl_eval(const double *src, const double *f, const double *w, const double *h,
                          int64_t ns, const double *trg, int64_t nt, double mu, double *out,
                          const stk_opts *opts, void *workspace, size_t workspace_bytes,
                          void *stream);
stk_status stokes_dl_eval(const double *src, const double *nrm, const double *phi,
                          const double *w, const double *h, int64_t ns, const double *trg,
                          int64_t nt, double *out, const stk_opts *opts, void *workspace,
                          size_t workspace_bytes, void *stream);
/* SL[f] + DL[phi] over one source set (Eq. "velocity_combined"). */
stk_status stokes_sldl_eval(const double *src, const double *f, const double *nrm,
                            const double *phi, const double *w, const double *h, int64_t ns,
                            const double *trg, int64_t nt, double mu, double *out,
                            const stk_opts *opts, void *workspace, size_t workspace_bytes,
                            void *stream);
/* kernels: 1 = SL, 2 = DL, 3 = SL + DL. */
stk_status stokes_direct_workspace_size(int64_t ns, int64_t nt, int32_t kernels,
                                        const stk_opts *opts, size_t *bytes);

/* ------------------------------------------------------------ FMM near field
 * P2P over octree U-lists (Sec. 3.1 "Far evaluation": the direct part of the
 * FMM).  pts [n][3] are sorted so that leaf l owns points
 * [leaf_ptr[l], leaf_ptr[l+1]); ulist_idx[ulist_ptr[l] .. ulist_ptr[l+1]) are
 * the leaves adjacent to l (l included).  Every point is a source and a
 * target: out_i = sum over sources in the leaves of U(leaf(i)).
 * kernels: 1 = SL (uses f), 2 = DL (uses nrm, phi), 3 = both.  Unused density
 * pointers may be NULL.  Leaves may hold at most 65535 points.
 * The call stays ordered on `stream` as every other: part of its work (the
 * packing of the sources) runs on a second stream the library keeps per host
 * thread and device (created on the first call outside a stream capture,
 * made again in a new context), forked from and joined back into `stream` by
 * events, which a stream capture follows.
 */
stk_status stokes_p2p_leaflists(const double *pts, const double *f, const double *phi,
                                const double *nrm, const double *w, const double *h, int64_t n,
                                const int32_t *leaf_ptr, int32_t nleaf, const int32_t *ulist_ptr,
                                const int32_t *ulist_idx, int64_t nulist, int32_t kernels,
                                double mu, double *out, const stk_opts *opts, void *workspace,
                                size_t workspace_bytes, void *stream);
stk_status stokes_p2p_workspace_size(int64_t n, int32_t nleaf, int32_t kernels,
                                     const stk_opts *opts, size_t *bytes);

/* ---------------------------------------------------- batched suspensions
 * S independent suspensions in one launch (Eq. "velocity_combined" per
 * suspension).  Suspension s owns points [susp_ptr[s], susp_ptr[s+1]); its
 * first n_cell[s] points are cell points carrying the single-layer density f,
 * the rest are vessel-wall points carrying the double-layer density phi.
 * Targets are all points of s: out_i = SL_cells(s)[f] + DL_wall(s)[phi].
 * susp_ptr [S+1] and n_cell [S] are device int64 arrays; susp_ptr[S] = n.
 */
stk_status stokes_batched_eval(const double *pts, const double *f, const double *phi,
                               const double *nrm, const double *w, const double *h, int64_t n,
                               const int64_t *susp_ptr, const int64_t *n_cell, int32_t nsusp,
                               double mu, double *out, const stk_opts *opts, void *workspace,
                               size_t workspace_bytes, void *stream);
stk_status stokes_batched_workspace_size(int64_t n, int32_t nsusp, const stk_opts *opts,
                                         size_t *bytes);

/* ------------------------------------------------- tuning and CUDA graphs
 * Work items (a warp's targets against its source segments) come in
 * stokes_tile_config_count() shapes; opts->tile_config picks one (-1: the
 * default).  The autotuners run every shape on the caller's own data (one
 * warm-up and three timed calls each; they synchronise the stream, write
 * `out`, and need a workspace from the matching *_workspace_size query) and
 * return the fastest id and its median time.
 * The *_graph_create calls capture one call with these arguments into an
 * executable CUDA graph (stream must not be the legacy default stream); the
 * graph replays with stokes_graph_launch on any stream, reading the same
 * device buffers, and is released with stokes_graph_destroy.  This is how a
 * batch of suspensions runs as one persistent launch per replay.
 */
int32_t stokes_tile_config_count(void);
stk_status stokes_autotune_p2p(const double *pts, const double *f, const double *phi,
                               const double *nrm, const double *w, const double *h, int64_t n,
                               const int32_t *leaf_ptr, int32_t nleaf, const int32_t *ulist_ptr,
                               const int32_t *ulist_idx, int64_t nulist, int32_t kernels,
                               double mu, double *out, const stk_opts *opts, void *workspace,
                               size_t workspace_bytes, void *stream, int32_t *best_config,
                               float *best_ms);
stk_status stokes_autotune_batched(const double *pts, const double *f, const double *phi,
                                   const double *nrm, const double *w, const double *h, int64_t n,
                                   const int64_t *susp_ptr, const int64_t *n_cell, int32_t nsusp,
                                   double mu, double *out, const stk_opts *opts, void *workspace,
                                   size_t workspace_bytes, void *stream, int32_t *best_config,
                                   float *best_ms);
stk_status stokes_p2p_graph_create(const double *pts, const double *f, const double *phi,
                                   const double *nrm, const double *w, const double *h, int64_t n,
                                   const int32_t *leaf_ptr, int32_t nleaf,
                                   const int32_t *ulist_ptr, const int32_t *ulist_idx,
                                   int64_t nulist, int32_t kernels, double mu, double *out,
                                   const stk_opts *opts, void *workspace, size_t workspace_bytes,
                                   void *stream, void **graph_exec);
stk_status stokes_batched_graph_create(const double *pts, const double *f, const double *phi,
                                       const double *nrm, const double *w, const double *h,
                                       int64_t n, const int64_t *susp_ptr, const int64_t *n_cell,
                                       int32_t nsusp, double mu, double *out,
                                       const stk_opts *opts, void *workspace,
                                       size_t workspace_bytes, void *stream, void **graph_exec);
/* A direct sum (kernels 1 = SL[f], 2 = DL[phi], 3 = SL[f] + DL[phi], the
 * arguments of stokes_sl_eval / stokes_dl_eval / stokes_sldl_eval) captured
 * into a graph: small sums are bound by the latency of their launches, which
 * a replay takes from the host. */
stk_status stokes_direct_graph_create(int32_t kernels, const double *src, const double *f,
                                      const double *nrm, const double *phi, const double *w,
                                      const double *h, int64_t ns, const double *trg, int64_t nt,
                                      double mu, double *out, const stk_opts *opts,
                                      void *workspace, size_t workspace_bytes, void *stream,
                                      void **graph_exec);
stk_status stokes_graph_launch(void *graph_exec, void *stream);
stk_status stokes_graph_destroy(void *graph_exec);

/* ----------------------------------------------------------------- adjoint
 * Gradients of L = sum_i g_i . u(x_i) with u = SL[f] + DL[phi] over one
 * source set (the kernels of Eq. "sl_stokes" and Sec. 2.1, differentiated
 * pair by pair; nothing O(ns nt) is stored, the pair terms are recomputed):
 *   grad_f [ns][3] = dL/df,  grad_phi [ns][3] = dL/dphi,
 *   grad_y [ns][3] = dL/d(source positions),  grad_n [ns][3] = dL/d(normals, as given),
 *   grad_x [nt][3] = dL/d(target positions).
 * g [nt][3] is the upstream gradient.  f or phi may be NULL (SL or DL only);
 * any output may be NULL to skip it.  Weights and spacings are constants.
 * When the targets are the sources, the caller adds grad_x to grad_y.
 * MIXED: FP32 pair terms in per-CTA local frames with two-sum accumulation;
 * pairs with |r| < near_ratio * h_j are listed per output point (up to 32;
 * a point with more is rescanned over all inputs, one thread per such point,
 * so inputs where most points are near each other are slow) and evaluated in
 * FP64 by a second pass, in input order, so results are deterministic.  FP64: all double.  The
 * workspace (stokes_grad_workspace_size) holds the packed records, the
 * Morton orders, the per-split partial gradients and, for MIXED, the near-pair
 * lists.
 */
stk_status stokes_sldl_grad(const double *src, const double *f, const double *nrm,
                            const double *phi, const double *w, const double *h, int64_t ns,
                            const double *trg, int64_t nt, const double *g, double mu,
                            double *grad_f, double *grad_phi, double *grad_y, double *grad_n,
                            double *grad_x, const stk_opts *opts, void *workspace,
                            size_t workspace_bytes, void *stream);
stk_status stokes_grad_workspace_size(int64_t ns, int64_t nt, const stk_opts *opts,
                                      size_t *bytes);

/* ------------------------------------------------- check-point quadrature
 * Layer potentials at targets on or near a patch surface by check-point
 * extrapolation (Sec. 3.1, "Singular and near-singular integral quadrature";
 * the steps are those of that passage, Eq. "quad_check_points" and
 * Eq. "sing-quad"):
 *   1. the density on each patch's (q+1) x (q+1) Clenshaw-Curtis nodes
 *      (u_i, v_j) = (cos(i pi/q), cos(j pi/q)), node index i (q+1) + j, is
 *      interpolated (tensor-product, degree q) to the fine discretisation:
 *      m x m sub-patches (m = 2^eta), sub-patch (su, sv) covering
 *      u in [-1 + 2 su/m, -1 + 2 (su+1)/m] (likewise v), each with the same
 *      node set; fine nodes are ordered patch, sub-patch (su m + sv), node;
 *   2. check points c_i = y - (R + i r) n, i = 0..p, from each target's
 *      closest surface point y and unit normal n there (y = x for a target
 *      on a node);
 *   3. the smooth quadrature sum (Eq. "smooth_double_layer_int_eq_patches_disc")
 *      of SL[f] (kernels 1), DL[phi] (2) or both (3) over the fine nodes at
 *      the check points, in opts->precision, as stokes_sl_eval etc. do;
 *   4. out(x) (+)= sum_i e_i u(c_i), e_i the Lagrange weights of the nodes
 *      t_i = R + i r at t = (y - x) . n.
 * f, phi: [npatch (q+1)^2][3] on the coarse nodes (the one not used may be
 * NULL).  fine_pts, fine_nrm [nf][3], fine_w, fine_h [nf] (h may be NULL):
 * the fine discretisation's nodes, outward unit normals, weights and
 * spacings, nf = npatch m^2 (q+1)^2 (the surface is fixed, so the caller
 * builds these once).  trg, cp_y, cp_n [nt][3].  Limits: 2 <= q <= 12,
 * 0 <= eta <= 3, 0 <= p <= 15, R > 0, r > 0.  Device pointers, caller-owned;
 * nothing is allocated and the stream is not synchronised.
 */
stk_status stokes_checkpoint_eval(int32_t kernels, const double *f, const double *phi,
                                  int32_t npatch, int32_t q, int32_t eta, const double *fine_pts,
                                  const double *fine_nrm, const double *fine_w,
                                  const double *fine_h, const double *trg, const double *cp_y,
                                  const double *cp_n, int64_t nt, double R, double r, int32_t p,
                                  double mu, double *out, const stk_opts *opts, void *workspace,
                                  size_t workspace_bytes, void *stream);
stk_status stokes_checkpoint_workspace_size(int32_t kernels, int32_t npatch, int32_t q,
                                            int32_t eta, int64_t nt, int32_t p,
                                            const stk_opts *opts, size_t *bytes);
/* The boundary-integral operator of Eq. "double_layer_int_eq" (discretised as
 * Eq. "int_eq_disc") applied to a double-layer density phi on the coarse nodes,
 * evaluated at the coarse nodes:
 *   out = (D - I/2) phi + N phi,
 * (D - I/2) phi being the limit of the double layer from the fluid side, taken
 * by stokes_checkpoint_eval with targets = closest points = the nodes and
 * normals nodes_n (check points y - (R + i r) n), and
 *   (N phi)(x) = sum_m w_m (n(x) . phi_m) n_m
 * the rank-completing operator (FP64, fixed-order reduction).  With this
 * library's kernel orientation (a constant density gives -c on the fluid
 * side, n pointing out of the fluid) the paper's +I/2 appears as -I/2.
 * nodes, nodes_n [npatch (q+1)^2][3], nodes_w [npatch (q+1)^2]; the fine
 * discretisation as for stokes_checkpoint_eval.  out is overwritten unless
 * opts->accumulate. */
stk_status stokes_bie_matvec(const double *phi, int32_t npatch, int32_t q, int32_t eta,
                             const double *nodes, const double *nodes_n, const double *nodes_w,
                             const double *fine_pts, const double *fine_nrm, const double *fine_w,
                             const double *fine_h, double R, double r, int32_t p, double *out,
                             const stk_opts *opts, void *workspace, size_t workspace_bytes,
                             void *stream);
stk_status stokes_bie_workspace_size(int32_t npatch, int32_t q, int32_t eta, int32_t p,
                                     const stk_opts *opts, size_t *bytes);
/* Step 1 alone: coarse [npatch (q+1)^2][ncomp] -> fine [npatch m^2 (q+1)^2][ncomp]
 * (FP64, ncomp 1..3), the upsampling operator U of Sec. 3.1. */
stk_status stokes_upsample_patches(const double *coarse, int32_t npatch, int32_t q, int32_t eta,
                                   int32_t ncomp, double *fine, void *stream);

/* ------------------------------------------------------ near-zone search
 * For each target x: the patch of a patch surface closest to x when x lies
 * within d_eps of it, the closest point y = P(u*, v*), the unit normal
 * (dP/du x dP/dv)/|...| there and the distance (Sec. 3.2, the closest-point
 * search, steps a-e: inflated patch boxes, a spatial hash of the boxes and the
 * targets, sorted keys, Newton's method with a backtracking line search per
 * candidate patch, the nearest patch kept).  A patch is the degree-q
 * tensor-product interpolant through its (q+1) x (q+1) Clenshaw-Curtis nodes,
 * ordered as for stokes_checkpoint_eval.  nodes [npatch (q+1)^2][3],
 * trg [nt][3]; outputs: patch [nt] (-1: none within d_eps), uv [nt][2],
 * y [nt][3], n [nt][3], dist [nt] (-1 for none).  Patch boxes are grown by
 * d_eps and 5% of their diagonal, so a target whose closest point lies
 * further outside its patch's node box than that is not found.  FP64.
 * 2 <= q <= 12. */
stk_status stokes_near_patch_search(const double *nodes, int32_t npatch, int32_t q,
                                    const double *trg, int64_t nt, double d_eps, int32_t *patch,
                                    double *uv, double *y, double *n, double *dist,
                                    void *workspace, size_t workspace_bytes, void *stream);
/* Workspace of stokes_near_patch_search for npatch patches of order q and nt
 * targets (0 <= nt <= 2^31 - 1): the patch boxes, the sorted (cell, patch)
 * keys and a list of nt target indices. */
stk_status stokes_near_search_workspace_size(int32_t npatch, int32_t q, int64_t nt,
                                             size_t *bytes);

/* ------------------------------------------------- FMM operators (host)
 * Set-up of the kernel-independent FMM of Sec. 3.1 ("Far evaluation"), host
 * only (no device memory, no stream).  Surface points: the boundary of a
 * p x p x p grid on [-1, 1]^3 (index i slowest, k fastest), count
 * p^3 - (p-2)^3; pts [count][3] may be NULL to query the count.
 * Check-to-equivalent operator of a box of half-width r: the pseudo-inverse
 * (one-sided Jacobi SVD, singular values below rcond * max dropped, FP64) of
 * the kernel matrix from equivalent points to check points.  upward != 0:
 * check points at 2.95 r, equivalent points at 1.05 r, densities of a force
 * and, when flux != 0, a point-source strength per point (out is
 * [(3 or 4) count][3 count], row-major); upward == 0: check at 1.05 r,
 * equivalent at 2.95 r, forces only (out [3 count][3 count]).  Check
 * velocities are [count][3], densities [count][3 or 4] in point order.
 * 2 <= p <= 12 for the operator (16 for the points); STK_EINVAL otherwise. */
stk_status stokes_fmm_surface(int32_t p, double *pts, int32_t *count);
stk_status stokes_fmm_check_to_equiv(int32_t p, double r, double mu, int32_t upward,
                                     int32_t flux, double rcond, double *out);
/* The check-to-equivalent operators of every depth 2..max_depth of a tree
 * whose root cube has side root_size, as stokes_fmm_far_eval takes them:
 * uc2e [max_depth - 1][(flux ? 4 : 3) ns][3 ns], dc2e [max_depth - 1][3 ns][3 ns]
 * (host arrays; nothing written for max_depth < 2).  A Stokeslet-only
 * operator of half-width r is r times that of half-width 1; with flux,
 * upward_scaled == 0 decomposes the upward operator at every depth,
 * upward_scaled != 0 scales the one of half-width 1, the source strengths in
 * units of r (an exact, not minimum-norm, operator). */
stk_status stokes_fmm_operators(int32_t p, double root_size, int32_t max_depth, double mu,
                                int32_t flux, double rcond, int32_t upward_scaled, double *uc2e,
                                double *dc2e);
/* The derived arrays of an FMM tree (host): from each box's depth, integer
 * anchor [nbox][3], parent (-1 for the root) and leaf number (-1 if none),
 * boxes numbered depth by depth with the root first and children in their
 * parents' order (checked, STK_EINVAL otherwise), it gives max_depth,
 * depth_ptr [max_depth + 2] (caller buffer of 23 entries), child_ptr
 * [nbox + 1], leaf_box [nleaf] and colleague [nbox][27] (the same-depth box
 * at anchor + (dx, dy, dz), entry (dx+1) 9 + (dy+1) 3 + (dz+1), -1 where there
 * is none) of stk_fmm_tree. */
stk_status stokes_fmm_tree_complete(int32_t nbox, int32_t nleaf, const int32_t *depth,
                                    const int32_t *anchor, const int32_t *parent,
                                    const int32_t *box_leaf, int32_t *max_depth,
                                    int32_t *depth_ptr, int32_t *child_ptr, int32_t *leaf_box,
                                    int32_t *colleague);
/* Kernel matrix [3 nx][ncomp ny] (row-major) from densities at y [ny][3] to
 * velocities at x [nx][3]: a force per point (Oseen tensor / (8 pi mu)) and,
 * for ncomp = 4, a point-source strength (d / (4 pi |d|^3)); coincident points
 * give zero.  With surface points placed by the caller it gives the FMM's
 * translation operators (M2M, M2L, L2L) on the host. */
stk_status stokes_fmm_kernel_matrix(const double *x, int32_t nx, const double *y, int32_t ny,
                                    double mu, int32_t ncomp, double *out);

/* Far field of the FMM on the GPU (Sec. 3.1, "Far evaluation"), FP64: the
 * velocity at every point of the sources outside its leaf's U-list, through
 * upward equivalent densities (S2M at the leaves, M2M), the interaction lists
 * (V: M2L; W: upward densities at a leaf's points; X: sources on a box's
 * downward check surface), downward equivalent densities (L2L) and L2T.  The
 * near field is stokes_p2p_leaflists over the same leaves; far + near is the
 * FMM's approximation of stokes_sldl_eval with targets = sources.
 *
 * The tree: nbox boxes numbered depth by depth (depth 0 = the root cube
 * [root_lo, root_lo + root_size]^3), Morton order within a depth, so the
 * children of box b are the boxes [child_ptr[b], child_ptr[b+1]).  A box of
 * depth d with integer index a = anchor[b] has centre root_lo + (a + 0.5)
 * root_size / 2^d.  Points are sorted by leaf: leaf l holds [leaf_ptr[l],
 * leaf_ptr[l+1]) and is box leaf_box[l]; box_leaf[b] is the leaf number of box
 * b or -1.  V, W and X are CSR lists over box numbers ([nbox + 1] pointers):
 *   V(B): children of the same-depth neighbours of B's parent that do not
 *         touch B (closed boxes); W(B), B a leaf: boxes below B's same-depth
 *         neighbours that do not touch B while their parent does; X(B): the
 *         leaves A with B in W(A).
 * colleague (optional, device [nbox][27]): the same-depth box at anchor +
 * (dx, dy, dz) for dx, dy, dz in {-1, 0, 1} (entry (dx+1) 9 + (dy+1) 3 +
 * (dz+1)), -1 where there is none; with it, Fourier-space M2L is blocked by
 * parent (each neighbour child's spectrum read once for all the parent's
 * children), without it summed per box over its V-list.
 * depth_ptr is a HOST array [max_depth + 2] (boxes of depth d are
 * [depth_ptr[d], depth_ptr[d+1])); every other array is in device memory and
 * must describe this one tree (its contents are not checked on the device).
 *
 * Operators: uc2e [max_depth - 1][(flux ? 4 : 3) ns][3 ns] and dc2e
 * [max_depth - 1][3 ns][3 ns] (device, depths 2..max_depth), the
 * check-to-equivalent operators of a box of half-width root_size / 2^(d+1)
 * as stokes_fmm_check_to_equiv returns them (same p, mu and flux); ns is the
 * surface count of p.  flux != 0: the upward density has a point-source
 * strength per surface point (needed for the double layer's far field).
 *
 * Every call clears the workspace's error word (the int32 at byte 8 of the
 * 256-byte aligned workspace, as for the other entry points); the mixed form's
 * kernels check each box, leaf and point index they read from the tree arrays
 * and record one out of range there (stokes_device_status then returns
 * STK_EINVAL) instead of using it.
 *
 * precision: STK_FP64 evaluates every pass in FP64; STK_MIXED packs points
 * (relative to their leaf's centre), densities, surfaces and spectra in FP32,
 * evaluates kernels and spectral products in FP32 with one FP64 difference of
 * box centres per pair of boxes, and forms the check-to-equivalent products
 * in double-FP32 arithmetic (operators split into FP32 pairs, exact FMA
 * products, two-sum accumulation: relative error about u + n u^2 k for a row
 * sum cancelling by k, u = 2^-24); operators cut at rcond ~ 1e-7 keep k small
 * enough for p >= 6.  n must
 * equal leaf_ptr[nleaf].
 * f or phi may be NULL (not both); nrm is needed with phi.  out [n][3] =
 * far field (accumulate != 0: out += far field).  2 <= p <= 12.  Boxes of
 * depth < 2 have no far field; a tree of max_depth < 2 gives zero.  Launches
 * 2 + 4 (max_depth - 1) kernels (3 more per depth with m2l_spectra; 2 more
 * with STK_MIXED, 3 with both) on the caller's stream; allocates nothing;
 * workspace from stokes_fmm_far_workspace_size.  STK_EINVAL for bad sizes,
 * NULL arrays or a depth_ptr that does not run from 0 to nbox. */
typedef struct {
  int32_t nbox, nleaf, max_depth;
  const int32_t *depth_ptr;  /* HOST */
  const int32_t *depth, *anchor, *parent, *child_ptr, *box_leaf, *leaf_box, *leaf_ptr;
  const int32_t *v_ptr, *v_idx, *w_ptr, *w_idx, *x_ptr, *x_idx;
  const int32_t *colleague;  /* optional [nbox][27]; see above */
  double root_lo[3];
  double root_size;
} stk_fmm_tree;
stk_status stokes_fmm_far_workspace_size(int32_t p, int32_t flux, int32_t fft_m2l,
                                         int32_t precision, int64_t n,
                                         const stk_fmm_tree *tree, size_t *bytes);
stk_status stokes_fmm_far_eval(const double *pts, const double *f, const double *phi,
                               const double *nrm, const double *w, int64_t n,
                               const stk_fmm_tree *tree, int32_t p, int32_t flux,
                               const double *uc2e, const double *dc2e,
                               const double *m2l_spectra, int32_t precision, double mu,
                               double *out, int32_t accumulate, void *workspace,
                               size_t workspace_bytes, void *stream);
/* Instrumentation of stokes_fmm_far_eval.  While events != NULL (capacity
 * cudaEvent_t handles created by the caller), the k-th kernel launch of each
 * later far-field call of this thread in the mixed form with p <= 8 records
 * events[2k] before and events[2k + 1] after it on the call's stream (for
 * k < capacity / 2), names[k] (may be NULL) receives a static string naming
 * its pass and *count (may be NULL) the number of launches recorded.  NULL
 * events switches it off.  STK_EINVAL for capacity < 2. */
stk_status stokes_fmm_set_pass_events(void **events, int32_t capacity, const char **names,
                                      int32_t *count);
/* Octree and interaction lists of the FMM (host, built once per point set;
 * Sec. 3.1, "Far evaluation" leaves the tree to the FMM library, so this is
 * one reading of it).  The root is the points' bounding cube grown by 1e-9;
 * a box splits into its 8 children while it holds more than max_leaf points
 * (to depth 21), a point going to the child whose half-open box holds it and
 * empty children dropped (no 2:1 balance).  Leaves are numbered depth-first in
 * Morton order; perm [n] maps leaf-sorted position to caller index, leaf_ptr
 * [nleaf + 1] gives each leaf's range.  U(B) [ulist_ptr/ulist_idx, over
 * leaves]: the leaves whose closed box meets B's (B included), the input of
 * stokes_p2p_leaflists.  Boxes (the leaves and their ancestors) are numbered
 * depth by depth, Morton order within a depth: box_depth [nbox], box_anchor
 * [nbox][3] (integer index at its depth), box_parent [nbox] (-1 for the root),
 * box_leaf [nbox] (leaf number or -1); V, W and X [nbox + 1 pointers] are the
 * lists of stk_fmm_tree, and colleague [nbox][27] its same-depth neighbours.  All lists ascending.  stokes_octree_build allocates
 * host memory owned by the returned handle (free it with
 * stokes_octree_destroy); stokes_octree_info gives the sizes, and
 * stokes_octree_export copies any of the arrays (NULL skips one) into caller
 * buffers of those sizes.  Points must be finite; STK_EINVAL otherwise,
 * STK_ENOMEM when host memory runs out. */
typedef struct stk_octree stk_octree;
typedef struct {
  int64_t n;
  int32_t nleaf, nbox, max_depth;
  int64_t nulist, nv, nw, nx;
  double root_lo[3];
  double root_size;
} stk_octree_info;
stk_status stokes_octree_build(const double *pts, int64_t n, int32_t max_leaf, stk_octree **tree);
stk_status stokes_octree_info(const stk_octree *tree, stk_octree_info *info);
stk_status stokes_octree_export(const stk_octree *tree, int64_t *perm, int32_t *leaf_ptr,
                                int32_t *ulist_ptr, int32_t *ulist_idx, int32_t *box_depth,
                                int32_t *box_anchor, int32_t *box_parent, int32_t *box_leaf,
                                int32_t *v_ptr, int32_t *v_idx, int32_t *w_ptr, int32_t *w_idx,
                                int32_t *x_ptr, int32_t *x_idx, int32_t *colleague);
void stokes_octree_destroy(stk_octree *tree);

/* Kernel spectra of M2L in Fourier space (host, FP64).  The upward
 * equivalent surface of a box and the downward check surface of a same-depth
 * box are the boundary of one p^3 lattice of spacing 2.1 r / (p - 1), so M2L
 * is a convolution over lattice index differences m with the kernel
 * K(delta m - 2 r o), o the source box's offset in box widths; zero-padded to
 * G = 2p points per axis it is a circular convolution, evaluated per
 * frequency.  out [343][G][G][p + 1][3][nc][2] (offset (ox+3) 49 + (oy+3) 7 +
 * (oz+3); frequencies kx, ky in [0, G), kz in [0, p]; velocity component,
 * density component; real, imaginary) holds the DFT (e^{-2 pi i m.k / G}) of
 * that kernel at half-width r = 1 (Oseen tensor / (8 pi mu) and, for flux != 0,
 * the source d / (4 pi |d|^3)); entries of neighbouring offsets are zero.
 * Passed to stokes_fmm_far_eval as m2l_spectra, it selects Fourier-space M2L
 * (the spectra scaled by 1 / r for forces and 1 / r^2 for sources at each
 * depth), with the workspace of fft_m2l != 0; NULL selects the dense M2L. */
stk_status stokes_fmm_m2l_spectra(int32_t p, double mu, int32_t flux, double *out);

/* ------------------------------------------------- no-allocation variant
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory when they need a velocity (an application
 * that owns every device allocation and hands out no scratch, a real-time
 * pipeline that forbids cudaMalloc after start-up because it can synchronise
 * the device, a process under a fixed memory budget).
 * Same single-layer sum and arguments as stokes_sl_eval, without a workspace:
 * the library uses a fixed 32 MiB device buffer of its own, held by every GPU
 * that loads the library until the process exits.  ns and nt may not exceed
 * 65536 (STK_EUNSUPPORTED otherwise); source splits are reduced if needed to
 * fit the buffer.  Allocates nothing.  The first call on a device looks up the
 * buffer's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  The address is cached per device and CUDA
 * context (a call in a new context, after cudaDeviceReset for instance, looks
 * it up again, and that call too should precede any capture).  All calls
 * share the buffer: calls whose kernels may overlap on the GPU race and must
 * be serialised by the caller.  A device wait that ran out during the last
 * call is reported by stokes_device_status(NULL, 0) after synchronising; the
 * next call clears it. */
stk_status stokes_sl_eval_noalloc(const double *src, const double *f, const double *w,
                                  const double *h, int64_t ns, const double *trg, int64_t nt,
                                  double mu, double *out, const stk_opts *opts, void *stream);

/* ----------------------------------------------------- pipe throughput
 * Throughput probes of the arithmetic pipes the summation kernels are bound
 * by, for rooflines against rates measured on the GPU at hand (the paper has
 * no counterpart; it names no GPU).  op: 0 FP32 FMA, 1 packed two-wide FP32
 * FMA (the engine's instruction), 2 FP64 FMA, 3 FP32 reciprocal square root
 * (rsqrt.approx, the MUFU unit).  One launch of SMs x 8 CTAs of 256 threads,
 * each thread running 8 independent chains of `iters` dependent operations
 * on the stream; *ops receives the work of the launch (flops for the FMA
 * forms: 2 per FMA, 4 per packed FMA; evaluations for rsqrt), to be divided
 * by the launch's duration timed by the caller.  sink: caller device memory
 * of stokes_pipe_probe_size bytes, written with the chains' sums. */
stk_status stokes_pipe_probe_size(size_t *sink_bytes);
stk_status stokes_pipe_probe(int32_t op, int32_t iters, void *sink, size_t sink_bytes,
                             double *ops, void *stream);

/* ------------------------------------------------ conversion self-check
 * The library converts between FP64 and FP32 with integer operations (IEEE
 * 754 round to nearest, ties to even, for results in the normal FP32 range;
 * exact widening of normal floats), because GB300 runs the conversion
 * instructions on its 1/64-rate FP64 pipe.  This call puts them beside
 * CUDA's own conversions for a check: for each in[i] (device, n values),
 * narrow_own[i] / narrow_cuda[i] receive the library's and CUDA's FP32
 * rounding of in[i], and widen_own[i] / widen_cuda[i] the library's and
 * CUDA's FP64 widening of narrow_cuda[i].  All pointers are device memory of
 * n elements, written on the stream; n = 0 does nothing. */
stk_status stokes_convert_check(const double *in, int64_t n, float *narrow_own,
                                float *narrow_cuda, double *widen_own, double *widen_cuda,
                                void *stream);

/* ----------------------------------------------------------------- status */
/* Reads the device error word kept in a workspace used by an earlier call.
 * The caller must have synchronised the stream.  Returns STK_OK or
 * STK_ETIMEOUT, and clears the word.  workspace == NULL reads the word of
 * stokes_sl_eval_noalloc's fixed buffer in the current CUDA context
 * (STK_EINVAL if that entry point has not run there). */
stk_status stokes_device_status(void *workspace, size_t workspace_bytes);
/* Instrumentation.  While both events are non-NULL (cudaEvent_t handles
 * created by the caller), every later call on this thread records `start`
 * immediately before and `stop` immediately after its engine kernel, on the
 * call's stream, so that the caller can time the dominant kernel alone.
 * Passing NULLs switches it off. */
stk_status stokes_set_engine_events(void *start_event, void *stop_event);
/* Wait policy of the later calls made on this thread (failure-path testing;
 * no device fault is involved).  The mixed engine stages sources through
 * bounded waits on shared-memory barriers; a wait that runs out records
 * STK_ETIMEOUT in the workspace's error word (stokes_device_status), the warp
 * then waits for the copy it already issued to land, bounded by at least the
 * default limit, and leaves the call with its work unfinished (the near-pair
 * pass skips the call; the results are incomplete).  limit_cycles: bound of
 * each wait in SM clock cycles (0 restores the default, 4e9 cycles, about
 * 2 s).  force_expire = 1: the first wait of every work item reports expiry
 * at once although its copy completes normally, so that a test can take the
 * failure path on any input; 0 switches it off.  STK_EINVAL for a negative
 * limit or another force_expire.  Graphs captured meanwhile keep the policy
 * they were captured with. */
stk_status stokes_set_wait_policy(int64_t limit_cycles, int32_t force_expire);
/* Number of kernels this thread has launched through the library so far.  A
 * graph capture adds nothing (its kernels are recorded, not run); each
 * stokes_graph_launch adds the kernels the graph holds. */
int64_t stokes_launch_count(void);
/* Message for the last error on the calling thread ("" if none). */
const char *stokes_last_error(void);
/* Library version string. */
const char *stokes_version(void);

#ifdef __cplusplus
}
#endif
#endif
