// fmm_ops.cu -- host-side operators of the kernel-independent FMM that
// evaluates the smooth quadrature at all targets at once (Sec. 3.1, "Far
// evaluation"): the equivalent and check surfaces of a box and the
// check-to-equivalent solves, computed once per plan in FP64.
//
// A box of half-width r gets the boundary points of a p x p x p grid on cubes
// of half-width 1.05 r (upward equivalent, downward check) and 2.95 r (upward
// check, downward equivalent).  The upward equivalent density has a force and,
// with flux, a point-source strength per surface point (a double layer has net
// flux through a closed surface, which Stokeslets cannot carry); the downward
// one a force.  The check-to-equivalent operator is the pseudo-inverse of the
// kernel matrix from equivalent to check points, truncated at rcond times the
// largest singular value, by a one-sided (Hestenes) Jacobi SVD.
//
// M2L in Fourier space: the upward equivalent surface of a box and the
// downward check surface of a same-depth box both sit at 1.05 r, so both are
// the boundary of one p^3 lattice of spacing 2.1 r / (p - 1) and the kernel
// between them depends only on the lattice index difference m and the boxes'
// offset o (in box widths): K(delta m - 2 r o).  Zero-padded to G = 2p points
// per axis, M2L is a circular convolution; its kernel spectrum per offset is
// computed here once, at half-width 1 (the Stokeslet scales as 1 / r, the
// point source as 1 / r^2 at other depths).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <utility>
#include <vector>

#include "../../include/stokesgpu.h"

namespace stk {
stk_status report_error(stk_status s, const char *msg);
}

namespace {

constexpr double kPiF = 3.14159265358979323846;
constexpr double kInner = 1.05, kOuter = 2.95;

int surface_count(int p) { return p * p * p - (p - 2) * (p - 2) * (p - 2); }

// boundary points of the p^3 grid on [-1, 1]^3, i slowest, k fastest
void surface(int p, std::vector<double> &s) {
  s.clear();
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j)
      for (int k = 0; k < p; ++k) {
        if (!(i == 0 || j == 0 || k == 0 || i == p - 1 || j == p - 1 || k == p - 1)) continue;
        const double c[3] = {-1.0 + 2.0 * i / (p - 1), -1.0 + 2.0 * j / (p - 1),
                             -1.0 + 2.0 * k / (p - 1)};
        s.insert(s.end(), c, c + 3);
      }
}

// Row-major [3 nx][ncomp ny] kernel matrix from densities at y to velocities
// at x: a force (Oseen tensor / (8 pi mu)) and, with ncomp = 4, a source
// d / (4 pi r^3).
void kernel_matrix(const std::vector<double> &x, const std::vector<double> &y, double mu,
                   int ncomp, std::vector<double> &K) {
  const size_t nx = x.size() / 3, ny = y.size() / 3, cols = (size_t)ncomp * ny;
  K.assign(3 * nx * cols, 0.0);
  for (size_t a = 0; a < nx; ++a)
    for (size_t b = 0; b < ny; ++b) {
      const double d[3] = {x[3 * a] - y[3 * b], x[3 * a + 1] - y[3 * b + 1],
                           x[3 * a + 2] - y[3 * b + 2]};
      const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (!(r2 > 0.0)) continue;
      const double ri = 1.0 / std::sqrt(r2), ri3 = ri * ri * ri;
      for (int i = 0; i < 3; ++i) {
        double *row = K.data() + (3 * a + i) * cols + (size_t)ncomp * b;
        for (int j = 0; j < 3; ++j)
          row[j] = ((i == j ? ri : 0.0) + d[i] * d[j] * ri3) / (8.0 * kPiF * mu);
        if (ncomp == 4) row[3] = d[i] * ri3 / (4.0 * kPiF);
      }
    }
}

// Pseudo-inverse of the row-major m x n matrix A (n x m, row-major), singular
// values below rcond * max truncated.  One-sided Jacobi on the columns of B,
// B = A^T when m < n (more columns than rows) and B = A otherwise.
void pinv(const std::vector<double> &A, int m, int n, double rcond, std::vector<double> &X) {
  const bool tr = m < n;
  const int rows = tr ? n : m, cols = tr ? m : n;
  // column-major copy of B
  std::vector<double> Bc((size_t)rows * cols), V((size_t)cols * cols, 0.0);
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < cols; ++c)
      Bc[(size_t)c * rows + r] = tr ? A[(size_t)c * n + r] : A[(size_t)r * n + c];
  for (int c = 0; c < cols; ++c) V[(size_t)c * cols + c] = 1.0;
  const double eps = 1e-15;
  for (int sweep = 0; sweep < 80; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < cols - 1; ++i)
      for (int j = i + 1; j < cols; ++j) {
        double *bi = &Bc[(size_t)i * rows], *bj = &Bc[(size_t)j * rows];
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int r = 0; r < rows; ++r) {
          al += bi[r] * bi[r];
          be += bj[r] * bj[r];
          ga += bi[r] * bj[r];
        }
        if (al == 0.0 || be == 0.0) continue;
        const double rel = std::fabs(ga) / std::sqrt(al * be);
        if (rel <= eps) continue;
        off = std::fmax(off, rel);
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = cs * t;
        for (int r = 0; r < rows; ++r) {
          const double u = bi[r], v = bj[r];
          bi[r] = cs * u - sn * v;
          bj[r] = sn * u + cs * v;
        }
        double *vi = &V[(size_t)i * cols], *vj = &V[(size_t)j * cols];
        for (int r = 0; r < cols; ++r) {
          const double u = vi[r], v = vj[r];
          vi[r] = cs * u - sn * v;
          vj[r] = sn * u + cs * v;
        }
      }
    if (off <= eps) break;
  }
  // B = U S V^T with U's columns b_c / s_c
  std::vector<double> s(cols);
  double smax = 0.0;
  for (int c = 0; c < cols; ++c) {
    double q = 0.0;
    for (int r = 0; r < rows; ++r) q += Bc[(size_t)c * rows + r] * Bc[(size_t)c * rows + r];
    s[c] = std::sqrt(q);
    smax = std::fmax(smax, s[c]);
  }
  // pinv(B) = V S^+ U^T  (cols x rows);  pinv(A) = pinv(B)^T when B = A^T
  X.assign((size_t)n * m, 0.0);
  for (int c = 0; c < cols; ++c) {
    if (!(s[c] > rcond * smax)) continue;
    const double inv2 = 1.0 / (s[c] * s[c]);  // U column = b_c / s_c, times 1 / s_c
    for (int a = 0; a < cols; ++a) {
      const double va = V[(size_t)c * cols + a] * inv2;
      if (va == 0.0) continue;
      const double *bc = &Bc[(size_t)c * rows];
      for (int r = 0; r < rows; ++r) {
        // pinv(B)[a][r] += V[a][c] / s_c^2 * b_c[r]
        if (tr)
          X[(size_t)r * m + a] += va * bc[r];  // pinv(A) = pinv(B)^T: n x m
        else
          X[(size_t)a * m + r] += va * bc[r];
      }
    }
  }
}

}  // namespace

extern "C" {

stk_status stokes_fmm_surface(int32_t p, double *pts, int32_t *count) {
  if (p < 2 || p > 16) return stk::report_error(STK_EINVAL, "p must be in [2, 16]");
  if (count) *count = surface_count(p);
  if (pts) {
    std::vector<double> s;
    surface(p, s);
    std::memcpy(pts, s.data(), sizeof(double) * s.size());
  }
  return STK_OK;
}

stk_status stokes_fmm_check_to_equiv(int32_t p, double r, double mu, int32_t upward,
                                     int32_t flux, double rcond, double *out) {
  if (p < 2 || p > 12) return stk::report_error(STK_EINVAL, "p must be in [2, 12]");
  if (!(r > 0.0) || !std::isfinite(r)) return stk::report_error(STK_EINVAL, "r must be > 0");
  if (!(mu > 0.0) || !std::isfinite(mu)) return stk::report_error(STK_EINVAL, "mu must be > 0");
  if (!(rcond >= 0.0 && rcond < 1.0)) return stk::report_error(STK_EINVAL, "rcond must be in [0, 1)");
  if (!out) return stk::report_error(STK_EINVAL, "out is NULL");
  std::vector<double> s, chk, eqv, K, X;
  surface(p, s);
  const int ns = surface_count(p);
  chk.resize(s.size());
  eqv.resize(s.size());
  const double rc = (upward ? kOuter : kInner) * r, re = (upward ? kInner : kOuter) * r;
  for (size_t i = 0; i < s.size(); ++i) {
    chk[i] = rc * s[i];
    eqv[i] = re * s[i];
  }
  const int ncomp = (upward && flux) ? 4 : 3;
  kernel_matrix(chk, eqv, mu, ncomp, K);
  pinv(K, 3 * ns, ncomp * ns, rcond, X);
  std::memcpy(out, X.data(), sizeof(double) * X.size());
  return STK_OK;
}

stk_status stokes_fmm_m2l_spectra(int32_t p, double mu, int32_t flux, double *out) {
  if (p < 2 || p > 12) return stk::report_error(STK_EINVAL, "p must be in [2, 12]");
  if (!(mu > 0.0) || !std::isfinite(mu)) return stk::report_error(STK_EINVAL, "mu must be > 0");
  if (!out) return stk::report_error(STK_EINVAL, "out is NULL");
  const int G = 2 * p, nz = p + 1, nc = flux ? 4 : 3, nic = 3 * nc;
  const size_t nfreq = (size_t)G * G * nz, per_offset = nfreq * nic * 2;
  const double delta = 2.0 * kInner / (p - 1);  // lattice spacing at half-width 1
  std::vector<double> cs(G), sn(G);
  for (int t = 0; t < G; ++t) {
    cs[t] = std::cos(2.0 * kPiF * t / G);
    sn[t] = std::sin(2.0 * kPiF * t / G);
  }
  // kernel on the lattice, then one 1-D DFT per axis (x, y, then the half
  // spectrum along z), complex values as (re, im)
  std::vector<double> T((size_t)G * G * G * nic), A((size_t)G * G * G * nic * 2),
      B((size_t)G * G * G * nic * 2);
  auto sgn = [G, p](int m) { return m < p ? m : m - G; };
  for (int ox = -3; ox <= 3; ++ox)
    for (int oy = -3; oy <= 3; ++oy)
      for (int oz = -3; oz <= 3; ++oz) {
        double *dst = out + (size_t)((ox + 3) * 49 + (oy + 3) * 7 + (oz + 3)) * per_offset;
        if (std::abs(ox) <= 1 && std::abs(oy) <= 1 && std::abs(oz) <= 1) {
          std::memset(dst, 0, sizeof(double) * per_offset);  // neighbours: never in a V-list
          continue;
        }
        for (int mx = 0; mx < G; ++mx)
          for (int my = 0; my < G; ++my)
            for (int mz = 0; mz < G; ++mz) {
              const double v[3] = {delta * sgn(mx) - 2.0 * ox, delta * sgn(my) - 2.0 * oy,
                                   delta * sgn(mz) - 2.0 * oz};
              const double r2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
              const double ri = 1.0 / std::sqrt(r2), ri3 = ri * ri * ri;
              double *t = T.data() + (((size_t)mx * G + my) * G + mz) * nic;
              for (int i = 0; i < 3; ++i) {
                for (int c = 0; c < 3; ++c)
                  t[i * nc + c] = ((i == c ? ri : 0.0) + v[i] * v[c] * ri3) / (8.0 * kPiF * mu);
                if (nc == 4) t[i * nc + 3] = v[i] * ri3 / (4.0 * kPiF);
              }
            }
        // x: A[kx][my][mz] = sum_mx T[mx][my][mz] e^{-2 pi i mx kx / G}
        for (int kx = 0; kx < G; ++kx)
          for (int my = 0; my < G; ++my)
            for (int mz = 0; mz < G; ++mz)
              for (int q = 0; q < nic; ++q) {
                double re = 0.0, im = 0.0;
                for (int mx = 0; mx < G; ++mx) {
                  const int t = (mx * kx) % G;
                  const double val = T[(((size_t)mx * G + my) * G + mz) * nic + q];
                  re += val * cs[t];
                  im -= val * sn[t];
                }
                double *a = A.data() + ((((size_t)kx * G + my) * G + mz) * nic + q) * 2;
                a[0] = re;
                a[1] = im;
              }
        // y: B[kx][ky][mz] = sum_my A[kx][my][mz] e^{-2 pi i my ky / G}
        for (int kx = 0; kx < G; ++kx)
          for (int ky = 0; ky < G; ++ky)
            for (int mz = 0; mz < G; ++mz)
              for (int q = 0; q < nic; ++q) {
                double re = 0.0, im = 0.0;
                for (int my = 0; my < G; ++my) {
                  const int t = (my * ky) % G;
                  const double *a = A.data() + ((((size_t)kx * G + my) * G + mz) * nic + q) * 2;
                  re += a[0] * cs[t] + a[1] * sn[t];
                  im += a[1] * cs[t] - a[0] * sn[t];
                }
                double *bb = B.data() + ((((size_t)kx * G + ky) * G + mz) * nic + q) * 2;
                bb[0] = re;
                bb[1] = im;
              }
        // z, half spectrum: out[kx][ky][kz <= p] = sum_mz B[kx][ky][mz] e^{-2 pi i mz kz / G}
        for (int kx = 0; kx < G; ++kx)
          for (int ky = 0; ky < G; ++ky)
            for (int kz = 0; kz < nz; ++kz)
              for (int q = 0; q < nic; ++q) {
                double re = 0.0, im = 0.0;
                for (int mz = 0; mz < G; ++mz) {
                  const int t = (mz * kz) % G;
                  const double *bb = B.data() + ((((size_t)kx * G + ky) * G + mz) * nic + q) * 2;
                  re += bb[0] * cs[t] + bb[1] * sn[t];
                  im += bb[1] * cs[t] - bb[0] * sn[t];
                }
                double *o = dst + ((((size_t)kx * G + ky) * nz + kz) * nic + q) * 2;
                o[0] = re;
                o[1] = im;
              }
      }
  return STK_OK;
}

stk_status stokes_fmm_kernel_matrix(const double *x, int32_t nx, const double *y, int32_t ny,
                                    double mu, int32_t ncomp, double *out) {
  if (nx < 0 || ny < 0) return stk::report_error(STK_EINVAL, "nx and ny must be >= 0");
  if (ncomp != 3 && ncomp != 4) return stk::report_error(STK_EINVAL, "ncomp must be 3 or 4");
  if (!(mu > 0.0) || !std::isfinite(mu)) return stk::report_error(STK_EINVAL, "mu must be > 0");
  if ((nx > 0 || ny > 0) && (!x || !y || !out)) return stk::report_error(STK_EINVAL, "NULL pointer");
  if (nx == 0 || ny == 0) return STK_OK;
  std::vector<double> X(x, x + 3 * (size_t)nx), Y(y, y + 3 * (size_t)ny), K;
  kernel_matrix(X, Y, mu, ncomp, K);
  std::memcpy(out, K.data(), sizeof(double) * K.size());
  return STK_OK;
}

// Check-to-equivalent operators of every depth 2..max_depth of a tree with
// root cube side root_size (the operators of one half-width r = root_size
// 2^-(d+1) per depth).  The Stokeslet is homogeneous of degree -1, so a
// Stokeslet-only operator of half-width r is r times that of half-width 1 (the
// cut-off is relative); the point source is homogeneous of degree -2: with
// flux, upward_scaled == 0 takes a pseudo-inverse at every depth (minimum-norm
// densities), upward_scaled != 0 takes the one of half-width 1 and measures
// source strengths in units of r (their rows scaled by r once more), an exact
// check-to-equivalent operator at every depth from one decomposition.
stk_status stokes_fmm_operators(int32_t p, double root_size, int32_t max_depth, double mu,
                                int32_t flux, double rcond, int32_t upward_scaled, double *uc2e,
                                double *dc2e) {
  if (p < 2 || p > 12) return stk::report_error(STK_EINVAL, "p must be in [2, 12]");
  if (!(root_size > 0.0) || !std::isfinite(root_size))
    return stk::report_error(STK_EINVAL, "root_size must be finite and > 0");
  if (max_depth < 0 || max_depth > 21) return stk::report_error(STK_EINVAL, "max_depth must be in [0, 21]");
  const int ns = surface_count(p), nc = flux ? 4 : 3;
  const int D = max_depth >= 2 ? max_depth - 1 : 0;
  if (D == 0) return STK_OK;
  if (!uc2e || !dc2e) return stk::report_error(STK_EINVAL, "uc2e/dc2e is NULL");
  const size_t nu = (size_t)nc * ns * 3 * ns, nd = (size_t)9 * ns * ns;
  std::vector<double> dc1(nd), uc1;
  stk_status st = stokes_fmm_check_to_equiv(p, 1.0, mu, 0, 0, rcond, dc1.data());
  if (st != STK_OK) return st;
  const bool one_upward = !flux || upward_scaled;
  if (one_upward) {
    uc1.resize(nu);
    st = stokes_fmm_check_to_equiv(p, 1.0, mu, 1, flux, rcond, uc1.data());
    if (st != STK_OK) return st;
  }
  for (int i = 0; i < D; ++i) {
    const double r = root_size / (double)(1 << (i + 2)) / 2;
    double *U = uc2e + (size_t)i * nu, *Dd = dc2e + (size_t)i * nd;
    for (size_t e = 0; e < nd; ++e) Dd[e] = r * dc1[e];
    if (!one_upward) {
      st = stokes_fmm_check_to_equiv(p, r, mu, 1, 1, rcond, U);
      if (st != STK_OK) return st;
    } else {
      for (size_t e = 0; e < nu; ++e) U[e] = r * uc1[e];
      if (flux)  // rows of source strengths (component 3 of each point): r once more
        for (int j = 0; j < ns; ++j)
          for (int c = 0; c < 3 * ns; ++c) U[((size_t)(4 * j + 3)) * 3 * ns + c] *= r;
    }
  }
  return STK_OK;
}

// Derived arrays of a tree given per box its depth, integer anchor, parent and
// leaf number (stk_fmm_tree's numbering: boxes depth by depth, children in
// their parents' order): depth_ptr [max_depth + 2], child_ptr [nbox + 1],
// leaf_box [nleaf] and each box's 27 same-depth neighbours (colleague,
// [nbox][27], -1 where there is none).  The order is checked.
stk_status stokes_fmm_tree_complete(int32_t nbox, int32_t nleaf, const int32_t *depth,
                                    const int32_t *anchor, const int32_t *parent,
                                    const int32_t *box_leaf, int32_t *max_depth,
                                    int32_t *depth_ptr, int32_t *child_ptr, int32_t *leaf_box,
                                    int32_t *colleague) {
  using stk::report_error;
  if (nbox < 1 || nleaf < 1 || nleaf > nbox) return report_error(STK_EINVAL, "need 1 <= nleaf <= nbox");
  if (!depth || !anchor || !parent || !box_leaf || !max_depth || !depth_ptr || !child_ptr ||
      !leaf_box || !colleague)
    return report_error(STK_EINVAL, "NULL array");
  if (depth[0] != 0 || parent[0] != -1 || (nbox > 1 && depth[1] == 0))
    return report_error(STK_EINVAL, "box 0 must be the root, the only box of depth 0");
  int32_t md = 0;
  for (int32_t b = 1; b < nbox; ++b) {
    if (depth[b] < depth[b - 1]) return report_error(STK_EINVAL, "boxes must be numbered depth by depth");
    const int32_t pb = parent[b];
    if (pb < 0 || pb >= nbox || depth[pb] != depth[b] - 1)
      return report_error(STK_EINVAL, "every box but the root needs a parent one depth up");
    if (b > 1 && pb < parent[b - 1])
      return report_error(STK_EINVAL, "children must be numbered in their parents' order");
    if (depth[b] > md) md = depth[b];
  }
  if (md > 21) return report_error(STK_EINVAL, "the tree is deeper than 21");
  *max_depth = md;
  for (int32_t d = 0, b = 0; d <= md + 1; ++d) {
    while (b < nbox && depth[b] < d) ++b;
    depth_ptr[d] = b;
  }
  std::vector<int32_t> cnt((size_t)nbox, 0);
  for (int32_t b = 1; b < nbox; ++b) ++cnt[parent[b]];
  child_ptr[0] = 1;
  for (int32_t b = 0; b < nbox; ++b) child_ptr[b + 1] = child_ptr[b] + cnt[b];
  for (int32_t l = 0; l < nleaf; ++l) leaf_box[l] = -1;
  int32_t seen = 0;
  for (int32_t b = 0; b < nbox; ++b) {
    const int32_t l = box_leaf[b];
    if (l < 0) continue;
    if (l >= nleaf || leaf_box[l] >= 0) return report_error(STK_EINVAL, "box_leaf must number every leaf exactly once");
    if (cnt[b] != 0) return report_error(STK_EINVAL, "a leaf box has children");
    leaf_box[l] = b;
    ++seen;
  }
  if (seen != nleaf) return report_error(STK_EINVAL, "box_leaf must number every leaf exactly once");
  // same-depth neighbours: per depth, the boxes' (i, j, k) keys sorted
  std::vector<std::pair<uint64_t, int32_t>> keys;
  auto key = [](int64_t i, int64_t j, int64_t k) {
    return ((uint64_t)i << 42) | ((uint64_t)j << 21) | (uint64_t)k;
  };
  for (int32_t d = 0; d <= md; ++d) {
    const int32_t lo = depth_ptr[d], hi = depth_ptr[d + 1];
    keys.clear();
    for (int32_t b = lo; b < hi; ++b) {
      const int32_t *a = anchor + 3 * (size_t)b;
      if (a[0] < 0 || a[1] < 0 || a[2] < 0 || a[0] >= (1 << d) || a[1] >= (1 << d) ||
          a[2] >= (1 << d))
        return report_error(STK_EINVAL, "an anchor lies outside its depth's grid");
      keys.emplace_back(key(a[0], a[1], a[2]), b);
    }
    std::sort(keys.begin(), keys.end());
    const int64_t m = (int64_t)1 << d;
    for (int32_t b = lo; b < hi; ++b) {
      const int32_t *a = anchor + 3 * (size_t)b;
      for (int o = 0; o < 27; ++o) {
        const int64_t i = a[0] + o / 9 - 1, j = a[1] + (o / 3) % 3 - 1, k = a[2] + o % 3 - 1;
        int32_t q = -1;
        if (i >= 0 && j >= 0 && k >= 0 && i < m && j < m && k < m) {
          const uint64_t kq = key(i, j, k);
          auto it = std::lower_bound(keys.begin(), keys.end(), std::make_pair(kq, (int32_t)-1));
          if (it != keys.end() && it->first == kq) q = it->second;
        }
        colleague[27 * (size_t)b + o] = q;
      }
    }
  }
  return STK_OK;
}

}  // extern "C"
