// fmm_passes.cuh -- the passes of the kernel-independent FMM's far field
// (Sec. 3.1, "Far evaluation": the smooth quadrature at all targets at once),
// one function per output value, so that each pass is "for every output e:
// compute e".  No output is written by two calls, so a pass needs no atomics
// and gives the same result in any execution order.
//
// The tree: boxes numbered depth by depth (depth 0 first), Morton order within
// a depth, so the children of a box are contiguous (child_ptr) and the boxes
// of one depth are one range (depth_ptr).  Points are sorted by leaf.  Lists
// (CSR over box numbers):
//   V(B): children of the same-depth neighbours of B's parent that do not
//         touch B (M2L);
//   W(B), B a leaf: boxes below B's same-depth neighbours that do not touch B
//         while their parent does (their upward densities at B's points);
//   X(B): leaves A with B in W(A) (their sources on B's downward check surface).
// The far field starts at depth 2 (a box of depth 1 touches every other).
//
// Surfaces: the boundary points of a p x p x p grid on a cube of half-width
// 1.05 r (upward equivalent, downward check) or 2.95 r (upward check,
// downward equivalent) about a box of half-width r.  The upward equivalent
// density has a force and, with flux, a point-source strength per point; the
// downward one a force.  Check-to-equivalent operators per depth are inputs.
//
// Steps, in order:
//   S2M    leaf sources -> upward check velocity (2.95 r);
//   M2M    children's upward densities -> parent's upward check velocity;
//   UC2E   upward check -> upward equivalent density, depth by depth upwards;
//   DCHK   V-list densities (M2L) + X-list sources + parent's downward
//          density (L2L, depth > 2) -> downward check velocity (1.05 r);
//          M2L either dense (kernel evaluations per surface-point pair) or,
//          given the kernel spectra, in Fourier space: UFFT (spectrum of each
//          box's upward density on the zero-padded (2p)^3 lattice, a direct
//          sum over its surface points, the only non-zero lattice values),
//          KMULP (per parent and frequency, blocked over the parent's
//          neighbours' children, given the colleague table; else KMUL, per
//          box and frequency over its V-list) and IFFT (back at the box's own
//          surface points);
//   DC2E   downward check -> downward equivalent density, depth by depth;
//   L2T    downward density of the point's leaf + W-list upward densities
//          -> velocity at every point.
// Each step exists in FP64 and in a mixed form (FP32 evaluations on local
// coordinates, double-FP32 check-to-equivalent products; see "mixed" below).
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>

#if defined(__CUDACC__)
#define FMM_HD __host__ __device__ inline
#else
#define FMM_HD inline
#endif
#if defined(__CUDA_ARCH__)
#define FMM_UNROLL _Pragma("unroll")
#else
#define FMM_UNROLL
#endif

// A host build with FMM_HOST_CHECKS checks every index before it is used.
#if defined(FMM_HOST_CHECKS)
void fmm_host_check_failed(const char *what, int64_t v, int64_t hi);
#define FMM_CHECK(v, hi, what)                                                 \
  do {                                                                         \
    if ((int64_t)(v) < 0 || (int64_t)(v) >= (int64_t)(hi))                     \
      fmm_host_check_failed(what, (int64_t)(v), (int64_t)(hi));                \
  } while (0)
#else
#define FMM_CHECK(v, hi, what) \
  do {                         \
  } while (0)
#endif

namespace stk {
namespace fmm {

constexpr double kPi = 3.14159265358979323846;
constexpr double kInner = 1.05;
constexpr double kOuter = 2.95;
constexpr int kFirstDepth = 2;  // shallowest depth with a far field
constexpr int kMaxTreeDepth = 21;

struct Tree {
  int32_t nbox, nleaf;
  const int32_t *depth;      // [nbox]
  const int32_t *anchor;     // [nbox][3] integer box index at its depth
  const int32_t *parent;     // [nbox], -1 for the root
  const int32_t *child_ptr;  // [nbox + 1]
  const int32_t *leaf_box;   // [nleaf] box number of each leaf
  const int32_t *leaf_ptr;   // [nleaf + 1] point ranges
  const int32_t *v_ptr, *v_idx, *w_ptr, *w_idx, *x_ptr, *x_idx;
  const int32_t *box_leaf;   // [nbox] leaf number or -1
  const int32_t *colleague;  // [nbox][27] same-depth box at anchor + (dx,dy,dz), -1 if none
                             // (index (dx+1) 9 + (dy+1) 3 + (dz+1)); NULL: V-list M2L
  double root_lo[3];
  double root_size;
};

// Everything one pass reads and writes.
struct Pass {
  Tree t;
  const double *pts, *f, *phi, *nrm, *w;  // [n][3] (w [n]); f or phi may be NULL
  int64_t n;
  double csl;   // 1 / (8 pi mu): single layer and the equivalent forces
  double cdl;   // 6 / (8 pi): double layer
  double csrc;  // 1 / (4 pi): equivalent point sources
  int32_t ns;   // points per surface
  int32_t nc;   // components of the upward density per point (3, or 4 with flux)
  double *surf;        // [ns][3] on [-1, 1]^3
  const double *uc2e;  // [depth - 2][nc ns][3 ns]
  const double *dc2e;  // [depth - 2][3 ns][3 ns]
  double *chk;         // [nbox][3 ns] check velocities (upward, then downward)
  double *up;          // [nbox][nc ns]
  double *dn;          // [nbox][3 ns]
  double *out;         // [n][3]
  int32_t accumulate;
  int32_t depth;       // depth of a per-depth pass; its boxes are [box0, box1)
  int32_t box0, box1;
  // Fourier-space M2L (spec != NULL): G = 2p lattice points per axis, the half
  // spectrum along z (p + 1 frequencies), nfreq = G G (p + 1)
  int32_t p;
  const double *spec;  // [343 offsets][nfreq][3][nc] complex, half-width 1
  int32_t *sidx;       // [ns][3] lattice index of each surface point
  double *tw;          // [G][2] cos, sin of 2 pi t / G
  double *uhat;        // [nbox][nfreq][nc] complex
  double *chat;        // [nbox][nfreq][3] complex
  double *m2l;         // [nbox][3 ns] M2L part of the downward check velocity
  // mixed precision (mixed != 0): FP32 copies; the FP64 chk, up, dn, tw, uhat,
  // chat and m2l are then unused (NULL)
  int32_t mixed;
  float *ploc;         // [n][3] point minus its leaf's centre
  float *qf, *pf, *nf; // [n][3] w f / (8 pi mu), w phi 6 / (8 pi), normals (NULL if unused)
  float *surf32;       // [ns][3]
  float *up32;         // [nbox][nc ns]
  float *dn32;         // [nbox][3 ns]
  float *tw32;         // [G][2]
  float *spec32;       // as spec
  float *uhat32, *chat32, *m2l32;
  float *chk32;             // [nbox][3 ns] check velocities (FP32 sums)
  float *ops_hi, *ops_lo;   // uc2e then dc2e as FP32 pairs
  int64_t n_uc2e, n_dc2e;   // entries of uc2e and dc2e
  // the CTA-blocked mixed kernels (fmm_fast.cu) add: the child in each octant
  // of a box, the boxes that are first children (flag and exclusive scan) and
  // the parents in that order, and the DFT matrices of the lattice
  int32_t *child8;     // [nbox][8] child box at octant (x&1) 4 + (y&1) 2 + (z&1), or -1
  int32_t *bflag;      // [nbox] 1 where the box is its parent's first child
  int32_t *bpos;       // [nbox + 1] exclusive scan of bflag (bpos[nbox] = total)
  int32_t *plist;      // [nbox] parents, in the order of their first children
  float *ftab;         // [ns][nfreq][2] forward DFT of the surface lattice (cos, -sin)
  float *fitab;        // inverse DFT over the half spectrum (weighted, / G^3) as the B table
                       // of the tensor-core product (fmm_fast.cu)
  int32_t *err;        // device error word (a tree index out of range), at workspace + 8 bytes
  float *uhh, *uhl;    // [nfreq][uslots][4][2] upward spectra of one depth split into TF32
                       // hi + lo parts, parent-major: slot 8 k + o holds the child in octant o
                       // of the depth's k-th parent (zero where there is none; fourth
                       // component zero without flux), operands of the tensor-core M2L
  int32_t uslots;      // slots of uhh / uhl per frequency (8 x the most parents of a depth)
  float *btab;         // [nfreq][52][hi, lo][48 x 32] kernel spectra of each neighbour
                       // direction and octant half in the tensor-core operand layout (see
                       // fmm_fast.cu)
  int32_t *vpar;       // [26][nbox] plist position of the neighbour in each direction of the
                       // parent at each plist position (-1 where it has no children)
  // work items of the blocked L2T (fmm_fast.cu): per leaf the item count,
  // log2 of the points per item and the exclusive scan of the counts; the
  // items as (leaf, block | log2 << 24) pairs
  int32_t *icnt, *ipb, *ioff, *items;
};

// Boundary points of the p^3 grid on [-1, 1]^3, i slowest, k fastest.
FMM_HD void fill_surface(int p, double *s) {
  int m = 0;
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j)
      for (int k = 0; k < p; ++k) {
        if (!(i == 0 || j == 0 || k == 0 || i == p - 1 || j == p - 1 || k == p - 1)) continue;
        s[3 * m + 0] = -1.0 + 2.0 * i / (p - 1);
        s[3 * m + 1] = -1.0 + 2.0 * j / (p - 1);
        s[3 * m + 2] = -1.0 + 2.0 * k / (p - 1);
        ++m;
      }
}

FMM_HD int surface_count(int p) { return p * p * p - (p - 2) * (p - 2) * (p - 2); }

FMM_HD int freq_count(int p) { return 4 * p * p * (p + 1); }

// Lattice indices of the surface points (the order of fill_surface) and the
// twiddles of the G-point DFT.
FMM_HD void fill_lattice(int p, int32_t *sidx, double *tw) {
  int m = 0;
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j)
      for (int k = 0; k < p; ++k) {
        if (!(i == 0 || j == 0 || k == 0 || i == p - 1 || j == p - 1 || k == p - 1)) continue;
        sidx[3 * m + 0] = i;
        sidx[3 * m + 1] = j;
        sidx[3 * m + 2] = k;
        ++m;
      }
  const int G = 2 * p;
  for (int t = 0; t < G; ++t) {
    tw[2 * t + 0] = cos(2.0 * kPi * t / G);
    tw[2 * t + 1] = sin(2.0 * kPi * t / G);
  }
}

// Centre and half-width of box b (depth d).
FMM_HD void box_geom(const Tree &t, int32_t b, int32_t d, double c[3], double &r) {
  const double size = t.root_size / (double)(1 << d);
  for (int q = 0; q < 3; ++q) c[q] = t.root_lo[q] + ((double)t.anchor[3 * b + q] + 0.5) * size;
  r = size / 2;
}

FMM_HD void surface_point(const Pass &P, const double c[3], double rad, int k, double x[3]) {
  for (int q = 0; q < 3; ++q) x[q] = c[q] + rad * P.surf[3 * k + q];
}

// Adds the single and double layer of the points [i0, i1) at x.
FMM_HD void add_sources(const Pass &P, const double x[3], int64_t i0, int64_t i1, double u[3]) {
  FMM_CHECK(i0, P.n + 1, "point range start");
  FMM_CHECK(i1, P.n + 1, "point range end");
  double us[3] = {0.0, 0.0, 0.0}, ud[3] = {0.0, 0.0, 0.0};
  for (int64_t i = i0; i < i1; ++i) {
    const double *y = P.pts + 3 * i;
    const double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (!(r2 > 0.0)) continue;
    const double r = sqrt(r2), ir = 1.0 / r;
    if (P.f) {
      const double q[3] = {P.w[i] * P.f[3 * i], P.w[i] * P.f[3 * i + 1], P.w[i] * P.f[3 * i + 2]};
      const double ir3 = ir / r2, dq = (d[0] * q[0] + d[1] * q[1] + d[2] * q[2]) * ir3;
      for (int a = 0; a < 3; ++a) us[a] += q[a] * ir + d[a] * dq;
    }
    if (P.phi) {
      const double *nn = P.nrm + 3 * i;
      const double s[3] = {P.w[i] * P.phi[3 * i], P.w[i] * P.phi[3 * i + 1],
                           P.w[i] * P.phi[3 * i + 2]};
      const double c = (d[0] * s[0] + d[1] * s[1] + d[2] * s[2]) *
                       (d[0] * nn[0] + d[1] * nn[1] + d[2] * nn[2]) / (r2 * r2 * r);
      for (int a = 0; a < 3; ++a) ud[a] += d[a] * c;
    }
  }
  for (int a = 0; a < 3; ++a) u[a] += P.csl * us[a] + P.cdl * ud[a];
}

// Adds at x the field of an equivalent density e on the surface of half-width
// rad about c: per point a force (Stokeslet) and, for nc = 4, a source.
FMM_HD void add_equivalent(const Pass &P, const double x[3], const double c[3], double rad,
                           const double *e, int nc, double u[3]) {
  double uf[3] = {0.0, 0.0, 0.0}, uq[3] = {0.0, 0.0, 0.0};
  for (int j = 0; j < P.ns; ++j) {
    double y[3];
    surface_point(P, c, rad, j, y);
    const double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (!(r2 > 0.0)) continue;
    const double ri = 1.0 / sqrt(r2), ri3 = ri * ri * ri;
    const double *ej = e + (size_t)nc * j;
    const double df = (d[0] * ej[0] + d[1] * ej[1] + d[2] * ej[2]) * ri3;
    for (int a = 0; a < 3; ++a) uf[a] += ej[a] * ri + d[a] * df;
    if (nc == 4)
      for (int a = 0; a < 3; ++a) uq[a] += d[a] * ej[3] * ri3;
  }
  for (int a = 0; a < 3; ++a) u[a] += P.csl * uf[a] + P.csrc * uq[a];
}

FMM_HD void store3(double *dst, const double u[3]) {
  dst[0] = u[0];
  dst[1] = u[1];
  dst[2] = u[2];
}

// S2M: e = leaf * ns + k.
struct S2M {
  FMM_HD void operator()(const Pass &P, int64_t e) const {
    const int64_t l = e / P.ns;
    const int k = (int)(e % P.ns);
    FMM_CHECK(l, P.t.nleaf, "leaf");
    const int32_t b = P.t.leaf_box[l];
    FMM_CHECK(b, P.t.nbox, "leaf box");
    const int32_t d = P.t.depth[b];
    if (d < kFirstDepth) return;
    double c[3], r, x[3], u[3] = {0.0, 0.0, 0.0};
    box_geom(P.t, b, d, c, r);
    surface_point(P, c, kOuter * r, k, x);
    add_sources(P, x, P.t.leaf_ptr[l], P.t.leaf_ptr[l + 1], u);
    store3(P.chk + (size_t)b * 3 * P.ns + 3 * k, u);
  }
};

// M2M: e = (box - box0) * ns + k over the boxes of one depth; leaves skip.
struct M2M {
  FMM_HD void operator()(const Pass &P, int64_t e) const {
    const int32_t b = P.box0 + (int32_t)(e / P.ns);
    const int k = (int)(e % P.ns);
    FMM_CHECK(b, P.box1, "m2m box");
    const int32_t c0 = P.t.child_ptr[b], c1 = P.t.child_ptr[b + 1];
    if (c0 >= c1) return;
    double c[3], r, x[3], u[3] = {0.0, 0.0, 0.0};
    box_geom(P.t, b, P.depth, c, r);
    surface_point(P, c, kOuter * r, k, x);
    for (int32_t ch = c0; ch < c1; ++ch) {
      FMM_CHECK(ch, P.t.nbox, "child");
      double cc[3], rc;
      box_geom(P.t, ch, P.depth + 1, cc, rc);
      add_equivalent(P, x, cc, kInner * rc, P.up + (size_t)ch * P.nc * P.ns, P.nc, u);
    }
    store3(P.chk + (size_t)b * 3 * P.ns + 3 * k, u);
  }
};

// Row i of a check-to-equivalent operator applied to box b's check velocity.
FMM_HD double apply_row(const double *M, int64_t i, const double *chk, int cols) {
  const double *row = M + (size_t)i * cols;
  double s = 0.0;
  for (int j = 0; j < cols; ++j) s += row[j] * chk[j];
  return s;
}

// UC2E: e = (box - box0) * nc ns + i.
struct UC2E {
  FMM_HD void operator()(const Pass &P, int64_t e) const {
    const int64_t rows = (int64_t)P.nc * P.ns;
    const int32_t b = P.box0 + (int32_t)(e / rows);
    const int64_t i = e % rows;
    FMM_CHECK(b, P.box1, "uc2e box");
    const double *M = P.uc2e + (size_t)(P.depth - kFirstDepth) * rows * 3 * P.ns;
    P.up[(size_t)b * rows + i] = apply_row(M, i, P.chk + (size_t)b * 3 * P.ns, 3 * P.ns);
  }
};

// DCHK: e = (box - box0) * ns + k over the boxes of one depth >= 2.
struct DCHK {
  FMM_HD void operator()(const Pass &P, int64_t e) const {
    const int32_t b = P.box0 + (int32_t)(e / P.ns);
    const int k = (int)(e % P.ns);
    FMM_CHECK(b, P.box1, "dchk box");
    double c[3], r, x[3], u[3] = {0.0, 0.0, 0.0};
    box_geom(P.t, b, P.depth, c, r);
    surface_point(P, c, kInner * r, k, x);
    if (P.spec)  // M2L done in Fourier space
      for (int q = 0; q < 3; ++q) u[q] = P.m2l[(size_t)b * 3 * P.ns + 3 * k + q];
    for (int32_t v = P.spec ? P.t.v_ptr[b + 1] : P.t.v_ptr[b]; v < P.t.v_ptr[b + 1]; ++v) {
      const int32_t a = P.t.v_idx[v];  // dense M2L
      FMM_CHECK(a, P.t.nbox, "V entry");
      double ca[3], ra;
      box_geom(P.t, a, P.t.depth[a], ca, ra);
      add_equivalent(P, x, ca, kInner * ra, P.up + (size_t)a * P.nc * P.ns, P.nc, u);
    }
    for (int32_t v = P.t.x_ptr[b]; v < P.t.x_ptr[b + 1]; ++v) {  // X-list sources
      const int32_t a = P.t.x_idx[v];
      FMM_CHECK(a, P.t.nbox, "X entry");
      const int32_t l = P.t.box_leaf[a];
      FMM_CHECK(l, P.t.nleaf, "X leaf");
      if (l < 0) continue;  // not a leaf: not an X-list entry
      add_sources(P, x, P.t.leaf_ptr[l], P.t.leaf_ptr[l + 1], u);
    }
    if (P.depth > kFirstDepth) {  // L2L
      const int32_t pb = P.t.parent[b];
      FMM_CHECK(pb, P.t.nbox, "parent");
      double cp[3], rp;
      box_geom(P.t, pb, P.depth - 1, cp, rp);
      add_equivalent(P, x, cp, kOuter * rp, P.dn + (size_t)pb * 3 * P.ns, 3, u);
    }
    store3(P.chk + (size_t)b * 3 * P.ns + 3 * k, u);
  }
};

// DC2E: e = (box - box0) * 3 ns + i.
struct DC2E {
  FMM_HD void operator()(const Pass &P, int64_t e) const {
    const int64_t rows = 3 * (int64_t)P.ns;
    const int32_t b = P.box0 + (int32_t)(e / rows);
    const int64_t i = e % rows;
    FMM_CHECK(b, P.box1, "dc2e box");
    const double *M = P.dc2e + (size_t)(P.depth - kFirstDepth) * rows * rows;
    P.dn[(size_t)b * rows + i] = apply_row(M, i, P.chk + (size_t)b * rows, (int)rows);
  }
};

// L2T + W-list: e = point (leaf order).
struct L2T {
  FMM_HD void operator()(const Pass &P, int64_t e) const {
    int32_t lo = 0, hi = P.t.nleaf;  // the last leaf whose range starts at or before e
    while (hi - lo > 1) {
      const int32_t mid = lo + (hi - lo) / 2;
      if (P.t.leaf_ptr[mid] <= e) lo = mid;
      else hi = mid;
    }
    const int32_t b = P.t.leaf_box[lo];
    FMM_CHECK(b, P.t.nbox, "point's leaf box");
    const int32_t d = P.t.depth[b];
    const double x[3] = {P.pts[3 * e], P.pts[3 * e + 1], P.pts[3 * e + 2]};
    double u[3] = {0.0, 0.0, 0.0};
    if (d >= kFirstDepth) {
      double c[3], r;
      box_geom(P.t, b, d, c, r);
      add_equivalent(P, x, c, kOuter * r, P.dn + (size_t)b * 3 * P.ns, 3, u);
    }
    for (int32_t v = P.t.w_ptr[b]; v < P.t.w_ptr[b + 1]; ++v) {
      const int32_t a = P.t.w_idx[v];
      FMM_CHECK(a, P.t.nbox, "W entry");
      double ca[3], ra;
      box_geom(P.t, a, P.t.depth[a], ca, ra);
      add_equivalent(P, x, ca, kInner * ra, P.up + (size_t)a * P.nc * P.ns, P.nc, u);
    }
    double *o = P.out + 3 * e;
    for (int a = 0; a < 3; ++a) o[a] = (P.accumulate ? o[a] : 0.0) + u[a];
  }
};

// Buffers of the FP64 (double) and mixed (float) forms.
template <class R>
struct Bufs;
template <>
struct Bufs<double> {
  static FMM_HD const double *up(const Pass &P) { return P.up; }
  static FMM_HD const double *tw(const Pass &P) { return P.tw; }
  static FMM_HD const double *spec(const Pass &P) { return P.spec; }
  static FMM_HD double *uhat(const Pass &P) { return P.uhat; }
  static FMM_HD double *chat(const Pass &P) { return P.chat; }
  static FMM_HD double *m2l(const Pass &P) { return P.m2l; }
};
template <>
struct Bufs<float> {
  static FMM_HD const float *up(const Pass &P) { return P.up32; }
  static FMM_HD const float *tw(const Pass &P) { return P.tw32; }
  static FMM_HD const float *spec(const Pass &P) { return P.spec32; }
  static FMM_HD float *uhat(const Pass &P) { return P.uhat32; }
  static FMM_HD float *chat(const Pass &P) { return P.chat32; }
  static FMM_HD float *m2l(const Pass &P) { return P.m2l32; }
};

// UFFT: e = ((box - box0) * nfreq + w) * nc + c; the spectrum of component c
// of the box's upward density, zero-padded to the G^3 lattice.
template <class R>
struct UFFTT {
  FMM_HD void operator()(const Pass &P, int64_t e) const {
    const int G = 2 * P.p, nz = P.p + 1, nf = freq_count(P.p);
    const int c = (int)(e % P.nc);
    const int64_t bw = e / P.nc;
    const int w = (int)(bw % nf);
    const int32_t b = P.box0 + (int32_t)(bw / nf);
    FMM_CHECK(b, P.box1, "ufft box");
    const int kx = w / (G * nz), ky = (w / nz) % G, kz = w % nz;
    const R *ub = Bufs<R>::up(P) + (size_t)b * P.nc * P.ns;
    const R *tw = Bufs<R>::tw(P);
    R re = 0, im = 0;
    for (int j = 0; j < P.ns; ++j) {
      const int t = (P.sidx[3 * j] * kx + P.sidx[3 * j + 1] * ky + P.sidx[3 * j + 2] * kz) % G;
      const R v = ub[(size_t)P.nc * j + c];
      re += v * tw[2 * t];
      im -= v * tw[2 * t + 1];
    }
    R *o = Bufs<R>::uhat(P) + (((size_t)b * nf + w) * P.nc + c) * 2;
    o[0] = re;
    o[1] = im;
  }
};

// KMUL: e = (box - box0) * nfreq + w; per velocity component the V-list sum of
// kernel spectrum (scaled to the depth) times source spectrum.
template <class R>
struct KMULT {
  FMM_HD void operator()(const Pass &P, int64_t e) const {
    const int nf = freq_count(P.p);
    const int w = (int)(e % nf);
    const int32_t b = P.box0 + (int32_t)(e / nf);
    FMM_CHECK(b, P.box1, "kmul box");
    double c[3], r;
    box_geom(P.t, b, P.depth, c, r);
    const R sf = (R)(1.0 / r), sq = (R)(1.0 / (r * r));  // Stokeslet 1 / r, source 1 / r^2
    const R *spec = Bufs<R>::spec(P);
    const R *uhat = Bufs<R>::uhat(P);
    R acc[6] = {0, 0, 0, 0, 0, 0};
    for (int32_t v = P.t.v_ptr[b]; v < P.t.v_ptr[b + 1]; ++v) {
      const int32_t a = P.t.v_idx[v];
      FMM_CHECK(a, P.t.nbox, "V entry");
      const int ox = P.t.anchor[3 * a] - P.t.anchor[3 * b];
      const int oy = P.t.anchor[3 * a + 1] - P.t.anchor[3 * b + 1];
      const int oz = P.t.anchor[3 * a + 2] - P.t.anchor[3 * b + 2];
      FMM_CHECK(ox + 3, 7, "V offset x");
      FMM_CHECK(oy + 3, 7, "V offset y");
      FMM_CHECK(oz + 3, 7, "V offset z");
      if (ox < -3 || ox > 3 || oy < -3 || oy > 3 || oz < -3 || oz > 3) continue;
      const int oi = (ox + 3) * 49 + (oy + 3) * 7 + (oz + 3);
      const R *S = spec + ((size_t)oi * nf + w) * 3 * P.nc * 2;
      const R *U = uhat + ((size_t)a * nf + w) * P.nc * 2;
      for (int cc = 0; cc < P.nc; ++cc) {
        const R sc = cc < 3 ? sf : sq;
        const R ur = U[2 * cc] * sc, ui = U[2 * cc + 1] * sc;
        for (int i = 0; i < 3; ++i) {
          const R kr = S[2 * (i * P.nc + cc)], ki = S[2 * (i * P.nc + cc) + 1];
          acc[2 * i] += kr * ur - ki * ui;
          acc[2 * i + 1] += kr * ui + ki * ur;
        }
      }
    }
    R *o = Bufs<R>::chat(P) + ((size_t)b * nf + w) * 3 * 2;
    for (int q = 0; q < 6; ++q) o[q] = acc[q];
  }
};

// IFFT: e = (box - box0) * ns + k; the inverse transform at surface point k
// (Hermitian half spectrum: planes kz = 0 and kz = p once, the others twice).
template <class R>
struct IFFTT {
  FMM_HD void operator()(const Pass &P, int64_t e) const {
    const int G = 2 * P.p, nz = P.p + 1, nf = freq_count(P.p);
    const int32_t b = P.box0 + (int32_t)(e / P.ns);
    const int k = (int)(e % P.ns);
    FMM_CHECK(b, P.box1, "ifft box");
    const int ix = P.sidx[3 * k], iy = P.sidx[3 * k + 1], iz = P.sidx[3 * k + 2];
    const R *C = Bufs<R>::chat(P) + (size_t)b * nf * 3 * 2;
    const R *tw = Bufs<R>::tw(P);
    R u[3] = {0, 0, 0};
    for (int w = 0; w < nf; ++w) {
      const int kx = w / (G * nz), ky = (w / nz) % G, kz = w % nz;
      const int t = (ix * kx + iy * ky + iz * kz) % G;
      const R cs = tw[2 * t], sn = tw[2 * t + 1];
      const R wt = (kz == 0 || kz == P.p) ? (R)1 : (R)2;
      for (int q = 0; q < 3; ++q)
        u[q] += wt * (C[(size_t)w * 6 + 2 * q] * cs - C[(size_t)w * 6 + 2 * q + 1] * sn);
    }
    const R inv = (R)(1.0 / ((double)G * G * G));
    for (int q = 0; q < 3; ++q) Bufs<R>::m2l(P)[(size_t)b * 3 * P.ns + 3 * k + q] = u[q] * inv;
  }
};

// KMULP: Fourier-space M2L blocked by parent.  e = w * (box1 - box0) + (parent
// - box0) over the parents of one depth (frequency-major, so that the threads
// of a warp share w and read the same kernel spectra).  For each of the 26
// neighbour directions of the parent, the source spectrum of each child of that
// neighbour is read once and applied to every child of the parent it does not
// touch, which enumerates exactly the V-lists of the parent's children (V(b):
// children of the neighbours of b's parent that do not touch b).  Writes the
// check spectra of all the parent's children at w.
template <class R>
struct KMULPT {
  FMM_HD void operator()(const Pass &P, int64_t e) const {
    const int nf = freq_count(P.p);
    const int64_t np = P.box1 - P.box0;
    const int w = (int)(e / np);
    const int32_t par = P.box0 + (int32_t)(e % np);
    FMM_CHECK(par, P.box1, "kmulp parent");
    const int32_t c0 = P.t.child_ptr[par], c1 = P.t.child_ptr[par + 1];
    if (c0 >= c1) return;
    FMM_CHECK(c1 - c0 - 1, 8, "children of a parent");
    double cc[3], r;
    box_geom(P.t, c0, P.depth, cc, r);  // the children's half-width
    const R sf = (R)(1.0 / r), sq = (R)(1.0 / (r * r));
    const R *spec = Bufs<R>::spec(P);
    const R *uhat = Bufs<R>::uhat(P);
    // fixed-size loops over the (up to 8) children and (up to 4) density
    // components keep the accumulators in registers
    const int nt = c1 - c0;
    int tpos[8][3];
    FMM_UNROLL
    for (int t = 0; t < 8; ++t)
      for (int q = 0; q < 3; ++q)
        tpos[t][q] = t < nt ? P.t.anchor[3 * (c0 + t) + q] - 2 * P.t.anchor[3 * par + q] : 0;
    R acc[8][6];
    FMM_UNROLL
    for (int t = 0; t < 8; ++t)
      for (int q = 0; q < 6; ++q) acc[t][q] = 0;
    for (int dir = 0; dir < 27; ++dir) {
      if (dir == 13) continue;  // the parent itself: its children touch each other
      const int32_t Q = P.t.colleague[27 * (size_t)par + dir];
      if (Q < 0) continue;
      FMM_CHECK(Q, P.t.nbox, "colleague");
      const int dx = dir / 9 - 1, dy = (dir / 3) % 3 - 1, dz = dir % 3 - 1;
      for (int32_t a = P.t.child_ptr[Q]; a < P.t.child_ptr[Q + 1]; ++a) {
        FMM_CHECK(a, P.t.nbox, "colleague child");
        const int sx = 2 * dx + P.t.anchor[3 * a] - 2 * P.t.anchor[3 * Q];
        const int sy = 2 * dy + P.t.anchor[3 * a + 1] - 2 * P.t.anchor[3 * Q + 1];
        const int sz = 2 * dz + P.t.anchor[3 * a + 2] - 2 * P.t.anchor[3 * Q + 2];
        const R *U = uhat + ((size_t)a * nf + w) * P.nc * 2;
        R u[8];
        FMM_UNROLL
        for (int c = 0; c < 4; ++c) {
          const R s = c < 3 ? sf : sq;
          u[2 * c] = c < P.nc ? U[2 * c] * s : (R)0;
          u[2 * c + 1] = c < P.nc ? U[2 * c + 1] * s : (R)0;
        }
        FMM_UNROLL
        for (int t = 0; t < 8; ++t) {
          if (t >= nt) continue;
          const int ox = sx - tpos[t][0], oy = sy - tpos[t][1], oz = sz - tpos[t][2];
          if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) continue;
          const int oi = (ox + 3) * 49 + (oy + 3) * 7 + (oz + 3);
          FMM_CHECK(oi, 343, "kmulp offset");
          const R *S = spec + ((size_t)oi * nf + w) * 3 * P.nc * 2;
          FMM_UNROLL
          for (int c = 0; c < 4; ++c) {
            if (c >= P.nc) continue;
            const R ur = u[2 * c], ui = u[2 * c + 1];
            FMM_UNROLL
            for (int i = 0; i < 3; ++i) {
              const R kr = S[2 * (i * P.nc + c)], ki = S[2 * (i * P.nc + c) + 1];
              acc[t][2 * i] += kr * ur - ki * ui;
              acc[t][2 * i + 1] += kr * ui + ki * ur;
            }
          }
        }
      }
    }
    FMM_UNROLL
    for (int t = 0; t < 8; ++t) {
      if (t >= nt) continue;
      R *o = Bufs<R>::chat(P) + ((size_t)(c0 + t) * nf + w) * 3 * 2;
      for (int q = 0; q < 6; ++q) o[q] = acc[t][q];
    }
  }
};

using UFFT = UFFTT<double>;
using KMUL = KMULT<double>;
using IFFT = IFFTT<double>;

// ------------------------------------------------------------------ mixed
// FP32 evaluations on local coordinates: points relative to their leaf's
// centre, surface points relative to their box's centre, and per pair of
// boxes one FP64 difference of centres rounded to FP32, so that no FP64
// operation runs per pair of points.  The check-to-equivalent operators are
// FP64 inputs, applied in double-FP32 arithmetic (below).

FMM_HD float frsqrt(float x) {
#if defined(__CUDA_ARCH__)
  return rsqrtf(x);
#else
  return 1.0f / sqrtf(x);
#endif
}

// centre of box a minus centre of box b, rounded to FP32
FMM_HD void centre_offset(const Pass &P, int32_t b, int32_t a, float off[3]) {
  double cb[3], ca[3], rb, ra;
  box_geom(P.t, b, P.t.depth[b], cb, rb);
  box_geom(P.t, a, P.t.depth[a], ca, ra);
  for (int q = 0; q < 3; ++q) off[q] = (float)(cb[q] - ca[q]);
}

// Adds at xs + off (relative to the centre of the sources' leaf) the single and
// double layer of the packed points [i0, i1).
FMM_HD void f_add_sources(const Pass &P, const float off[3], const float xs[3], int64_t i0,
                          int64_t i1, float u[3]) {
  FMM_CHECK(i0, P.n + 1, "point range start");
  FMM_CHECK(i1, P.n + 1, "point range end");
  const float x0 = off[0] + xs[0], x1 = off[1] + xs[1], x2 = off[2] + xs[2];
  for (int64_t i = i0; i < i1; ++i) {
    const float *y = P.ploc + 3 * i;
    const float d0 = x0 - y[0], d1 = x1 - y[1], d2 = x2 - y[2];
    const float r2 = d0 * d0 + d1 * d1 + d2 * d2;
    if (!(r2 > 0.0f)) continue;
    const float ri = frsqrt(r2), ri2 = ri * ri;
    if (P.qf) {
      const float *q = P.qf + 3 * i;
      const float dq = (d0 * q[0] + d1 * q[1] + d2 * q[2]) * ri2 * ri;
      u[0] += q[0] * ri + d0 * dq;
      u[1] += q[1] * ri + d1 * dq;
      u[2] += q[2] * ri + d2 * dq;
    }
    if (P.pf) {
      const float *s = P.pf + 3 * i, *nn = P.nf + 3 * i;
      const float c = (d0 * s[0] + d1 * s[1] + d2 * s[2]) * (d0 * nn[0] + d1 * nn[1] + d2 * nn[2]) *
                      ri2 * ri2 * ri;
      u[0] += d0 * c;
      u[1] += d1 * c;
      u[2] += d2 * c;
    }
  }
}

// Adds at xs + off (relative to the centre of the source box) the field of the
// FP32 equivalent density e on the source box's surface of half-width rad.
FMM_HD void f_add_equivalent(const Pass &P, const float off[3], const float xs[3], float rad,
                             const float *e, int nc, float u[3]) {
  const float x0 = off[0] + xs[0], x1 = off[1] + xs[1], x2 = off[2] + xs[2];
  const float csl = (float)P.csl, csrc = (float)P.csrc;
  float uf[3] = {0.0f, 0.0f, 0.0f}, uq[3] = {0.0f, 0.0f, 0.0f};
  for (int j = 0; j < P.ns; ++j) {
    const float *sj = P.surf32 + 3 * j;
    const float d0 = x0 - rad * sj[0], d1 = x1 - rad * sj[1], d2 = x2 - rad * sj[2];
    const float r2 = d0 * d0 + d1 * d1 + d2 * d2;
    if (!(r2 > 0.0f)) continue;
    const float ri = frsqrt(r2), ri3 = ri * ri * ri;
    const float *ej = e + (size_t)nc * j;
    const float df = (d0 * ej[0] + d1 * ej[1] + d2 * ej[2]) * ri3;
    uf[0] += ej[0] * ri + d0 * df;
    uf[1] += ej[1] * ri + d1 * df;
    uf[2] += ej[2] * ri + d2 * df;
    if (nc == 4) {
      const float s = ej[3] * ri3;
      uq[0] += d0 * s;
      uq[1] += d1 * s;
      uq[2] += d2 * s;
    }
  }
  for (int a = 0; a < 3; ++a) u[a] += csl * uf[a] + csrc * uq[a];
}

FMM_HD int32_t leaf_of_point(const Tree &t, int64_t e) {
  int32_t lo = 0, hi = t.nleaf;  // the last leaf whose range starts at or before e
  while (hi - lo > 1) {
    const int32_t mid = lo + (hi - lo) / 2;
    if (t.leaf_ptr[mid] <= e) lo = mid;
    else hi = mid;
  }
  return lo;
}

// PACK: e = point; local coordinates and pre-scaled FP32 densities.
struct PACK {
  FMM_HD void operator()(const Pass &P, int64_t e) const {
    const int32_t b = P.t.leaf_box[leaf_of_point(P.t, e)];
    FMM_CHECK(b, P.t.nbox, "point's leaf box");
    double c[3], r;
    box_geom(P.t, b, P.t.depth[b], c, r);
    for (int q = 0; q < 3; ++q) {
      P.ploc[3 * e + q] = (float)(P.pts[3 * e + q] - c[q]);
      if (P.qf) P.qf[3 * e + q] = (float)(P.csl * (P.w[e] * P.f[3 * e + q]));
      if (P.pf) {
        P.pf[3 * e + q] = (float)(P.cdl * (P.w[e] * P.phi[3 * e + q]));
        P.nf[3 * e + q] = (float)P.nrm[3 * e + q];
      }
    }
  }
};

// SPEC32: e = value; the kernel spectra rounded to FP32.
struct SPEC32 {
  FMM_HD void operator()(const Pass &P, int64_t e) const { P.spec32[e] = (float)P.spec[e]; }
};

// S2M, mixed: e = leaf * ns + k.
struct S2MF {
  FMM_HD void operator()(const Pass &P, int64_t e) const {
    const int64_t l = e / P.ns;
    const int k = (int)(e % P.ns);
    FMM_CHECK(l, P.t.nleaf, "leaf");
    const int32_t b = P.t.leaf_box[l];
    FMM_CHECK(b, P.t.nbox, "leaf box");
    const int32_t d = P.t.depth[b];
    if (d < kFirstDepth) return;
    double c[3], r;
    box_geom(P.t, b, d, c, r);
    const float rad = (float)(kOuter * r), off[3] = {0.0f, 0.0f, 0.0f};
    const float xs[3] = {rad * P.surf32[3 * k], rad * P.surf32[3 * k + 1],
                         rad * P.surf32[3 * k + 2]};
    float u[3] = {0.0f, 0.0f, 0.0f};
    f_add_sources(P, off, xs, P.t.leaf_ptr[l], P.t.leaf_ptr[l + 1], u);
    for (int q = 0; q < 3; ++q) P.chk32[(size_t)b * 3 * P.ns + 3 * k + q] = u[q];
  }
};

// M2M, mixed: e = (box - box0) * ns + k.
struct M2MF {
  FMM_HD void operator()(const Pass &P, int64_t e) const {
    const int32_t b = P.box0 + (int32_t)(e / P.ns);
    const int k = (int)(e % P.ns);
    FMM_CHECK(b, P.box1, "m2m box");
    const int32_t c0 = P.t.child_ptr[b], c1 = P.t.child_ptr[b + 1];
    if (c0 >= c1) return;
    double c[3], r;
    box_geom(P.t, b, P.depth, c, r);
    const float rad = (float)(kOuter * r);
    const float xs[3] = {rad * P.surf32[3 * k], rad * P.surf32[3 * k + 1],
                         rad * P.surf32[3 * k + 2]};
    const float rc = (float)(kInner * r / 2);  // children have half the half-width
    float u[3] = {0.0f, 0.0f, 0.0f};
    for (int32_t ch = c0; ch < c1; ++ch) {
      FMM_CHECK(ch, P.t.nbox, "child");
      float off[3];
      centre_offset(P, b, ch, off);
      f_add_equivalent(P, off, xs, rc, P.up32 + (size_t)ch * P.nc * P.ns, P.nc, u);
    }
    for (int q = 0; q < 3; ++q) P.chk32[(size_t)b * 3 * P.ns + 3 * k + q] = u[q];
  }
};

// Check-to-equivalent, mixed.  The operators' entries are large (1e3 to 1e8)
// and their row products cancel, so FP32 alone would not do; FP64 runs at
// 1/64 of the FP32 rate here.  Each operator entry is split into an FP32 pair
// (hi + lo, 48 bits), products are formed exactly by FMA (Dekker's product
// with FMA) and summed into a pair by Knuth's two-sum: the error stays below
// 2 u |result| + 4 n u^2 sum |terms| (u = 2^-24), i.e. about u + n u^2 k
// relative for a sum cancelling by k (k ~ 2e4 at p = 4, ~5e5 at p = 6 with
// operators cut at 1e-7).
FMM_HD float fma_f(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}

// Rounded FP32 operations the compiler may not fuse (the two-sum below is
// exact only if every product and sum is rounded on its own).
FMM_HD float mul_rn(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
FMM_HD float add_rn(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
FMM_HD float sub_rn(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}

// Row i of (hi + lo) times x, x exact in FP32 (the check velocities of the
// mixed passes are FP32 sums).  The operator is stored column by column
// (entry (i, j) at j * rows + i), so that the threads of a warp, which take
// consecutive rows, read consecutive addresses.
FMM_HD float apply_row_df(const float *hi, const float *lo, int64_t i, int64_t rows,
                          const float *x, int cols) {
  float sh = 0.0f, sl = 0.0f;
  for (int j = 0; j < cols; ++j) {
    const float ah = hi[(size_t)j * rows + i], al = lo[(size_t)j * rows + i];
    const float p = mul_rn(ah, x[j]);
    const float err = fma_f(al, x[j], fma_f(ah, x[j], -p));  // ah x = p + exact rest
    const float t = add_rn(sh, p), bv = sub_rn(t, sh);      // two-sum of sh and p
    sl = add_rn(sl, add_rn(add_rn(sub_rn(sh, sub_rn(t, bv)), sub_rn(p, bv)), err));
    sh = t;
  }
  return add_rn(sh, sl);
}

// OPSPLIT: e = operator entry (uc2e then dc2e, all depths, row-major as
// given); its hi and lo parts, stored transposed within each depth's matrix.
struct OPSPLIT {
  FMM_HD void operator()(const Pass &P, int64_t e) const {
    const int64_t nu = P.n_uc2e, cols = 3 * (int64_t)P.ns;
    const bool up = e < nu;
    const int64_t rows = up ? (int64_t)P.nc * P.ns : cols, m = up ? e : e - nu;
    const int64_t per = rows * cols, base = (up ? 0 : nu) + (m / per) * per;
    const int64_t i = (m % per) / cols, j = m % cols;
    const double v = up ? P.uc2e[e] : P.dc2e[e - nu];
    const float h = (float)v;
    P.ops_hi[base + j * rows + i] = h;
    P.ops_lo[base + j * rows + i] = (float)(v - (double)h);
  }
};

struct UC2EF {
  FMM_HD void operator()(const Pass &P, int64_t e) const {
    const int64_t rows = (int64_t)P.nc * P.ns;
    const int32_t b = P.box0 + (int32_t)(e / rows);
    const int64_t i = e % rows;
    FMM_CHECK(b, P.box1, "uc2e box");
    const size_t off = (size_t)(P.depth - kFirstDepth) * rows * 3 * P.ns;
    P.up32[(size_t)b * rows + i] = apply_row_df(P.ops_hi + off, P.ops_lo + off, i, rows,
                                                P.chk32 + (size_t)b * 3 * P.ns, 3 * P.ns);
  }
};

struct DC2EF {
  FMM_HD void operator()(const Pass &P, int64_t e) const {
    const int64_t rows = 3 * (int64_t)P.ns;
    const int32_t b = P.box0 + (int32_t)(e / rows);
    const int64_t i = e % rows;
    FMM_CHECK(b, P.box1, "dc2e box");
    const size_t off = (size_t)P.n_uc2e + (size_t)(P.depth - kFirstDepth) * rows * rows;
    P.dn32[(size_t)b * rows + i] = apply_row_df(P.ops_hi + off, P.ops_lo + off, i, rows,
                                                P.chk32 + (size_t)b * rows, (int)rows);
  }
};

// DCHK, mixed: e = (box - box0) * ns + k.
struct DCHKF {
  FMM_HD void operator()(const Pass &P, int64_t e) const {
    const int32_t b = P.box0 + (int32_t)(e / P.ns);
    const int k = (int)(e % P.ns);
    FMM_CHECK(b, P.box1, "dchk box");
    double c[3], r;
    box_geom(P.t, b, P.depth, c, r);
    const float rad = (float)(kInner * r);
    const float xs[3] = {rad * P.surf32[3 * k], rad * P.surf32[3 * k + 1],
                         rad * P.surf32[3 * k + 2]};
    float u[3] = {0.0f, 0.0f, 0.0f};
    if (P.spec)  // M2L done in Fourier space
      for (int q = 0; q < 3; ++q) u[q] = P.m2l32[(size_t)b * 3 * P.ns + 3 * k + q];
    for (int32_t v = P.spec ? P.t.v_ptr[b + 1] : P.t.v_ptr[b]; v < P.t.v_ptr[b + 1]; ++v) {
      const int32_t a = P.t.v_idx[v];  // dense M2L: same depth, same radius
      FMM_CHECK(a, P.t.nbox, "V entry");
      float off[3];
      centre_offset(P, b, a, off);
      f_add_equivalent(P, off, xs, rad, P.up32 + (size_t)a * P.nc * P.ns, P.nc, u);
    }
    for (int32_t v = P.t.x_ptr[b]; v < P.t.x_ptr[b + 1]; ++v) {  // X-list sources
      const int32_t a = P.t.x_idx[v];
      FMM_CHECK(a, P.t.nbox, "X entry");
      const int32_t l = P.t.box_leaf[a];
      FMM_CHECK(l, P.t.nleaf, "X leaf");
      if (l < 0) continue;
      float off[3];
      centre_offset(P, b, a, off);
      f_add_sources(P, off, xs, P.t.leaf_ptr[l], P.t.leaf_ptr[l + 1], u);
    }
    if (P.depth > kFirstDepth) {  // L2L
      const int32_t pb = P.t.parent[b];
      FMM_CHECK(pb, P.t.nbox, "parent");
      float off[3];
      centre_offset(P, b, pb, off);
      f_add_equivalent(P, off, xs, (float)(kOuter * 2.0 * r), P.dn32 + (size_t)pb * 3 * P.ns, 3, u);
    }
    for (int q = 0; q < 3; ++q) P.chk32[(size_t)b * 3 * P.ns + 3 * k + q] = u[q];
  }
};

// L2T + W-list, mixed: e = point (leaf order).
struct L2TF {
  FMM_HD void operator()(const Pass &P, int64_t e) const {
    const int32_t b = P.t.leaf_box[leaf_of_point(P.t, e)];
    FMM_CHECK(b, P.t.nbox, "point's leaf box");
    const int32_t d = P.t.depth[b];
    const float xs[3] = {P.ploc[3 * e], P.ploc[3 * e + 1], P.ploc[3 * e + 2]};
    float u[3] = {0.0f, 0.0f, 0.0f};
    if (d >= kFirstDepth) {
      double c[3], r;
      box_geom(P.t, b, d, c, r);
      const float off[3] = {0.0f, 0.0f, 0.0f};
      f_add_equivalent(P, off, xs, (float)(kOuter * r), P.dn32 + (size_t)b * 3 * P.ns, 3, u);
    }
    for (int32_t v = P.t.w_ptr[b]; v < P.t.w_ptr[b + 1]; ++v) {
      const int32_t a = P.t.w_idx[v];
      FMM_CHECK(a, P.t.nbox, "W entry");
      double ca[3], ra;
      box_geom(P.t, a, P.t.depth[a], ca, ra);
      float off[3];
      centre_offset(P, b, a, off);
      f_add_equivalent(P, off, xs, (float)(kInner * ra), P.up32 + (size_t)a * P.nc * P.ns, P.nc,
                       u);
    }
    double *o = P.out + 3 * e;
    for (int a = 0; a < 3; ++a) o[a] = (P.accumulate ? o[a] : 0.0) + (double)u[a];
  }
};

// Workspace layout.  FP64 form: surface, per-box check, upward and downward
// arrays, and with Fourier-space M2L the lattice, twiddles and spectra.  Mixed
// form: the check array stays FP64 (input of the FP64 operators); points,
// surfaces, densities and spectra are FP32.
struct Layout {
  size_t counters;  // int32 [4] at offset 0; [2] is the device error word
  size_t surf, chk, up, dn, sidx, tw, uhat, chat, m2l;
  size_t ploc, qf, pf, nf, surf32, up32, dn32, tw32, spec32, uhat32, chat32, m2l32;
  size_t chk32, ops_hi, ops_lo;
  size_t child8, bflag, bpos, plist, ftab, fitab, vpar, uhh, uhl, btab;
  int64_t uslots;
  size_t icnt, ipb, ioff, items;
  size_t total;
};

// Entries of the per-depth operators (depths 2..max_depth).
inline int64_t op_entries(int p, int nc, int max_depth, bool upward) {
  const int64_t ns = surface_count(p), D = max_depth >= kFirstDepth ? max_depth - 1 : 0;
  return D * (upward ? nc * ns : 3 * ns) * 3 * ns;
}

inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Slots of the parent-major source spectra of one depth: 8 per parent with
// children there; depth d has at most min(boxes at d - 1, boxes at d) of them.
inline int64_t spectrum_slots(const int32_t *depth_ptr, int max_depth) {
  int64_t m = 1;
  for (int d = 1; d <= max_depth; ++d) {
    const int64_t a = depth_ptr[d] - depth_ptr[d - 1], b = depth_ptr[d + 1] - depth_ptr[d];
    const int64_t c = a < b ? a : b;
    m = c > m ? c : m;
  }
  return 8 * m;
}

inline Layout layout(int64_t nbox, int p, int nc, bool fft, bool mixed, int64_t n,
                     int max_depth, const int32_t *depth_ptr) {
  const int ns = surface_count(p);
  const size_t nf = (size_t)freq_count(p), B = (size_t)nbox, N = (size_t)n;
  Layout L;
  size_t o = 0;
  auto take = [&o](size_t bytes) {
    const size_t at = o;
    o += align256(bytes);
    return at;
  };
  const size_t none = 0;
  L.counters = take(sizeof(int32_t) * 4);
  L.surf = take(sizeof(double) * 3 * ns);
  L.sidx = take(sizeof(int32_t) * 3 * ns);
  L.chk = L.up = L.dn = L.tw = L.uhat = L.chat = L.m2l = none;
  L.ploc = L.qf = L.pf = L.nf = L.surf32 = L.up32 = L.dn32 = L.tw32 = L.spec32 = L.uhat32 =
      L.chat32 = L.m2l32 = L.chk32 = L.ops_hi = L.ops_lo = none;
  L.child8 = L.bflag = L.bpos = L.plist = L.ftab = L.fitab = L.vpar = L.uhh = L.uhl = L.btab =
      none;
  L.uslots = spectrum_slots(depth_ptr, max_depth);
  L.icnt = L.ipb = L.ioff = L.items = none;
  if (!mixed) {
    L.chk = take(sizeof(double) * 3 * ns * B);
    L.up = take(sizeof(double) * nc * ns * B);
    L.dn = take(sizeof(double) * 3 * ns * B);
    L.tw = take(sizeof(double) * 4 * p);
    if (fft) {
      L.uhat = take(sizeof(double) * 2 * nf * nc * B);
      L.chat = take(sizeof(double) * 2 * nf * 3 * B);
      L.m2l = take(sizeof(double) * 3 * ns * B);
    }
  } else {
    const size_t nops = (size_t)(op_entries(p, nc, max_depth, true) +
                                 op_entries(p, nc, max_depth, false));
    L.chk32 = take(sizeof(float) * 3 * ns * B);
    L.ops_hi = take(sizeof(float) * nops);
    L.ops_lo = take(sizeof(float) * nops);
    L.ploc = take(sizeof(float) * 3 * N);
    L.qf = take(sizeof(float) * 3 * N);
    L.pf = take(sizeof(float) * 3 * N);
    L.nf = take(sizeof(float) * 3 * N);
    L.surf32 = take(sizeof(float) * 3 * ns);
    L.up32 = take(sizeof(float) * nc * ns * B);
    L.dn32 = take(sizeof(float) * 3 * ns * B);
    L.tw32 = take(sizeof(float) * 4 * p);
    if (fft) {
      L.spec32 = take(sizeof(float) * 343 * nf * 3 * nc * 2);
      L.uhat32 = take(sizeof(float) * 2 * nf * nc * B);
      L.chat32 = take(sizeof(float) * 2 * nf * 3 * B);
      L.m2l32 = take(sizeof(float) * 3 * ns * B);
      L.ftab = take(sizeof(float) * 2 * ns * nf);
      L.fitab = take(sizeof(float) * 2 * 64 * 32 * (size_t)((ns + 63) / 64) *
                     ((2 * nf + 31) / 32));  // the inverse-DFT product's B table
      L.vpar = take(sizeof(int32_t) * 26 * B);
      L.uhh = take(sizeof(float) * 8 * nf * (size_t)L.uslots);
      L.uhl = take(sizeof(float) * 8 * nf * (size_t)L.uslots);
      L.btab = take(sizeof(float) * nf * 52 * 2 * 48 * 32);
    }
    L.child8 = take(sizeof(int32_t) * 8 * B);
    L.bflag = take(sizeof(int32_t) * B);
    L.bpos = take(sizeof(int32_t) * (B + 1));
    L.plist = take(sizeof(int32_t) * B);
    // L2T items: at most ceil(points / 8) per leaf
    L.icnt = take(sizeof(int32_t) * B);  // B >= leaves
    L.ipb = take(sizeof(int32_t) * B);
    L.ioff = take(sizeof(int32_t) * (B + 1));
    L.items = take(sizeof(int32_t) * 2 * (B + (N + 7) / 8 + 1));
  }
  L.total = o + 256;  // slack for aligning the caller's base
  return L;
}

// Points the Pass at its buffers in a workspace (base aligned to 256 bytes).
inline void bind(Pass &P, char *ws, const Layout &L, bool fft, bool mixed) {
  auto d = [ws](size_t off) { return reinterpret_cast<double *>(ws + off); };
  auto f = [ws](size_t off) { return reinterpret_cast<float *>(ws + off); };
  P.surf = d(L.surf);
  P.sidx = reinterpret_cast<int32_t *>(ws + L.sidx);
  P.mixed = mixed ? 1 : 0;
  P.chk = mixed ? nullptr : d(L.chk);
  P.chk32 = mixed ? f(L.chk32) : nullptr;
  P.ops_hi = mixed ? f(L.ops_hi) : nullptr;
  P.ops_lo = mixed ? f(L.ops_lo) : nullptr;
  P.up = mixed ? nullptr : d(L.up);
  P.dn = mixed ? nullptr : d(L.dn);
  P.tw = mixed ? nullptr : d(L.tw);
  P.uhat = (fft && !mixed) ? d(L.uhat) : nullptr;
  P.chat = (fft && !mixed) ? d(L.chat) : nullptr;
  P.m2l = (fft && !mixed) ? d(L.m2l) : nullptr;
  P.ploc = mixed ? f(L.ploc) : nullptr;
  P.qf = (mixed && P.f) ? f(L.qf) : nullptr;
  P.pf = (mixed && P.phi) ? f(L.pf) : nullptr;
  P.nf = (mixed && P.phi) ? f(L.nf) : nullptr;
  P.surf32 = mixed ? f(L.surf32) : nullptr;
  P.up32 = mixed ? f(L.up32) : nullptr;
  P.dn32 = mixed ? f(L.dn32) : nullptr;
  P.tw32 = mixed ? f(L.tw32) : nullptr;
  P.spec32 = (fft && mixed) ? f(L.spec32) : nullptr;
  P.uhat32 = (fft && mixed) ? f(L.uhat32) : nullptr;
  P.chat32 = (fft && mixed) ? f(L.chat32) : nullptr;
  P.m2l32 = (fft && mixed) ? f(L.m2l32) : nullptr;
  auto i32 = [ws](size_t off) { return reinterpret_cast<int32_t *>(ws + off); };
  P.err = i32(L.counters) + 2;
  P.child8 = mixed ? i32(L.child8) : nullptr;
  P.bflag = mixed ? i32(L.bflag) : nullptr;
  P.bpos = mixed ? i32(L.bpos) : nullptr;
  P.plist = mixed ? i32(L.plist) : nullptr;
  P.ftab = (fft && mixed) ? f(L.ftab) : nullptr;
  P.fitab = (fft && mixed) ? f(L.fitab) : nullptr;
  P.vpar = (fft && mixed) ? i32(L.vpar) : nullptr;
  P.uslots = (int32_t)L.uslots;
  P.uhh = (fft && mixed) ? f(L.uhh) : nullptr;
  P.uhl = (fft && mixed) ? f(L.uhl) : nullptr;
  P.btab = (fft && mixed) ? f(L.btab) : nullptr;
  P.icnt = mixed ? i32(L.icnt) : nullptr;
  P.ipb = mixed ? i32(L.ipb) : nullptr;
  P.ioff = mixed ? i32(L.ioff) : nullptr;
  P.items = mixed ? i32(L.items) : nullptr;
}

// Surface points, lattice indices and twiddles (one thread; set-up of a call).
FMM_HD void fill_setup(const Pass &P) {
  fill_surface(P.p, P.surf);
  double tw[2 * 2 * 12];  // G = 2p <= 24 twiddles
  fill_lattice(P.p, P.sidx, tw);
  for (int t = 0; t < 2 * 2 * P.p; ++t) {
    if (P.tw) P.tw[t] = tw[t];
    if (P.tw32) P.tw32[t] = (float)tw[t];
  }
  if (P.surf32)
    for (int q = 0; q < 3 * P.ns; ++q) P.surf32[q] = (float)P.surf[q];
}

// The spectral products of one depth: blocked by parent when the colleague
// table is given, else per box over its V-list.
template <class Exec, class R>
void m2l_products(Exec &ex, Pass P, const int32_t *depth_ptr, int64_t per_box_count) {
  if (P.t.colleague) {
    P.box0 = depth_ptr[P.depth - 1];
    P.box1 = depth_ptr[P.depth];
    ex.template run<KMULPT<R>>(P, (int64_t)(P.box1 - P.box0) * freq_count(P.p));
  } else {
    ex.template run<KMULT<R>>(P, per_box_count);
  }
}

// The pass sequence; Exec::run<F>(P, count) calls F on every output of a pass
// (a kernel launch on the GPU).  depth_ptr is the host copy of the depth
// ranges of the boxes.
template <class Exec>
void far_field(Exec &ex, Pass P, const int32_t *depth_ptr, int32_t max_depth) {
  const int64_t ns = P.ns;
  const bool mixed = P.mixed != 0;
  if (mixed) {
    ex.template run<PACK>(P, P.n);
    ex.template run<OPSPLIT>(P, P.n_uc2e + P.n_dc2e);
    if (P.spec) ex.template run<SPEC32>(P, (int64_t)343 * freq_count(P.p) * 3 * P.nc * 2);
    ex.template run<S2MF>(P, (int64_t)P.t.nleaf * ns);
  } else {
    ex.template run<S2M>(P, (int64_t)P.t.nleaf * ns);
  }
  for (int32_t d = max_depth; d >= kFirstDepth; --d) {
    P.depth = d;
    P.box0 = depth_ptr[d];
    P.box1 = depth_ptr[d + 1];
    const int64_t nb = P.box1 - P.box0;
    if (mixed) {
      if (d < max_depth) ex.template run<M2MF>(P, nb * ns);
      ex.template run<UC2EF>(P, nb * P.nc * ns);
    } else {
      if (d < max_depth) ex.template run<M2M>(P, nb * ns);
      ex.template run<UC2E>(P, nb * P.nc * ns);
    }
  }
  for (int32_t d = kFirstDepth; d <= max_depth; ++d) {
    P.depth = d;
    P.box0 = depth_ptr[d];
    P.box1 = depth_ptr[d + 1];
    const int64_t nb = P.box1 - P.box0;
    const int64_t nf = freq_count(P.p);
    if (mixed) {
      if (P.spec) {
        ex.template run<UFFTT<float>>(P, nb * nf * P.nc);
        m2l_products<Exec, float>(ex, P, depth_ptr, nb * nf);
        ex.template run<IFFTT<float>>(P, nb * ns);
      }
      ex.template run<DCHKF>(P, nb * ns);
      ex.template run<DC2EF>(P, nb * 3 * ns);
    } else {
      if (P.spec) {
        ex.template run<UFFT>(P, nb * nf * P.nc);
        m2l_products<Exec, double>(ex, P, depth_ptr, nb * nf);
        ex.template run<IFFT>(P, nb * ns);
      }
      ex.template run<DCHK>(P, nb * ns);
      ex.template run<DC2E>(P, nb * 3 * ns);
    }
  }
  if (mixed) ex.template run<L2TF>(P, P.n);
  else ex.template run<L2T>(P, P.n);
}

}  // namespace fmm
}  // namespace stk
