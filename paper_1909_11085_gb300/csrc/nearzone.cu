// nearzone.cu -- near-zone search on a patch surface (Sec. 3.2, the closest-
// point search, steps a-e): for each target x, the patch of the surface
// closest to x when x lies within d_eps of it, with the closest point
// y = P(u*, v*), the unit normal there and the distance.
//
// A patch is the image of [-1, 1]^2 under the degree-q tensor-product
// interpolant through its (q+1) x (q+1) Clenshaw-Curtis nodes
// (u_i, v_j) = (cos(i pi/q), cos(j pi/q)), node index i (q+1) + j.
//  a. k_nz_boxes: each patch's node box, grown by d_eps and by 5% of its
//     diagonal (the interpolant may leave the nodes' box);
//  b. k_nz_grid / k_nz_cells: a spatial hash -- a uniform grid whose spacing
//     H is at least every box side, so that each box covers at most 2 x 2 x 2
//     cells -- and the (cell, patch) keys of every box;
//  c. the keys sorted (the library's radix sort); a target's cell key then
//     finds the patches whose boxes cover its cell (binary search), and the
//     exact box test keeps those whose box contains it;
//  d. for each of those, the closest point by Newton's method on
//     |x - P(u, v)|^2 with the Gauss-Newton Hessian, a backtracking (Armijo)
//     line search and projection onto [-1, 1]^2, started at the nearest node;
//  e. the nearest patch (ties to the lower index) is kept if its distance is
//     at most d_eps.
// Few targets lie near the surface, and the FP64 Newton iteration runs on
// GB300's FP64 pipe (1/64 of the FP32 rate), which charges a warp instruction
// in full however few of its lanes are active.  So k_nz_mark first lists the
// targets that lie in at least one grown box (and writes "none" for the
// rest), and k_nz_search runs one listed target per thread.
// All of it in FP64; the normal is (dP/du x dP/dv) / |dP/du x dP/dv|.
#include <cfloat>
#include <cmath>

#include "../../include/stokesgpu.h"
#include "common.cuh"
#include "prep.cuh"

namespace stk {
stk_status report_error(stk_status s, const char *msg);
}

namespace {

using namespace stk;

constexpr int kNzMaxN1 = 13;  // q <= 12
constexpr int kNzCells = 8;   // cells per patch box
constexpr int kNzThreads = 128;

struct NzGrid {
  double org[3];
  double H;
  int64_t dims[3];
};

__global__ void __launch_bounds__(kNzThreads) k_nz_boxes(const double *__restrict__ nodes,
                                                         int n1sq, double d_eps,
                                                         double *__restrict__ boxes,
                                                         double *__restrict__ rp) {
  __shared__ double s[6][kNzThreads];
  __shared__ double sr[kNzThreads];
  const int p = blockIdx.x;
  // the largest distance between two corners of a node cell: every point of
  // the patch lies within it of a node, up to the interpolant's small
  // deviation from the bilinear cell
  const int n1 = (int)lrint(sqrt((double)n1sq));
  double cm = 0.0;
  for (int e = threadIdx.x; e < (n1 - 1) * (n1 - 1); e += blockDim.x) {
    const int i = e / (n1 - 1), j = e % (n1 - 1);
    const double *c00 = nodes + ((size_t)p * n1sq + i * n1 + j) * 3;
    const double *c01 = c00 + 3, *c10 = c00 + 3 * n1, *c11 = c10 + 3;
    const double *cs[4] = {c00, c01, c10, c11};
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b) {
        const double dx = cs[a][0] - cs[b][0], dy = cs[a][1] - cs[b][1], dz = cs[a][2] - cs[b][2];
        cm = fmax(cm, dx * dx + dy * dy + dz * dz);
      }
  }
  sr[threadIdx.x] = cm;
  double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
  for (int e = threadIdx.x; e < n1sq; e += blockDim.x)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double v = nodes[((size_t)p * n1sq + e) * 3 + k];
      lo[k] = fmin(lo[k], v);
      hi[k] = fmax(hi[k], v);
    }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    s[k][threadIdx.x] = lo[k];
    s[3 + k][threadIdx.x] = hi[k];
  }
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        s[k][threadIdx.x] = fmin(s[k][threadIdx.x], s[k][threadIdx.x + o]);
        s[3 + k][threadIdx.x] = fmax(s[3 + k][threadIdx.x], s[3 + k][threadIdx.x + o]);
      }
      sr[threadIdx.x] = fmax(sr[threadIdx.x], sr[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    rp[p] = 1.1 * sqrt(sr[0]);
    const double dx = s[3][0] - s[0][0], dy = s[4][0] - s[1][0], dz = s[5][0] - s[2][0];
    const double grow = d_eps + 0.05 * sqrt(dx * dx + dy * dy + dz * dz);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      boxes[6 * p + k] = s[k][0] - grow;
      boxes[6 * p + 3 + k] = s[3 + k][0] + grow;
    }
  }
}

__global__ void __launch_bounds__(kNzThreads) k_nz_grid(const double *__restrict__ boxes,
                                                        int npatch, NzGrid *__restrict__ g) {
  __shared__ double s[7][kNzThreads];
  double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX}, side = 0.0;
  for (int p = threadIdx.x; p < npatch; p += blockDim.x)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      lo[k] = fmin(lo[k], boxes[6 * p + k]);
      hi[k] = fmax(hi[k], boxes[6 * p + 3 + k]);
      side = fmax(side, boxes[6 * p + 3 + k] - boxes[6 * p + k]);
    }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    s[k][threadIdx.x] = lo[k];
    s[3 + k][threadIdx.x] = hi[k];
  }
  s[6][threadIdx.x] = side;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        s[k][threadIdx.x] = fmin(s[k][threadIdx.x], s[k][threadIdx.x + o]);
        s[3 + k][threadIdx.x] = fmax(s[3 + k][threadIdx.x], s[3 + k][threadIdx.x + o]);
      }
      s[6][threadIdx.x] = fmax(s[6][threadIdx.x], s[6][threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double H = s[6][0] > 0.0 ? s[6][0] * (1.0 + 1e-9) : 1.0;
    // cell keys c0 + d0 (c1 + d1 c2) must fit 64 bits: a coarser grid only
    // puts more boxes in a cell
    double d[3];
    while (true) {
#pragma unroll
      for (int k = 0; k < 3; ++k) d[k] = floor((s[3 + k][0] - s[k][0]) / H) + 1.0;
      if (d[0] * d[1] * d[2] <= 4.0e18) break;
      H *= 2.0;
    }
    g->H = H;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      g->org[k] = s[k][0];
      g->dims[k] = (int64_t)d[k];
    }
  }
}

__device__ __forceinline__ bool nz_cell(const NzGrid &g, const double x[3], int64_t c[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double f = floor((x[k] - g.org[k]) / g.H);
    if (!(f >= 0.0) || f >= (double)g.dims[k]) return false;
    c[k] = (int64_t)f;
  }
  return true;
}

__global__ void k_nz_cells(const double *__restrict__ boxes, int npatch,
                           const NzGrid *__restrict__ gp, uint64_t *__restrict__ keys,
                           int32_t *__restrict__ vals) {
  const NzGrid g = *gp;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < npatch * kNzCells;
       e += gridDim.x * blockDim.x) {
    const int p = e / kNzCells, c = e % kNzCells;
    int64_t cl[3], ch[3], cc[3];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cl[k] = (int64_t)floor((boxes[6 * p + k] - g.org[k]) / g.H);
      ch[k] = (int64_t)floor((boxes[6 * p + 3 + k] - g.org[k]) / g.H);
      cl[k] = cl[k] < 0 ? 0 : cl[k];
      ch[k] = ch[k] >= g.dims[k] ? g.dims[k] - 1 : ch[k];
      cc[k] = cl[k] + ((c >> k) & 1);
      ok = ok && cc[k] <= ch[k];
    }
    keys[e] = ok ? (uint64_t)(cc[0] + g.dims[0] * (cc[1] + g.dims[1] * cc[2])) : ~0ull;
    vals[e] = p;
  }
}

// Lagrange basis on the CC nodes and its derivative at t (barycentric form;
// at a node, the differentiation matrix row).
__device__ void nz_basis(int n1, const double *xk, const double *wk, double t, double *L,
                         double *D) {
  int hit = -1;
  for (int k = 0; k < n1; ++k)
    if (fabs(t - xk[k]) < 1e-14) hit = k;
  if (hit >= 0) {
    double dd = 0.0;
    for (int k = 0; k < n1; ++k) {
      L[k] = k == hit ? 1.0 : 0.0;
      D[k] = 0.0;
      if (k != hit) {
        D[k] = (wk[k] / wk[hit]) / (xk[hit] - xk[k]);
        dd -= D[k];
      }
    }
    D[hit] = dd;
    return;
  }
  // l_k = (w_k / (t - x_k)) / S and l_k' = l_k (sum_m w_m / (t - x_m)^2 / S - 1 / (t - x_k)),
  // with D[] holding 1 / (t - x_k) until the end
  double S = 0.0, S2 = 0.0;
  for (int k = 0; k < n1; ++k) {
    const double r = 1.0 / (t - xk[k]);
    const double a = wk[k] * r;
    L[k] = a;
    D[k] = r;
    S += a;
    S2 += a * r;
  }
  const double iS = 1.0 / S, sig = S2 * iS;
  for (int k = 0; k < n1; ++k) {
    L[k] *= iS;
    D[k] = L[k] * (sig - D[k]);
  }
}

// P(u, v), dP/du, dP/dv of one patch.
__device__ void nz_eval(int n1, const double *__restrict__ X, const double *xk, const double *wk,
                        double u, double v, double P[3], double Pu[3], double Pv[3]) {
  double Lu[kNzMaxN1], Du[kNzMaxN1], Lv[kNzMaxN1], Dv[kNzMaxN1];
  nz_basis(n1, xk, wk, u, Lu, Du);
  nz_basis(n1, xk, wk, v, Lv, Dv);
#pragma unroll
  for (int c = 0; c < 3; ++c) P[c] = Pu[c] = Pv[c] = 0.0;
  for (int i = 0; i < n1; ++i) {
    double T[3] = {0.0, 0.0, 0.0}, Tv[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < n1; ++j) {
      const double *xp = X + 3 * (i * n1 + j);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T[c] = fma(Lv[j], xp[c], T[c]);
        Tv[c] = fma(Dv[j], xp[c], Tv[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      P[c] = fma(Lu[i], T[c], P[c]);
      Pu[c] = fma(Du[i], T[c], Pu[c]);
      Pv[c] = fma(Lu[i], Tv[c], Pv[c]);
    }
  }
}

// The node of a patch nearest to x: squared distance and its (u, v).
__device__ double nz_nearest_node(int n1, const double *__restrict__ X, const double *xk,
                                  const double x[3], double &u, double &v) {
  double best = DBL_MAX;
  for (int e = 0; e < n1 * n1; ++e) {
    const double *xp = X + 3 * e;
    const double d = (xp[0] - x[0]) * (xp[0] - x[0]) + (xp[1] - x[1]) * (xp[1] - x[1]) +
                     (xp[2] - x[2]) * (xp[2] - x[2]);
    if (d < best) {
      best = d;
      u = xk[e / n1];
      v = xk[e % n1];
    }
  }
  return best;
}

// Closest point of a patch to x, from the start (u, v).
__device__ double nz_closest(int n1, const double *__restrict__ X, const double *xk,
                             const double *wk, const double x[3], double &u, double &v,
                             double y[3], double nn[3]) {
  double P[3], Pu[3], Pv[3];
  nz_eval(n1, X, xk, wk, u, v, P, Pu, Pv);
  double f = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) f += (P[c] - x[c]) * (P[c] - x[c]);
  for (int it = 0; it < 40; ++it) {
    double gu = 0.0, gv = 0.0, huu = 0.0, huv = 0.0, hvv = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double r = P[c] - x[c];
      gu += r * Pu[c];
      gv += r * Pv[c];
      huu += Pu[c] * Pu[c];
      huv += Pu[c] * Pv[c];
      hvv += Pv[c] * Pv[c];
    }
    // active set: a parameter on its bound whose gradient points out of the
    // square stays there, and the step solves for the other one alone
    const bool fu = (u <= -1.0 && gu > 0.0) || (u >= 1.0 && gu < 0.0);
    const bool fv = (v <= -1.0 && gv > 0.0) || (v >= 1.0 && gv < 0.0);
    if (fu && fv) break;  // a corner that is a constrained minimum
    const double det = huu * hvv - huv * huv;
    double su, sv;
    if (fu) {
      su = 0.0;
      sv = hvv > 1e-300 ? -gv / hvv : -gv;
    } else if (fv) {
      su = huu > 1e-300 ? -gu / huu : -gu;
      sv = 0.0;
    } else if (det > 1e-300) {
      su = -(hvv * gu - huv * gv) / det;
      sv = -(huu * gv - huv * gu) / det;
    } else {
      su = -gu;
      sv = -gv;
    }
    const double slope = gu * su + gv * sv;  // half the directional derivative of f
    double a = 1.0, un = u, vn = v, Pn[3], Pun[3], Pvn[3], fn = f;
    bool moved = false;
    for (int ls = 0; ls < 40; ++ls) {
      un = fmin(1.0, fmax(-1.0, u + a * su));
      vn = fmin(1.0, fmax(-1.0, v + a * sv));
      nz_eval(n1, X, xk, wk, un, vn, Pn, Pun, Pvn);
      fn = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c) fn += (Pn[c] - x[c]) * (Pn[c] - x[c]);
      // Armijo decrease.  Near the minimum the decrease a step buys is below
      // the rounding of |x - P|^2 (about 1e-16 |x|^2; the distance is flat
      // along the surface), so a full Newton step shorter than 1e-6 in the
      // parameters is taken without the test
      if (fn <= f + 2e-4 * a * slope || (ls == 0 && fabs(su) + fabs(sv) < 1e-6)) {
        moved = true;
        break;
      }
      a *= 0.5;
    }
    if (!moved) break;
    const double step = fabs(un - u) + fabs(vn - v);
    u = un;
    v = vn;
    f = fn;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      P[c] = Pn[c];
      Pu[c] = Pun[c];
      Pv[c] = Pvn[c];
    }
    // converged: the parameters are in [-1, 1] and a step below 1e-12 is at
    // the level of the rounding in the gradient (coordinates of order 1e2)
    if (step < 1e-12) break;
  }
  const double cx = Pu[1] * Pv[2] - Pu[2] * Pv[1], cy = Pu[2] * Pv[0] - Pu[0] * Pv[2],
               cz = Pu[0] * Pv[1] - Pu[1] * Pv[0];
  const double cl = sqrt(cx * cx + cy * cy + cz * cz);
  nn[0] = cx / cl;
  nn[1] = cy / cl;
  nn[2] = cz / cl;
#pragma unroll
  for (int c = 0; c < 3; ++c) y[c] = P[c];
  return sqrt(f);
}

// Lists the targets inside at least one grown patch box; the others get
// "none" (patch -1, distance -1, zero parameters, point and normal).
__global__ void __launch_bounds__(kNzThreads) k_nz_mark(
    const double *__restrict__ boxes, const NzGrid *__restrict__ gp,
    const uint64_t *__restrict__ keys, const int32_t *__restrict__ vals, int64_t nkeys,
    const double *__restrict__ trg, int64_t nt, int32_t *__restrict__ list,
    int32_t *__restrict__ nlist, int32_t *__restrict__ patch_out, double *__restrict__ uv_out,
    double *__restrict__ y_out, double *__restrict__ n_out, double *__restrict__ dist_out) {
  const NzGrid g = *gp;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt;
       t += (int64_t)gridDim.x * blockDim.x) {
    const double x[3] = {trg[3 * t], trg[3 * t + 1], trg[3 * t + 2]};
    bool any = false;
    int64_t c[3];
    if (nz_cell(g, x, c)) {
      const uint64_t key = (uint64_t)(c[0] + g.dims[0] * (c[1] + g.dims[1] * c[2]));
      int64_t lo = 0, hi = nkeys;  // first entry with keys[i] >= key
      while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (keys[mid] < key) lo = mid + 1;
        else hi = mid;
      }
      for (int64_t i = lo; i < nkeys && keys[i] == key && !any; ++i) {
        const double *b = boxes + 6 * vals[i];
        any = x[0] >= b[0] && x[1] >= b[1] && x[2] >= b[2] && x[0] <= b[3] && x[1] <= b[4] &&
              x[2] <= b[5];
      }
    }
    if (any) {
      list[atomicAdd(nlist, 1)] = (int32_t)t;
    } else {
      patch_out[t] = -1;
      uv_out[2 * t] = uv_out[2 * t + 1] = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) y_out[3 * t + k] = n_out[3 * t + k] = 0.0;
      dist_out[t] = -1.0;
    }
  }
}

__global__ void __launch_bounds__(kNzThreads) k_nz_search(
    const double *__restrict__ nodes, int q, const double *__restrict__ boxes,
    const NzGrid *__restrict__ gp, const uint64_t *__restrict__ keys,
    const int32_t *__restrict__ vals, int64_t nkeys, const double *__restrict__ trg,
    const int32_t *__restrict__ list, const int32_t *__restrict__ nlist,
    const double *__restrict__ rp, double d_eps, int32_t *__restrict__ patch_out,
    double *__restrict__ uv_out,
    double *__restrict__ y_out, double *__restrict__ n_out, double *__restrict__ dist_out) {
  __shared__ double xk[kNzMaxN1], wk[kNzMaxN1];
  const int n1 = q + 1;
  if (threadIdx.x < n1) {
    xk[threadIdx.x] = cos(3.14159265358979323846 * threadIdx.x / q);
    wk[threadIdx.x] = ((threadIdx.x & 1) ? -1.0 : 1.0) * ((threadIdx.x == 0 || threadIdx.x == q) ? 0.5 : 1.0);
  }
  __syncthreads();
  const NzGrid g = *gp;
  const int64_t nl = *nlist;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nl;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = list[j];
    const double x[3] = {trg[3 * t], trg[3 * t + 1], trg[3 * t + 2]};
    int bp = -1;
    double bd = DBL_MAX, bu = 0.0, bv = 0.0, by[3] = {0.0, 0.0, 0.0}, bn[3] = {0.0, 0.0, 0.0};
    int64_t c[3];
    if (nz_cell(g, x, c)) {
      const uint64_t key = (uint64_t)(c[0] + g.dims[0] * (c[1] + g.dims[1] * c[2]));
      int64_t lo = 0, hi = nkeys;  // first entry with keys[i] >= key
      while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (keys[mid] < key) lo = mid + 1;
        else hi = mid;
      }
      for (int64_t i = lo; i < nkeys && keys[i] == key; ++i) {
        const int p = vals[i];
        const double *b = boxes + 6 * p;
        if (x[0] < b[0] || x[1] < b[1] || x[2] < b[2] || x[0] > b[3] || x[1] > b[4] ||
            x[2] > b[5])
          continue;
        const double *X = nodes + (size_t)p * n1 * n1 * 3;
        double u, v, y[3], nn[3];
        // every point of the patch lies within rp of a node: skip a patch that
        // cannot come within d_eps or beat the best so far
        const double lb = sqrt(nz_nearest_node(n1, X, xk, x, u, v)) - rp[p];
        if (lb > d_eps || lb > bd) continue;
        const double d = nz_closest(n1, X, xk, wk, x, u, v, y, nn);
        if (d < bd || (d == bd && p < bp)) {
          bd = d;
          bp = p;
          bu = u;
          bv = v;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            by[k] = y[k];
            bn[k] = nn[k];
          }
        }
      }
    }
    const bool near = bp >= 0 && bd <= d_eps;
    patch_out[t] = near ? bp : -1;
    uv_out[2 * t] = near ? bu : 0.0;
    uv_out[2 * t + 1] = near ? bv : 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      y_out[3 * t + k] = near ? by[k] : 0.0;
      n_out[3 * t + k] = near ? bn[k] : 0.0;
    }
    dist_out[t] = near ? bd : -1.0;
  }
}

struct NzLayout {
  size_t boxes, rp, grid, ka, va, kb, vb, hist, hist_scan, list, nlist, total;
};

NzLayout nz_layout(int32_t npatch, int64_t nt) {
  NzLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  const size_t nk = (size_t)npatch * kNzCells;
  L.boxes = take(sizeof(double) * 6 * (size_t)npatch);
  L.rp = take(sizeof(double) * (size_t)npatch);
  L.grid = take(sizeof(NzGrid));
  L.ka = take(sizeof(uint64_t) * nk);
  L.va = take(sizeof(int32_t) * nk);
  L.kb = take(sizeof(uint64_t) * nk);
  L.vb = take(sizeof(int32_t) * nk);
  const size_t he = radix_hist_entries((int64_t)nk);
  L.hist = take(sizeof(int32_t) * he);
  L.hist_scan = take(sizeof(int32_t) * (he + 1));
  L.list = take(sizeof(int32_t) * (size_t)(nt > 0 ? nt : 1));
  L.nlist = take(sizeof(int32_t));
  L.total = off + 256;
  return L;
}

}  // namespace

extern "C" {

stk_status stokes_near_search_workspace_size(int32_t npatch, int32_t q, int64_t nt,
                                             size_t *bytes) {
  if (!bytes) return report_error(STK_EINVAL, "bytes is NULL");
  if (npatch < 0) return report_error(STK_EINVAL, "npatch must be >= 0");
  if (nt < 0 || nt > 0x7fffffff) return report_error(STK_EINVAL, "nt must be in [0, 2^31 - 1]");
  if (q < 2 || q > kNzMaxN1 - 1) return report_error(STK_EUNSUPPORTED, "q must be in [2, 12]");
  *bytes = nz_layout(npatch, nt).total;
  return STK_OK;
}

stk_status stokes_near_patch_search(const double *nodes, int32_t npatch, int32_t q,
                                    const double *trg, int64_t nt, double d_eps, int32_t *patch,
                                    double *uv, double *y, double *n, double *dist,
                                    void *workspace, size_t workspace_bytes, void *stream) {
  size_t need = 0;
  stk_status s = stokes_near_search_workspace_size(npatch, q, nt, &need);
  if (s != STK_OK) return s;
  if (!(d_eps >= 0.0) || !std::isfinite(d_eps))
    return report_error(STK_EINVAL, "d_eps must be finite and >= 0");
  if (nt == 0) return STK_OK;
  if (!trg || !patch || !uv || !y || !n || !dist)
    return report_error(STK_EINVAL, "trg or an output is NULL");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (npatch == 0) {
    // no surface: nothing is near
    if (cudaMemsetAsync(patch, 0xff, sizeof(int32_t) * (size_t)nt, st) != cudaSuccess)
      return report_error(STK_ECUDA, "cudaMemsetAsync failed");
    return STK_OK;
  }
  if (!nodes) return report_error(STK_EINVAL, "nodes is NULL");
  if (!workspace || workspace_bytes < need) return report_error(STK_ENOMEM, "workspace too small");
  const NzLayout L = nz_layout(npatch, nt);
  const uintptr_t u = reinterpret_cast<uintptr_t>(workspace);
  char *ws = reinterpret_cast<char *>((u + 255) & ~(uintptr_t)255);
  double *boxes = reinterpret_cast<double *>(ws + L.boxes);
  NzGrid *grid = reinterpret_cast<NzGrid *>(ws + L.grid);
  uint64_t *ka = reinterpret_cast<uint64_t *>(ws + L.ka), *kb = reinterpret_cast<uint64_t *>(ws + L.kb);
  int32_t *va = reinterpret_cast<int32_t *>(ws + L.va), *vb = reinterpret_cast<int32_t *>(ws + L.vb);
  const int n1 = q + 1;
  double *rp = reinterpret_cast<double *>(ws + L.rp);
  k_nz_boxes<<<npatch, kNzThreads, 0, st>>>(nodes, n1 * n1, d_eps, boxes, rp);
  k_nz_grid<<<1, kNzThreads, 0, st>>>(boxes, npatch, grid);
  const int64_t nk = (int64_t)npatch * kNzCells;
  k_nz_cells<<<(int)((nk + 255) / 256), 256, 0, st>>>(boxes, npatch, grid, ka, va);
  count_launches(3);
  const int which = radix_sort(ka, va, kb, vb, nk, 64, reinterpret_cast<int32_t *>(ws + L.hist),
                               reinterpret_cast<int32_t *>(ws + L.hist_scan), st);
  const uint64_t *keys = which ? kb : ka;
  const int32_t *vals = which ? vb : va;
  int32_t *list = reinterpret_cast<int32_t *>(ws + L.list);
  int32_t *nlist = reinterpret_cast<int32_t *>(ws + L.nlist);
  if (cudaMemsetAsync(nlist, 0, sizeof(int32_t), st) != cudaSuccess)
    return report_error(STK_ECUDA, "cudaMemsetAsync failed");
  int64_t blocks = (nt + kNzThreads - 1) / kNzThreads;
  if (blocks > 65535) blocks = 65535;
  k_nz_mark<<<(int)blocks, kNzThreads, 0, st>>>(boxes, grid, keys, vals, nk, trg, nt, list, nlist,
                                                patch, uv, y, n, dist);
  k_nz_search<<<(int)blocks, kNzThreads, 0, st>>>(nodes, q, boxes, grid, keys, vals, nk, trg, list,
                                                  nlist, rp, d_eps, patch, uv, y, n, dist);
  count_launches(2);
  if (cudaGetLastError() != cudaSuccess) return report_error(STK_ECUDA, "near-zone search launch failed");
  return STK_OK;
}

}  // extern "C"
