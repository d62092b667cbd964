// Host build of the GPU far-field passes (paper_1909_11085_gb300/csrc/
// fmm_passes.cuh) for the CPU tests: the same per-output functions and the
// same pass sequence, run by plain loops over host arrays, with every index
// checked before it is used.  It is test infrastructure: the library does not
// contain or call it.
#include <cstdint>
#include <cstdio>
#include <vector>

#define FMM_HOST_CHECKS 1
#include "../../paper_1909_11085_gb300/csrc/fmm_passes.cuh"

static int g_bad = 0;
static char g_msg[256] = "";

void fmm_host_check_failed(const char *what, int64_t v, int64_t hi) {
  if (!g_bad) std::snprintf(g_msg, sizeof(g_msg), "%s: index %lld outside [0, %lld)", what,
                            (long long)v, (long long)hi);
  g_bad = 1;
}

namespace {
struct HostExec {
  int64_t launches = 0;
  template <class F>
  void run(const stk::fmm::Pass &P, int64_t n) {
    if (n <= 0) return;
    ++launches;
    for (int64_t e = 0; e < n && !g_bad; ++e) F()(P, e);
  }
};
}  // namespace

extern "C" {

const char *fmm_host_message(void) { return g_msg; }

// One row product of the mixed check-to-equivalent step: (hi + lo) . x (a
// one-row operator, so its column-by-column storage is the row itself).
float fmm_host_row_df(const float *hi, const float *lo, const float *x, int n) {
  return stk::fmm::apply_row_df(hi, lo, 0, 1, x, n);
}

// Returns the number of passes run (>= 0), or -1 when an index check failed.
long long fmm_host_far_eval(const double *pts, const double *f, const double *phi,
                            const double *nrm, const double *w, long long n, int nbox, int nleaf,
                            int max_depth, const int *depth_ptr, const int *depth,
                            const int *anchor, const int *parent, const int *child_ptr,
                            const int *box_leaf, const int *leaf_box, const int *leaf_ptr,
                            const int *v_ptr, const int *v_idx, const int *w_ptr,
                            const int *w_idx, const int *x_ptr, const int *x_idx,
                            const int *colleague, const double *root_lo, double root_size,
                            int p, int flux,
                            const double *uc2e, const double *dc2e, const double *spec,
                            int mixed, double mu, double *out, int accumulate) {
  g_bad = 0;
  g_msg[0] = 0;
  stk::fmm::Pass P;
  stk::fmm::Tree &T = P.t;
  T.nbox = nbox;
  T.nleaf = nleaf;
  T.depth = depth;
  T.anchor = anchor;
  T.parent = parent;
  T.child_ptr = child_ptr;
  T.box_leaf = box_leaf;
  T.leaf_box = leaf_box;
  T.leaf_ptr = leaf_ptr;
  T.v_ptr = v_ptr;
  T.v_idx = v_idx;
  T.w_ptr = w_ptr;
  T.w_idx = w_idx;
  T.x_ptr = x_ptr;
  T.x_idx = x_idx;
  T.colleague = colleague;
  for (int q = 0; q < 3; ++q) T.root_lo[q] = root_lo[q];
  T.root_size = root_size;
  const int ns = stk::fmm::surface_count(p), nc = flux ? 4 : 3;
  P.pts = pts;
  P.f = f;
  P.phi = phi;
  P.nrm = nrm;
  P.w = w;
  P.n = n;
  P.csl = 1.0 / (8.0 * stk::fmm::kPi * mu);
  P.cdl = 6.0 / (8.0 * stk::fmm::kPi);
  P.csrc = 1.0 / (4.0 * stk::fmm::kPi);
  P.ns = ns;
  P.nc = nc;
  P.uc2e = uc2e;
  P.dc2e = dc2e;
  P.out = out;
  P.accumulate = accumulate;
  P.depth = 0;
  P.box0 = P.box1 = 0;
  P.p = p;
  P.spec = spec;
  P.n_uc2e = stk::fmm::op_entries(p, nc, max_depth, true);
  P.n_dc2e = stk::fmm::op_entries(p, nc, max_depth, false);
  // the library's workspace layout, in one buffer aligned as the library aligns it
  const stk::fmm::Layout L =
      stk::fmm::layout(nbox, p, nc, spec != nullptr, mixed != 0, n, max_depth, depth_ptr);
  std::vector<char> buf(L.total + 256);
  char *ws = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(buf.data()) + 255) &
                                      ~(uintptr_t)255);
  stk::fmm::bind(P, ws, L, spec != nullptr, mixed != 0);
  stk::fmm::fill_setup(P);
  HostExec ex;
  stk::fmm::far_field(ex, P, depth_ptr, max_depth);
  return g_bad ? -1 : ex.launches;
}

}  // extern "C"
