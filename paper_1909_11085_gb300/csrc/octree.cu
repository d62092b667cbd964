// octree.cu -- host-side octree and interaction lists of the FMM (Sec. 3.1,
// "Far evaluation"): the tree the U-list P2P sum (stokes_p2p_leaflists) and
// the far field (stokes_fmm_far_eval) take.  The paper leaves the tree to its
// FMM library; this one is:
//   * root: the bounding cube of the points grown by 1e-9 (relative), so that
//     every point lies strictly inside;
//   * a box splits into its 8 children while it holds more than max_leaf
//     points (down to depth 21); a point belongs to the child whose half-open
//     box contains it (its integer cell on the depth-21 grid); empty children
//     are dropped; no 2:1 balance;
//   * leaves numbered depth-first in Morton order, points permuted so that each
//     leaf is one range;
//   * U(B) = the leaves whose closed box meets B's (B included);
//   * boxes numbered depth by depth, Morton order within a depth;
//   * V(B), depth >= 2: children of the same-depth neighbours of B's parent
//     that do not touch B; W(B), B a leaf: boxes below B's same-depth
//     neighbours that do not touch B while their parent does; X(B): the leaves
//     A with B in W(A).  All lists ascending.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <unordered_map>
#include <vector>

#include "../../include/stokesgpu.h"

namespace stk {
stk_status report_error(stk_status s, const char *msg);
}

namespace {

constexpr int kMaxDepth = 21;

uint64_t spread3(uint64_t v) {  // two zero bits between the low 21 bits
  v &= 0x1FFFFFull;
  v = (v | (v << 32)) & 0x1F00000000FFFFull;
  v = (v | (v << 16)) & 0x1F0000FF0000FFull;
  v = (v | (v << 8)) & 0x100F00F00F00F00Full;
  v = (v | (v << 4)) & 0x10C30C30C30C30C3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}

uint64_t morton(int64_t i, int64_t j, int64_t k) {
  return (spread3((uint64_t)i) << 2) | (spread3((uint64_t)j) << 1) | spread3((uint64_t)k);
}

struct Box {
  int32_t depth;
  int64_t a[3];  // integer index at its depth
};

// Closed boxes meet (exact, in depth-21 units).
bool touch(const Box &x, const Box &y) {
  const int64_t sx = (int64_t)1 << (kMaxDepth - x.depth), sy = (int64_t)1 << (kMaxDepth - y.depth);
  for (int q = 0; q < 3; ++q)
    if (!(x.a[q] * sx <= (y.a[q] + 1) * sy && y.a[q] * sy <= (x.a[q] + 1) * sx)) return false;
  return true;
}

}  // namespace

struct stk_octree {
  int64_t n = 0;
  double root_lo[3] = {0, 0, 0}, root_size = 0;
  std::vector<int64_t> perm;
  std::vector<int32_t> leaf_ptr, leaf_depth, ulist_ptr, ulist_idx;
  std::vector<int64_t> leaf_anchor;  // [nleaf][3]
  std::vector<int32_t> box_depth, box_anchor, box_parent, box_leaf;
  std::vector<int32_t> v_ptr, v_idx, w_ptr, w_idx, x_ptr, x_idx;
  std::vector<int32_t> colleague;  // [nbox][27]
};

namespace {

void csr(const std::vector<std::vector<int32_t>> &lists, std::vector<int32_t> &ptr,
         std::vector<int32_t> &idx) {
  ptr.assign(lists.size() + 1, 0);
  for (size_t b = 0; b < lists.size(); ++b) ptr[b + 1] = ptr[b] + (int32_t)lists[b].size();
  idx.clear();
  idx.reserve(ptr.back());
  for (const auto &l : lists) {
    std::vector<int32_t> s(l);
    std::sort(s.begin(), s.end());
    idx.insert(idx.end(), s.begin(), s.end());
  }
}

stk_status build(const double *pts, int64_t n, int32_t max_leaf, stk_octree &T) {
  // root cube and integer cells (the same operations, in the same order, as
  // the definition above spells out)
  double cmin[3], cmax[3];
  for (int q = 0; q < 3; ++q) cmin[q] = cmax[q] = pts[q];
  for (int64_t i = 1; i < n; ++i)
    for (int q = 0; q < 3; ++q) {
      cmin[q] = std::fmin(cmin[q], pts[3 * i + q]);
      cmax[q] = std::fmax(cmax[q], pts[3 * i + q]);
    }
  double ext = 0.0;
  for (int q = 0; q < 3; ++q) ext = std::fmax(ext, cmax[q] - cmin[q]);
  if (ext == 0.0) ext = 1.0;
  const double size = ext * (1.0 + 1e-9) + 1e-300;
  for (int q = 0; q < 3; ++q) T.root_lo[q] = 0.5 * (cmin[q] + cmax[q]) - 0.5 * size;
  T.root_size = size;
  const double scale = (double)(1 << kMaxDepth);
  const int64_t top = ((int64_t)1 << kMaxDepth) - 1;
  std::vector<uint64_t> key(n);
  for (int64_t i = 0; i < n; ++i) {
    int64_t c[3];
    for (int q = 0; q < 3; ++q) {
      const double v = std::floor((pts[3 * i + q] - T.root_lo[q]) / size * scale);
      c[q] = v < 0.0 ? 0 : (v > (double)top ? top : (int64_t)v);
    }
    key[i] = morton(c[0], c[1], c[2]);
  }
  T.perm.resize(n);
  for (int64_t i = 0; i < n; ++i) T.perm[i] = i;
  std::stable_sort(T.perm.begin(), T.perm.end(),
                   [&key](int64_t a, int64_t b) { return key[a] < key[b]; });
  std::vector<uint64_t> sk(n);
  for (int64_t i = 0; i < n; ++i) sk[i] = key[T.perm[i]];

  // depth-first split in Morton order
  struct Node {
    int64_t a, b;
    int32_t d;
    uint64_t prefix;
  };
  std::vector<Node> leaves, stack{{0, n, 0, 0}};
  while (!stack.empty()) {
    const Node nd = stack.back();
    stack.pop_back();
    if (nd.b - nd.a <= max_leaf || nd.d == kMaxDepth) {
      leaves.push_back(nd);
      continue;
    }
    const int shift = 3 * (kMaxDepth - nd.d - 1);
    std::vector<Node> kids;
    for (uint64_t c = 0; c < 8; ++c) {
      const uint64_t child = (nd.prefix << 3) | c;
      const uint64_t klo = child << shift, khi = (child + 1) << shift;
      const int64_t ca = std::lower_bound(sk.begin() + nd.a, sk.begin() + nd.b, klo) - sk.begin();
      const int64_t cb = std::lower_bound(sk.begin() + nd.a, sk.begin() + nd.b, khi) - sk.begin();
      if (cb > ca) kids.push_back({ca, cb, nd.d + 1, child});
    }
    for (auto it = kids.rbegin(); it != kids.rend(); ++it) stack.push_back(*it);
  }
  std::sort(leaves.begin(), leaves.end(), [](const Node &x, const Node &y) { return x.a < y.a; });
  const int64_t L = (int64_t)leaves.size();
  if (L > 0x7fffffffLL) return stk::report_error(STK_EUNSUPPORTED, "too many leaves");
  T.leaf_ptr.resize(L + 1);
  T.leaf_depth.resize(L);
  T.leaf_anchor.resize(3 * L);
  for (int64_t l = 0; l < L; ++l) {
    const Node &nd = leaves[l];
    T.leaf_ptr[l] = (int32_t)nd.a;
    T.leaf_depth[l] = nd.d;
    int64_t ix = 0, iy = 0, iz = 0;
    for (int lv = 0; lv < nd.d; ++lv) {
      const uint64_t bits = (nd.prefix >> (3 * (nd.d - 1 - lv))) & 7;
      ix = (ix << 1) | ((bits >> 2) & 1);
      iy = (iy << 1) | ((bits >> 1) & 1);
      iz = (iz << 1) | (bits & 1);
    }
    T.leaf_anchor[3 * l] = ix;
    T.leaf_anchor[3 * l + 1] = iy;
    T.leaf_anchor[3 * l + 2] = iz;
  }
  T.leaf_ptr[L] = (int32_t)n;

  // every box (the leaves' ancestors), depth by depth, Morton order; one map
  // from Morton code to box number per depth (a depth-21 code has 63 bits)
  std::vector<std::unordered_map<uint64_t, int32_t>> num(kMaxDepth + 1);
  struct Entry {
    int32_t depth;
    uint64_t code;
    Box b;
  };
  std::vector<Entry> order;
  for (int64_t l = 0; l < L; ++l) {
    const int32_t d = T.leaf_depth[l];
    for (int32_t k = 0; k <= d; ++k) {
      Box b{k, {T.leaf_anchor[3 * l] >> (d - k), T.leaf_anchor[3 * l + 1] >> (d - k),
                T.leaf_anchor[3 * l + 2] >> (d - k)}};
      const uint64_t code = morton(b.a[0], b.a[1], b.a[2]);
      if (num[k].emplace(code, -1).second) order.push_back({k, code, b});
    }
  }
  std::sort(order.begin(), order.end(), [](const Entry &x, const Entry &y) {
    return x.depth != y.depth ? x.depth < y.depth : x.code < y.code;
  });
  if (order.size() > 0x7fffffffULL) return stk::report_error(STK_EUNSUPPORTED, "too many boxes");
  const int32_t M = (int32_t)order.size();
  std::vector<Box> box(M);
  for (int32_t i = 0; i < M; ++i) {
    box[i] = order[i].b;
    num[order[i].depth][order[i].code] = i;
  }
  auto find = [&num](int32_t d, int64_t i, int64_t j, int64_t k) -> int32_t {
    const int64_t m = (int64_t)1 << d;
    if (d < 0 || d > kMaxDepth || i < 0 || j < 0 || k < 0 || i >= m || j >= m || k >= m)
      return -1;
    const auto it = num[d].find(morton(i, j, k));
    return it == num[d].end() ? -1 : it->second;
  };
  T.box_depth.resize(M);
  T.box_anchor.resize(3 * (size_t)M);
  T.box_parent.resize(M);
  T.box_leaf.assign(M, -1);
  std::vector<std::vector<int32_t>> kids(M);
  for (int32_t i = 0; i < M; ++i) {
    const Box &b = box[i];
    T.box_depth[i] = b.depth;
    for (int q = 0; q < 3; ++q) T.box_anchor[3 * i + q] = (int32_t)b.a[q];
    T.box_parent[i] = b.depth ? find(b.depth - 1, b.a[0] >> 1, b.a[1] >> 1, b.a[2] >> 1) : -1;
    if (T.box_parent[i] >= 0) kids[T.box_parent[i]].push_back(i);
  }
  for (int64_t l = 0; l < L; ++l)
    T.box_leaf[find(T.leaf_depth[l], T.leaf_anchor[3 * l], T.leaf_anchor[3 * l + 1],
                    T.leaf_anchor[3 * l + 2])] = (int32_t)l;

  // U-lists: descend from the root into every box that touches the leaf
  std::vector<std::vector<int32_t>> U(L);
  for (int64_t l = 0; l < L; ++l) {
    const Box me{T.leaf_depth[l], {T.leaf_anchor[3 * l], T.leaf_anchor[3 * l + 1],
                                   T.leaf_anchor[3 * l + 2]}};
    std::vector<int32_t> st{0};
    while (!st.empty()) {
      const int32_t q = st.back();
      st.pop_back();
      if (!touch(box[q], me)) continue;
      if (T.box_leaf[q] >= 0) U[l].push_back(T.box_leaf[q]);
      else
        for (int32_t c : kids[q]) st.push_back(c);
    }
  }
  csr(U, T.ulist_ptr, T.ulist_idx);

  // V, W, X
  std::vector<std::vector<int32_t>> V(M), W(M), X(M);
  auto colleagues = [&](int32_t b) {
    std::vector<int32_t> out;
    const Box &x = box[b];
    for (int di = -1; di <= 1; ++di)
      for (int dj = -1; dj <= 1; ++dj)
        for (int dk = -1; dk <= 1; ++dk) {
          const int32_t q = find(x.depth, x.a[0] + di, x.a[1] + dj, x.a[2] + dk);
          if (q >= 0) out.push_back(q);
        }
    return out;
  };
  for (int32_t b = 0; b < M; ++b) {
    if (box[b].depth < 2) continue;
    for (int32_t q : colleagues(T.box_parent[b]))
      for (int32_t c : kids[q])
        if (!touch(box[c], box[b])) V[b].push_back(c);
  }
  for (int32_t b = 0; b < M; ++b) {
    if (T.box_leaf[b] < 0) continue;
    std::vector<int32_t> st;
    for (int32_t q : colleagues(b))
      if (q != b && T.box_leaf[q] < 0) st.push_back(q);
    while (!st.empty()) {
      const int32_t q = st.back();
      st.pop_back();
      for (int32_t c : kids[q]) {
        if (!touch(box[c], box[b])) W[b].push_back(c);
        else if (T.box_leaf[c] < 0) st.push_back(c);
      }
    }
    for (int32_t a : W[b]) X[a].push_back(b);
  }
  csr(V, T.v_ptr, T.v_idx);
  csr(W, T.w_ptr, T.w_idx);
  csr(X, T.x_ptr, T.x_idx);
  T.colleague.resize(27 * (size_t)M);
  for (int32_t b = 0; b < M; ++b)
    for (int o = 0; o < 27; ++o)
      T.colleague[27 * (size_t)b + o] =
          find(box[b].depth, box[b].a[0] + o / 9 - 1, box[b].a[1] + (o / 3) % 3 - 1,
               box[b].a[2] + o % 3 - 1);
  T.n = n;
  return STK_OK;
}

template <class A, class B>
void copy_out(const std::vector<A> &v, B *dst) {
  if (dst)
    for (size_t i = 0; i < v.size(); ++i) dst[i] = (B)v[i];
}

}  // namespace

extern "C" {

stk_status stokes_octree_build(const double *pts, int64_t n, int32_t max_leaf, stk_octree **tree) {
  if (!tree) return stk::report_error(STK_EINVAL, "tree is NULL");
  *tree = nullptr;
  if (n < 1 || n > 0x7fffffffLL) return stk::report_error(STK_EINVAL, "n must be in [1, 2^31-1]");
  if (!pts) return stk::report_error(STK_EINVAL, "pts is NULL");
  if (max_leaf < 1) return stk::report_error(STK_EINVAL, "max_leaf must be >= 1");
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!std::isfinite(pts[i])) return stk::report_error(STK_EINVAL, "a point is not finite");
  stk_octree *t = new (std::nothrow) stk_octree;
  if (!t) return stk::report_error(STK_ENOMEM, "out of host memory");
  stk_status s;
  try {
    s = build(pts, n, max_leaf, *t);
  } catch (const std::bad_alloc &) {
    s = stk::report_error(STK_ENOMEM, "out of host memory");
  }
  if (s != STK_OK) {
    delete t;
    return s;
  }
  *tree = t;
  return STK_OK;
}

stk_status stokes_octree_info(const stk_octree *t, stk_octree_info *info) {
  if (!t || !info) return stk::report_error(STK_EINVAL, "tree/info is NULL");
  info->n = t->n;
  info->nleaf = (int32_t)t->leaf_depth.size();
  info->nbox = (int32_t)t->box_depth.size();
  info->max_depth = t->box_depth.empty() ? 0 : t->box_depth.back();
  info->nulist = (int64_t)t->ulist_idx.size();
  info->nv = (int64_t)t->v_idx.size();
  info->nw = (int64_t)t->w_idx.size();
  info->nx = (int64_t)t->x_idx.size();
  for (int q = 0; q < 3; ++q) info->root_lo[q] = t->root_lo[q];
  info->root_size = t->root_size;
  return STK_OK;
}

stk_status stokes_octree_export(const stk_octree *t, int64_t *perm, int32_t *leaf_ptr,
                                int32_t *ulist_ptr, int32_t *ulist_idx, int32_t *box_depth,
                                int32_t *box_anchor, int32_t *box_parent, int32_t *box_leaf,
                                int32_t *v_ptr, int32_t *v_idx, int32_t *w_ptr, int32_t *w_idx,
                                int32_t *x_ptr, int32_t *x_idx, int32_t *colleague) {
  if (!t) return stk::report_error(STK_EINVAL, "tree is NULL");
  copy_out(t->perm, perm);
  copy_out(t->leaf_ptr, leaf_ptr);
  copy_out(t->ulist_ptr, ulist_ptr);
  copy_out(t->ulist_idx, ulist_idx);
  copy_out(t->box_depth, box_depth);
  copy_out(t->box_anchor, box_anchor);
  copy_out(t->box_parent, box_parent);
  copy_out(t->box_leaf, box_leaf);
  copy_out(t->v_ptr, v_ptr);
  copy_out(t->v_idx, v_idx);
  copy_out(t->w_ptr, w_ptr);
  copy_out(t->w_idx, w_idx);
  copy_out(t->x_ptr, x_ptr);
  copy_out(t->x_idx, x_idx);
  copy_out(t->colleague, colleague);
  return STK_OK;
}

void stokes_octree_destroy(stk_octree *t) { delete t; }

}  // extern "C"
