// stokes_abi.cu -- the C ABI declared in include/stokesgpu.h: argument
// validation, workspace planning and the launch sequence of every form.
//
// Launch sequence (all on the caller's stream, nothing allocated):
//   1. zero the workspace counters (item count, engine and near-pair queue
//      heads, error word);
//   2. pack the sources (mixed 64-byte or FP64 96-byte records);
//   3. MIXED direct/batched: bounding box + Morton keys + stable radix sort of
//      the targets, so that every 128-target work item is spatially compact;
//   4. build work items (direct: target chunks x source splits; near field:
//      leaf chunks x U-list; batched: suspension chunks x {cells, wall}) and,
//      where items are uneven, radix-sort them by descending cost;
//   5. one persistent engine launch (SMs x resident CTAs, 4 warps each);
//      MIXED: then k_near adds the near pairs the engine left out, in FP64;
//   6. reduce the source splits in fixed order and scatter to caller order.
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>

#include "../../include/stokesgpu.h"
#include "common.cuh"
#include "prep.cuh"

using namespace stk;

namespace stk {
unsigned long long context_id();  // noalloc.cu
}

namespace {

thread_local std::string g_err;
thread_local cudaEvent_t g_ev_start = nullptr, g_ev_stop = nullptr;
// Wait policy of later calls on this thread (stokes_set_wait_policy): the
// bound of the engine's chunk waits (0 = default) and forced expiry.
thread_local int64_t g_wait_limit = 0;
thread_local int32_t g_force_expire = 0;

// Kernels recorded in each executable graph the library captured, so that a
// replay adds them to the launch count (any thread may replay a graph).
std::mutex g_graph_mu;
std::unordered_map<void *, int64_t> g_graph_kernels;

stk_status fail(stk_status s, const char *msg) {
  g_err = msg;
  return s;
}

#define CU(x)                                                                        \
  do {                                                                               \
    cudaError_t e_ = (x);                                                            \
    if (e_ != cudaSuccess) {                                                         \
      g_err = std::string(#x) + ": " + cudaGetErrorString(e_);                       \
      return STK_ECUDA;                                                              \
    }                                                                                \
  } while (0)

constexpr double kPi = 3.14159265358979323846;
constexpr int64_t kMaxN = 0x7fffffffLL;
constexpr int64_t kSpinLimit = 4000000000LL;  // SM cycles, about 2 s at 2 GHz

struct DevInfo {
  int dev = -1;
  int sms = 0;
  int occ_mixed = 0;
  int occ_fp64 = 0;
};

cudaError_t dev_info(DevInfo &di) {
  static thread_local DevInfo cache[16];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 16) return cudaErrorInvalidDevice;
  DevInfo &c = cache[dev];
  if (c.dev != dev) {
    DevInfo n;
    n.dev = dev;
    e = cudaDeviceGetAttribute(&n.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = engine_mixed_occupancy(&n.occ_mixed);
    if (e != cudaSuccess) return e;
    e = engine_fp64_occupancy(&n.occ_fp64);
    if (e != cudaSuccess) return e;
    if (n.occ_mixed < 1) n.occ_mixed = 1;
    if (n.occ_fp64 < 1) n.occ_fp64 = 1;
    c = n;
  }
  di = c;
  return cudaSuccess;
}

// ------------------------------------------------------------ workspace plan
struct Alloc {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  }
};

enum Form { F_DIRECT, F_P2P, F_BATCHED };

struct Plan {
  Form form;
  bool mixed;
  int64_t ns, nt;
  int32_t nsplit = 1;
  int64_t max_items = 0;
  TileConfig tile = {kItemMax, 0};
  int32_t nseg_ranges = 0;  // entries of range_ptr minus one
  bool sort_targets = false;
  bool sort_items = false;
  bool small = false;  // the one-launch small direct form (direct_small.cu)
  int32_t ngroup = 0;
  // offsets (the counters always sit at offset 0 of the aligned workspace)
  size_t counters, rec, keys_a, keys_b, vals_a, vals_b, ikeys_a, ikeys_b, ivals_a, ivals_b, hist,
      hist_scan, bbox_part, bbox, items, range, cnt, offs, part, frames = 0, xloc = 0,
      cand_list = 0, cand_cnt = 0, total;
};

// Candidate sources the engine lists per item for k_near (items with more are
// rescanned by k_near).
constexpr int32_t kCandCap = 512;

int auto_splits(int64_t nt, int64_t ns, const DevInfo &di, int occ) {
  const int64_t chunks = (nt + kItemMax - 1) / kItemMax;
  if (chunks <= 0) return 1;
  const int64_t warps = (int64_t)di.sms * occ * kWarpsPerCta;
  int64_t s = (2 * warps + chunks - 1) / chunks;
  const int64_t cap = ns / 64 > 1 ? ns / 64 : 1;  // at least 64 sources per split
  if (s > cap) s = cap;
  if (s > 64) s = 64;
  if (s < 1) s = 1;
  return (int)s;
}

void layout(Plan &p) {
  Alloc a;
  p.counters = a.take(sizeof(int32_t) * 4);
  if (p.small) {  // partial results per source split and a counter per target block
    p.cnt = a.take(sizeof(int32_t) * (size_t)direct_small_blocks(p.nt));
    p.part = a.take(sizeof(double) * 3 * (size_t)p.nt * (size_t)p.nsplit);
    p.total = a.off + 256;
    return;
  }
  p.rec = a.take((size_t)p.ns * (p.mixed ? sizeof(SrcRec) : sizeof(SrcRec64)));
  const int64_t nsort = p.sort_targets ? p.nt : 0;
  const int64_t nitem = p.sort_items ? p.max_items : 0;
  p.keys_a = a.take(sizeof(uint64_t) * (size_t)nsort);
  p.keys_b = a.take(sizeof(uint64_t) * (size_t)nsort);
  p.vals_a = a.take(sizeof(int32_t) * (size_t)nsort);
  p.vals_b = a.take(sizeof(int32_t) * (size_t)nsort);
  p.ikeys_a = a.take(sizeof(uint64_t) * (size_t)nitem);
  p.ikeys_b = a.take(sizeof(uint64_t) * (size_t)nitem);
  p.ivals_a = a.take(sizeof(int32_t) * (size_t)nitem);
  p.ivals_b = a.take(sizeof(int32_t) * (size_t)nitem);
  const size_t he = radix_hist_entries(nsort > nitem ? nsort : nitem);
  p.hist = a.take(sizeof(int32_t) * he);
  p.hist_scan = a.take(sizeof(int32_t) * (he + 1));
  p.bbox_part = a.take(sizeof(double) * 6 * 1024);
  p.bbox = a.take(sizeof(double) * 6);
  p.items = a.take(sizeof(Item) * (size_t)(p.max_items > 0 ? p.max_items : 1));
  p.range = a.take(sizeof(int64_t) * (size_t)(p.nseg_ranges + 1));
  p.cnt = a.take(sizeof(int32_t) * (size_t)(p.ngroup + 1));
  p.offs = a.take(sizeof(int32_t) * (size_t)(p.ngroup + 2));
  p.part = a.take(sizeof(double) * 3 * (size_t)p.nt * (size_t)p.nsplit);
  if (p.mixed) {
    const size_t mi = (size_t)(p.max_items > 0 ? p.max_items : 1);
    p.frames = a.take(sizeof(float) * 12 * mi);
    p.xloc = a.take(sizeof(float) * 3 * (size_t)(p.nt > 0 ? p.nt : 1));
    p.cand_list = a.take(sizeof(int32_t) * (size_t)kCandCap * mi);
    p.cand_cnt = a.take(sizeof(int32_t) * mi);
  }
  p.total = a.off + 256;  // slack for re-alignment of an unaligned base
}

stk_status plan_direct(int64_t ns, int64_t nt, const stk_opts *o, Plan &p) {
  DevInfo di;
  CU(dev_info(di));
  p.form = F_DIRECT;
  p.mixed = o->precision == STK_MIXED;
  p.tile = tile_config(o->tile_config < 0 ? 0 : o->tile_config);
  p.ns = ns;
  p.nt = nt;
  // small mixed sums with the default options: one launch and the finish
  if (p.mixed && o->source_splits == 0 && o->tile_config < 0 && ns > 0 && nt > 0 &&
      (double)ns * (double)nt <= (double)kSmallPairs) {
    p.small = true;
    p.nsplit = direct_small_splits(ns, nt, di.sms);
    layout(p);
    return STK_OK;
  }
  const int occ = p.mixed ? di.occ_mixed : di.occ_fp64;
  p.nsplit = o->source_splits > 0 ? o->source_splits : auto_splits(nt, ns, di, occ);
  if (p.nsplit > ns && ns > 0) p.nsplit = (int32_t)ns;
  if (p.nsplit < 1) p.nsplit = 1;
  p.max_items = ((nt + kMinItemMax - 1) / kMinItemMax) * p.nsplit;
  p.nseg_ranges = p.nsplit;
  p.sort_targets = p.mixed;
  p.sort_items = false;
  p.ngroup = 0;
  layout(p);
  return STK_OK;
}

stk_status plan_p2p(int64_t n, int32_t nleaf, const stk_opts *o, Plan &p) {
  p.form = F_P2P;
  p.mixed = o->precision == STK_MIXED;
  p.tile = tile_config(o->tile_config < 0 ? 0 : o->tile_config);
  p.ns = p.nt = n;
  p.nsplit = 1;
  p.max_items = (int64_t)nleaf + n / kMinItemMax + 1;
  p.nseg_ranges = nleaf;
  p.sort_targets = false;
  p.sort_items = true;
  p.ngroup = nleaf;
  layout(p);
  return STK_OK;
}

stk_status plan_batched(int64_t n, int32_t nsusp, const stk_opts *o, Plan &p) {
  p.form = F_BATCHED;
  p.mixed = o->precision == STK_MIXED;
  p.tile = tile_config(o->tile_config < 0 ? 0 : o->tile_config);
  p.ns = p.nt = n;
  p.nsplit = 1;
  p.max_items = (int64_t)nsusp + n / kMinItemMax + 1;
  p.nseg_ranges = 2 * nsusp;
  p.sort_targets = p.mixed;
  p.sort_items = true;
  p.ngroup = nsusp;
  layout(p);
  return STK_OK;
}

constexpr int64_t kMaxMixed = (int64_t)1 << 30;

stk_status check_opts(const stk_opts *o) {
  if (!o) return fail(STK_EINVAL, "opts is NULL");
  if (o->precision != STK_FP64 && o->precision != STK_MIXED)
    return fail(STK_EINVAL, "opts->precision must be STK_FP64 or STK_MIXED");
  if (!(o->near_ratio >= 0.0) || !std::isfinite(o->near_ratio))
    return fail(STK_EINVAL, "opts->near_ratio must be finite and >= 0");
  if (o->source_splits < 0 || o->source_splits > 1024)
    return fail(STK_EINVAL, "opts->source_splits must be in [0, 1024]");
  if (o->tile_config < -1 || o->tile_config >= kNumTileConfigs)
    return fail(STK_EINVAL, "opts->tile_config must be -1 or a configuration id");
  return STK_OK;
}

template <class T>
T *at(void *ws, size_t off) {
  return reinterpret_cast<T *>(reinterpret_cast<char *>(ws) + off);
}

void *align_ws(void *ws) {
  const uintptr_t u = reinterpret_cast<uintptr_t>(ws);
  return reinterpret_cast<void *>((u + 255) & ~(uintptr_t)255);
}

// A second stream per host thread and device, for the part of a call that can
// run beside the caller's stream: a fork event recorded on the caller's
// stream, the work on this stream, a join event the caller's stream waits on
// (graph capture follows the fork and the join).  The handles belong to one
// context and are made again in another; none is made while the caller's
// stream is being captured.
struct SideStream {
  unsigned long long ctx = 0;
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
constexpr int kSideDevices = 64;
thread_local SideStream t_side[kSideDevices];

SideStream *side_stream(bool create) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kSideDevices) {
    cudaGetLastError();
    return nullptr;
  }
  SideStream &sd = t_side[dev];
  const unsigned long long ctx = stk::context_id();
  if (ctx == 0) return nullptr;
  if (sd.s && sd.ctx == ctx) return &sd;
  if (!create) return nullptr;
  sd = SideStream{};  // handles of an earlier context went with it
  cudaStream_t st = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&a, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b, cudaEventDisableTiming) != cudaSuccess) {
    if (b) cudaEventDestroy(b);
    if (a) cudaEventDestroy(a);
    if (st) cudaStreamDestroy(st);
    cudaGetLastError();
    return nullptr;
  }
  sd.ctx = ctx;
  sd.s = st;
  sd.fork = a;
  sd.join = b;
  return &sd;
}

// Forks the side stream off st: returns it with its work ordered after st's
// work so far, or nullptr (the call then runs on st alone).
SideStream *fork_side(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  SideStream *sd = side_stream(cs == cudaStreamCaptureStatusNone);
  if (!sd) return nullptr;
  if (cudaEventRecord(sd->fork, st) != cudaSuccess ||
      cudaStreamWaitEvent(sd->s, sd->fork, 0) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return sd;
}

// Engine launch common to all forms.
// direct_out (optional): with one part and targets in caller order, the
// engines write the caller's output instead of the partial buffer (no finish).
stk_status run_engine(const Plan &p, void *ws, EngineParams &P, cudaStream_t st,
                      double *direct_out = nullptr) {
  DevInfo di;
  CU(dev_info(di));
  int32_t *counters = at<int32_t>(ws, p.counters);
  P.n_items = counters + 0;
  P.item_counter = counters + 1;
  P.err_flag = counters + 2;
  P.near_counter = counters + 3;
  P.spin_limit = g_wait_limit > 0 ? g_wait_limit : kSpinLimit;
  P.drain_limit = P.spin_limit > kSpinLimit ? P.spin_limit : kSpinLimit;
  P.force_expire = g_force_expire;
  P.policy = p.tile.policy;
  P.part_out = direct_out ? direct_out : at<double>(ws, p.part);
  P.nt = (int32_t)p.nt;
  const int occ = p.mixed ? di.occ_mixed : di.occ_fp64;
  int64_t grid = (int64_t)di.sms * occ;
  const int64_t need = (p.max_items + kWarpsPerCta - 1) / kWarpsPerCta;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  if (g_ev_start && g_ev_stop) CU(cudaEventRecord(g_ev_start, st));
  if (p.mixed) {
    P.rec = at<SrcRec>(ws, p.rec);
    P.frames = at<float>(ws, p.frames);
    P.xloc = at<float>(ws, p.xloc);
    P.cand_list = at<int32_t>(ws, p.cand_list);
    P.cand_cnt = at<int32_t>(ws, p.cand_cnt);
    P.cand_cap = kCandCap;
    CU(launch_engine_mixed(P, (int)grid, st));
  } else {
    P.rec64 = at<SrcRec64>(ws, p.rec);
    CU(launch_engine_fp64(P, (int)grid, st));
  }
  if (g_ev_start && g_ev_stop) CU(cudaEventRecord(g_ev_stop, st));
  if (p.mixed) {
    launch_near(P, di.sms, p.max_items, st);
    CU(cudaGetLastError());
  }
  return STK_OK;
}

stk_status pack(const Plan &p, void *ws, const double *src, const double *f, const double *nrm,
                const double *phi, const double *w, const double *h, double mu, double alpha,
                cudaStream_t st) {
  const double csl = 1.0 / (8.0 * kPi * mu), cdl = 6.0 / (8.0 * kPi);
  if (p.mixed)
    launch_pack_mixed(p.ns, src, f, nrm, phi, w, h, alpha, csl, cdl, src, at<SrcRec>(ws, p.rec),
                      st);
  else
    launch_pack_fp64(p.ns, src, f, nrm, phi, w, csl, cdl, at<SrcRec64>(ws, p.rec), st);
  CU(cudaGetLastError());
  return STK_OK;
}

// Morton sort of the targets; returns the sorted -> caller permutation.
const int32_t *sort_targets(const Plan &p, void *ws, const double *trg, const int64_t *group_ptr,
                            int32_t ngroup, cudaStream_t st) {
  launch_bbox(p.nt, trg, at<double>(ws, p.bbox_part), at<double>(ws, p.bbox), st);
  uint64_t *ka = at<uint64_t>(ws, p.keys_a), *kb = at<uint64_t>(ws, p.keys_b);
  int32_t *va = at<int32_t>(ws, p.vals_a), *vb = at<int32_t>(ws, p.vals_b);
  launch_morton(p.nt, trg, at<double>(ws, p.bbox), group_ptr, ngroup, ka, va, st);
  int bits = 30;
  if (group_ptr) {
    int gb = 0;
    while ((1LL << gb) < ngroup) ++gb;
    bits += gb;
  }
  const int which = radix_sort(ka, va, kb, vb, p.nt, bits, at<int32_t>(ws, p.hist),
                               at<int32_t>(ws, p.hist_scan), st);
  return which ? vb : va;
}

// Builds items with cost keys through `emit` and returns the processing order
// (descending cost).  The item count is only known on the device, so the sort
// runs over the upper bound; unused key slots hold the maximum key and sort last.
template <class Emit>
const int32_t *build_sorted_items(const Plan &p, void *ws, cudaStream_t st, Emit emit) {
  uint64_t *ka = at<uint64_t>(ws, p.ikeys_a), *kb = at<uint64_t>(ws, p.ikeys_b);
  int32_t *va = at<int32_t>(ws, p.ivals_a), *vb = at<int32_t>(ws, p.ivals_b);
  cudaMemsetAsync(ka, 0xff, sizeof(uint64_t) * (size_t)p.max_items, st);
  cudaMemsetAsync(va, 0xff, sizeof(int32_t) * (size_t)p.max_items, st);
  emit(ka, va);
  // rank per item in the first half of kb's storage, order in vb
  launch_bucket_order(p.max_items, ka, va, at<int32_t>(ws, p.hist), at<int32_t>(ws, p.hist_scan),
                      reinterpret_cast<int32_t *>(kb), vb, st);
  return vb;
}

stk_status direct_common(int32_t kinds, const double *src, const double *f, const double *nrm,
                         const double *phi, const double *w, const double *h, int64_t ns,
                         const double *trg, int64_t nt, double mu, double *out, const stk_opts *o,
                         void *workspace, size_t wbytes, void *stream) {
  stk_status s = check_opts(o);
  if (s != STK_OK) return s;
  if (ns < 0 || nt < 0 || ns > kMaxN || nt > kMaxN)
    return fail(STK_EINVAL, "ns and nt must be in [0, 2^31-1]");
  if (o->precision == STK_MIXED && ns >= kMaxMixed)
    return fail(STK_EUNSUPPORTED, "the mixed form supports fewer than 2^30 sources");
  if (nt > 0 && (!trg || !out)) return fail(STK_EINVAL, "trg/out is NULL");
  if (ns > 0 && nt > 0) {
    if (!src || !w) return fail(STK_EINVAL, "src/w is NULL");
    if ((kinds & K_SL) && !f) return fail(STK_EINVAL, "f is NULL");
    if ((kinds & K_DL) && (!nrm || !phi)) return fail(STK_EINVAL, "nrm/phi is NULL");
    if ((kinds & K_SL) && !(mu > 0.0 && std::isfinite(mu)))
      return fail(STK_EINVAL, "mu must be finite and > 0");
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (nt == 0) return STK_OK;
  if (ns == 0) {
    if (!o->accumulate) CU(cudaMemsetAsync(out, 0, sizeof(double) * 3 * (size_t)nt, st));
    return STK_OK;
  }
  Plan p;
  s = plan_direct(ns, nt, o, p);
  if (s != STK_OK) return s;
  if (!workspace || wbytes < p.total) return fail(STK_ENOMEM, "workspace too small");
  void *ws = align_ws(workspace);
  if (p.small) {
    CU(cudaMemsetAsync(at<int32_t>(ws, p.counters), 0, sizeof(int32_t) * 4, st));
    CU(cudaMemsetAsync(at<int32_t>(ws, p.cnt), 0,
                       sizeof(int32_t) * (size_t)direct_small_blocks(nt), st));
    const double csl = (kinds & K_SL) ? 1.0 / (8.0 * kPi * mu) : 0.0, cdl = 6.0 / (8.0 * kPi);
    CU(launch_direct_small(kinds, src, (kinds & K_SL) ? f : nullptr, nrm,
                           (kinds & K_DL) ? phi : nullptr, w, h, ns, trg, nt, o->near_ratio, csl,
                           cdl, p.nsplit, o->accumulate ? 1 : 0, at<double>(ws, p.part),
                           at<int32_t>(ws, p.cnt), out, st));
    return STK_OK;
  }
  launch_zero_ints(at<int32_t>(ws, p.counters), 4, st);
  s = pack(p, ws, src, (kinds & K_SL) ? f : nullptr, nrm, (kinds & K_DL) ? phi : nullptr, w, h,
           (kinds & K_SL) ? mu : 1.0, o->near_ratio, st);
  if (s != STK_OK) return s;
  EngineParams P;
  std::memset(&P, 0, sizeof(P));
  P.src64 = src;
  P.trg64 = trg;
  P.self_index = (trg == src) ? 1 : 0;
  P.tperm = p.sort_targets ? sort_targets(p, ws, trg, nullptr, 0, st) : nullptr;
  launch_items_direct((int32_t)nt, ns, p.nsplit, p.tile.item_max, at<Item>(ws, p.items),
                      at<int64_t>(ws, p.range), at<int32_t>(ws, p.counters), st);
  CU(cudaGetLastError());
  P.items = at<Item>(ws, p.items);
  P.item_order = nullptr;
  P.seg_list = nullptr;
  P.range_ptr = at<int64_t>(ws, p.range);
  P.kind = kinds;
  P.kind_alternating = 0;
  s = run_engine(p, ws, P, st);
  if (s != STK_OK) return s;
  launch_finish(nt, p.nsplit, at<double>(ws, p.part), P.tperm, o->accumulate, out, st);
  CU(cudaGetLastError());
  return STK_OK;
}


// ------------------------------------------------------------------ adjoint
struct GradPlan {
  bool mixed;
  int64_t ns, nt;
  int32_t nsplit_src, nsplit_trg;
  size_t srec, trec, ska, skb, sva, svb, tka, tkb, tva, tvb, hist, hist_scan, bbox_part, bbox,
      part_src, part_trg, counters, near_cnt = 0, near_idx = 0, oframe = 0, total;
};

int32_t adj_splits(int64_t nout, int64_t nin, const DevInfo &di) {
  const int64_t tiles = (nout + 127) / 128;
  if (tiles <= 0) return 1;
  int64_t s = ((int64_t)di.sms * 8 + tiles - 1) / tiles;
  const int64_t cap = nin / 256 > 1 ? nin / 256 : 1;
  if (s > cap) s = cap;
  if (s > 64) s = 64;
  return (int32_t)(s < 1 ? 1 : s);
}

stk_status plan_grad(int64_t ns, int64_t nt, const stk_opts *o, GradPlan &p) {
  DevInfo di;
  CU(dev_info(di));
  p.mixed = o->precision == STK_MIXED;
  p.ns = ns;
  p.nt = nt;
  p.nsplit_src = adj_splits(ns, nt, di);
  p.nsplit_trg = adj_splits(nt, ns, di);
  Alloc a;
  p.counters = a.take(sizeof(int32_t) * 4);
  const size_t rb = p.mixed ? sizeof(SrcRec) : sizeof(SrcRec64);
  p.srec = a.take(rb * (size_t)ns);
  p.trec = a.take(rb * (size_t)nt);
  p.ska = a.take(8 * (size_t)ns);
  p.skb = a.take(8 * (size_t)ns);
  p.sva = a.take(4 * (size_t)ns);
  p.svb = a.take(4 * (size_t)ns);
  p.tka = a.take(8 * (size_t)nt);
  p.tkb = a.take(8 * (size_t)nt);
  p.tva = a.take(4 * (size_t)nt);
  p.tvb = a.take(4 * (size_t)nt);
  const size_t he = radix_hist_entries(ns > nt ? ns : nt);
  p.hist = a.take(4 * he);
  p.hist_scan = a.take(4 * (he + 1));
  p.bbox_part = a.take(sizeof(double) * 6 * 1024);
  p.bbox = a.take(sizeof(double) * 6);
  p.part_src = a.take(sizeof(double) * 12 * (size_t)ns * (size_t)p.nsplit_src);
  p.part_trg = a.take(sizeof(double) * 3 * (size_t)nt * (size_t)p.nsplit_trg);
  if (p.mixed) {  // near-pair lists of one pass at a time (the larger point set)
    const size_t nmax = (size_t)(ns > nt ? ns : nt);
    p.near_cnt = a.take(sizeof(int32_t) * nmax);
    p.near_idx = a.take(sizeof(int32_t) * nmax * (size_t)kAdjNearCap);
    p.oframe = a.take(sizeof(float) * 9 * nmax);
  }
  p.total = a.off + 256;
  return STK_OK;
}

// Morton order of n points (permutation sorted -> caller index).
const int32_t *morton_perm(int64_t n, const double *pts, void *ws, size_t ka, size_t kb,
                           size_t va, size_t vb, size_t hist, size_t hist_scan, size_t bpart,
                           size_t bbox, cudaStream_t st) {
  launch_bbox(n, pts, at<double>(ws, bpart), at<double>(ws, bbox), st);
  uint64_t *k0 = at<uint64_t>(ws, ka), *k1 = at<uint64_t>(ws, kb);
  int32_t *v0 = at<int32_t>(ws, va), *v1 = at<int32_t>(ws, vb);
  launch_morton(n, pts, at<double>(ws, bbox), nullptr, 0, k0, v0, st);
  const int which = radix_sort(k0, v0, k1, v1, n, 30, at<int32_t>(ws, hist),
                               at<int32_t>(ws, hist_scan), st);
  return which ? v1 : v0;
}
}  // namespace

namespace stk {
// Records `msg` as the calling thread's last error and returns `s` (used by
// the other translation units of the library).
stk_status report_error(stk_status s, const char *msg) { return fail(s, msg); }
// noalloc.cu: the fixed buffer of stokes_sl_eval_noalloc in the current context.
stk_status noalloc_scratch(void **addr, size_t *bytes);
}  // namespace stk

extern "C" {

void stokes_default_opts(stk_opts *o) {
  if (!o) return;
  o->precision = STK_MIXED;
  o->near_ratio = 1.0;
  o->accumulate = 0;
  o->source_splits = 0;
  o->tile_config = -1;
}

const char *stokes_last_error(void) { return g_err.c_str(); }

stk_status stokes_set_engine_events(void *start_event, void *stop_event) {
  g_ev_start = reinterpret_cast<cudaEvent_t>(start_event);
  g_ev_stop = reinterpret_cast<cudaEvent_t>(stop_event);
  return STK_OK;
}

int64_t stokes_launch_count(void) { return stk::launch_count(); }

stk_status stokes_set_wait_policy(int64_t limit_cycles, int32_t force_expire) {
  if (limit_cycles < 0) return fail(STK_EINVAL, "limit_cycles must be >= 0");
  if (force_expire != 0 && force_expire != 1) return fail(STK_EINVAL, "force_expire must be 0 or 1");
  g_wait_limit = limit_cycles;
  g_force_expire = force_expire;
  return STK_OK;
}

const char *stokes_version(void) { return "stokesgpu 0.1 (sm_103a)"; }

stk_status stokes_direct_workspace_size(int64_t ns, int64_t nt, int32_t kernels,
                                        const stk_opts *opts, size_t *bytes) {
  stk_status s = check_opts(opts);
  if (s != STK_OK) return s;
  if (!bytes) return fail(STK_EINVAL, "bytes is NULL");
  if (ns < 0 || nt < 0 || ns > kMaxN || nt > kMaxN) return fail(STK_EINVAL, "bad sizes");
  if (kernels < 1 || kernels > 3) return fail(STK_EINVAL, "kernels must be 1, 2 or 3");
  Plan p;
  s = plan_direct(ns, nt, opts, p);
  if (s != STK_OK) return s;
  *bytes = p.total;
  return STK_OK;
}

stk_status stokes_sl_eval(const double *src, const double *f, const double *w, const double *h,
                          int64_t ns, const double *trg, int64_t nt, double mu, double *out,
                          const stk_opts *opts, void *workspace, size_t workspace_bytes,
                          void *stream) {
  return direct_common(K_SL, src, f, nullptr, nullptr, w, h, ns, trg, nt, mu, out, opts, workspace,
                       workspace_bytes, stream);
}

stk_status stokes_dl_eval(const double *src, const double *nrm, const double *phi,
                          const double *w, const double *h, int64_t ns, const double *trg,
                          int64_t nt, double *out, const stk_opts *opts, void *workspace,
                          size_t workspace_bytes, void *stream) {
  return direct_common(K_DL, src, nullptr, nrm, phi, w, h, ns, trg, nt, 1.0, out, opts, workspace,
                       workspace_bytes, stream);
}

stk_status stokes_sldl_eval(const double *src, const double *f, const double *nrm,
                            const double *phi, const double *w, const double *h, int64_t ns,
                            const double *trg, int64_t nt, double mu, double *out,
                            const stk_opts *opts, void *workspace, size_t workspace_bytes,
                            void *stream) {
  return direct_common(K_SLDL, src, f, nrm, phi, w, h, ns, trg, nt, mu, out, opts, workspace,
                       workspace_bytes, stream);
}

stk_status stokes_p2p_workspace_size(int64_t n, int32_t nleaf, int32_t kernels,
                                     const stk_opts *opts, size_t *bytes) {
  stk_status s = check_opts(opts);
  if (s != STK_OK) return s;
  if (!bytes) return fail(STK_EINVAL, "bytes is NULL");
  if (n < 0 || n > kMaxN || nleaf < 0) return fail(STK_EINVAL, "bad sizes");
  if (kernels < 1 || kernels > 3) return fail(STK_EINVAL, "kernels must be 1, 2 or 3");
  Plan p;
  s = plan_p2p(n, nleaf, opts, p);
  if (s != STK_OK) return s;
  *bytes = p.total;
  return STK_OK;
}

stk_status stokes_p2p_leaflists(const double *pts, const double *f, const double *phi,
                                const double *nrm, const double *w, const double *h, int64_t n,
                                const int32_t *leaf_ptr, int32_t nleaf, const int32_t *ulist_ptr,
                                const int32_t *ulist_idx, int64_t nulist, int32_t kernels,
                                double mu, double *out, const stk_opts *opts, void *workspace,
                                size_t workspace_bytes, void *stream) {
  stk_status s = check_opts(opts);
  if (s != STK_OK) return s;
  if (n < 0 || n > kMaxN || nleaf < 0 || nulist < 0 || nulist > kMaxN)
    return fail(STK_EINVAL, "bad sizes");
  if (opts->precision == STK_MIXED && n >= kMaxMixed)
    return fail(STK_EUNSUPPORTED, "the mixed form supports fewer than 2^30 points");
  if (kernels < 1 || kernels > 3) return fail(STK_EINVAL, "kernels must be 1, 2 or 3");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (n == 0) return STK_OK;
  if (nleaf == 0) return fail(STK_EINVAL, "points without leaves");
  if (!pts || !w || !out || !leaf_ptr || !ulist_ptr || (nulist > 0 && !ulist_idx))
    return fail(STK_EINVAL, "NULL pointer");
  if ((kernels & K_SL) && !f) return fail(STK_EINVAL, "f is NULL");
  if ((kernels & K_DL) && (!nrm || !phi)) return fail(STK_EINVAL, "nrm/phi is NULL");
  if ((kernels & K_SL) && !(mu > 0.0 && std::isfinite(mu)))
    return fail(STK_EINVAL, "mu must be finite and > 0");
  Plan p;
  s = plan_p2p(n, nleaf, opts, p);
  if (s != STK_OK) return s;
  if (!workspace || workspace_bytes < p.total) return fail(STK_ENOMEM, "workspace too small");
  void *ws = align_ws(workspace);
  launch_zero_ints(at<int32_t>(ws, p.counters), 4, st);
  // the packing runs beside the item build (they meet at the engine)
  SideStream *sd = fork_side(st);
  s = pack(p, ws, pts, (kernels & K_SL) ? f : nullptr, nrm, (kernels & K_DL) ? phi : nullptr, w,
           h, (kernels & K_SL) ? mu : 1.0, opts->near_ratio, sd ? sd->s : st);
  if (s != STK_OK) return s;
  if (sd) CU(cudaEventRecord(sd->join, sd->s));
  int64_t *range = at<int64_t>(ws, p.range);
  launch_widen((int64_t)nleaf + 1, leaf_ptr, range, st);
  int32_t *counters = at<int32_t>(ws, p.counters);
  const int32_t *order = build_sorted_items(p, ws, st, [&](uint64_t *keys, int32_t *vals) {
    launch_p2p_items(nleaf, leaf_ptr, ulist_ptr, ulist_idx, p.tile.item_max, at<int32_t>(ws, p.cnt),
                     at<int32_t>(ws, p.offs), counters, at<Item>(ws, p.items), keys, vals, st);
  });
  CU(cudaGetLastError());
  if (sd) CU(cudaStreamWaitEvent(st, sd->join, 0));
  EngineParams P;
  std::memset(&P, 0, sizeof(P));
  P.src64 = pts;
  P.trg64 = pts;
  P.self_index = 1;
  P.tperm = nullptr;
  P.items = at<Item>(ws, p.items);
  P.item_order = order;
  P.seg_list = ulist_idx;
  P.range_ptr = range;
  P.kind = kernels;
  P.kind_alternating = 0;
  // points are targets in caller order and there is one part: without
  // accumulation the engines write out directly
  const bool direct = !opts->accumulate;
  s = run_engine(p, ws, P, st, direct ? out : nullptr);
  if (s != STK_OK) return s;
  if (!direct) launch_finish(n, 1, at<double>(ws, p.part), nullptr, opts->accumulate, out, st);
  CU(cudaGetLastError());
  return STK_OK;
}

stk_status stokes_batched_workspace_size(int64_t n, int32_t nsusp, const stk_opts *opts,
                                         size_t *bytes) {
  stk_status s = check_opts(opts);
  if (s != STK_OK) return s;
  if (!bytes) return fail(STK_EINVAL, "bytes is NULL");
  if (n < 0 || n > kMaxN || nsusp < 0 || nsusp > (1 << 24)) return fail(STK_EINVAL, "bad sizes");
  Plan p;
  s = plan_batched(n, nsusp, opts, p);
  if (s != STK_OK) return s;
  *bytes = p.total;
  return STK_OK;
}

stk_status stokes_batched_eval(const double *pts, const double *f, const double *phi,
                               const double *nrm, const double *w, const double *h, int64_t n,
                               const int64_t *susp_ptr, const int64_t *n_cell, int32_t nsusp,
                               double mu, double *out, const stk_opts *opts, void *workspace,
                               size_t workspace_bytes, void *stream) {
  stk_status s = check_opts(opts);
  if (s != STK_OK) return s;
  if (n < 0 || n > kMaxN || nsusp < 0 || nsusp > (1 << 24)) return fail(STK_EINVAL, "bad sizes");
  if (opts->precision == STK_MIXED && n >= kMaxMixed)
    return fail(STK_EUNSUPPORTED, "the mixed form supports fewer than 2^30 points");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (n == 0 || nsusp == 0) return STK_OK;
  if (!pts || !f || !phi || !nrm || !w || !out || !susp_ptr || !n_cell)
    return fail(STK_EINVAL, "NULL pointer");
  if (!(mu > 0.0 && std::isfinite(mu))) return fail(STK_EINVAL, "mu must be finite and > 0");
  Plan p;
  s = plan_batched(n, nsusp, opts, p);
  if (s != STK_OK) return s;
  if (!workspace || workspace_bytes < p.total) return fail(STK_ENOMEM, "workspace too small");
  void *ws = align_ws(workspace);
  launch_zero_ints(at<int32_t>(ws, p.counters), 4, st);
  s = pack(p, ws, pts, f, nrm, phi, w, h, mu, opts->near_ratio, st);
  if (s != STK_OK) return s;
  EngineParams P;
  std::memset(&P, 0, sizeof(P));
  P.src64 = pts;
  P.trg64 = pts;
  P.self_index = 1;
  P.tperm = p.sort_targets ? sort_targets(p, ws, pts, susp_ptr, nsusp, st) : nullptr;
  int32_t *counters = at<int32_t>(ws, p.counters);
  const int32_t *order = build_sorted_items(p, ws, st, [&](uint64_t *keys, int32_t *vals) {
    launch_batched_items(nsusp, susp_ptr, n_cell, p.tile.item_max, at<int32_t>(ws, p.cnt),
                         at<int32_t>(ws, p.offs),
                         counters, at<Item>(ws, p.items), at<int64_t>(ws, p.range), keys, vals,
                         st);
  });
  CU(cudaGetLastError());
  P.items = at<Item>(ws, p.items);
  P.item_order = order;
  P.seg_list = nullptr;
  P.range_ptr = at<int64_t>(ws, p.range);
  P.kind = K_SLDL;
  P.kind_alternating = 1;
  s = run_engine(p, ws, P, st);
  if (s != STK_OK) return s;
  launch_finish(n, 1, at<double>(ws, p.part), P.tperm, opts->accumulate, out, st);
  CU(cudaGetLastError());
  return STK_OK;
}


stk_status stokes_grad_workspace_size(int64_t ns, int64_t nt, const stk_opts *opts,
                                      size_t *bytes) {
  stk_status s = check_opts(opts);
  if (s != STK_OK) return s;
  if (!bytes) return fail(STK_EINVAL, "bytes is NULL");
  if (ns < 0 || nt < 0 || ns > kMaxN || nt > kMaxN) return fail(STK_EINVAL, "bad sizes");
  GradPlan p;
  s = plan_grad(ns, nt, opts, p);
  if (s != STK_OK) return s;
  *bytes = p.total;
  return STK_OK;
}

stk_status stokes_sldl_grad(const double *src, const double *f, const double *nrm,
                            const double *phi, const double *w, const double *h, int64_t ns,
                            const double *trg, int64_t nt, const double *g, double mu,
                            double *grad_f, double *grad_phi, double *grad_y, double *grad_n,
                            double *grad_x, const stk_opts *opts, void *workspace,
                            size_t workspace_bytes, void *stream) {
  stk_status s = check_opts(opts);
  if (s != STK_OK) return s;
  if (ns < 0 || nt < 0 || ns > kMaxN || nt > kMaxN) return fail(STK_EINVAL, "bad sizes");
  if (!f && !phi) return fail(STK_EINVAL, "f and phi are both NULL");
  if (f && !(mu > 0.0 && std::isfinite(mu))) return fail(STK_EINVAL, "mu must be finite and > 0");
  if (phi && !nrm) return fail(STK_EINVAL, "nrm is NULL");
  if (grad_f && !f) return fail(STK_EINVAL, "grad_f requested without f");
  if ((grad_phi || grad_n) && !phi) return fail(STK_EINVAL, "grad_phi/grad_n requested without phi");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const bool want_src = grad_f || grad_phi || grad_y || grad_n;
  if (ns == 0 || nt == 0 || (!want_src && !grad_x)) {
    if (ns > 0 && want_src) {
      if (grad_f) CU(cudaMemsetAsync(grad_f, 0, 24 * (size_t)ns, st));
      if (grad_phi) CU(cudaMemsetAsync(grad_phi, 0, 24 * (size_t)ns, st));
      if (grad_y) CU(cudaMemsetAsync(grad_y, 0, 24 * (size_t)ns, st));
      if (grad_n) CU(cudaMemsetAsync(grad_n, 0, 24 * (size_t)ns, st));
    }
    if (nt > 0 && grad_x) CU(cudaMemsetAsync(grad_x, 0, 24 * (size_t)nt, st));
    return STK_OK;
  }
  if (!src || !w || !trg || !g) return fail(STK_EINVAL, "NULL pointer");
  if (opts->precision == STK_MIXED && (ns >= kMaxMixed || nt >= kMaxMixed))
    return fail(STK_EUNSUPPORTED, "the mixed form supports fewer than 2^30 points");
  GradPlan p;
  s = plan_grad(ns, nt, opts, p);
  if (s != STK_OK) return s;
  if (!workspace || workspace_bytes < p.total) return fail(STK_ENOMEM, "workspace too small");
  void *ws = align_ws(workspace);
  const double csl = f ? 1.0 / (8.0 * kPi * mu) : 0.0, cdl = 6.0 / (8.0 * kPi);
  if (p.mixed) {
    launch_pack_mixed(ns, src, f, nrm, phi, w, h, opts->near_ratio, csl, cdl, src,
                      at<SrcRec>(ws, p.srec), st);
    launch_pack_mixed(nt, trg, g, nullptr, nullptr, nullptr, nullptr, 0.0, 1.0, 0.0, src,
                      at<SrcRec>(ws, p.trec), st);
  } else {
    launch_pack_fp64(ns, src, f, nrm, phi, w, csl, cdl, at<SrcRec64>(ws, p.srec), st);
    launch_pack_fp64(nt, trg, g, nullptr, nullptr, nullptr, 1.0, 0.0, at<SrcRec64>(ws, p.trec),
                     st);
  }
  CU(cudaGetLastError());
  const int32_t *sperm = morton_perm(ns, src, ws, p.ska, p.skb, p.sva, p.svb, p.hist, p.hist_scan,
                                     p.bbox_part, p.bbox, st);
  const int32_t *tperm = morton_perm(nt, trg, ws, p.tka, p.tkb, p.tva, p.tvb, p.hist, p.hist_scan,
                                     p.bbox_part, p.bbox, st);
  CU(cudaGetLastError());
  AdjParams A;
  A.near_cnt = p.mixed ? at<int32_t>(ws, p.near_cnt) : nullptr;
  A.near_idx = p.mixed ? at<int32_t>(ws, p.near_idx) : nullptr;
  A.near_cap = kAdjNearCap;
  A.oframe = p.mixed ? at<float>(ws, p.oframe) : nullptr;
  A.has_sl = f ? 1 : 0;
  A.has_dl = phi ? 1 : 0;
  if (want_src) {
    A.out_rec = at<void>(ws, p.srec);
    A.in_rec = at<void>(ws, p.trec);
    A.operm = sperm;
    A.iperm = tperm;
    A.nout = ns;
    A.nin = nt;
    A.nsplit = p.nsplit_src;
    A.out64 = src;
    A.in64 = trg;
    A.partial = at<double>(ws, p.part_src);
    if (g_ev_start && g_ev_stop) CU(cudaEventRecord(g_ev_start, st));
    CU(launch_adjoint(p.mixed, true, A, st));
    launch_adj_finish(true, ns, p.nsplit_src, A.partial, w, csl, cdl, grad_f, grad_phi, grad_n,
                      grad_y, nullptr, st);
  }
  if (grad_x) {
    A.out_rec = at<void>(ws, p.trec);
    A.in_rec = at<void>(ws, p.srec);
    A.operm = tperm;
    A.iperm = sperm;
    A.nout = nt;
    A.nin = ns;
    A.nsplit = p.nsplit_trg;
    A.out64 = trg;
    A.in64 = src;
    A.partial = at<double>(ws, p.part_trg);
    CU(launch_adjoint(p.mixed, false, A, st));
    if (g_ev_start && g_ev_stop) CU(cudaEventRecord(g_ev_stop, st));
    launch_adj_finish(false, nt, p.nsplit_trg, A.partial, nullptr, 0.0, 0.0, nullptr, nullptr,
                      nullptr, nullptr, grad_x, st);
  } else if (g_ev_start && g_ev_stop) {
    CU(cudaEventRecord(g_ev_stop, st));
  }
  CU(cudaGetLastError());
  return STK_OK;
}

stk_status stokes_device_status(void *workspace, size_t workspace_bytes) {
  if (!workspace) {  // the fixed buffer of stokes_sl_eval_noalloc in the current context
    const stk_status s = stk::noalloc_scratch(&workspace, &workspace_bytes);
    if (s != STK_OK) return s;
  }
  if (workspace_bytes < 512) return fail(STK_EINVAL, "workspace is too small");
  int32_t *counters = at<int32_t>(align_ws(workspace), 0);
  int32_t err = 0;
  CU(cudaMemcpy(&err, counters + 2, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (err != 0) {
    const int32_t zero = 0;
    CU(cudaMemcpy(counters + 2, &zero, sizeof(int32_t), cudaMemcpyHostToDevice));
    if (err == 6)
      return fail(STK_EINVAL, "an index read from the tree arrays on the device was out of range; "
                              "results of that call are incomplete");
    return fail(STK_ETIMEOUT, "a bounded device wait ran out; results of that call are incomplete");
  }
  return STK_OK;
}

}  // extern "C"

// ------------------------------------------------------------- autotuning
namespace {
// Times `call` on the caller's data for every tile configuration (one
// warm-up and three timed calls each, median) and returns the fastest.
template <class Call>
stk_status tune_configs(cudaStream_t st, Call call, int32_t *best, float *best_ms) {
  if (!best) return fail(STK_EINVAL, "best is NULL");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CU(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(STK_ECUDA, "cudaEventCreate failed");
  }
  const cudaEvent_t save0 = g_ev_start, save1 = g_ev_stop;
  g_ev_start = g_ev_stop = nullptr;
  stk_status s = STK_OK;
  float bestv = 3.0e38f;
  int32_t bestc = 0;
  for (int32_t c = 0; c < kNumTileConfigs && s == STK_OK; ++c) {
    s = call(c);
    float t[3];
    for (int r = 0; r < 3 && s == STK_OK; ++r) {
      if (cudaEventRecord(e0, st) != cudaSuccess) {
        s = fail(STK_ECUDA, "cudaEventRecord failed");
        break;
      }
      s = call(c);
      if (s == STK_OK &&
          (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
           cudaEventElapsedTime(&t[r], e0, e1) != cudaSuccess))
        s = fail(STK_ECUDA, "tuning run failed");
    }
    if (s != STK_OK) break;
    const float med = fmaxf(fminf(t[0], t[1]), fminf(fmaxf(t[0], t[1]), t[2]));
    if (med < bestv) {
      bestv = med;
      bestc = c;
    }
  }
  g_ev_start = save0;
  g_ev_stop = save1;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != STK_OK) return s;
  *best = bestc;
  if (best_ms) *best_ms = bestv;
  return STK_OK;
}

// Captures one call into an executable CUDA graph.  Kernels recorded during
// the capture do not run, so they leave the launch count as it was and are
// counted at each replay instead.
template <class Call>
stk_status capture_graph(cudaStream_t st, Call call, void **graph_exec) {
  if (!graph_exec) return fail(STK_EINVAL, "graph_exec is NULL");
  if (!st) return fail(STK_EINVAL, "capture needs a stream other than the legacy default stream");
  DevInfo di;
  CU(dev_info(di));  // one-time per-device set-up stays outside the capture
  side_stream(true);
  const cudaEvent_t save0 = g_ev_start, save1 = g_ev_stop;
  g_ev_start = g_ev_stop = nullptr;
  CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  const int64_t c0 = launch_count();
  const stk_status s = call();
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &graph);
  const int64_t recorded = launch_count() - c0;
  count_launches(-(int)recorded);
  g_ev_start = save0;
  g_ev_stop = save1;
  if (s != STK_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess || !graph) return fail(STK_ECUDA, "stream capture failed");
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) return fail(STK_ECUDA, "cudaGraphInstantiate failed");
  *graph_exec = reinterpret_cast<void *>(exec);
  std::lock_guard<std::mutex> lock(g_graph_mu);
  g_graph_kernels[*graph_exec] = recorded;
  return STK_OK;
}
}  // namespace

extern "C" {

int32_t stokes_tile_config_count(void) { return kNumTileConfigs; }

stk_status stokes_autotune_p2p(const double *pts, const double *f, const double *phi,
                               const double *nrm, const double *w, const double *h, int64_t n,
                               const int32_t *leaf_ptr, int32_t nleaf, const int32_t *ulist_ptr,
                               const int32_t *ulist_idx, int64_t nulist, int32_t kernels,
                               double mu, double *out, const stk_opts *opts, void *workspace,
                               size_t workspace_bytes, void *stream, int32_t *best_config,
                               float *best_ms) {
  stk_status s = check_opts(opts);
  if (s != STK_OK) return s;
  stk_opts o = *opts;
  o.accumulate = 0;
  return tune_configs(reinterpret_cast<cudaStream_t>(stream), [&](int32_t c) {
    o.tile_config = c;
    return stokes_p2p_leaflists(pts, f, phi, nrm, w, h, n, leaf_ptr, nleaf, ulist_ptr, ulist_idx,
                                nulist, kernels, mu, out, &o, workspace, workspace_bytes, stream);
  }, best_config, best_ms);
}

stk_status stokes_autotune_batched(const double *pts, const double *f, const double *phi,
                                   const double *nrm, const double *w, const double *h, int64_t n,
                                   const int64_t *susp_ptr, const int64_t *n_cell, int32_t nsusp,
                                   double mu, double *out, const stk_opts *opts, void *workspace,
                                   size_t workspace_bytes, void *stream, int32_t *best_config,
                                   float *best_ms) {
  stk_status s = check_opts(opts);
  if (s != STK_OK) return s;
  stk_opts o = *opts;
  o.accumulate = 0;
  return tune_configs(reinterpret_cast<cudaStream_t>(stream), [&](int32_t c) {
    o.tile_config = c;
    return stokes_batched_eval(pts, f, phi, nrm, w, h, n, susp_ptr, n_cell, nsusp, mu, out, &o,
                               workspace, workspace_bytes, stream);
  }, best_config, best_ms);
}

stk_status stokes_p2p_graph_create(const double *pts, const double *f, const double *phi,
                                   const double *nrm, const double *w, const double *h, int64_t n,
                                   const int32_t *leaf_ptr, int32_t nleaf,
                                   const int32_t *ulist_ptr, const int32_t *ulist_idx,
                                   int64_t nulist, int32_t kernels, double mu, double *out,
                                   const stk_opts *opts, void *workspace, size_t workspace_bytes,
                                   void *stream, void **graph_exec) {
  return capture_graph(reinterpret_cast<cudaStream_t>(stream), [&]() {
    return stokes_p2p_leaflists(pts, f, phi, nrm, w, h, n, leaf_ptr, nleaf, ulist_ptr, ulist_idx,
                                nulist, kernels, mu, out, opts, workspace, workspace_bytes,
                                stream);
  }, graph_exec);
}

stk_status stokes_batched_graph_create(const double *pts, const double *f, const double *phi,
                                       const double *nrm, const double *w, const double *h,
                                       int64_t n, const int64_t *susp_ptr, const int64_t *n_cell,
                                       int32_t nsusp, double mu, double *out,
                                       const stk_opts *opts, void *workspace,
                                       size_t workspace_bytes, void *stream, void **graph_exec) {
  return capture_graph(reinterpret_cast<cudaStream_t>(stream), [&]() {
    return stokes_batched_eval(pts, f, phi, nrm, w, h, n, susp_ptr, n_cell, nsusp, mu, out, opts,
                               workspace, workspace_bytes, stream);
  }, graph_exec);
}

stk_status stokes_direct_graph_create(int32_t kernels, const double *src, const double *f,
                                      const double *nrm, const double *phi, const double *w,
                                      const double *h, int64_t ns, const double *trg, int64_t nt,
                                      double mu, double *out, const stk_opts *opts,
                                      void *workspace, size_t workspace_bytes, void *stream,
                                      void **graph_exec) {
  if (kernels < 1 || kernels > 3) return fail(STK_EINVAL, "kernels must be 1, 2 or 3");
  return capture_graph(reinterpret_cast<cudaStream_t>(stream), [&]() {
    return direct_common(kernels, src, f, nrm, phi, w, h, ns, trg, nt, kernels & K_SL ? mu : 1.0,
                         out, opts, workspace, workspace_bytes, stream);
  }, graph_exec);
}

stk_status stokes_graph_launch(void *graph_exec, void *stream) {
  if (!graph_exec) return fail(STK_EINVAL, "graph_exec is NULL");
  CU(cudaGraphLaunch(reinterpret_cast<cudaGraphExec_t>(graph_exec),
                     reinterpret_cast<cudaStream_t>(stream)));
  int64_t k = 0;
  {
    std::lock_guard<std::mutex> lock(g_graph_mu);
    const auto it = g_graph_kernels.find(graph_exec);
    if (it != g_graph_kernels.end()) k = it->second;
  }
  count_launches((int)k);
  return STK_OK;
}

stk_status stokes_graph_destroy(void *graph_exec) {
  if (!graph_exec) return STK_OK;
  {
    std::lock_guard<std::mutex> lock(g_graph_mu);
    g_graph_kernels.erase(graph_exec);
  }
  CU(cudaGraphExecDestroy(reinterpret_cast<cudaGraphExec_t>(graph_exec)));
  return STK_OK;
}

}  // extern "C"
