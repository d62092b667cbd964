// engine_mixed.cu -- mixed FP32/FP64 evaluation of the Stokes single- and
// double-layer sums (Eq. "sl_stokes" and the double-layer kernel of Sec. 2.1,
// summed as in Sec. 3.1, Eq. "smooth_double_layer_int_eq_patches_disc").
//
// Design (GB300, sm_103a):
//  * Work unit = one warp-item: up to 128 spatially sorted targets held in
//    registers (T = 1..4 per lane) against a list of source segments.  Four
//    independent warps per CTA; a persistent grid pulls items from an atomic
//    queue in cost order, so uneven items balance without output atomics.
//  * Sources arrive as 80-byte records in chunks of 64, staged into each
//    warp's shared memory by a 1-D bulk async copy (cp.async.bulk) completing
//    on an mbarrier; the copy of chunk c+1 overlaps the arithmetic of chunk c.
//  * Local frames: positions are stored hi/lo relative to a frame centre;
//    each item re-centres targets and sources on the item's own origin with
//    FP32 adds, so FP32 differences are accurate relative to |x - y| plus
//    the item extent, not the absolute coordinates.
//  * Each staged source is classified against the item's bounding box: far
//    sources (box distance >= alpha h_j) run a branch-free FP32 loop;
//    candidates run a masked loop that routes pairs with |r| < alpha h_j to a
//    per-lane queue, drained with all lanes active: x - y and 1/|r| in FP64,
//    products in FP32.  Pairs at zero distance contribute nothing.
//  * Accumulation: plain FP32 within a chunk (<= 64 terms per lane), then a
//    two-sum into per-target (hi, lo).
#include "common.cuh"

namespace stk {

struct __align__(16) WarpSmem {
  SrcRec raw[kChunk];          // bulk-copy destination
  float4 Y[kChunk];            // local position + hh
  float4 Q[kChunk];            // SL density (scaled) + source index bits
  float4 N[kChunk];            // normal
  float4 Pd[kChunk];           // DL density (scaled)
  float acc[2 * 4 * 3][kWarp]; // per-lane compensated sums (hi, lo), lane-minor
  uint8_t queue[kWarp][kQCap]; // near pairs: k | t << 6
  unsigned long long mbar;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bounded wait on the warp's mbarrier; every lane polls.  `limit` is in SM
// clock cycles (about 2 s by default); on expiry the caller records an error.
__device__ __forceinline__ bool wait_chunk(WarpSmem &sm, uint32_t parity, int64_t limit) {
  if (mbar_try_wait(&sm.mbar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try_wait(&sm.mbar, parity)) return true;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void issue_chunk(WarpSmem &sm, const SrcRec *rec, int64_t s, int n,
                                            int lane) {
  if (lane == 0) {
    fence_proxy_async();  // order earlier generic reads of raw[] before the async write
    const uint32_t bytes = (uint32_t)n * (uint32_t)sizeof(SrcRec);
    mbar_expect_tx(&sm.mbar, bytes);
    bulk_g2s(sm.raw, rec + s, bytes, &sm.mbar);
  }
}

// ---------------------------------------------------------------- pair math
// Adds the far-field contribution of one staged source to T targets.
// SL:   q/r + d (d.q)/r^3             (q pre-scaled by w / (8 pi mu))
// DL:   d (d.psi)(d.n)/r^5            (psi pre-scaled by 6 w / (8 pi))
// SLDL: q/r + d [(d.q)/r^3 + (d.psi)(d.n)/r^5]
template <int T, int KIND, bool MASKED>
__device__ __forceinline__ void pair_block(const float (&x)[T][3], float (&ps)[T][3], float4 Y,
                                           float4 Q, float4 N, float4 Pd, unsigned &nm) {
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const float dx = x[t][0] - Y.x, dy = x[t][1] - Y.y, dz = x[t][2] - Y.z;
    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (MASKED) {
      const bool nr = r2 < Y.w;
      nm |= (unsigned)nr << t;
      r2 = nr ? __int_as_float(0x7f800000) : r2;  // rsqrt(+inf) = 0: pair removed here
    }
    const float ri = rsqrtf(r2);
    const float ri2 = ri * ri;
    if (KIND == K_SL) {
      const float dq = fmaf(dx, Q.x, fmaf(dy, Q.y, dz * Q.z));
      const float c = dq * ri2;
      ps[t][0] = fmaf(fmaf(dx, c, Q.x), ri, ps[t][0]);
      ps[t][1] = fmaf(fmaf(dy, c, Q.y), ri, ps[t][1]);
      ps[t][2] = fmaf(fmaf(dz, c, Q.z), ri, ps[t][2]);
    } else if (KIND == K_DL) {
      const float dp = fmaf(dx, Pd.x, fmaf(dy, Pd.y, dz * Pd.z));
      const float dn = fmaf(dx, N.x, fmaf(dy, N.y, dz * N.z));
      const float c = (dp * dn) * (ri2 * ri2 * ri);
      ps[t][0] = fmaf(dx, c, ps[t][0]);
      ps[t][1] = fmaf(dy, c, ps[t][1]);
      ps[t][2] = fmaf(dz, c, ps[t][2]);
    } else {
      const float dq = fmaf(dx, Q.x, fmaf(dy, Q.y, dz * Q.z));
      const float dp = fmaf(dx, Pd.x, fmaf(dy, Pd.y, dz * Pd.z));
      const float dn = fmaf(dx, N.x, fmaf(dy, N.y, dz * N.z));
      const float c = fmaf(dp * dn, ri2, dq) * ri2;
      ps[t][0] = fmaf(fmaf(dx, c, Q.x), ri, ps[t][0]);
      ps[t][1] = fmaf(fmaf(dy, c, Q.y), ri, ps[t][1]);
      ps[t][2] = fmaf(fmaf(dz, c, Q.z), ri, ps[t][2]);
    }
  }
}

// Near pair: d and 1/|r| in FP64 (one Newton step on the FP32 estimate),
// kernel products in FP32 written through the unit vector e = d/|r| so that
// they stay in range however close the pair is:
//   SL: (q + e (e.q)) / r      DL: e (e.psi)(e.n) / r^2
// Returns false for a zero-distance pair.
template <int KIND>
__device__ __forceinline__ bool near_pair(const double *xt, const double *ys, float4 Q, float4 N,
                                          float4 Pd, float (&c)[3]) {
  const double dx = xt[0] - ys[0], dy = xt[1] - ys[1], dz = xt[2] - ys[2];
  const double r2 = dx * dx + dy * dy + dz * dz;
  if (!(r2 > 0.0)) return false;
  double rid;
  const float r2f = __double2float_rn(r2);
  if (r2f > 1e-30f && r2f < 1e30f) {
    const double y0 = (double)rsqrtf(r2f);
    rid = y0 * (1.5 - 0.5 * r2 * y0 * y0);
  } else {
    rid = 1.0 / sqrt(r2);
  }
  const float ri = __double2float_rn(rid);
  const float ex = __double2float_rn(dx * rid), ey = __double2float_rn(dy * rid),
              ez = __double2float_rn(dz * rid);
  if (KIND == K_SL) {
    const float eq = fmaf(ex, Q.x, fmaf(ey, Q.y, ez * Q.z));
    c[0] = fmaf(ex, eq, Q.x) * ri;
    c[1] = fmaf(ey, eq, Q.y) * ri;
    c[2] = fmaf(ez, eq, Q.z) * ri;
  } else if (KIND == K_DL) {
    const float ep = fmaf(ex, Pd.x, fmaf(ey, Pd.y, ez * Pd.z));
    const float en = fmaf(ex, N.x, fmaf(ey, N.y, ez * N.z));
    const float cc = (ep * en) * (ri * ri);
    c[0] = ex * cc;
    c[1] = ey * cc;
    c[2] = ez * cc;
  } else {
    const float eq = fmaf(ex, Q.x, fmaf(ey, Q.y, ez * Q.z));
    const float ep = fmaf(ex, Pd.x, fmaf(ey, Pd.y, ez * Pd.z));
    const float en = fmaf(ex, N.x, fmaf(ey, N.y, ez * N.z));
    const float cc = fmaf(ep * en, ri, eq);
    c[0] = fmaf(ex, cc, Q.x) * ri;
    c[1] = fmaf(ey, cc, Q.y) * ri;
    c[2] = fmaf(ez, cc, Q.z) * ri;
  }
  return true;
}

struct ItemCtx {
  int lane, b, G, tgl, sg, tn;
  int32_t t0;
};

template <int T, int KIND>
__device__ __forceinline__ void drain_queue(WarpSmem &sm, const EngineParams &P, const ItemCtx &ic,
                                         int &qcnt, float (&ps)[T][3]) {
  const int maxc = __reduce_max_sync(kFull, qcnt);
  for (int r = 0; r < maxc; ++r) {
    if (r < qcnt) {
      const unsigned e = sm.queue[ic.lane][r];
      const int k = (int)(e & 63u), t = (int)(e >> 6);
      const float4 Q = sm.Q[k];
      const float4 N = sm.N[k];
      const float4 Pd = sm.Pd[k];
      const int j = __float_as_int(Q.w);
      const int gi = ic.t0 + ic.tgl + ic.G * t;
      const int ci = P.tperm ? P.tperm[gi] : gi;
      float c[3];
      if (near_pair<KIND>(P.trg64 + 3 * (size_t)ci, P.src64 + 3 * (size_t)j, Q, N, Pd, c)) {
#pragma unroll
        for (int tt = 0; tt < T; ++tt)
          if (tt == t) {
            ps[tt][0] += c[0];
            ps[tt][1] += c[1];
            ps[tt][2] += c[2];
          }
      }
    }
  }
  qcnt = 0;
}

template <int T, int KIND>
__device__ __forceinline__ void chunk_compute(WarpSmem &sm, const EngineParams &P,
                                              const ItemCtx &ic, int n, int nfar,
                                              const float (&x)[T][3], float (&ps)[T][3]) {
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  // far sources: no per-pair test
#pragma unroll 2
  for (int k = ic.sg; k < nfar; k += ic.b) {
    const float4 Y = sm.Y[k];
    const float4 Q = (KIND & K_SL) ? sm.Q[k] : z4;
    const float4 N = (KIND & K_DL) ? sm.N[k] : z4;
    const float4 Pd = (KIND & K_DL) ? sm.Pd[k] : z4;
    unsigned nm = 0;
    pair_block<T, KIND, false>(x, ps, Y, Q, N, Pd, nm);
  }
  // candidates: per-pair near test, near pairs queued for the FP64 pass
  int qcnt = 0;
  for (int kk = nfar; kk < n; kk += ic.b) {
    const int k = kk + ic.sg;
    if (k < n) {
      const float4 Y = sm.Y[k];
      const float4 Q = (KIND & K_SL) ? sm.Q[k] : z4;
      const float4 N = (KIND & K_DL) ? sm.N[k] : z4;
      const float4 Pd = (KIND & K_DL) ? sm.Pd[k] : z4;
      unsigned nm = 0;
      pair_block<T, KIND, true>(x, ps, Y, Q, N, Pd, nm);
      if (nm) {
#pragma unroll
        for (int t = 0; t < T; ++t)
          if ((nm >> t) & 1u) sm.queue[ic.lane][qcnt++] = (uint8_t)(k | (t << 6));
      }
    }
    if (__any_sync(kFull, qcnt > kQCap - T)) drain_queue<T, KIND>(sm, P, ic, qcnt, ps);
  }
  if (__any_sync(kFull, qcnt > 0)) drain_queue<T, KIND>(sm, P, ic, qcnt, ps);
}

// Converts the staged raw chunk to local coordinates, far sources first.
__device__ __forceinline__ int convert_chunk(WarpSmem &sm, int n, const float (&oh)[3],
                                             const float (&ol)[3], const float (&blo)[3],
                                             const float (&bhi)[3], int lane) {
  int nfar = 0, ncand = 0;
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < kChunk / kWarp; ++r) {
    const int k = r * kWarp + lane;
    const bool valid = k < n;
    bool cand = false;
    float4 Y = make_float4(0.f, 0.f, 0.f, 0.f), q = Y, nn = Y, pp = Y;
    float idx = 0.f;
    if (valid) {
      const float4 yh = sm.raw[k].yh, yl = sm.raw[k].yl;
      q = sm.raw[k].q;
      nn = sm.raw[k].n;
      pp = sm.raw[k].p;
      Y.x = to_local(yh.x, yl.x, oh[0], ol[0]);
      Y.y = to_local(yh.y, yl.y, oh[1], ol[1]);
      Y.z = to_local(yh.z, yl.z, oh[2], ol[2]);
      Y.w = yh.w;
      idx = yl.w;
      const float ex = fmaxf(fmaxf(blo[0] - Y.x, Y.x - bhi[0]), 0.f);
      const float ey = fmaxf(fmaxf(blo[1] - Y.y, Y.y - bhi[1]), 0.f);
      const float ez = fmaxf(fmaxf(blo[2] - Y.z, Y.z - bhi[2]), 0.f);
      const float bd2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
      cand = !(bd2 >= Y.w);
    }
    const unsigned bc = __ballot_sync(kFull, valid && cand);
    const unsigned bf = __ballot_sync(kFull, valid && !cand);
    if (valid) {
      const int dst = cand ? (n - 1 - (ncand + __popc(bc & lt))) : (nfar + __popc(bf & lt));
      sm.Y[dst] = Y;
      sm.Q[dst] = make_float4(q.x, q.y, q.z, idx);
      sm.N[dst] = nn;
      sm.Pd[dst] = pp;
    }
    nfar += __popc(bf);
    ncand += __popc(bc);
  }
  return nfar;
}

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

struct Cursor {
  int e;
  int sid;
  int64_t s, end;
};

__device__ __forceinline__ bool cursor_next(const EngineParams &P, const Item &it, Cursor &c) {
  while (c.s >= c.end) {
    if (++c.e >= it.seg1) return false;
    c.sid = P.seg_list ? P.seg_list[c.e] : c.e;
    c.s = P.range_ptr[c.sid];
    c.end = P.range_ptr[c.sid + 1];
  }
  return true;
}

template <int T>
__device__ __forceinline__ void dispatch_compute(int kind, WarpSmem &sm, const EngineParams &P,
                                                 const ItemCtx &ic, int n, int nfar,
                                                 const float (&x)[T][3], float (&ps)[T][3]) {
  if (kind == K_SL)
    chunk_compute<T, K_SL>(sm, P, ic, n, nfar, x, ps);
  else if (kind == K_DL)
    chunk_compute<T, K_DL>(sm, P, ic, n, nfar, x, ps);
  else
    chunk_compute<T, K_SLDL>(sm, P, ic, n, nfar, x, ps);
}

// One work item with T targets per lane and b source slices per warp.
template <int T>
__device__ bool run_item(const EngineParams &P, const Item &it, WarpSmem &sm, int b,
                         uint32_t &phase, int lane) {
  ItemCtx ic;
  ic.lane = lane;
  ic.b = b;
  ic.G = kWarp / b;
  ic.tgl = lane % ic.G;
  ic.sg = lane / ic.G;
  ic.tn = it.tn_part & 0xFF;
  ic.t0 = it.t0;
  const int part = it.tn_part >> 8;

  const double cx = P.src64[0], cy = P.src64[1], cz = P.src64[2];
  // item origin: centre of the targets' bounding box
  const int c0 = P.tperm ? P.tperm[it.t0] : it.t0;
  const double x0 = P.trg64[3 * (size_t)c0], y0 = P.trg64[3 * (size_t)c0 + 1],
               z0 = P.trg64[3 * (size_t)c0 + 2];
  bool valid[T];
  float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int li = ic.tgl + ic.G * t;
    valid[t] = li < ic.tn;
    if (valid[t]) {
      const int gi = it.t0 + li;
      const double *xp = P.trg64 + 3 * (size_t)(P.tperm ? P.tperm[gi] : gi);
      const float rx = __double2float_rn(xp[0] - x0), ry = __double2float_rn(xp[1] - y0),
                  rz = __double2float_rn(xp[2] - z0);
      mn[0] = fminf(mn[0], rx); mx[0] = fmaxf(mx[0], rx);
      mn[1] = fminf(mn[1], ry); mx[1] = fmaxf(mx[1], ry);
      mn[2] = fminf(mn[2], rz); mx[2] = fmaxf(mx[2], rz);
    }
  }
  float oh[3], ol[3];
  {
    const double org[3] = {x0 + 0.5 * ((double)warp_min(mn[0]) + (double)warp_max(mx[0])),
                           y0 + 0.5 * ((double)warp_min(mn[1]) + (double)warp_max(mx[1])),
                           z0 + 0.5 * ((double)warp_min(mn[2]) + (double)warp_max(mx[2]))};
    split_hl(org[0] - cx, oh[0], ol[0]);
    split_hl(org[1] - cy, oh[1], ol[1]);
    split_hl(org[2] - cz, oh[2], ol[2]);
  }
  float x[T][3];
  float blo[3] = {INFINITY, INFINITY, INFINITY}, bhi[3] = {-INFINITY, -INFINITY, -INFINITY};
  const double cc[3] = {cx, cy, cz};
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int li = ic.tgl + ic.G * t;
    const int gi = it.t0 + (valid[t] ? li : 0);
    const double *xp = P.trg64 + 3 * (size_t)(P.tperm ? P.tperm[gi] : gi);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (valid[t]) {
        float vh, vl;
        split_hl(xp[k] - cc[k], vh, vl);
        x[t][k] = to_local(vh, vl, oh[k], ol[k]);
        blo[k] = fminf(blo[k], x[t][k]);
        bhi[k] = fmaxf(bhi[k], x[t][k]);
      } else {
        x[t][k] = 1e30f;  // padding slot: far from everything, never written
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    blo[k] = warp_min(blo[k]);
    bhi[k] = warp_max(bhi[k]);
  }

  float ps[T][3];
#pragma unroll
  for (int t = 0; t < T; ++t)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      ps[t][k] = 0.f;
      sm.acc[t * 3 + k][lane] = 0.f;
      sm.acc[(T + t) * 3 + k][lane] = 0.f;
    }

  Cursor cur;
  cur.e = it.seg0 - 1;
  cur.sid = 0;
  cur.s = cur.end = 0;
  bool have = cursor_next(P, it, cur);
  int n_cur = 0, kind_cur = 0;
  if (have) {
    n_cur = (int)min((int64_t)kChunk, cur.end - cur.s);
    kind_cur = seg_kind(P, cur.sid);
    issue_chunk(sm, P.rec, cur.s, n_cur, lane);
    cur.s += n_cur;
  }
  bool ok = true;
  while (have) {
    if (!wait_chunk(sm, phase, P.spin_limit)) {
      set_error(P.err_flag, 4);
      ok = false;
      // wait (bounded) for the copy in flight before giving up on the item
      wait_chunk(sm, phase, P.spin_limit);
      break;
    }
    phase ^= 1u;
    const int nfar = convert_chunk(sm, n_cur, oh, ol, blo, bhi, lane);
    __syncwarp();
    const bool have_next = cursor_next(P, it, cur);
    int n_next = 0, kind_next = 0;
    if (have_next) {
      n_next = (int)min((int64_t)kChunk, cur.end - cur.s);
      kind_next = seg_kind(P, cur.sid);
      issue_chunk(sm, P.rec, cur.s, n_next, lane);
      cur.s += n_next;
    }
    dispatch_compute<T>(kind_cur, sm, P, ic, n_cur, nfar, x, ps);
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        float h = sm.acc[t * 3 + k][lane], l = sm.acc[(T + t) * 3 + k][lane];
        two_sum_acc(h, l, ps[t][k]);
        sm.acc[t * 3 + k][lane] = h;
        sm.acc[(T + t) * 3 + k][lane] = l;
        ps[t][k] = 0.f;
      }
    __syncwarp();
    have = have_next;
    n_cur = n_next;
    kind_cur = kind_next;
  }
  if (!ok) return false;
  float hi[T][3], lo[T][3];
#pragma unroll
  for (int t = 0; t < T; ++t)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      hi[t][k] = sm.acc[t * 3 + k][lane];
      lo[t][k] = sm.acc[(T + t) * 3 + k][lane];
    }

  // combine the b source slices (lanes tgl, tgl + G, ...)
  for (int o = ic.G; o < kWarp; o <<= 1) {
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float h2 = __shfl_xor_sync(kFull, hi[t][k], o);
        const float l2 = __shfl_xor_sync(kFull, lo[t][k], o);
        two_sum_acc(hi[t][k], lo[t][k], h2);
        lo[t][k] += l2;
      }
  }
  if (ic.sg == 0) {
    double *out = P.part_out + ((size_t)part * (size_t)P.nt + (size_t)it.t0) * 3;
#pragma unroll
    for (int t = 0; t < T; ++t) {
      if (valid[t]) {
        const int li = ic.tgl + ic.G * t;
#pragma unroll
        for (int k = 0; k < 3; ++k) out[3 * li + k] = (double)hi[t][k] + (double)lo[t][k];
      }
    }
  }
  return true;
}

__global__ void __launch_bounds__(kWarpsPerCta *kWarp, 4) k_engine_mixed(EngineParams P) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  WarpSmem &sm = reinterpret_cast<WarpSmem *>(smem_raw)[threadIdx.x / kWarp];
  const int lane = threadIdx.x & (kWarp - 1);
  if (lane == 0) {
    mbar_init(&sm.mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_proxy_async();
  }
  __syncwarp();
  uint32_t phase = 0;
  const int n_items = *P.n_items;
  while (true) {
    int idx = 0;
    if (lane == 0) idx = atomicAdd(P.item_counter, 1);
    idx = __shfl_sync(kFull, idx, 0);
    if (idx >= n_items) break;
    const int id = P.item_order ? P.item_order[idx] : idx;
    const Item it = P.items[id];
    const int tn = it.tn_part & 0xFF;
    bool ok;
    if (tn <= 8)
      ok = run_item<1>(P, it, sm, 4, phase, lane);
    else if (tn <= 16)
      ok = run_item<2>(P, it, sm, 4, phase, lane);
    else if (tn <= 24)
      ok = run_item<3>(P, it, sm, 4, phase, lane);
    else if (tn <= 32)
      ok = run_item<4>(P, it, sm, 4, phase, lane);
    else if (tn <= 48)
      ok = run_item<3>(P, it, sm, 2, phase, lane);
    else if (tn <= 64)
      ok = run_item<4>(P, it, sm, 2, phase, lane);
    else if (tn <= 96)
      ok = run_item<3>(P, it, sm, 1, phase, lane);
    else
      ok = run_item<4>(P, it, sm, 1, phase, lane);
    if (!ok) break;
  }
}

size_t engine_mixed_smem_bytes() { return sizeof(WarpSmem) * kWarpsPerCta; }

// The dynamic shared memory (> 48 KB) needs the opt-in attribute on every
// device; engine_mixed_occupancy() sets it and runs once per device before
// the first launch there.
cudaError_t launch_engine_mixed(const EngineParams &P, int grid, cudaStream_t stream) {
  k_engine_mixed<<<grid, kWarpsPerCta * kWarp, engine_mixed_smem_bytes(), stream>>>(P);
  return cudaGetLastError();
}

cudaError_t engine_mixed_occupancy(int *blocks_per_sm) {
  const size_t smem = engine_mixed_smem_bytes();
  cudaError_t e =
      cudaFuncSetAttribute(k_engine_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_engine_mixed,
                                                       kWarpsPerCta * kWarp, smem);
}

}  // namespace stk
