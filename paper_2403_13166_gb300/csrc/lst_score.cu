// lst_score.cu -- T5-DNN (arXiv 2403.13166, Sections 2-3): the 38 input features of each
// quintuplet and the 38 -> 32 -> ... -> 1 network (ReLU hidden layers, sigmoid output),
// FP32 on the CUDA cores. Output candidates are exported as hit-index tuples here too.
//
// The FP32 path keeps the score within 1e-6 of an FP64 evaluation for trained networks,
// which move the score by ~1e-6 for a single FP32 rounding of one input or one hidden
// activation: the features are computed in float-float (lst_ff.cuh) and every layer is a
// compensated dot product of FP32 weights with float-float activations (Dot2: each
// product split exactly by an FMA, the running sum's rounding errors collected and added
// back), so that only the final sigmoid rounds to FP32.
#include "lst_features.cuh"

namespace lstk {

// One neuron: bias + sum_i w[i] (xh[i] + xl[i]), compensated (Dot2 of Ogita, Rump and
// Oishi with the activations' low parts folded into the error term).
template <int N>
__device__ __forceinline__ ff dot2(const float *__restrict__ w, float bias, const float *xh, const float *xl) {
  float s = bias, c = 0.0f;
#pragma unroll
  for (int i = 0; i < N; i++) {
    const ff p = two_prod(w[i], xh[i]);
    const ff q = two_sum(s, p.hi);
    s = q.hi;
    c = __fmaf_rn(w[i], xl[i], c + (q.lo + p.lo));
  }
  return two_sum(s, c);
}

// Four neurons o0..o0+3 of one layer at once (rows of N weights, biases b), ReLU: each
// input is read once for the four, and the four compensated sums are independent.
template <int N>
__device__ __forceinline__ void dot2x4_relu(const float *__restrict__ w, const float *__restrict__ b, int o0,
                                            const float *xh, const float *xl, float *oh, float *ol) {
  float s[4], c[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    s[k] = b[o0 + k];
    c[k] = 0.0f;
  }
#pragma unroll
  for (int i = 0; i < N; i++) {
    const float xhi = xh[i], xlo = xl[i];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const float wk = w[(o0 + k) * N + i];
      const ff p = two_prod(wk, xhi);
      const ff q = two_sum(s[k], p.hi);
      s[k] = q.hi;
      c[k] = __fmaf_rn(wk, xlo, c[k] + (q.lo + p.lo));
    }
  }
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const ff v = two_sum(s[k], c[k]);
    oh[o0 + k] = v.hi > 0.0f ? v.hi : 0.0f;
    ol[o0 + k] = v.hi > 0.0f ? v.lo : 0.0f;
  }
}

// The network on float-float inputs with the weights in shared memory (flat layout of
// lst_mlp); hidden activations stay float-float.
__device__ __forceinline__ float mlp_ff(const float *__restrict__ w, int n_hidden, const float *fh, const float *fl) {
  float hh[NHID], hl[NHID], th[NHID], tl[NHID];
#pragma unroll 1
  for (int o = 0; o < NHID; o += 4) dot2x4_relu<NFEAT>(w, w + NHID * NFEAT, o, fh, fl, hh, hl);
  const float *p = w + NHID * NFEAT + NHID;
  for (int l = 1; l < n_hidden; l++) {
#pragma unroll 1
    for (int o = 0; o < NHID; o += 4) dot2x4_relu<NHID>(p, p + NHID * NHID, o, hh, hl, th, tl);
#pragma unroll
    for (int o = 0; o < NHID; o++) {
      hh[o] = th[o];
      hl[o] = tl[o];
    }
    p += NHID * NHID + NHID;
  }
  const ff v = dot2<NHID>(p, p[NHID], hh, hl);
  // exp(-(hi + lo)) = exp(-hi) (1 - lo + ...), |lo| <= ulp(hi) / 2
  const float E = expf(-v.hi);
  const float Ec = E < 3.0e38f ? __fmaf_rn(-E, v.lo, E) : E;
  return 1.0f / (1.0f + Ec);
}

__host__ __device__ constexpr int mlp_floats(int n_hidden) {
  return NHID * NFEAT + NHID + (n_hidden - 1) * (NHID * NHID + NHID) + NHID + 1;
}

// Fused features + FP32 network over every T5 of every event of the batch.
__global__ void __launch_bounds__(256) k_score_fp32(const EvDesc *__restrict__ evs, int n_events,
                                                   DevGeom g, lst_cuts c, const float *__restrict__ wts,
                                                   int n_hidden) {
  extern __shared__ __align__(16) float s_w[];
  __shared__ int s_pref[MAX_EVENTS + 1];
  const int nw = mlp_floats(n_hidden);
  for (int i = threadIdx.x; i < nw; i += blockDim.x) s_w[i] = wts[i];
  block_event_prefix(n_events, [&](int e) {
    const EvDesc &ev = evs[e];
    return ev_void(ev) ? 0 : clamp_count(ev.cnt[C_T5], ev.t5_cap);
  }, s_pref);
  const int total = s_pref[n_events];
  const int lane = threadIdx.x & 31;
  // warp-uniform trip count so that the ballot below sees the full warp
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total; base += stride) {
    const int u = base + lane;
    bool sel = false;
    int e = 0;
    if (u < total) {
      e = find_event(s_pref, n_events, u);
      const EvDesc &ev = evs[e];
      const int t = u - s_pref[e];
      float fh[NFEAT], fl[NFEAT];
      t5_features_ff(ev, g, t, c.k_field, fh, fl);
      const float s = mlp_ff(s_w, n_hidden, fh, fl);
      sel = c.t5_chi2_max > 0.0f || s >= c.wp;     // pre-DNN mode: the chi2 cut selected it
      ev.t5_score[t] = s;
      ev.t5_sel[t] = sel ? 1 : 0;
    }
    // count selected per event: lanes of one warp may straddle events
    const unsigned act = __ballot_sync(FULL, u < total);
    if (u < total) {
      const unsigned same = __match_any_sync(act, e);
      const unsigned sb = __ballot_sync(act, sel) & same;
      if ((same & lanemask_lt()) == 0 && sb) atomicAdd(evs[e].cnt + C_NSEL, __popc(sb));
    }
  }
}

// Feature export [n][38] of one event (lst_get_t5_features): the FP32 features the
// tensor-core score paths read, so that lst_score_t5 on them reproduces those scores.
__global__ void k_features(const EvDesc *__restrict__ ev_p, DevGeom g, float k_field, float *out, int n) {
  const EvDesc &ev = *ev_p;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    float f[NFEAT];
    t5_features(ev, g, t, k_field, f);
#pragma unroll
    for (int i = 0; i < NFEAT; i++) out[(size_t)t * NFEAT + i] = f[i];
  }
}

// Standalone scoring of precomputed features (lst_score_t5), FP32.
__global__ void __launch_bounds__(256) k_score_feat_fp32(const float *__restrict__ feat, int64_t n,
                                                        const float *__restrict__ wts, int n_hidden,
                                                        float *__restrict__ out) {
  extern __shared__ __align__(16) float s_w[];
  const int nw = mlp_floats(n_hidden);
  for (int i = threadIdx.x; i < nw; i += blockDim.x) s_w[i] = wts[i];
  __syncthreads();
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    float f[NFEAT], fl[NFEAT];
#pragma unroll
    for (int i = 0; i < NFEAT; i++) {
      f[i] = feat[t * NFEAT + i];
      fl[i] = 0.0f;
    }
    out[t] = mlp_ff(s_w, n_hidden, f, fl);
  }
}

// Hit-index tuples of one object kind of one event.
__global__ void k_gather(const EvDesc *__restrict__ ev_p, int kind, int n, int32_t *out, float *score,
                         uint8_t *sel) {
  const EvDesc &ev = *ev_p;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    if (kind == LST_MD) {
      const int2 h = ev.md_hits[t];
      out[2 * (size_t)t] = h.x;
      out[2 * (size_t)t + 1] = h.y;
    } else if (kind == LST_LS) {
      const int4 L = ev.lsu[t];
      const int2 a = ev.md_hits[L.x], b = ev.md_hits[L.y];
      int32_t *o = out + 4 * (size_t)t;
      o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    } else if (kind == LST_T3) {
      const int4 m = ev.t3_md[t];
      const int2 a = ev.md_hits[m.x], b = ev.md_hits[m.y], c = ev.md_hits[m.z];
      int32_t *o = out + 6 * (size_t)t;
      o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y; o[4] = c.x; o[5] = c.y;
    } else {
      const int4 a = ev.t5_a[t], b = ev.t5_b[t];
      const int md[5] = {a.x, a.y, a.z, a.w, b.x};
      int32_t *o = out + 10 * (size_t)t;
#pragma unroll
      for (int i = 0; i < 5; i++) {
        const int2 h = ev.md_hits[md[i]];
        o[2 * i] = h.x;
        o[2 * i + 1] = h.y;
      }
      if (score) score[t] = ev.t5_score[t];
      if (sel) sel[t] = ev.t5_sel[t];
    }
  }
}

// Hit-index tuples, scores and selection flags of the track candidates of one event, in
// no particular order (counter: one int on the device, zeroed by the caller; cap: the rows
// the output holds, the event's candidate count: a row past it is not written, so a counter
// that did not start at zero can never send a write out of the buffer).
__global__ void k_gather_tc(const EvDesc *__restrict__ ev_p, int n_t5, int *counter, int32_t *out, float *score,
                            uint8_t *sel, int64_t cap) {
  const EvDesc &ev = *ev_p;
  const int lane = threadIdx.x & 31;
  for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n_t5; base += gridDim.x * blockDim.x) {
    const int t = base + lane;
    const bool keep = t < n_t5 && ev.t5_tc[t];
    const unsigned bal = __ballot_sync(FULL, keep);
    int o0 = 0;
    if (lane == 0 && bal) o0 = atomicAdd(counter, __popc(bal));
    o0 = __shfl_sync(FULL, o0, 0);
    const int o = o0 + __popc(bal & lanemask_lt());
    if (keep && o >= 0 && o < cap) {
      const int4 a = ev.t5_a[t], b = ev.t5_b[t];
      const int md[5] = {a.x, a.y, a.z, a.w, b.x};
#pragma unroll
      for (int i = 0; i < 5; i++) {
        const int2 h = ev.md_hits[md[i]];
        out[10 * (size_t)o + 2 * i] = h.x;
        out[10 * (size_t)o + 2 * i + 1] = h.y;
      }
      if (score) score[o] = ev.t5_score[t];
      if (sel) sel[o] = ev.t5_sel[t];
    }
  }
}

// LS graph of one event (MD nodes, LS edges from inner to outer MD): CSR row offsets by one
// CTA, row_off[n_md] = number of edges.
__global__ void k_graph_rows(const EvDesc *__restrict__ ev_p, int n_md, int32_t *row_off) {
  const EvDesc &ev = *ev_p;
  block_exclusive_scan(ev.ls_cnt, row_off, n_md);
  if (threadIdx.x == 0) row_off[n_md] = n_md ? row_off[n_md - 1] + ev.ls_cnt[n_md - 1] : 0;
}

// ... then the edges of every MD (its LS range) and the node / edge features.
__global__ void k_graph_fill(const EvDesc *__restrict__ ev_p, DevGeom g, int n_md, const int32_t *row_off,
                             int32_t *col, float *node_feat, float *edge_feat) {
  const EvDesc &ev = *ev_p;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n_md; m += gridDim.x * blockDim.x) {
    const float4 A = ev.md_anchor[m];
    const int beg = ev.ls_start[m], cnt = ev.ls_cnt[m], o = row_off[m];
    for (int k = 0; k < cnt; k++) {
      const int b = ev.ls_to[beg + k];
      col[o + k] = b;
      if (edge_feat) {
        const float4 B = ev.md_anchor[b];
        edge_feat[2 * (size_t)(o + k)] = ls_curvature(A, B);
        edge_feat[2 * (size_t)(o + k) + 1] = A.z - A.w * ((B.z - A.z) / (B.w - A.w));   // z at r = 0
      }
    }
    if (node_feat) {
      float *f = node_feat + 6 * (size_t)m;
      f[0] = A.x; f[1] = A.y; f[2] = A.z; f[3] = A.w;
      f[4] = ev.md_kappa[m].x;
      f[5] = (float)g.layer[ev.md_mod[m]];
    }
  }
}

// Zero the per-event counters, sensor histogram and the per-MD range counts (units whose
// MD range was dropped after an overflow must read as empty).
__global__ void k_reset(const EvDesc *__restrict__ evs, DevGeom g) {
  const EvDesc &ev = evs[blockIdx.y];
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
  if (tid < C_NCOUNTERS) ev.cnt[tid] = 0;
  for (int i = tid; i < 2 * g.n_mod; i += st) ev.sens_cnt[i] = 0;
  for (int i = tid; i < ev.md_cap; i += st) {
    ev.ls_cnt[i] = 0;
    ev.lso_cnt[i] = 0;
    ev.t3_cnt[i] = 0;
    ev.tc_cnt[i] = 0;
  }
  for (int i = tid; i < g.n_mod; i += st) ev.md_cnt[i] = 0;
}

}  // namespace lstk
