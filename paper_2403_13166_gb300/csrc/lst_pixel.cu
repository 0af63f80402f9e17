// lst_pixel.cu -- pixel seeds on the GPU: Table 1 steps 0 and 5-8 (pT5, T5, pT3 and pLS
// track candidates) for one finished event.
//
// A pixel seed (pLS) is four inner-tracker hits H1..H4 made upstream (step 0). It is matched
// to an outer object -- a track-candidate T5 by its first T3, then a T3 -- whose first anchors
// are P0, P1 and whose curvature is ko, when both lie on one helix (Section 1): the azimuth
// and r-z slope windows, the seed's curvature against ko, the circle through H1, H4, P0
// against ko, and H4's z against its interpolation between H1 and P0 along the arc (FP32,
// the expression trees of the oracle). Matching is one-to-one with preference to the better
// (rz residual, curvature difference): the edges in ascending (residual, difference, seed
// index, object hit tuple) order, each taken when both ends are free. On the GPU that
// greedy result is reached in rounds: every free object finds its best free seed, every free
// seed its best free object, and the pairs that chose each other are taken (such an edge is
// the minimum at both its ends, so the greedy pass takes it too); rounds repeat until none
// is taken.
//
// Seeds are binned by the azimuth of H4 and their r-z slope; a warp scans the bins of an
// object's windows (one contiguous run of azimuth bins per slope row), so a pair that passes
// the window test is always met. The seeds that the pT5s took are binned out before the T3
// stage (they can match nothing there), which shrinks its windows about fivefold.
#include "lst_internal.cuh"

namespace lstk {

constexpr float PIX_MMAX = 6.0f;                // slope bins cover [-6, 6]; the end bins take the rest
constexpr float PIX_PI = 3.14159265358979f;

__device__ __forceinline__ float pix_curv3(float ax0, float ay0, float bx0, float by0, float cx0, float cy0) {
  const float d01x = bx0 - ax0, d01y = by0 - ay0;
  const float d12x = cx0 - bx0, d12y = cy0 - by0;
  const float d02x = cx0 - ax0, d02y = cy0 - ay0;
  const float a = sqrtf(d01x * d01x + d01y * d01y);
  const float b = sqrtf(d12x * d12x + d12y * d12y);
  const float c = sqrtf(d02x * d02x + d02y * d02y);
  const float cr = d01x * d02y - d01y * d02x;
  return 2.0f * cr / (a * b * c);
}

__device__ __forceinline__ bool pix_kappa_ok(float k1, float k2, const lst_pixel_cuts &pc) {
  return fabsf(k1 - k2) <= pc.kappa_rel * 0.5f * (fabsf(k1) + fabsf(k2)) + pc.kappa_abs;
}

// The seed / object match: A = (x1, y1, z1, kp), B = (x4, y4, z4, r4), mp the seed's slope;
// P0, P1 the object's first two anchors, mo = (P1.z - P0.z) / (P1.w - P0.w), ko its curvature.
__device__ __forceinline__ bool pix_match(const float4 A, const float4 B, float mp, const float4 P0, float mo,
                                          float ko, const lst_pixel_cuts &pc, float &res, float &dk) {
  if (!(B.x * P0.x + B.y * P0.y > 0.0f)) return false;                              // azimuth
  if (!(fabsf(B.x * P0.y - B.y * P0.x) <= (pc.dphi0 + pc.dphi_cm * (P0.w - B.w)) * (B.w * P0.w))) return false;
  if (!(fabsf(mp - mo) <= pc.dm_abs + pc.dm_rel * fabsf(mo))) return false;          // slope
  if (!pix_kappa_ok(A.w, ko, pc)) return false;                                     // pT
  const float kx = pix_curv3(A.x, A.y, B.x, B.y, P0.x, P0.y);
  if (!pix_kappa_ok(kx, ko, pc)) return false;                                      // circle
  const float kbar = 0.5f * (kx + ko);
  const float ax = B.x - A.x, ay = B.y - A.y, bx = P0.x - B.x, by = P0.y - B.y;
  const float a = sqrtf(ax * ax + ay * ay), b = sqrtf(bx * bx + by * by);
  const float s14 = a * (1.0f + a * a * kbar * kbar / 24.0f);
  const float s40 = b * (1.0f + b * b * kbar * kbar / 24.0f);
  const float zp = A.z + (P0.z - A.z) * s14 / (s14 + s40);
  res = fabsf(B.z - zp);
  if (!(res <= pc.rz_tol)) return false;                                            // rz
  dk = fabsf(kx - ko);
  return true;
}

__device__ __forceinline__ int pix_mbin(float m) {
  const float v = fminf(fmaxf((m + PIX_MMAX) * (PIX_NM / (2.0f * PIX_MMAX)), 0.0f), (float)(PIX_NM - 1));
  return (int)v;                     // NaN -> 0
}
__device__ __forceinline__ int pix_phibin(float y, float x) {
  int b = (int)floorf((atan2f(y, x) + PIX_PI) * (PIX_NPHI / (2.0f * PIX_PI)));
  return ((b % PIX_NPHI) + PIX_NPHI) % PIX_NPHI;
}

// the seed's derived values, the oracle's expressions: r1, r4, slope, curvature through H1, H3, H4
__device__ __forceinline__ void pix_seed(const float *H, float4 &A, float4 &B, float &mp) {
  const float r1 = sqrtf(H[0] * H[0] + H[1] * H[1]);
  const float r4 = sqrtf(H[9] * H[9] + H[10] * H[10]);
  mp = (H[11] - H[2]) / (r4 - r1);
  A = make_float4(H[0], H[1], H[2], pix_curv3(H[0], H[1], H[6], H[7], H[9], H[10]));
  B = make_float4(H[9], H[10], H[11], r4);
}

// Seeds into their (slope row, azimuth bin) cells: counts and ranks. With rebin (between the
// stages) only the seeds still free are binned again: the seeds the pT5s took leave the scans
// of stage 7, the per-seed state and the smallest seed radius stay as they are (the windows
// drawn from the smaller radius of all seeds stay wide enough).
__global__ void k_pix_bin(const PixDesc *Ps, int rebin) {
  const PixDesc &P = Ps[blockIdx.y];
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P.n_pls; p += gridDim.x * blockDim.x) {
    if (rebin) {
      if (P.pmatch[p] < 0) P.rank[p] = atomicAdd(P.cell_cnt + P.cell[p], 1);
      continue;
    }
    float4 A, B;
    float mp;
    pix_seed(P.hits + 12 * (size_t)p, A, B, mp);
    const int c = pix_mbin(mp) * PIX_NPHI + pix_phibin(B.y, B.x);
    if (B.w >= 0.0f) atomicMin(P.ctr + 3, __float_as_int(B.w));   // smallest r4 (non-negative: int order)
    P.cell[p] = c;
    P.rank[p] = atomicAdd(P.cell_cnt + c, 1);
    P.pkey[p] = ~0ull;
    P.pcnt[p] = 0;
    P.pobj[p] = -1;
    P.pmatch[p] = -1;
  }
}

__global__ void k_pix_rebin_clear(const PixDesc *Ps) {
  const PixDesc &P = Ps[blockIdx.y];
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < PIX_NCELL; c += gridDim.x * blockDim.x) P.cell_cnt[c] = 0;
}

__global__ void k_pix_scan(const PixDesc *Ps) {
  const PixDesc &P = Ps[blockIdx.y];
  block_exclusive_scan(P.cell_cnt, P.cell_off, PIX_NCELL);
  __syncthreads();
  if (threadIdx.x == 0) P.cell_off[PIX_NCELL] = P.cell_off[PIX_NCELL - 1] + P.cell_cnt[PIX_NCELL - 1];
}

__global__ void k_pix_scatter(const PixDesc *Ps, int rebin) {
  const PixDesc &P = Ps[blockIdx.y];
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P.n_pls; p += gridDim.x * blockDim.x) {
    if (rebin && P.pmatch[p] >= 0) continue;
    float4 A, B;
    float mp;
    pix_seed(P.hits + 12 * (size_t)p, A, B, mp);
    const int q = P.cell_off[P.cell[p]] + P.rank[p];
    P.sa[q] = A;
    P.sb[q] = B;
    P.sm[q] = mp;
    P.sk[q] = A.w;
    P.sidx[q] = p;
  }
}

// Object o of the stage: T5 (stage 5; only track-candidate T5s) or T3 (stage 7; not made of
// MDs of pT5 quintuplets). Fills its first two anchors and curvature; false if it takes no part.
__device__ __forceinline__ bool pix_object(const EvDesc &ev, const PixDesc &P, int stage, int o, float4 &P0,
                                           float4 &P1, float &ko) {
  int m0, m1;
  if (stage == 5) {
    if (!ev.t5_tc[o]) return false;
    const int4 a = ev.t5_a[o];
    m0 = a.x;
    m1 = a.y;
    ko = ev.t3_kappa[ev.t5_b[o].y];
  } else {
    const int4 t = ev.t3_md[o];
    if (P.mdflag[t.x] && P.mdflag[t.y] && P.mdflag[t.z]) return false;
    m0 = t.x;
    m1 = t.y;
    ko = ev.t3_kappa[o];
  }
  P0 = ev.md_anchor[m0];
  P1 = ev.md_anchor[m1];
  return true;
}

// Whether object o takes part in the stage at all (what pix_object decides first).
__device__ __forceinline__ bool pix_eligible(const EvDesc &ev, const PixDesc &P, int stage, int o) {
  if (stage == 5) return ev.t5_tc[o] != 0;
  const int4 t = ev.t3_md[o];
  return !(P.mdflag[t.x] && P.mdflag[t.y] && P.mdflag[t.z]);
}

// Visit every free seed in the object's windows that matches it: f(hit, p, res, dk) is called
// on every lane of the warp (warp-uniform, so f may vote), hit telling whether the lane's seed
// p matched. The azimuth window is the turn the cut allows at this radius from the smallest
// seed radius r4min (its sine bound, arcsine, plus one bin for rounding); the slope window its
// rows plus one on each side. The scan runs in two passes: the seeds of the window are tested
// on the packed curvatures alone -- the pT test, which rejects about 85% of a window -- and
// the survivors go into the warp's queue (PIX_QCAP seed positions in shared memory), from
// which the full match runs on full warps, 32 seeds at a time. The run bounds of 32 slope rows
// are loaded at once, a lane per row; then either the warp walks the non-empty runs one after
// another, 128 seeds at a time, or (sparse windows: cheaper when the longest run is short)
// every lane walks its own row's runs, four seeds a step.
template <typename F>
__device__ __forceinline__ void pix_scan_object(const PixDesc &P, const float4 P0, const float4 P1, float ko,
                                                const lst_pixel_cuts &pc, float r4min, int *queue, F f) {
  const int lane = threadIdx.x & 31;
  const float mo = (P1.z - P0.z) / (P1.w - P0.w);
  const float w = pc.dm_abs + pc.dm_rel * fabsf(mo);
  const int m_lo = max(0, pix_mbin(mo - w) - 1), m_hi = min(PIX_NM - 1, pix_mbin(mo + w) + 1);
  const bool all_m = !(w <= 1e30f);              // an infinite or NaN window: every row
  const int r0 = all_m ? 0 : m_lo, r1 = all_m ? PIX_NM - 1 : m_hi;
  const float sb = pc.dphi0 + pc.dphi_cm * (P0.w - r4min);
  const float turn = sb >= 1.0f || !(sb == sb) ? 0.5f * PIX_PI : asinf(fmaxf(sb, 0.0f));
  const int dphi_bins = (int)(turn * (PIX_NPHI / (2.0f * PIX_PI))) + 2;
  const int c0 = pix_phibin(P0.y, P0.x);
  const int span = min(2 * dphi_bins + 1, PIX_NPHI);
  const int first = ((c0 - dphi_bins) % PIX_NPHI + PIX_NPHI) % PIX_NPHI;
  // the azimuth bins [first, first + span) modulo PIX_NPHI: [first, e0), and [0, e1) if it wraps
  const bool wrap = first + span > PIX_NPHI;
  const int e0 = min(first + span, PIX_NPHI), e1 = first + span - PIX_NPHI;
  int qn = 0;                                    // seed positions in the queue (warp-uniform)
  // the full match on queue entries [j, j + 32); lanes at or past `upto` take no seed
  auto match = [&](int j, int upto) {
    const int t = j + lane;
    bool hit = false;
    int p = -1;
    float res = 0.0f, dk = 0.0f;
    if (t < upto) {
      const int q = queue[t];
      p = P.sidx[q];
      hit = P.pmatch[p] < 0 && pix_match(P.sa[q], P.sb[q], P.sm[q], P0, mo, ko, pc, res, dk);
    }
    f(hit, p, res, dk);
  };
  // append the lane's survivors (bit s of m: position qs[s]) to the queue; match full warps of it
  auto enqueue = [&](unsigned m, const int (&qs)[4]) {
    const int c = __popc(m);
    int x = c;                                   // inclusive prefix of the survivor counts
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(FULL, x, d);
      if (lane >= d) x += y;
    }
    int at = qn + x - c;
#pragma unroll
    for (int s = 0; s < 4; s++)
      if (m >> s & 1u) queue[at++] = qs[s];
    qn += __shfl_sync(FULL, x, 31);
    __syncwarp();
    if (qn >= 32) {
      int j = 0;
      for (; j + 32 <= qn; j += 32) match(j, qn);
      const int rem = qn - j;                    // below 32: to the front of the queue
      const int v = lane < rem ? queue[j + lane] : 0;
      __syncwarp();
      if (lane < rem) queue[lane] = v;
      __syncwarp();
      qn = rem;
    }
  };
  for (int rb = r0; rb <= r1; rb += 32) {
    const int row = rb + lane;
    int a0 = 0, la = 0, b0 = 0, lb = 0;
    if (row <= r1) {
      const int *co = P.cell_off + row * PIX_NPHI;
      a0 = co[first];
      la = co[e0] - a0;
      if (wrap) {
        b0 = co[0];
        lb = co[e1] - b0;
      }
    }
    const int len = la + lb;
    const int maxlen = __reduce_max_sync(FULL, (unsigned)len);
    // steps of the two walks: the longest run's, four seeds a step; the non-empty runs' one by one
    const int n_runs = __popc(__ballot_sync(FULL, la > 0)) + __popc(__ballot_sync(FULL, lb > 0));
    const int total = __reduce_add_sync(FULL, (unsigned)len);
    if ((maxlen + 3) / 4 <= n_runs + total / 128) {
      for (int t = 0; t < maxlen; t += 4) {
        int qs[4];
        float kv[4];
#pragma unroll
        for (int s = 0; s < 4; s++) {
          const int u = t + s;
          qs[s] = u < la ? a0 + u : b0 + (u - la);
          kv[s] = u < len ? P.sk[qs[s]] : 0.0f;
        }
        unsigned m = 0;
#pragma unroll
        for (int s = 0; s < 4; s++)
          if (t + s < len && pix_kappa_ok(kv[s], ko, pc)) m |= 1u << s;
        enqueue(m, qs);
      }
    } else {
      for (int k = 0; k < 2; k++) {
        unsigned nonempty = __ballot_sync(FULL, (k == 0 ? la : lb) > 0);
        while (nonempty) {
          const int src = __ffs(nonempty) - 1;
          nonempty &= nonempty - 1;
          const int q0 = __shfl_sync(FULL, k == 0 ? a0 : b0, src);
          const int q1 = q0 + __shfl_sync(FULL, k == 0 ? la : lb, src);
          for (int qb = q0; qb < q1; qb += 128) {
            int qs[4];
            float kv[4];
#pragma unroll
            for (int s = 0; s < 4; s++) {
              qs[s] = qb + 32 * s + lane;
              kv[s] = P.sk[min(qs[s], q1 - 1)];  // in range: q1 > qb
            }
            unsigned m = 0;
#pragma unroll
            for (int s = 0; s < 4; s++)
              if (qs[s] < q1 && pix_kappa_ok(kv[s], ko, pc)) m |= 1u << s;
            enqueue(m, qs);
          }
        }
      }
    }
  }
  if (qn > 0) match(0, qn);
}

__device__ __forceinline__ unsigned long long pix_key(float res, float dk) {
  return ((unsigned long long)__float_as_uint(res) << 32) | __float_as_uint(dk);
}

// Round, part 1: each free object's best free seed (rank, then seed index) and, at each seed,
// the best rank over its free objects. A warp takes G consecutive objects at a time (32, or
// fewer when the objects would not give every warp that many). The first round of a stage
// scans each object's windows (the whole warp, one object after another) and caches its
// candidates (PIX_OCAP at most; an object with more keeps scanning); later rounds and part 2
// read the cache, a lane per object, dropping seeds taken since (seeds only leave the free
// pool and the match of a pair does not change, so the candidates are the same as a scan's).
__global__ void __launch_bounds__(PIX_SCAN_THREADS, 4) k_pix_propose(const EvDesc *__restrict__ evs, const PixDesc *Ps, int stage, lst_pixel_cuts pc) {
  const EvDesc &ev = evs[blockIdx.y];
  const PixDesc &P = Ps[blockIdx.y];
  if (P.ctr[PIX_DONE]) return;
  const int lane = threadIdx.x & 31;
  const int n = stage == 5 ? P.n_t5 : P.n_t3, base = stage == 5 ? 0 : P.n_t5;
  const float r4min = __int_as_float(P.ctr[3]);
  __shared__ int s_queue[(PIX_SCAN_THREADS / 32) * PIX_QCAP];
  int *queue = s_queue + (threadIdx.x >> 5) * PIX_QCAP;
  const int W = (gridDim.x * blockDim.x) >> 5;
  const int G = min(32, max(1, n / W));           // objects per warp and step (W warps: balance)
  for (int ob = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * G; ob < n; ob += G * W) {
    const int o = ob + lane, g = base + o;
    bool active = lane < G && o < n && P.omatch[g] == -1;   // not taken, not out
    const int cached = active ? P.ocnt[g] : 0;
    if (active && cached == -1 && !pix_eligible(ev, P, stage, o)) {   // first round: out for good
      P.okey[g] = ~0ull;
      P.op[g] = -1;
      P.omatch[g] = -2;
      active = false;
    }
    const bool from_cache = active && cached >= 0 && cached <= PIX_OCAP;
    if (from_cache) {
      unsigned long long best = ~0ull;
      int bp = 0x7fffffff;
      for (int j = 0; j < cached; j++) {
        const int p = P.oseed[(size_t)g * PIX_OCAP + j];
        if (P.pmatch[p] >= 0) continue;
        const unsigned long long k = P.okeys[(size_t)g * PIX_OCAP + j];
        atomicMin(P.pkey + p, k);
        if (k < best || (k == best && p < bp)) { best = k; bp = p; }
      }
      P.okey[g] = best;
      P.op[g] = best == ~0ull ? -1 : bp;
      // no free seed matches it now, so none will later (seeds only leave): out for good
      if (best == ~0ull) P.omatch[g] = -2;
    }
    unsigned to_scan = __ballot_sync(FULL, active && !from_cache);
    while (to_scan) {
      const int src = __ffs(to_scan) - 1;
      to_scan &= to_scan - 1;
      const int so = ob + src, sg = base + so;
      const bool build = __shfl_sync(FULL, cached, src) == -1;
      unsigned long long best = ~0ull;
      int bp = 0x7fffffff;
      float4 P0, P1;
      float ko;
      if (pix_object(ev, P, stage, so, P0, P1, ko)) {
        int cnt = 0;
        pix_scan_object(P, P0, P1, ko, pc, r4min, queue, [&](bool hit, int p, float res, float dk) {
          const unsigned long long k = pix_key(res, dk);
          if (hit) {
            atomicMin(P.pkey + p, k);
            if (k < best || (k == best && p < bp)) { best = k; bp = p; }
          }
          if (build) {
            const unsigned m = __ballot_sync(FULL, hit);
            const int at = cnt + __popc(m & lanemask_lt());
            if (hit && at < PIX_OCAP) {
              P.oseed[(size_t)sg * PIX_OCAP + at] = p;
              P.okeys[(size_t)sg * PIX_OCAP + at] = k;
            }
            cnt += __popc(m);
          }
        });
        if (build && lane == 0) P.ocnt[sg] = min(cnt, PIX_OCAP + 1);
      }
#pragma unroll
      for (int s = 16; s; s >>= 1) {               // the warp's minimum of (rank, seed)
        const unsigned long long ob2 = __shfl_xor_sync(FULL, best, s);
        const int op2 = __shfl_xor_sync(FULL, bp, s);
        if (ob2 < best || (ob2 == best && op2 < bp)) { best = ob2; bp = op2; }
      }
      if (lane == 0) {
        P.okey[sg] = best;
        P.op[sg] = best == ~0ull ? -1 : bp;
        if (best == ~0ull) P.omatch[sg] = -2;
      }
    }
  }
}

// Round, part 2: the objects that reach a seed's best rank list themselves at that seed; as
// in part 1, a lane per cached object and the whole warp for an object that scans.
__global__ void __launch_bounds__(PIX_SCAN_THREADS, 4) k_pix_ties(const EvDesc *__restrict__ evs, const PixDesc *Ps, int stage, lst_pixel_cuts pc) {
  const EvDesc &ev = evs[blockIdx.y];
  const PixDesc &P = Ps[blockIdx.y];
  if (P.ctr[PIX_DONE]) return;
  const int lane = threadIdx.x & 31;
  const int n = stage == 5 ? P.n_t5 : P.n_t3, base = stage == 5 ? 0 : P.n_t5;
  const float r4min = __int_as_float(P.ctr[3]);
  __shared__ int s_queue[(PIX_SCAN_THREADS / 32) * PIX_QCAP];
  int *queue = s_queue + (threadIdx.x >> 5) * PIX_QCAP;
  const int W = (gridDim.x * blockDim.x) >> 5;
  auto list_at = [&](int o, int p, unsigned long long k) {
    if (k != P.pkey[p]) return;
    const int s = atomicAdd(P.pcnt + p, 1);
    if (s < PIX_TIES)
      P.plist[PIX_TIES * (size_t)p + s] = o;
    else
      atomicOr(P.ctr + 2, 1);
  };
  const int G = min(32, max(1, n / W));           // objects per warp and step (W warps: balance)
  for (int ob = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * G; ob < n; ob += G * W) {
    const int o = ob + lane, g = base + o;
    // a free seed matches it (okey set by part 1) and it is still free
    const bool active = lane < G && o < n && P.okey[g] != ~0ull && P.omatch[g] == -1;
    const int cached = active ? P.ocnt[g] : 0;
    const bool from_cache = active && cached >= 0 && cached <= PIX_OCAP;
    if (from_cache) {
      for (int j = 0; j < cached; j++) {
        const int p = P.oseed[(size_t)g * PIX_OCAP + j];
        if (P.pmatch[p] < 0) list_at(o, p, P.okeys[(size_t)g * PIX_OCAP + j]);
      }
    }
    unsigned to_scan = __ballot_sync(FULL, active && !from_cache);
    while (to_scan) {
      const int src = __ffs(to_scan) - 1;
      to_scan &= to_scan - 1;
      const int so = ob + src;
      float4 P0, P1;
      float ko;
      if (!pix_object(ev, P, stage, so, P0, P1, ko)) continue;
      pix_scan_object(P, P0, P1, ko, pc, r4min, queue, [&](bool hit, int p, float res, float dk) {
        if (hit) list_at(so, p, pix_key(res, dk));
      });
    }
  }
}

// lexicographic comparison of two objects' hit tuples (original hit indices of their MDs)
__device__ __forceinline__ bool pix_tuple_less(const EvDesc &ev, int stage, int a, int b) {
  int ma[5], mb[5];
  int nm;
  if (stage == 5) {
    const int4 a1 = ev.t5_a[a], b1 = ev.t5_a[b];
    ma[0] = a1.x; ma[1] = a1.y; ma[2] = a1.z; ma[3] = a1.w; ma[4] = ev.t5_b[a].x;
    mb[0] = b1.x; mb[1] = b1.y; mb[2] = b1.z; mb[3] = b1.w; mb[4] = ev.t5_b[b].x;
    nm = 5;
  } else {
    const int4 a1 = ev.t3_md[a], b1 = ev.t3_md[b];
    ma[0] = a1.x; ma[1] = a1.y; ma[2] = a1.z;
    mb[0] = b1.x; mb[1] = b1.y; mb[2] = b1.z;
    nm = 3;
  }
  for (int i = 0; i < nm; i++) {
    const int2 ha = ev.md_hits[ma[i]], hb = ev.md_hits[mb[i]];
    if (ha.x != hb.x) return ha.x < hb.x;
    if (ha.y != hb.y) return ha.y < hb.y;
  }
  return false;
}

// Round, part 3: each seed's choice among the objects of its best rank: the smallest hit tuple.
__global__ void k_pix_pick(const EvDesc *__restrict__ evs, const PixDesc *Ps, int stage) {
  const EvDesc &ev = evs[blockIdx.y];
  const PixDesc &P = Ps[blockIdx.y];
  if (P.ctr[PIX_DONE]) return;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P.n_pls; p += gridDim.x * blockDim.x) {
    const int n = min(P.pcnt[p], PIX_TIES);
    if (n == 0) continue;
    int best = P.plist[PIX_TIES * (size_t)p];
    for (int i = 1; i < n; i++) {
      const int o = P.plist[PIX_TIES * (size_t)p + i];
      if (pix_tuple_less(ev, stage, o, best)) best = o;
    }
    P.pobj[p] = best;
  }
}

// Round, part 4: take the pairs that chose each other; clear the round's seed state.
__global__ void k_pix_accept(const PixDesc *Ps, int stage) {
  const PixDesc &P = Ps[blockIdx.y];
  if (P.ctr[PIX_DONE]) return;
  const int n = stage == 5 ? P.n_t5 : P.n_t3, base = stage == 5 ? 0 : P.n_t5;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n; o += gridDim.x * blockDim.x) {
    const int p = P.op[base + o];
    if (p >= 0 && P.pobj[p] == o) {
      P.omatch[base + o] = p;
      P.pmatch[p] = base + o;
      atomicAdd(P.ctr, 1);
    }
  }
}
__global__ void k_pix_clear(const PixDesc *Ps) {
  const PixDesc &P = Ps[blockIdx.y];
  if (P.ctr[PIX_DONE]) return;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P.n_pls; p += gridDim.x * blockDim.x) {
    P.pkey[p] = ~0ull;
    P.pcnt[p] = 0;
    P.pobj[p] = -1;
  }
}

// MDs of the pT5 quintuplets
__global__ void k_pix_mark(const EvDesc *__restrict__ evs, const PixDesc *Ps) {
  const EvDesc &ev = evs[blockIdx.y];
  const PixDesc &P = Ps[blockIdx.y];
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < P.n_t5; o += gridDim.x * blockDim.x) {
    if (P.omatch[o] < 0) continue;
    const int4 a = ev.t5_a[o];
    P.mdflag[a.x] = 1; P.mdflag[a.y] = 1; P.mdflag[a.z] = 1; P.mdflag[a.w] = 1;
    P.mdflag[ev.t5_b[o].x] = 1;
  }
}

// Track candidates as rows (type, seed, object): 5 pT5, 6 T5 without a seed, 7 pT3, 8 pLS.
__global__ void k_pix_rows(const EvDesc *__restrict__ evs, const PixDesc *Ps) {
  const EvDesc &ev = evs[blockIdx.y];
  const PixDesc &P = Ps[blockIdx.y];
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
  auto emit = [&](int t, int p, int o) {
    const int r = atomicAdd(P.ctr + 1, 1);
    atomicAdd(P.ctr + t - 1, 1);
    P.rows[3 * (size_t)r] = t;
    P.rows[3 * (size_t)r + 1] = p;
    P.rows[3 * (size_t)r + 2] = o;
  };
  for (int o = tid; o < P.n_t5; o += st)
    if (ev.t5_tc[o]) emit(P.omatch[o] >= 0 ? 5 : 6, max(P.omatch[o], -1), o);
  for (int u = tid; u < P.n_t3; u += st)
    if (P.omatch[P.n_t5 + u] >= 0) emit(7, P.omatch[P.n_t5 + u], u);
  for (int p = tid; p < P.n_pls; p += st)
    if (P.pmatch[p] < 0) emit(8, p, -1);
}

// Stage bookkeeping per event (a thread per event): at the start of a stage an event takes
// part unless it has no seeds or no objects of the stage; after each round an event whose
// round took no pair is done with the stage (a further round would find the same), and
// flags[e] reports done (1) and a tie-list overflow (2) to the host.
__global__ void k_pix_stage_begin(const PixDesc *Ps, int n_events, int stage) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_events; e += gridDim.x * blockDim.x) {
    const PixDesc &P = Ps[e];
    P.ctr[0] = 0;
    P.ctr[PIX_DONE] = P.n_pls == 0 || (stage == 5 ? P.n_t5 : P.n_t3) == 0;
  }
}
__global__ void k_pix_round_end(const PixDesc *Ps, int n_events, int stage, int *flags) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_events; e += gridDim.x * blockDim.x) {
    const PixDesc &P = Ps[e];
    if (!P.ctr[PIX_DONE]) {
      P.ctr[stage == 5 ? PIX_ROUNDS5 : PIX_ROUNDS7]++;
      if (P.ctr[0] == 0) P.ctr[PIX_DONE] = 1;
      P.ctr[0] = 0;
    }
    flags[e] = (P.ctr[PIX_DONE] ? 1 : 0) | (P.ctr[2] ? 2 : 0);
  }
}

// Host-side launch helpers for n events (all on `st`, grid x `grid` per event); rounds are
// driven by the caller.
cudaError_t pix_launch_bin(const PixDesc *Ps, int n, bool any_seeds, int grid, cudaStream_t st) {
  if (any_seeds) k_pix_bin<<<dim3(grid, n), 256, 0, st>>>(Ps, 0);
  k_pix_scan<<<dim3(1, n), 1024, 0, st>>>(Ps);
  if (any_seeds) k_pix_scatter<<<dim3(grid, n), 256, 0, st>>>(Ps, 0);
  return cudaGetLastError();
}
cudaError_t pix_launch_rebin(const PixDesc *Ps, int n, bool any_seeds, int grid, cudaStream_t st) {
  if (!any_seeds) return cudaSuccess;
  k_pix_rebin_clear<<<dim3(grid, n), 256, 0, st>>>(Ps);
  k_pix_bin<<<dim3(grid, n), 256, 0, st>>>(Ps, 1);
  k_pix_scan<<<dim3(1, n), 1024, 0, st>>>(Ps);
  k_pix_scatter<<<dim3(grid, n), 256, 0, st>>>(Ps, 1);
  return cudaGetLastError();
}
cudaError_t pix_launch_stage_begin(const PixDesc *Ps, int n, int stage, cudaStream_t st) {
  k_pix_stage_begin<<<(n + 255) / 256, 256, 0, st>>>(Ps, n, stage);
  return cudaGetLastError();
}
cudaError_t pix_launch_round(const EvDesc *dd, const PixDesc *Ps, int n, int stage, lst_pixel_cuts pc, int grid,
                             int *flags, cudaStream_t st) {
  k_pix_propose<<<dim3(4 * grid, n), PIX_SCAN_THREADS, 0, st>>>(dd, Ps, stage, pc);
  k_pix_ties<<<dim3(4 * grid, n), PIX_SCAN_THREADS, 0, st>>>(dd, Ps, stage, pc);
  k_pix_pick<<<dim3(grid, n), 256, 0, st>>>(dd, Ps, stage);
  k_pix_accept<<<dim3(grid, n), 256, 0, st>>>(Ps, stage);
  k_pix_clear<<<dim3(grid, n), 256, 0, st>>>(Ps);
  k_pix_round_end<<<(n + 255) / 256, 256, 0, st>>>(Ps, n, stage, flags);
  return cudaGetLastError();
}
cudaError_t pix_launch_mark(const EvDesc *dd, const PixDesc *Ps, int n, int grid, cudaStream_t st) {
  k_pix_mark<<<dim3(grid, n), 256, 0, st>>>(dd, Ps);
  return cudaGetLastError();
}
cudaError_t pix_launch_rows(const EvDesc *dd, const PixDesc *Ps, int n, int grid, cudaStream_t st) {
  k_pix_rows<<<dim3(grid, n), 256, 0, st>>>(dd, Ps);
  return cudaGetLastError();
}

}  // namespace lstk
