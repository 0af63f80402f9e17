// lst_features.cuh -- the 38 T5-DNN input features of a quintuplet (arXiv 2403.13166,
// Section 2), shared by the FP32 and the tensor-core score kernels.
#pragma once
#include "lst_ff.cuh"

namespace lstk {

constexpr float KAPPA_FLOOR = 1e-7f;   // radii above 1e7 cm count as 1e7 cm in the log features
constexpr float INV_PI = 0.318309886183790672f;

// Section 2: for each of the 5 MDs the anchor hit's r, phi, z, eta, layer (+ the MD's
// curvature estimate), the pT and radius of each T3's circle, the T5's pT, eta and phi,
// and the radius of the bridge T3 (middle three MDs).
__device__ __forceinline__ void t5_features(const EvDesc &ev, const DevGeom &g, int t, float k_field, float *f) {
  const int4 a = ev.t5_a[t], b = ev.t5_b[t];
  const int md[5] = {a.x, a.y, a.z, a.w, b.x};
  float4 P[5];
#pragma unroll
  for (int i = 0; i < 5; i++) {
    P[i] = ev.md_anchor[md[i]];
    const float r = P[i].w;
    f[6 * i + 0] = r * 0.01f;
    f[6 * i + 1] = atan2f(P[i].y, P[i].x) * INV_PI;
    f[6 * i + 2] = P[i].z * 0.01f;
    f[6 * i + 3] = asinhf(P[i].z / r) * 0.4f;
    f[6 * i + 4] = (float)g.layer[ev.md_mod[md[i]]] / 11.0f;
    f[6 * i + 5] = 100.0f * ev.md_kappa[md[i]].y;
  }
  const float ka = curv3_acc(P[0], P[1], P[2]);
  const float kb = curv3_acc(P[2], P[3], P[4]);
  const float la = log10f(fmaxf(fabsf(ka), KAPPA_FLOOR));
  const float lb = log10f(fmaxf(fabsf(kb), KAPPA_FLOOR));
  const float lk = log10f(k_field);
  f[30] = lk - la;
  f[31] = -la;
  f[32] = lk - lb;
  f[33] = -lb;
  const float k5 = curv3_acc(P[0], P[2], P[4]);
  f[34] = lk - log10f(fmaxf(fabsf(k5), KAPPA_FLOOR));
  const float kbar = 0.5f * (ka + kb);
  float S4 = 0.0f;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const ff dx = two_diff(P[i + 1].x, P[i].x), dy = two_diff(P[i + 1].y, P[i].y);
    const float d = sqrtf(dx.hi * dx.hi + dy.hi * dy.hi);
    S4 += d * (1.0f + d * d * kbar * kbar * (1.0f / 24.0f));
  }
  const ff dz = two_diff(P[4].z, P[0].z);
  f[35] = asinhf(dz.hi / S4) * 0.4f;
  const ff ex = two_diff(P[4].x, P[0].x), ey = two_diff(P[4].y, P[0].y);
  f[36] = atan2f(ey.hi, ex.hi) * INV_PI;
  const float kbr = curv3_acc(P[1], P[2], P[3]);
  f[37] = -log10f(fmaxf(fabsf(kbr), KAPPA_FLOOR));
}


// The same 38 features in float-float (hi + lo), for the FP32 score path: every feature
// within about 1e-9 of its exact value given the FP32 hit coordinates, the azimuths (to
// which the networks are insensitive) excepted, which keep the FP32 form above. Same
// definitions and operation order as above; the MD curvature estimate is recomputed from
// the MD's two hits instead of read back as a float.
__device__ __forceinline__ ff curv3_ff(const float4 P0, const float4 P1, const float4 P2) {
  const ff ax = two_diff(P1.x, P0.x), ay = two_diff(P1.y, P0.y);
  const ff bx = two_diff(P2.x, P1.x), by = two_diff(P2.y, P1.y);
  const ff cx = two_diff(P2.x, P0.x), cy = two_diff(P2.y, P0.y);
  const ff cr = ff_sub(ff_mul(ax, cy), ff_mul(ay, cx));
  const ff abc = ff_mul(ff_mul(ff_sqrt(ff_norm2(ax, ay)), ff_sqrt(ff_norm2(bx, by))), ff_sqrt(ff_norm2(cx, cy)));
  return ff_div(ff_mulf(cr, 2.0f), abc);
}
// log10 max(|k|, 1e-7), the floor as the float-float nearest to 1e-7
__device__ __forceinline__ ff log10_kabs_ff(ff k) {
  const ff floor7 = {1e-7f, -1.1686097e-15f};
  const ff a = ff_abs(k);
  return ff_log10(ff_lt(a, floor7) || !(a.hi == a.hi) ? floor7 : a);
}
static __device__ __noinline__ void t5_features_ff(const EvDesc &ev, const DevGeom &g, int t, float k_field, float *fh,
                                            float *fl) {
  const int4 a = ev.t5_a[t], b = ev.t5_b[t];
  const int md[5] = {a.x, a.y, a.z, a.w, b.x};
  float4 P[5];
  auto put = [&](int j, ff v) {
    fh[j] = v.hi;
    fl[j] = v.lo;
  };
#pragma unroll 1
  for (int i = 0; i < 5; i++) {
    P[i] = ev.md_anchor[md[i]];
    const ff r = ff_sqrt(ff_add(two_prod(P[i].x, P[i].x), two_prod(P[i].y, P[i].y)));
    put(6 * i + 0, ff_divf(r, 100.0f));
    put(6 * i + 1, ff_make(atan2f(P[i].y, P[i].x) * INV_PI));
    put(6 * i + 2, ff_divf(ff_make(P[i].z), 100.0f));
    put(6 * i + 3, ff_divf(ff_asinh(ff_div(ff_make(P[i].z), r)), 2.5f));
    const int mod = ev.md_mod[md[i]];
    put(6 * i + 4, ff_divf(ff_make((float)g.layer[mod]), 11.0f));
    ff mk = {0.0f, 0.0f};
    if (g.subdet[mod] == 0) {
      // 2 sin(angle(L, U - L)) / rL of the MD's lower and upper hits
      const int2 h = ev.md_hits[md[i]];
      const float lx = ev.x[h.x], ly = ev.y[h.x];
      const ff dx = two_diff(ev.x[h.y], lx), dy = two_diff(ev.y[h.y], ly);
      const ff dT = ff_sqrt(ff_norm2(dx, dy));
      const ff rL = ff_sqrt(ff_add(two_prod(lx, lx), two_prod(ly, ly)));
      const ff cr = ff_sub(ff_mulf(dy, lx), ff_mulf(dx, ly));
      mk = ff_div(ff_mulf(ff_div(cr, ff_mul(rL, dT)), 2.0f), rL);
    }
    put(6 * i + 5, ff_mulf(mk, 100.0f));
  }
  const ff ka = curv3_ff(P[0], P[1], P[2]);
  const ff kb = curv3_ff(P[2], P[3], P[4]);
  const ff la = log10_kabs_ff(ka), lb = log10_kabs_ff(kb);
  const ff lk = ff_log10(ff_make(k_field));
  put(30, ff_sub(lk, la));
  put(31, ff_neg(la));
  put(32, ff_sub(lk, lb));
  put(33, ff_neg(lb));
  put(34, ff_sub(lk, log10_kabs_ff(curv3_ff(P[0], P[2], P[4]))));
  const ff kbar = ff_mulf(ff_add(ka, kb), 0.5f);
  const ff kbar2 = ff_mul(kbar, kbar);
  ff S4 = {0.0f, 0.0f};
#pragma unroll 1
  for (int i = 0; i < 4; i++) {
    const ff dx = two_diff(P[i + 1].x, P[i].x), dy = two_diff(P[i + 1].y, P[i].y);
    const ff d2 = ff_norm2(dx, dy);
    const ff d = ff_sqrt(d2);
    S4 = ff_add(S4, ff_mul(d, ff_add(ff_make(1.0f), ff_divf(ff_mul(d2, kbar2), 24.0f))));
  }
  put(35, ff_divf(ff_asinh(ff_div(two_diff(P[4].z, P[0].z), S4)), 2.5f));
  const ff ex = two_diff(P[4].x, P[0].x), ey = two_diff(P[4].y, P[0].y);
  put(36, ff_make(atan2f(ey.hi, ex.hi) * INV_PI));
  put(37, ff_neg(log10_kabs_ff(curv3_ff(P[1], P[2], P[3]))));
}

}  // namespace lstk
