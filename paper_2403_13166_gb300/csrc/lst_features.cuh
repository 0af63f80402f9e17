// lst_features.cuh -- the 38 T5-DNN input features of a quintuplet (arXiv 2403.13166,
// Section 2), shared by the FP32 and the tensor-core score kernels.
#pragma once
#include "lst_internal.cuh"

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

}  // namespace lstk
