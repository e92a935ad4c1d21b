// Strip-point interpolation (Section 3.4), shared by k_interp and the row DFT kernel that
// assembles the extension with the strip values computed in place:
//   value = sum_a wth[a] sum_b weta[b] F[(pb + a) mod B][s + b],
// with the weights, the first normal pb and the first fine node s of each strip point
// precomputed at plan time (k_interp_weights).  MM > 0: compile-time M.  VEC (float F,
// ldF a multiple of 4, ldF >= Cr + 12, F 16-byte aligned): the M values s..s+M-1 of a
// normal come from the three aligned float4 at s & ~3, weighted by the eta weights
// shifted once by s & 3 into a 12-entry window.
#pragma once
#include "fc2d_kernels.cuh"
#include "plan_internal.h"

#if defined(__CUDACC__)
namespace fc2d {

template <int MM, typename TW>
struct InterpPoint {
  TW eta[MM > 0 ? MM : kMaxM];
  TW th[MM > 0 ? MM : kMaxM];
  int pb, s;
};

// The weights and indices of strip point n (plan constants).
template <int MM, typename TW>
__device__ __forceinline__ InterpPoint<MM, TW> interp_load(const InterpArgs& a, int n) {
  InterpPoint<MM, TW> q;
  const int M = MM > 0 ? MM : a.M, ns = a.n_strip;
  const TW* w = reinterpret_cast<const TW*>(a.w);
  q.pb = __ldg(a.pb + n);
  q.s = __ldg(a.sb + n);
#pragma unroll
  for (int b = 0; b < (MM > 0 ? MM : kMaxM); ++b) {
    if (b < M) q.eta[b] = __ldg(w + (size_t)(M + b) * ns + n);
    if (b < M) q.th[b] = __ldg(w + (size_t)b * ns + n);
  }
  return q;
}

// The value of a strip point from the strip values Ff of one function ([B][ldF]); Ff
// may be global or shared memory (plain loads).  WRAP false: the M normals pb .. pb+M-1
// lie inside Ff without the cyclic wrap (a CTA's local tile), so its rows are one base
// pointer plus multiples of ldF.
template <int MM, typename TF, typename TW, typename TA, bool VEC, bool WRAP = true>
__device__ __forceinline__ TA interp_apply(const InterpArgs& a, const TF* __restrict__ Ff,
                                           const InterpPoint<MM, TW>& q) {
  const int M = MM > 0 ? MM : a.M;
  const int B = a.B, ld = a.ldF;
  TA acc = 0;
  if constexpr (VEC) {
    static_assert(MM > 0 && MM <= 9, "vector path needs a compile-time M <= 9");
    const int s0 = q.s & ~3, sh = q.s & 3;
    TA ws[12];
#pragma unroll
    for (int b = 0; b < 12; ++b) {
      const TA w0 = b < MM ? (TA)q.eta[b] : (TA)0;
      const TA w1 = (b >= 1 && b - 1 < MM) ? (TA)q.eta[b >= 1 ? b - 1 : 0] : (TA)0;
      const TA w2 = (b >= 2 && b - 2 < MM) ? (TA)q.eta[b >= 2 ? b - 2 : 0] : (TA)0;
      const TA w3 = (b >= 3 && b - 3 < MM) ? (TA)q.eta[b >= 3 ? b - 3 : 0] : (TA)0;
      ws[b] = sh == 0 ? w0 : sh == 1 ? w1 : sh == 2 ? w2 : w3;
    }
    const TF* row0 = Ff + q.pb * ld + s0;  // used without the wrap
#pragma unroll
    for (int ai = 0; ai < MM; ++ai) {
      int pr = q.pb + ai;
      pr = pr < 0 ? pr + B : (pr >= B ? pr - B : pr);
      const float4* row = reinterpret_cast<const float4*>(
          WRAP ? Ff + (size_t)pr * ld + s0 : row0 + ai * ld);
      TA v = 0;
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const float4 x = row[u];
        v = fma(ws[4 * u], (TA)x.x, v);
        v = fma(ws[4 * u + 1], (TA)x.y, v);
        v = fma(ws[4 * u + 2], (TA)x.z, v);
        v = fma(ws[4 * u + 3], (TA)x.w, v);
      }
      acc = fma((TA)q.th[ai], v, acc);
    }
  } else {
#pragma unroll
    for (int ai = 0; ai < (MM > 0 ? MM : kMaxM); ++ai) {
      if (ai >= M) break;
      int pr = q.pb + ai;
      pr = pr < 0 ? pr + B : (pr >= B ? pr - B : pr);
      const TF* row = Ff + (size_t)pr * ld + q.s;
      TA v = 0;
#pragma unroll
      for (int b = 0; b < (MM > 0 ? MM : kMaxM); ++b)
        if (b < M) v = fma((TA)q.eta[b], (TA)row[b], v);
      acc = fma((TA)q.th[ai], v, acc);
    }
  }
  return acc;
}

}  // namespace fc2d
#endif
