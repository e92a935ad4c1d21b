// Power-of-two DFT kernels (eq. (3.1)): compile-time radix, one shared buffer.
//
// A transform of N = 2^LOGN complex points is done by NT = N/E threads, each holding
// E complex values in registers (E = 16 for float, 8 for double).  Every Stockham
// stage (radix R dividing E; R = E except a smaller last stage) is:
//   read the thread's E inputs x[j + r N/R] from shared memory, barrier,
//   twiddle by exp(-2 pi i r (j mod Ns)/(Ns R)) (table lookups), length-R DFT,
//   write y[(j/Ns) Ns R + (j mod Ns) + r Ns], barrier,
// so one buffer of N values suffices.  Shared indices are padded by one element per
// E to break the bank conflicts of the strided first-stage writes.
//
// k_fft_rows_p2: one block per (row, function): the extension row (fused load from
// f and the strip values, or a plain grid row) as nx/2 complex pairs, the length-nx/2
// transform, the even/odd split to X_k, k = 0..nx/2, written to the intermediate.
// k_fft_cols_p2: one block per (CB columns, function): length-ny column transforms,
// scaled by 1/(nx ny), written to the half spectrum [ny][nx/2+1].
#include <cuda.h>  // CUtensorMap and its enums (the encoder is reached through the runtime)
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "fc2d_kernels.cuh"
#include "plan_internal.h"

namespace fc2d {
namespace p2 {

template <typename T> struct Cx;
template <> struct Cx<double> { using type = double2; };
template <> struct Cx<float> { using type = float2; };

template <typename C> __device__ __forceinline__ C add(C a, C b) { return {a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C sub(C a, C b) { return {a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C mul(C a, C b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C> __device__ __forceinline__ C mul_mi(C a) { return {a.y, -a.x}; }

// L2 residency hints (PTX eviction priorities; no value changes).  The grid values f
// are read once per call: they bypass L1 and go first when L2 evicts, so that the row
// transforms' output (the intermediate, read again by both column passes) stays in L2.
// The intermediate's stores ask L2 to keep their lines; the spectrum, written once,
// asks it to evict its lines first.  Bits: 1 f loads, 2 intermediate stores, 4 spectrum
// stores.
#ifndef FC2D_L2_HINTS
#define FC2D_L2_HINTS 1
#endif
__device__ __forceinline__ uint64_t l2_keep() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t l2_drop() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ double2 ld_stream(const double2* p, uint64_t pol) {
#if FC2D_L2_HINTS & 1
  double2 v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
      : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol));
  return v;
#else
  return __ldg(p);
#endif
}
// store with an L2 policy (FP32 complex); other types store plainly
template <int BIT, typename C> __device__ __forceinline__ void st_hint(C* p, C v, uint64_t pol) {
  if constexpr (sizeof(C) == 8 && (FC2D_L2_HINTS & BIT)) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;"
                 ::"l"(p), "f"(v.x), "f"(v.y), "l"(pol) : "memory");
  } else {
    *p = v;
  }
}

// exp(-2 pi i m/16), m = 0..15
template <typename T, typename C>
__device__ __forceinline__ C w16(int m) {
  const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;
  const T h = (T)0.70710678118654752440;
  switch (m & 15) {
    case 0: return C{(T)1, (T)0};
    case 1: return C{c1, -s1};
    case 2: return C{h, -h};
    case 3: return C{s1, -c1};
    case 4: return C{(T)0, (T)-1};
    case 5: return C{-s1, -c1};
    case 6: return C{-h, -h};
    case 7: return C{-c1, -s1};
    case 8: return C{(T)-1, (T)0};
    case 9: return C{-c1, s1};
    case 10: return C{-h, h};
    case 11: return C{-s1, c1};
    case 12: return C{(T)0, (T)1};
    case 13: return C{s1, c1};
    case 14: return C{h, h};
    default: return C{c1, s1};
  }
}

template <typename C> __device__ __forceinline__ void dft2(C* v) {
  C a = v[0], b = v[1];
  v[0] = add(a, b);
  v[1] = sub(a, b);
}

template <typename C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
  C t0 = add(a0, a2), t1 = sub(a0, a2), t2 = add(a1, a3), t3 = mul_mi(sub(a1, a3));
  a0 = add(t0, t2);
  a2 = sub(t0, t2);
  a1 = add(t1, t3);
  a3 = sub(t1, t3);
}

template <typename T, typename C> __device__ __forceinline__ void dft8(C* v) {
  const T s = (T)0.70710678118654752440;
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4(e0, e1, e2, e3);
  dft4(o0, o1, o2, o3);
  C w1 = {s * (o1.x + o1.y), s * (o1.y - o1.x)};
  C w2 = mul_mi(o2);
  C w3 = {s * (o3.y - o3.x), -s * (o3.x + o3.y)};
  v[0] = add(e0, o0);
  v[4] = sub(e0, o0);
  v[1] = add(e1, w1);
  v[5] = sub(e1, w1);
  v[2] = add(e2, w2);
  v[6] = sub(e2, w2);
  v[3] = add(e3, w3);
  v[7] = sub(e3, w3);
}

// 16-point DFT as 4 x 4: inner DFT4 over n1 for each n2, twiddle w16^(n2 k1), outer
// DFT4 over n2; X[k1 + 4 k2] lands in v[k1 + 4 k2].
template <typename T, typename C> __device__ __forceinline__ void dft16(C* v) {
  C a[16];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    C x0 = v[n2], x1 = v[4 + n2], x2 = v[8 + n2], x3 = v[12 + n2];
    dft4(x0, x1, x2, x3);  // x_k1 = sum_n1 v[4 n1 + n2] w4^(n1 k1)
    a[4 * n2 + 0] = x0;
    a[4 * n2 + 1] = n2 ? mul(x1, w16<T, C>(n2)) : x1;
    a[4 * n2 + 2] = n2 ? mul(x2, w16<T, C>(2 * n2)) : x2;
    a[4 * n2 + 3] = n2 ? mul(x3, w16<T, C>(3 * n2)) : x3;
  }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C y0 = a[k1], y1 = a[4 + k1], y2 = a[8 + k1], y3 = a[12 + k1];
    dft4(y0, y1, y2, y3);
    v[k1] = y0;
    v[k1 + 4] = y1;
    v[k1 + 8] = y2;
    v[k1 + 12] = y3;
  }
}

template <typename T, typename C> __device__ __forceinline__ void dft3(C* v) {
  const T c1 = (T)-0.5, s1 = (T)0.86602540378443864676;  // exp(-2 pi i/3) = c1 - i s1
  const C a = v[0], sbc = add(v[1], v[2]), dbc = sub(v[1], v[2]);
  v[0] = add(a, sbc);
  const C m = {a.x + c1 * sbc.x, a.y + c1 * sbc.y};
  const C r = {s1 * dbc.y, -s1 * dbc.x};  // -i s1 (b - c)
  v[1] = add(m, r);
  v[2] = sub(m, r);
}

template <typename T, typename C> __device__ __forceinline__ void dft5(C* v) {
  const T c1 = (T)0.30901699437494742410, s1 = (T)0.95105651629515357212;  // 2 pi/5
  const T c2 = (T)-0.80901699437494742410, s2 = (T)0.58778525229247312917;  // 4 pi/5
  const C a = v[0];
  const C s14 = add(v[1], v[4]), d14 = sub(v[1], v[4]);
  const C s23 = add(v[2], v[3]), d23 = sub(v[2], v[3]);
  v[0] = add(a, add(s14, s23));
  const C m1 = {a.x + c1 * s14.x + c2 * s23.x, a.y + c1 * s14.y + c2 * s23.y};
  const C m2 = {a.x + c2 * s14.x + c1 * s23.x, a.y + c2 * s14.y + c1 * s23.y};
  const C r1 = {s1 * d14.y + s2 * d23.y, -(s1 * d14.x + s2 * d23.x)};
  const C r2 = {s2 * d14.y - s1 * d23.y, -(s2 * d14.x - s1 * d23.x)};
  v[1] = add(m1, r1);
  v[4] = sub(m1, r1);
  v[2] = add(m2, r2);
  v[3] = sub(m2, r2);
}

template <typename T, typename C, int R> __device__ __forceinline__ void dft(C* v) {
  if constexpr (R == 2) dft2(v);
  else if constexpr (R == 3) dft3<T, C>(v);
  else if constexpr (R == 5) dft5<T, C>(v);
  else if constexpr (R == 4) dft4(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) dft8<T, C>(v);
  else dft16<T, C>(v);
}

// Length R1 R2 DFT in registers (Cooley-Tukey, n = R2 n1 + n2, k = k1 + R1 k2):
// R2 DFTs of length R1, the twiddles w_{R1 R2}^(n2 k1) (wt[t * ws] = w_{R1 R2}^t), R1
// DFTs of length R2.  x holds the input in natural order and receives the output.
template <int R1, int R2>
__device__ __forceinline__ void dft_ct(float2* x, const float2* __restrict__ wt, int ws) {
  float2 a[R1 * R2];
#pragma unroll
  for (int n2 = 0; n2 < R2; ++n2) {
    float2 v[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) v[n1] = x[R2 * n1 + n2];
    dft<float, float2, R1>(v);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1)
      a[n2 * R1 + k1] = (n2 * k1) ? mul(v[k1], __ldg(wt + (n2 * k1) * ws)) : v[k1];
  }
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) {
    float2 u[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) u[n2] = a[n2 * R1 + k1];
    dft<float, float2, R2>(u);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) x[k1 + R1 * k2] = u[k2];
  }
}

// Round-to-nearest-even double -> float on the integer pipe (the FP64 pipe that the
// conversion instruction uses is narrow on this part), for doubles whose exponent e lies
// in [897, 1148] (float exponents 1..252, so no overflow even after rounding up): add
// 2^28 - 1 plus bit 29 to the 64-bit pattern (round half to even at bit 29; a mantissa
// carry moves into the exponent), keep bits 29..60 (e's low 9 bits over the top 23
// mantissa bits), rebase the exponent by 896 (mod 2^32) and put the sign back.  Other
// values (zero, subnormal, huge, inf, NaN) take the hardware conversion.
__device__ __forceinline__ bool d2f_in_range(unsigned hi) {
  return (hi & 0x7FF00000u) - (897u << 20) <= (251u << 20);
}
__device__ __forceinline__ float d2f_in(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned long long u = b + 0x0FFFFFFFull + ((b >> 29) & 1ull);
  const unsigned r = (unsigned)(u >> 29) - (896u << 23);
  return __uint_as_float(r | ((unsigned)(b >> 32) & 0x80000000u));
}
__device__ __forceinline__ float d2f_rn(double x) {
  return d2f_in_range((unsigned)__double2hiint(x)) ? d2f_in(x) : __double2float_rn(x);
}
// both values of a pair, one range test
__device__ __forceinline__ float2 d2f2_rn(double2 v) {
  if (d2f_in_range((unsigned)__double2hiint(v.x)) && d2f_in_range((unsigned)__double2hiint(v.y)))
    return float2{d2f_in(v.x), d2f_in(v.y)};
  return float2{__double2float_rn(v.x), __double2float_rn(v.y)};
}
template <typename T> __device__ __forceinline__ T from_double(double x) { return (T)x; }
template <> __device__ __forceinline__ float from_double<float>(double x) { return d2f_rn(x); }

// One pad element per E = elems<T>() elements: the first stage writes at stride E
// (index E j + r), which the pad spreads over all banks; the other stages access
// contiguous runs of the thread index, which the pad leaves contiguous.
template <typename T> __host__ __device__ constexpr int pad_shift() { return sizeof(T) == 4 ? 4 : 3; }
template <typename T> __device__ __forceinline__ int pad(int i) { return i + (i >> pad_shift<T>()); }
template <typename T> __host__ __device__ constexpr int padded(int n) { return n + (n >> pad_shift<T>()); }
// pad(i + r S) for r = 0..R-1 as pad(i) plus a compile-time offset, which the shared
// memory instructions take as an immediate: exact when S is a multiple of the pad unit
// U (then pad(i + r S) = pad(i) + r (S + S / U)), or when S = 1, R divides U and i is a
// multiple of R (then i and i + R - 1 lie in one unit).
template <typename T, int S, int R> __host__ __device__ constexpr bool pad_affine() {
  return S % (1 << pad_shift<T>()) == 0 || (S == 1 && (1 << pad_shift<T>()) % R == 0);
}
template <typename T, int S> __host__ __device__ constexpr int pad_step() {
  return S % (1 << pad_shift<T>()) == 0 ? S + S / (1 << pad_shift<T>()) : S;
}

// Offset of the twiddle block of the stage with sub-transform length NS in the
// per-stage table (blocks of R x NS entries for every stage with NS > 1, in order).
__host__ __device__ constexpr int stage_off(int N, int E, int NS) {
  int off = 0, ns = 1;
  while (ns < NS) {
    const int R = (N / ns >= E) ? E : N / ns;
    if (ns > 1) off += R * ns;
    ns *= R;
  }
  return off;
}

// One Stockham stage of radix R on buffer `buf` (padded), NT threads, butterflies
// j = t + m NT, m < E/R.  Ns = product of the earlier radices.
template <typename T, int LOGN, int E, int R, int NS>
__device__ __forceinline__ void stage(typename Cx<T>::type* buf, int t, bool active,
                                      const typename Cx<T>::type* __restrict__ tw, int tws) {
  using C = typename Cx<T>::type;
  constexpr int N = 1 << LOGN;
  constexpr int NT = N / E;
  constexpr int NR = N / R;
  constexpr int M = E / R;
  C v[E];
  if (active) {
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const int j = t + m * NT;
      if constexpr (NR % (1 << pad_shift<T>()) == 0) {
        const C* src = buf + pad<T>(j);
#pragma unroll
        for (int r = 0; r < R; ++r) v[m * R + r] = src[r * pad_step<T, NR>()];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) v[m * R + r] = buf[pad<T>(j + r * NR)];
      }
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int j = t + m * NT;
    const int k = j & (NS - 1);
    if (NS > 1) {
      constexpr int OFF = stage_off(N, E, NS);
#pragma unroll
      for (int r = 1; r < R; ++r) v[m * R + r] = mul(v[m * R + r], __ldg(tw + OFF + r * NS + k));
    }
    dft<T, C, R>(v + m * R);
    const int base = (j / NS) * NS * R + k;
    if constexpr (pad_affine<T, NS, R>()) {
      C* dst = buf + pad<T>(base);
#pragma unroll
      for (int r = 0; r < R; ++r) dst[r * pad_step<T, NS>()] = v[m * R + r];
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) buf[pad<T>(base + r * NS)] = v[m * R + r];
    }
  }
  }
  __syncthreads();
}

// Whole transform of N = 2^LOGN points in buf (padded), threads t < NT = N/E.
// Threads with active == false take part in the barriers only.
template <typename T, int LOGN, int E, int NS = 1>
__device__ __forceinline__ void block_fft(typename Cx<T>::type* buf, int t, bool active,
                                          const typename Cx<T>::type* __restrict__ tw, int tws) {
  constexpr int N = 1 << LOGN;
  if constexpr (NS < N) {
    constexpr int R = (N / NS >= E) ? E : N / NS;
    stage<T, LOGN, E, R, NS>(buf, t, active, tw, tws);
    block_fft<T, LOGN, E, NS * R>(buf, t, active, tw, tws);
  }
}

// All stages but the last one (the stages of block_fft with NS * R < N).
template <typename T, int LOGN, int E, int NS = 1>
__device__ __forceinline__ void block_fft_head(typename Cx<T>::type* buf, int t, bool active,
                                               const typename Cx<T>::type* __restrict__ tw,
                                               int tws) {
  constexpr int N = 1 << LOGN;
  constexpr int R = (N / NS >= E) ? E : N / NS;
  if constexpr (NS * R < N) {
    stage<T, LOGN, E, R, NS>(buf, t, active, tw, tws);
    block_fft_head<T, LOGN, E, NS * R>(buf, t, active, tw, tws);
  }
}

// Sub-transform length NS of the last stage of block_fft.
template <int LOGN, int E> __host__ __device__ constexpr int last_ns() {
  int ns = 1;
  while (true) {
    const int R = ((1 << LOGN) / ns >= E) ? E : (1 << LOGN) / ns;
    if (ns * R == (1 << LOGN)) return ns;
    ns *= R;
  }
}

// The real row's spectrum from the complex transform Z of its pairs (as
// even_odd_split; FP32 only: rtw is followed by its halved copy), with the last
// Stockham stage done in registers: thread t takes the
// butterflies j = t and j = NS - t (thread 0: 0 and NS/2), whose outputs are Z_k,
// k = j + NS r, and their partners Z_{NH-k}, so the split needs no exchange.  Needs
// NS = 2 NT (true for nx/2 = 2048 with E = 16 or 8).  buf holds the input of the last
// stage; X_k, k = 0..NH, go to out.
template <typename T, int LOGN, int E>
__device__ __forceinline__ void last_stage_split(const typename Cx<T>::type* buf, int t,
                                                 const typename Cx<T>::type* __restrict__ tw,
                                                 const typename Cx<T>::type* __restrict__ rtw,
                                                 typename Cx<T>::type* __restrict__ out) {
  using C = typename Cx<T>::type;
  constexpr int N = 1 << LOGN, NS = last_ns<LOGN, E>(), R = N / NS;
  constexpr int OFF = stage_off(N, E, NS);
  static_assert(NS == 2 * (N / E), "last_stage_split: NS must be twice the thread count");
  const int j1 = t, j2 = t ? NS - t : NS / 2;
  C a[R], b[R];
  static_assert(pad_affine<T, NS, R>() && NS > 1, "last_stage_split: NS a multiple of the pad unit");
  const C* s1 = buf + pad<T>(j1);
  const C* s2 = buf + pad<T>(j2);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    a[r] = s1[r * pad_step<T, NS>()];
    b[r] = s2[r * pad_step<T, NS>()];
  }
#pragma unroll
  for (int r = 1; r < R; ++r) {
    a[r] = mul(a[r], __ldg(tw + OFF + r * NS + j1));
    b[r] = mul(b[r], __ldg(tw + OFF + r * NS + j2));
  }
  dft<T, C, R>(a);
  dft<T, C, R>(b);
  // X_ks and X_kl (kl = NH - ks) from zk = Z_ks and zl = Z_kl: with e2 = 2e, o2 = 2o and
  // the halved table rtwh = rtw/2 (exact), w o = rtwh o2 and e = e2/2 enters through a
  // fused multiply-add: the same values as (e, o, rtw) with fewer instructions
  const C* rtwh = rtw + N + 1;
  const uint64_t pol = l2_keep();
  auto put = [&](int ks, int kl, C zk, C zl) {
    zl.y = -zl.y;
    const C e2 = {zk.x + zl.x, zk.y + zl.y};
    const C o2 = {zk.x - zl.x, zk.y - zl.y};
    const C wo = mul(__ldg(rtwh + ks), o2);
    st_hint<2>(out + ks, C{fma((T)0.5, e2.x, wo.y), fma((T)0.5, e2.y, -wo.x)}, pol);
    if (ks != kl) st_hint<2>(out + kl, C{fma((T)0.5, e2.x, -wo.y), fma((T)-0.5, e2.y, -wo.x)}, pol);
  };
  if (t) {
    // k = j1 + r NS and its partner N - k = j2 + (R - 1 - r) NS (never equal for t > 0),
    // addressed from four base pointers with compile-time offsets
    C* o_up = out + j1;
    C* o_dn = out + (N - j1);
    const C* w_up = rtwh + j1;
    const C* w_dn = rtwh + (N - j1);
    auto put2 = [&](C* ok, C* ol, const C* wk, C zk, C zl) {
      zl.y = -zl.y;
      const C e2 = {zk.x + zl.x, zk.y + zl.y};
      const C o2 = {zk.x - zl.x, zk.y - zl.y};
      const C wo = mul(__ldg(wk), o2);
      st_hint<2>(ok, C{fma((T)0.5, e2.x, wo.y), fma((T)0.5, e2.y, -wo.x)}, pol);
      st_hint<2>(ol, C{fma((T)0.5, e2.x, -wo.y), fma((T)-0.5, e2.y, -wo.x)}, pol);
    };
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r < R / 2) put2(o_up + r * NS, o_dn - r * NS, w_up + r * NS, a[r], b[R - 1 - r]);
      else put2(o_dn - r * NS, o_up + r * NS, w_dn - r * NS, b[R - 1 - r], a[r]);
    }
  } else {
    put(0, N, a[0], a[0]);
#pragma unroll
    for (int r = 1; r < R / 2; ++r) put(r * NS, N - r * NS, a[r], a[R - r]);
    put(N / 2, N / 2, a[R / 2], a[R / 2]);
#pragma unroll
    for (int r = 0; r < R / 2; ++r) put(NS / 2 + r * NS, N - NS / 2 - r * NS, b[r], b[R - 1 - r]);
  }
}

// lanes served by one shared-memory wavefront for complex values of type T
template <typename T> __host__ __device__ constexpr int col_lanes() { return sizeof(T) == 4 ? 16 : 8; }

// complex values per thread: 16 for float (radix-16 stages, three for 4096 points),
// 8 for double (register pressure of FP64 complex values)
template <typename T> __host__ __device__ constexpr int elems() { return sizeof(T) == 4 ? 16 : 8; }

// First stage (Ns = 1, radix R) straight from global memory: x[j + r N/R] at stride
// `stride`, length-R DFT, written to the shared buffer, then a barrier.
template <typename T, int LOGN, int E, int R>
__device__ __forceinline__ void stage_first_global(const typename Cx<T>::type* __restrict__ src,
                                                   size_t stride, typename Cx<T>::type* buf,
                                                   int t) {
  using C = typename Cx<T>::type;
  constexpr int N = 1 << LOGN;
  constexpr int NT = N / E;
  constexpr int NR = N / R;
  constexpr int M = E / R;
  C v[E];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int j = t + m * NT;
#pragma unroll
    for (int r = 0; r < R; ++r) v[m * R + r] = __ldg(src + (size_t)(j + r * NR) * stride);
  }
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int j = t + m * NT;
    dft<T, C, R>(v + m * R);
    if constexpr (pad_affine<T, 1, R>()) {
      C* dst = buf + pad<T>(j * R);
#pragma unroll
      for (int r = 0; r < R; ++r) dst[r] = v[m * R + r];
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) buf[pad<T>(j * R + r)] = v[m * R + r];
    }
  }
  __syncthreads();
}

// Last stage (Ns * R = N) from the shared buffer straight to global memory, scaled.
template <typename T, int LOGN, int E, int R, int NS>
__device__ __forceinline__ void stage_last_global(const typename Cx<T>::type* buf, int t,
                                                  const typename Cx<T>::type* __restrict__ tw,
                                                  typename Cx<T>::type* __restrict__ dst,
                                                  size_t stride, T scale, bool store) {
  using C = typename Cx<T>::type;
  constexpr int N = 1 << LOGN;
  constexpr int NT = N / E;
  constexpr int NR = N / R;
  constexpr int M = E / R;
  C v[E];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int j = t + m * NT;
    if constexpr (NR % (1 << pad_shift<T>()) == 0) {
      const C* src = buf + pad<T>(j);
#pragma unroll
      for (int r = 0; r < R; ++r) v[m * R + r] = src[r * pad_step<T, NR>()];
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) v[m * R + r] = buf[pad<T>(j + r * NR)];
    }
  }
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int j = t + m * NT;
    const int k = j & (NS - 1);
    constexpr int OFF = stage_off(N, E, NS);
#pragma unroll
    for (int r = 1; r < R; ++r) v[m * R + r] = mul(v[m * R + r], __ldg(tw + OFF + r * NS + k));
    dft<T, C, R>(v + m * R);
    const int base = (j / NS) * NS * R + k;
    if (store) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const C x = v[m * R + r];
        dst[(size_t)(base + r * NS) * stride] = C{x.x * scale, x.y * scale};
      }
    }
  }
}

// Stages after the first: shared-memory stages, the last one to global memory.
template <typename T, int LOGN, int E, int NS>
__device__ __forceinline__ void fft_rest_to_global(typename Cx<T>::type* buf, int t,
                                                   const typename Cx<T>::type* __restrict__ tw,
                                                   typename Cx<T>::type* __restrict__ dst,
                                                   size_t stride, T scale, bool store) {
  constexpr int N = 1 << LOGN;
  constexpr int R = (N / NS >= E) ? E : N / NS;
  if constexpr (NS * R == N) {
    stage_last_global<T, LOGN, E, R, NS>(buf, t, tw, dst, stride, scale, store);
  } else {
    stage<T, LOGN, E, R, NS>(buf, t, true, tw, 1);
    fft_rest_to_global<T, LOGN, E, NS * R>(buf, t, tw, dst, stride, scale, store);
  }
}

// The extended row j of function f as NH complex pairs z_n = x_{2n} + i x_{2n+1} in the
// padded shared buffer: mode 0 from an extended grid; mode 1 assembled (zeros, the
// inside reals of f, the strip values).  Ends with a barrier.  It makes the kernel's
// dependent-launch wait: in mode 0 before anything else; in the assembled modes only
// before the strip values, which the previous kernel (the blend + interpolation) writes.
// f itself was written before that kernel's own wait returned, and this kernel was
// launched after that kernel triggered, so f may be read before the wait.
// NTHR: the block size (blockDim.x) when known at compile time, else 0
template <typename T, typename TV, int NTHR = 0>
__device__ __forceinline__ void assemble_row(const RowArgs& ra, int mode, int NH, int j, int f,
                                             const T* __restrict__ ext,
                                             const double* __restrict__ f_grid,
                                             const TV* __restrict__ vals,
                                             typename Cx<T>::type* buf) {
  using C = typename Cx<T>::type;
  const int nx = 2 * NH;
  const int nthr = NTHR ? NTHR : (int)blockDim.x;
  auto put = [&](int i, T v) { reinterpret_cast<T*>(&buf[pad<T>(i >> 1)])[i & 1] = v; };
  if (mode == 0) {
    pdl_wait();
    pdl_trigger();
    const T* src = ext + (size_t)f * ra.grid_stride + (size_t)j * nx;
    for (int n = threadIdx.x; n < NH; n += nthr) {
      const C v = reinterpret_cast<const C*>(src)[n];
      buf[pad<T>(n)] = v;
    }
  } else {
    // mode 1: element i of the row at fg[i]; mode 2 (compact): at fin[coff_k + i - lo_k]
    const double* fg = mode == 1 ? f_grid + (size_t)f * ra.grid_stride + (size_t)j * nx
                                 : f_grid + (size_t)f * ra.grid_stride;
    const int iv0 = __ldg(ra.row_iv_off + j), iv1 = __ldg(ra.row_iv_off + j + 1);
    if (NTHR > 0 && NTHR % (1 << pad_shift<T>()) == 0 && NH % NTHR == 0) {
      C* z = buf + pad<T>(threadIdx.x);  // n = t + i NTHR: pad(n) = pad(t) + i pad_step
      for (int i = 0; i < NH / (NTHR > 0 ? NTHR : 1); ++i)
        z[i * pad_step<T, (NTHR > 0 ? NTHR : 1)>()] = C{(T)0, (T)0};
    } else {
      for (int n = threadIdx.x; n < NH; n += nthr) buf[pad<T>(n)] = C{(T)0, (T)0};
    }
    __syncthreads();
    // inside intervals [lo, hi]: the pairs n with lo <= 2n and 2n + 1 <= hi as one
    // 16-byte load each when the source is 16-byte aligned at even i (eight loads in
    // flight per thread), the odd ends element by element
    for (int k = iv0; k < iv1; ++k) {
      const int lo = __ldg(ra.row_iv + 2 * k), hi = __ldg(ra.row_iv + 2 * k + 1);
      const double* src = mode == 1 ? fg : fg + ((int64_t)__ldg(ra.row_iv_coff + k) - lo);
      const bool vec = (reinterpret_cast<uintptr_t>(src) & 15) == 0;
      if (vec) {
        const int p0 = (lo + 1) >> 1, p1 = (hi + 1) >> 1;  // pairs p0 .. p1 - 1
        const double2* fg2 = reinterpret_cast<const double2*>(src);
        const uint64_t pol = l2_drop();
        for (int n0 = p0 + threadIdx.x; n0 < p1; n0 += 8 * nthr) {
          // pairs n0 + u nthr from two base pointers (with a compile-time block size that
          // is a multiple of the pad unit, pad(n0 + u nthr) = pad(n0) + u pad_step)
          constexpr bool affine = NTHR > 0 && NTHR % (1 << pad_shift<T>()) == 0;
          const double2* s2 = fg2 + n0;
          C* d2 = buf + pad<T>(n0);
          double2 d[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int n = n0 + u * nthr;
            d[u] = n < p1 ? ld_stream(s2 + u * nthr, pol) : make_double2(0.0, 0.0);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int n = n0 + u * nthr;
            if (n < p1) {
              C* dst = affine ? d2 + u * pad_step<T, (NTHR > 0 ? NTHR : 1)>() : buf + pad<T>(n);
              if constexpr (sizeof(T) == 4) *dst = d2f2_rn(d[u]);
              else *dst = C{d[u].x, d[u].y};
            }
          }
        }
        if (threadIdx.x == 0 && (lo & 1)) put(lo, from_double<T>(__ldg(src + lo)));
        if (threadIdx.x == 0 && !(hi & 1)) put(hi, from_double<T>(__ldg(src + hi)));
      } else {
        for (int i = lo + threadIdx.x; i <= hi; i += nthr) put(i, from_double<T>(__ldg(src + i)));
      }
    }
    const int s0 = __ldg(ra.row_strip_off + j), s1 = __ldg(ra.row_strip_off + j + 1);
    const int base = j * nx;
    const TV* v = vals + (size_t)f * ra.n_strip;
    pdl_wait();
    pdl_trigger();
    for (int k = s0 + threadIdx.x; k < s1; k += nthr) put(__ldg(ra.s_lin + k) - base, (T)__ldg(v + k));
  }
  __syncthreads();
}

// The real row's spectrum X_k, k = 0..NH, from the complex transform Z of the pairs (in
// the padded buffer): X_k and X_{NH-k} from Z_k and Z_{NH-k} (k = 0..NH/2; k = 0 pairs
// with NH): e' = conj(e), o' = -conj(o), rtw_{NH-k} = -conj(rtw_k), so w'o' = conj(w o).
template <typename T>
__device__ __forceinline__ void even_odd_split(const typename Cx<T>::type* buf, int NH,
                                               const typename Cx<T>::type* __restrict__ rtw,
                                               typename Cx<T>::type* __restrict__ out) {
  using C = typename Cx<T>::type;
  for (int k = threadIdx.x; k <= NH / 2; k += blockDim.x) {
    const C zk = buf[pad<T>(k)];
    C zc = buf[pad<T>(k == 0 ? 0 : NH - k)];
    zc.y = -zc.y;
    const C e = {(T)0.5 * (zk.x + zc.x), (T)0.5 * (zk.y + zc.y)};
    const C o = {(T)0.5 * (zk.x - zc.x), (T)0.5 * (zk.y - zc.y)};
    const C wo = mul(__ldg(rtw + k), o);
    out[k] = C{e.x + wo.y, e.y - wo.x};
    if (k != NH - k) out[NH - k] = C{e.x - wo.y, -e.y - wo.x};
  }
}

// Blocks per SM asked of the compiler for FP32 kernels of `threads` threads: about 1024
// resident threads (at most 64 registers each), at most 32 blocks.  FP64 kernels, bound
// by their FP64 pipe, keep `fp64` (more registers, fewer shared-memory passes).
__host__ __device__ constexpr int fp32_blocks(int threads) {
  return 1024 / threads < 1 ? 1 : (1024 / threads > 32 ? 32 : 1024 / threads);
}

// rows: nx = 2^(LOGNH+1); the transform's NT = 2^LOGNH / E threads, the block at least
// one warp (row_threads: the launch's block size, which assemble_row's loops assume)
template <typename T, int LOGNH> __host__ __device__ constexpr int row_threads() {
  return (1 << LOGNH) / elems<T>() < 32 ? 32 : (1 << LOGNH) / elems<T>();
}
template <typename T, typename TV, int LOGNH>
__global__ void __launch_bounds__(row_threads<T, LOGNH>(),
                                  sizeof(T) == 4 ? fp32_blocks(row_threads<T, LOGNH>()) : 1)
k_fft_rows_p2(FftArgs fa, RowArgs ra, int mode, const T* __restrict__ ext,
              const double* __restrict__ f_grid, const TV* __restrict__ vals,
              typename Cx<T>::type* __restrict__ inter) {
  using C = typename Cx<T>::type;
  constexpr int E = elems<T>();
  constexpr int NH = 1 << LOGNH;
  constexpr int NT = NH / E < 1 ? 1 : NH / E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int j = blockIdx.x, f = blockIdx.y, t = threadIdx.x;
  assemble_row<T, TV, row_threads<T, LOGNH>()>(ra, mode, NH, j, f, ext, f_grid, vals, buf);
  const C* tw = reinterpret_cast<const C*>(fa.tsx);
  C* out = inter + ((size_t)f * fa.ny + j) * fa.pitch;
  // FP32: the last stage and the split in registers (for FP64, bound by its FP64 pipe,
  // the extra registers cost more than the saved shared-memory passes)
  if constexpr (sizeof(T) == 4 && NH / E >= 32 && last_ns<LOGNH, E>() == 2 * (NH / E)) {
    block_fft_head<T, LOGNH, E>(buf, t, true, tw, 1);
    last_stage_split<T, LOGNH, E>(buf, t, tw, reinterpret_cast<const C*>(fa.rtw), out);
  } else {
    block_fft<T, LOGNH, E>(buf, t, t < NT, tw, 1);
    even_odd_split<T>(buf, NH, reinterpret_cast<const C*>(fa.rtw), out);
  }
}

// rows of NH = 64 N2 complex pairs (N2 = 3, 5, 6, 10, 12: the non-power-of-two row
// lengths), FP32, one block of 128 threads per (row, function), in shared memory:
//   n = N2 n1 + n2, k = k1 + 64 k2;
//   step 1: for each n2 (a group of 8 lanes, 8 values each): the 64-point DFT over n1
//           (length-8 DFT in registers, twiddles w_64^(l m), exchange inside the group,
//           length-8 DFT), the twiddle w_NH^(n2 k1), back in place at N2 k1 + n2;
//   step 2: for each k1 (64 threads): the N2-point DFT over n2 in registers, written to
//           k1 + 64 k2 (natural order), then the even/odd split to the spectrum.
// Twiddles from the row table w_NH^t (w_64^k = w[N2 k], w_N2^k = w[64 k]).
template <int N2> __device__ __forceinline__ void dft_len(float2* x, const float2* __restrict__ w) {
  if constexpr (N2 == 3 || N2 == 5) dft<float, float2, N2>(x);
  else if constexpr (N2 == 6) dft_ct<2, 3>(x, w, 64);
  else if constexpr (N2 == 10) dft_ct<2, 5>(x, w, 64);
  else dft_ct<4, 3>(x, w, 64);  // 12
}

template <int N2>
__global__ void __launch_bounds__(128, fp32_blocks(128))
k_rows_64n(FftArgs fa, RowArgs ra, int mode, const float* __restrict__ ext,
           const double* __restrict__ f_grid, const float* __restrict__ vals,
           float2* __restrict__ inter) {
  constexpr int NH = 64 * N2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* buf = reinterpret_cast<float2*>(smem_raw);
  float2* ex = buf + padded<float>(NH);  // [N2][8][9] exchange tiles
  const int j = blockIdx.x, f = blockIdx.y, t = threadIdx.x;
  const float2* w = reinterpret_cast<const float2*>(fa.twx);
  assemble_row<float, float>(ra, mode, NH, j, f, ext, f_grid, vals, buf);
  if (t < 8 * N2) {
    const int n2 = t >> 3, l = t & 7;
    float2* e = ex + n2 * 72;
    float2 a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = buf[pad<float>(N2 * (l + 8 * i) + n2)];
    dft<float, float2, 8>(a);
#pragma unroll
    for (int m = 1; m < 8; ++m) a[m] = mul(a[m], __ldg(w + ((l * m) & 63) * N2));
#pragma unroll
    for (int m = 0; m < 8; ++m) e[m * 9 + l] = a[m];
    __syncwarp(0xFFu << (t & 24));
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = e[l * 9 + k];
    dft<float, float2, 8>(a);
#pragma unroll
    for (int m2 = 0; m2 < 8; ++m2) {
      const int k1 = l + 8 * m2;
      buf[pad<float>(N2 * k1 + n2)] = mul(a[m2], __ldg(w + n2 * k1));  // n2 k1 < NH
    }
  }
  __syncthreads();
  float2 x[N2];
  if (t < 64) {
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) x[n2] = buf[pad<float>(N2 * t + n2)];
    dft_len<N2>(x, w);
  }
  __syncthreads();
  if (t < 64) {
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) buf[pad<float>(t + 64 * k2)] = x[k2];
  }
  __syncthreads();
  even_odd_split<float>(buf, NH, reinterpret_cast<const float2*>(fa.rtw),
                        inter + ((size_t)f * fa.ny + j) * fa.pitch);
}

template <int N2>
static void rows64n_launch(const FftArgs& fa, const RowArgs& ra, int n_f, int mode, const void* ext,
                           const double* fg, const void* vals, void* inter, cudaStream_t s) {
  const size_t sm = ((size_t)padded<float>(64 * N2) + 72 * N2) * sizeof(float2);
  auto k = k_rows_64n<N2>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  launch_pdl(k, dim3(fa.ny, n_f), dim3(128), sm, s, fa, ra, mode, (const float*)ext, fg,
             (const float*)vals, (float2*)inter);
}

// cols: ny = 2^LOGNY, CB columns per block, block = CB * NT threads.  Thread
// (c = tid % CB, t = tid / CB): the CB columns of a row are read by neighbouring
// threads.  First stage from the intermediate, last stage to the spectrum.
template <typename T, int LOGNY, int CB>
__global__ void __launch_bounds__(CB * ((1 << LOGNY) / elems<T>()),
                                  sizeof(T) == 4 ? fp32_blocks(CB * ((1 << LOGNY) / elems<T>()))
                                  : (CB * ((1 << LOGNY) / elems<T>()) <= 512 ? 2 : 1))
k_fft_cols_p2(FftArgs fa, const typename Cx<T>::type* __restrict__ inter,
              typename Cx<T>::type* __restrict__ fhat) {
  using C = typename Cx<T>::type;
  constexpr int E = elems<T>();
  constexpr int N = 1 << LOGNY;
  constexpr int PN = padded<T>(N);
  constexpr int R1 = N >= E ? E : N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int ncol = fa.nx / 2 + 1;
  const int c = threadIdx.x % CB, t = threadIdx.x / CB;
  const int kx = blockIdx.x * CB + c, f = blockIdx.y;
  // kx < pitch always (pitch = nx/2+1 rounded up to 16, CB divides 16): reads stay in the
  // intermediate row; columns beyond nx/2 are computed and not stored
  const C* src = inter + (size_t)f * N * fa.pitch + kx;
  // column c starts c * W/CB elements after c * PN (W = lanes per shared-memory
  // wavefront: 16 for 8-byte, 8 for 16-byte elements), so that the CB interleaved
  // columns served by one wavefront fall in disjoint banks (no conflicts in the
  // first-stage writes and the stage reads, for every size and CB launched below)
  C* col = buf + c * PN + c * (col_lanes<T>() / CB);
  pdl_wait();
  pdl_trigger();
  stage_first_global<T, LOGNY, E, R1>(src, fa.pitch, col, t);
  const C* tw = reinterpret_cast<const C*>(fa.tsy);
  fft_rest_to_global<T, LOGNY, E, R1>(col, t, tw, fhat + (size_t)f * N * ncol + kx, ncol,
                                      (T)fa.scale, kx < ncol);
}

// ------------------------------------------------------------------------- //
// Columns of 4096 points (FP32) in two passes, N = 64 x 64 ("four-step"):
//   j = 64 j1 + j2, m = m1 + 64 m2,
//   pass A: Y[m1][j2] = w_4096^(j2 m1) sum_j1 x[64 j1 + j2] w_64^(j1 m1), written in
//           place to row 64 m1 + j2 of the intermediate;
//   pass B: X[m1 + 64 m2] = sum_j2 Y[m1][j2] w_64^(j2 m2), scaled, to the spectrum.
// A block of 128 threads serves 16 adjacent columns; thread (c = tid % 16, l = tid / 16)
// holds the 8 values of input index l + 8 i of its column.  Each 64-point DFT is a
// length-8 DFT over i in registers, the twiddles w_64^(l m'), an exchange through
// shared memory and a length-8 DFT over l, after which thread (c, L) holds the outputs
// L + 8 m'.  Consecutive lanes take consecutive columns, so a warp's load or store is
// two rows of 16 columns (two 128-byte lines).  Blocks need 8 KB of shared memory, so
// many are resident per SM, and the 67 MB intermediate of a 4096^2 grid can stay in L2
// between the passes.
// ------------------------------------------------------------------------- //
constexpr int kC4Cols = 16;   // columns per block (mixed-radix passes; the 4096-point
                              // passes take the width tuned at plan time, tune_plan)

// 64-point DFT of a[i] = x[l + 8 i] held by the threads (c, l = 0..7) of column c;
// on return a[m'] = X[l + 8 m'].  ex: the block's [8][8][CC] exchange buffer; w: the
// table w_N^t of the column length N = 64 n2 (w_64^k = w[n2 k]).
template <int CC = kC4Cols>
__device__ __forceinline__ void dft64_cols(float2* a, int c, int l, float2* ex,
                                           const float2* __restrict__ w, int n2 = 64) {
  dft<float, float2, 8>(a);
#pragma unroll
  for (int m = 1; m < 8; ++m) a[m] = mul(a[m], __ldg(w + (l * m) * n2));  // l m <= 49
#pragma unroll
  for (int m = 0; m < 8; ++m) ex[(m * 8 + l) * CC + c] = a[m];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = ex[(l * 8 + k) * CC + c];
  dft<float, float2, 8>(a);
}

// CC adjacent columns per block of 8 CC threads (16, 32 or 64: every width computes the
// same values; wider blocks read longer contiguous row segments).
// Row offsets within one function's slab (4096 x pitch < 2^32 elements) in 32-bit
// unsigned arithmetic: one multiply and one wide add per access.
template <int CC>
__global__ void __launch_bounds__(8 * CC, 2048 / (8 * CC)) k_cols4k_a(FftArgs fa, float2* __restrict__ inter) {
  __shared__ float2 ex[64 * CC];
  const int c = threadIdx.x & (CC - 1), l = threadIdx.x / CC;
  const int ncol = fa.nx / 2 + 1;
  const int kx = blockIdx.x * CC + c;
  const int j2 = blockIdx.y, f = blockIdx.z;
  const bool live = kx < ncol;
  const float2* w = reinterpret_cast<const float2*>(fa.twy);
  float2* col = inter + (size_t)f * 4096 * fa.pitch + kx;
  pdl_wait();
  pdl_trigger();
  float2 a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
    a[i] = live ? col[(unsigned)(64 * (l + 8 * i) + j2) * (unsigned)fa.pitch] : make_float2(0.f, 0.f);
  const uint64_t pol = l2_keep();
  dft64_cols<CC>(a, c, l, ex, w);
#pragma unroll
  for (int m2 = 0; m2 < 8; ++m2) {
    const int m1 = l + 8 * m2;
    const float2 y = mul(a[m2], __ldg(w + j2 * m1));  // j2 m1 <= 63 * 63
    if (live) st_hint<2>(col + (unsigned)(64 * m1 + j2) * (unsigned)fa.pitch, y, pol);
  }
}

template <int CC>
__global__ void __launch_bounds__(8 * CC, 2048 / (8 * CC)) k_cols4k_b(FftArgs fa, int drop,
                                                      float2* __restrict__ inter,
                                                      float2* __restrict__ fhat) {
  __shared__ float2 ex[64 * CC];
  const int c = threadIdx.x & (CC - 1), l = threadIdx.x / CC;
  const int ncol = fa.nx / 2 + 1;
  const int kx = blockIdx.x * CC + c;
  const int m1 = blockIdx.y, f = blockIdx.z;
  const bool live = kx < ncol;
  const float2* w = reinterpret_cast<const float2*>(fa.twy);
  float2* col = inter + (size_t)f * 4096 * fa.pitch + kx;
  pdl_wait();
  pdl_trigger();
  float2 a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
    a[i] = live ? col[(unsigned)(64 * m1 + l + 8 * i) * (unsigned)fa.pitch] : make_float2(0.f, 0.f);
  dft64_cols<CC>(a, c, l, ex, w);
  // the intermediate is scratch and this block was the last reader of its 64 rows x CC
  // columns (every load completed before the transform's barrier): drop the lines from
  // L2 without writing them back (each row of 16 columns is one 128-byte line; `drop` is
  // set only when the host has checked the 128-byte alignment of the buffer and the
  // pitch), one line per thread.  Only lines of live columns: a wide block's columns past
  // the last one would name the next row's lines.
  if (drop && (int)threadIdx.x < 64 * (CC / 16)) {
    const int r = threadIdx.x & 63, g = threadIdx.x >> 6;
    const int kx0 = blockIdx.x * CC + 16 * g;
    if (kx0 < ncol)
      asm volatile("discard.global.L2 [%0], 128;" ::"l"(inter + (size_t)f * 4096 * fa.pitch +
                                                         (unsigned)(64 * m1 + r) * (unsigned)fa.pitch + kx0)
                   : "memory");
  }
  const float sc = (float)fa.scale;
  float2* out = fhat + (size_t)f * 4096 * ncol + kx;
  if (live) {
    const uint64_t pol = l2_drop();
#pragma unroll
    for (int m2p = 0; m2p < 8; ++m2p) {
      const int m2 = l + 8 * m2p;
      st_hint<4>(out + (unsigned)(m1 + 64 * m2) * (unsigned)ncol, make_float2(a[m2p].x * sc, a[m2p].y * sc), pol);
    }
  }
}

// ------------------------------------------------------------------------- //
// FP32 columns of N = 64 N2 points (N2 = 6, 10, 12, 24: non-power-of-two sizes; N2 = 32:
// 2048 points, whose one-pass blocks would read 16 bytes per row), in the
// same two passes: j = N2 j1 + j2, m = m1 + 64 m2,
//   pass A: 64-point DFTs over j1 (rows N2 j1 + j2, as k_cols4k_a with stride N2), the
//           twiddle w_N^(j2 m1), in place to row N2 m1 + j2;
//   pass B: N2-point DFTs over the N2 consecutive rows N2 m1 + j2, one per thread
//           (16 columns x 8 values of m1 per block), scaled, to the spectrum rows
//           m1 + 64 m2; then the intermediate's lines are dropped from L2.
// ------------------------------------------------------------------------- //

// (row offsets within one function's slab in 32-bit unsigned arithmetic, as the
// 4096-point passes)
__global__ void __launch_bounds__(128, fp32_blocks(128)) k_cols64_a(FftArgs fa, int n2, float2* __restrict__ inter) {
  __shared__ float2 ex[64 * kC4Cols];
  const int c = threadIdx.x & (kC4Cols - 1), l = threadIdx.x / kC4Cols;
  const int ncol = fa.nx / 2 + 1, N = fa.ny;
  const int kx = blockIdx.x * kC4Cols + c;
  const int j2 = blockIdx.y, f = blockIdx.z;
  const bool live = kx < ncol;
  const float2* w = reinterpret_cast<const float2*>(fa.twy);
  float2* col = inter + (size_t)f * N * fa.pitch + kx;
  pdl_wait();
  pdl_trigger();
  float2 a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
    a[i] = live ? col[(unsigned)(n2 * (l + 8 * i) + j2) * (unsigned)fa.pitch] : make_float2(0.f, 0.f);
  dft64_cols(a, c, l, ex, w, n2);
#pragma unroll
  for (int m2 = 0; m2 < 8; ++m2) {
    const int m1 = l + 8 * m2;
    const float2 y = mul(a[m2], __ldg(w + j2 * m1));  // j2 m1 < N
    if (live) col[(unsigned)(n2 * m1 + j2) * (unsigned)fa.pitch] = y;
  }
}

template <int R1, int R2>
__global__ void __launch_bounds__(128, R1 * R2 >= 24 ? 4 : fp32_blocks(128)) k_cols64_b(FftArgs fa, int drop, float2* __restrict__ inter,
                                                   float2* __restrict__ fhat) {
  constexpr int N2 = R1 * R2;
  const int c = threadIdx.x & (kC4Cols - 1);
  const int ncol = fa.nx / 2 + 1, N = fa.ny;
  const int kx = blockIdx.x * kC4Cols + c;
  const int m1 = blockIdx.y * 8 + threadIdx.x / kC4Cols, f = blockIdx.z;
  const bool live = kx < ncol;
  const float2* w = reinterpret_cast<const float2*>(fa.twy);
  float2* col = inter + (size_t)f * N * fa.pitch + kx;
  pdl_wait();
  pdl_trigger();
  float2 x[N2];
#pragma unroll
  for (int j2 = 0; j2 < N2; ++j2)
    x[j2] = live ? col[(unsigned)(N2 * m1 + j2) * (unsigned)fa.pitch] : make_float2(0.f, 0.f);
  dft_ct<R1, R2>(x, w, 64);  // w_N2^t = w_N^(64 t)
  const float sc = (float)fa.scale;
  float2* out = fhat + (size_t)f * N * ncol + kx;
  if (live) {
#pragma unroll
    for (int m2 = 0; m2 < N2; ++m2)
      out[(unsigned)(m1 + 64 * m2) * (unsigned)ncol] = make_float2(x[m2].x * sc, x[m2].y * sc);
  }
  // last reader of the intermediate: drop its lines (one 128-byte line per row of the
  // block's 16 columns; `drop` only when the host checked the alignment)
  if (drop && c == 0) {
#pragma unroll
    for (int j2 = 0; j2 < N2; ++j2)
      asm volatile("discard.global.L2 [%0], 128;" ::"l"(col + (unsigned)(N2 * m1 + j2) * (unsigned)fa.pitch)
                   : "memory");
  }
}

template <int R1, int R2>
static void cols64_launch(const FftArgs& fa, int n_f, void* inter, void* fhat, cudaStream_t s) {
  const int ncol = fa.nx / 2 + 1;
  const int groups = (ncol + kC4Cols - 1) / kC4Cols;
  const int drop = (reinterpret_cast<uintptr_t>(inter) % 128 == 0 && fa.pitch % 16 == 0) ? 1 : 0;
  launch_pdl(k_cols64_a, dim3(groups, R1 * R2, n_f), dim3(128), 0, s, fa, R1 * R2, (float2*)inter);
  launch_pdl(k_cols64_b<R1, R2>, dim3(groups, 8, n_f), dim3(128), 0, s, fa, drop, (float2*)inter,
             (float2*)fhat);
}

template <int CC>
static void cols4k_launch_cc(const FftArgs& fa, int n_f, void* inter, void* fhat, cudaStream_t s) {
  const int ncol = fa.nx / 2 + 1;
  const dim3 grid((ncol + CC - 1) / CC, 64, n_f);
  const int drop = (reinterpret_cast<uintptr_t>(inter) % 128 == 0 && fa.pitch % 16 == 0) ? 1 : 0;
  launch_pdl(k_cols4k_a<CC>, grid, dim3(8 * CC), 0, s, fa, (float2*)inter);
  launch_pdl(k_cols4k_b<CC>, grid, dim3(8 * CC), 0, s, fa, drop, (float2*)inter, (float2*)fhat);
}

// ------------------------------------------------------------------------- //
// The same two 4096-point passes with TMA-pipelined loads.  Persistent blocks (as many
// as fit on the GPU) take the tiles t = blockIdx.x + k gridDim.x, a tile being the
// 64 rows x CC columns one direct-form block reads, in that form's block order (column
// block fastest, then j2 or m1, then the function).  Thread 0 keeps the next tiles in
// flight: each is one tensor-map copy (cp.async.bulk.tensor) into one of S shared-memory
// stages, completing on that stage's mbarrier with the tile's byte count.  The block
// reads a stage once its barrier's phase completes.  The transform's exchange runs in
// place in the stage: thread (c, l) reads the rows l + 8 i of its column and writes its
// exchange values to the rows 8 m + l, the same rows, so no other thread's input is
// overwritten and no barrier is needed before the writes; after the block's barrier
// each thread reads the rows 8 l .. 8 l + 7.  The barrier of tile k also tells thread 0
// that every thread has finished with the stage of tile k - 1, which it refills with
// tile k - 1 + S.  One barrier per tile, no exchange buffer: S tiles of shared
// memory per block, so 1024 threads fit on an SM with S - 1 tiles in flight per block
// during the transforms, and the loads no longer wait in the computing warps'
// registers.  Each thread holds the same values as in the direct form and runs the same
// arithmetic (dft64_cols's steps), so both forms give the same results bit for bit; the
// stores, their L2 policies and pass B's L2 discard are the direct form's.  The
// generic-proxy writes of the exchange are ordered before the copy that later refills
// their stage by a proxy fence in each writing thread and the block's barrier.
//
// Tensor maps (8-byte elements, zero fill past the last column): pass A views one
// function's slab as [f][j1][j2][kx] (extents n_f, 64, 64, nx/2+1; a box of CC x 1 x 64 x 1
// lands as [j1][c]); pass B as [f][row][kx] (extents n_f, 4096, nx/2+1; a box of
// CC x 64 x 1 lands as [row][c]).  The host builds them only when the intermediate is
// 16-byte aligned and its pitch a multiple of 16 bytes (the encoder checks both again).
//
// Every wait is bounded: a stage whose copy has not landed after kTileSpin polls sets
// FC2D_ERR_TIMEOUT in the status word; the block then agrees at its barrier to stop,
// thread 0 waits (bounded again) for the copies it issued, and the block returns.
// ------------------------------------------------------------------------- //
constexpr uint32_t kTileSpin = 1u << 22;

__device__ __forceinline__ uint32_t sm_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ bool stage_ready(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool stage_wait(uint32_t mbar, uint32_t parity, int* status) {
  for (uint32_t it = 0; it < kTileSpin; ++it)
    if (stage_ready(mbar, parity)) return true;
  if (status) atomicExch(status, (int)FC2D_ERR_TIMEOUT);
  return false;
}

// thread 0: tile k of this block into stage k % S, completing on that stage's barrier
template <int PASS, int CC, int S>
__device__ __forceinline__ void tile_issue(const CUtensorMap* tm, int k, int ncb,
                                           float2* stage, uint64_t* full) {
  const int t = blockIdx.x + k * gridDim.x;
  const int cb = t % ncb, r = (t / ncb) & 63, f = t / (ncb * 64);
  const uint32_t mb = sm_addr(full + k % S), dst = sm_addr(stage + (k % S) * (64 * CC));
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
               ::"r"(mb), "r"((uint32_t)(64 * CC * sizeof(float2))) : "memory");
  const uint64_t map = reinterpret_cast<uint64_t>(tm);
  if constexpr (PASS == 0)
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(dst), "l"(map), "r"(cb * CC), "r"(r), "r"(0), "r"(f), "r"(mb) : "memory");
  else
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"(map), "r"(cb * CC), "r"(64 * r), "r"(f), "r"(mb) : "memory");
}

template <int CC, int S>
constexpr size_t cols_tma_smem() {
  return 128 + (size_t)S * 64 * CC * sizeof(float2) + S * sizeof(uint64_t);
}

// (resident blocks: S = 3 tiles of shared memory allow eight blocks of 16 columns or
// four of 32 per SM, 1024 threads either way, which leaves each thread 64 registers)
template <int PASS, int CC, int S>
__global__ void __launch_bounds__(8 * CC, 128 / CC)
    k_cols4k_tma(const __grid_constant__ CUtensorMap tm, FftArgs fa, int n_f, int drop,
                 float2* __restrict__ inter, float2* __restrict__ fhat) {
  constexpr int TILE = 64 * CC;
  extern __shared__ __align__(128) unsigned char smem_tma[];
  // the stages start on a 128-byte boundary (the copies' destination alignment), which
  // the launch's 128 extra bytes allow whatever the base
  unsigned char* base = smem_tma + ((128u - (sm_addr(smem_tma) & 127u)) & 127u);
  float2* stage = reinterpret_cast<float2*>(base);                     // [S][64][CC]
  uint64_t* full = reinterpret_cast<uint64_t*>(stage + S * TILE);      // [S]
  const int tid = threadIdx.x, c = tid & (CC - 1), l = tid / CC;
  const int ncol = fa.nx / 2 + 1, ncb = (ncol + CC - 1) / CC;
  const int n_tiles = ncb * 64 * n_f;
  const int n_my = (int)blockIdx.x < n_tiles
                       ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const float2* w = reinterpret_cast<const float2*>(fa.twy);
  if (tid == 0) {
    for (int q = 0; q < S; ++q)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sm_addr(full + q)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  pdl_wait();
  pdl_trigger();
  if (tid == 0)
    for (int k = 0; k < S && k < n_my; ++k) tile_issue<PASS, CC, S>(&tm, k, ncb, stage, full);
  const uint64_t pol = PASS == 0 ? l2_keep() : l2_drop();
  for (int k = 0; k < n_my; ++k) {
    const int t = blockIdx.x + k * gridDim.x;
    const int cb = t % ncb, r = (t / ncb) & 63, f = t / (ncb * 64);
    const int kx = cb * CC + c;
    const bool ok = stage_wait(sm_addr(full + k % S), (uint32_t)(k / S) & 1u, fa.status);
    float2* st = stage + (k % S) * TILE;
    float2 a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = st[(l + 8 * i) * CC + c];
    // dft64_cols's steps, the exchange in place (rows 8 m + l: this thread's own rows)
    dft<float, float2, 8>(a);
#pragma unroll
    for (int m = 1; m < 8; ++m) a[m] = mul(a[m], __ldg(w + (l * m) * 64));  // l m <= 49
#pragma unroll
    for (int m = 0; m < 8; ++m) st[(m * 8 + l) * CC + c] = a[m];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (!__syncthreads_and(ok)) {
      // a copy did not land: wait (bounded) for every copy this block issued, then stop
      if (tid == 0) {
        const int issued = min(n_my, k == 0 ? S : k - 1 + S);
        for (int q = k; q < issued; ++q)
          stage_wait(sm_addr(full + q % S), (uint32_t)(q / S) & 1u, fa.status);
      }
      return;
    }
    // every thread has read the previous tile's stage: refill it
    if (tid == 0 && k >= 1 && k - 1 + S < n_my)
      tile_issue<PASS, CC, S>(&tm, k - 1 + S, ncb, stage, full);
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = st[(l * 8 + q) * CC + c];
    dft<float, float2, 8>(a);
    if constexpr (PASS == 0) {
      if (kx < ncol) {
        float2* col = inter + (size_t)f * 4096 * fa.pitch + kx;
#pragma unroll
        for (int m2 = 0; m2 < 8; ++m2) {
          const int m1 = l + 8 * m2;
          const float2 y = mul(a[m2], __ldg(w + r * m1));  // j2 m1 <= 63 * 63
          st_hint<2>(col + (unsigned)(64 * m1 + r) * (unsigned)fa.pitch, y, pol);
        }
      }
    } else {
      // this block was the intermediate's last reader of the tile (its copy has
      // landed): drop the tile's lines from L2, one line per thread, live columns only
      if (drop && tid < 64 * (CC / 16)) {
        const int rr = tid & 63, g = tid >> 6;
        const int kx0 = cb * CC + 16 * g;
        if (kx0 < ncol)
          asm volatile("discard.global.L2 [%0], 128;" ::"l"(inter + (size_t)f * 4096 * fa.pitch +
                                                             (unsigned)(64 * r + rr) * (unsigned)fa.pitch + kx0)
                       : "memory");
      }
      if (kx < ncol) {
        const float sc = (float)fa.scale;
        float2* out = fhat + (size_t)f * 4096 * ncol + kx;
#pragma unroll
        for (int m2p = 0; m2p < 8; ++m2p) {
          const int m2 = l + 8 * m2p;
          st_hint<4>(out + (unsigned)(r + 64 * m2) * (unsigned)ncol,
                     make_float2(a[m2p].x * sc, a[m2p].y * sc), pol);
        }
      }
    }
  }
}

// The driver's tensor-map encoder, reached through the runtime (no link against the
// driver library); null when the driver does not offer it.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// The tensor map of pass A (pass 0) or B over n_f functions of the intermediate, tiles of
// cc columns; false when the layout allows none (then the direct form runs).
static bool cols_tma_map(int pass, int cc, const FftArgs& fa, int n_f, void* inter,
                         CUtensorMap* tm) {
  const EncodeTiledFn enc = encode_tiled();
  const cuuint64_t ncol = (cuuint64_t)(fa.nx / 2 + 1), rowb = (cuuint64_t)fa.pitch * sizeof(float2);
  if (!enc || fa.ny != 4096 || (reinterpret_cast<uintptr_t>(inter) & 15) || (rowb & 15))
    return false;
  const cuuint32_t unit[4] = {1, 1, 1, 1};
  const CUtensorMapL2promotion prom =
      cc >= 32 ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B : CU_TENSOR_MAP_L2_PROMOTION_L2_128B;
  CUresult r;
  if (pass == 0) {
    const cuuint64_t dim[4] = {ncol, 64, 64, (cuuint64_t)n_f};  // kx, j2, j1, f
    const cuuint64_t str[3] = {rowb, 64 * rowb, 4096 * rowb};
    const cuuint32_t box[4] = {(cuuint32_t)cc, 1, 64, 1};
    r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, inter, dim, str, box, unit,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, prom,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    const cuuint64_t dim[3] = {ncol, 4096, (cuuint64_t)n_f};  // kx, row, f
    const cuuint64_t str[2] = {rowb, 4096 * rowb};
    const cuuint32_t box[3] = {(cuuint32_t)cc, 64, 1};
    r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, inter, dim, str, box, unit,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, prom,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  return r == CUDA_SUCCESS;
}

// Resident blocks per SM of one TMA pass on the current device (its shared-memory
// limit raised once per device) and the device's SM count; 0 when it cannot run.
template <int PASS, int CC, int S>
static int cols_tma_blocks(int* n_sm) {
  constexpr int kDev = 64;
  static std::mutex mu;
  static int nb[kDev], nsm[kDev];
  static bool done[kDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDev) {
    cudaGetLastError();
    return 0;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!done[dev]) {
    const size_t sm = cols_tma_smem<CC, S>();
    int b = 0, n = 0;
    if (cudaFuncSetAttribute(k_cols4k_tma<PASS, CC, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_cols4k_tma<PASS, CC, S>, 8 * CC, sm) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      b = 0;
    }
    nb[dev] = b;
    nsm[dev] = n;
    done[dev] = true;
  }
  *n_sm = nsm[dev];
  return nb[dev];
}

// Both passes in the TMA form (S stages of CC columns); false (nothing launched) when
// the form cannot run on this intermediate.
template <int CC, int S>
static bool cols4k_tma_launch_cc(const FftArgs& fa, int n_f, void* inter, void* fhat,
                                 cudaStream_t s) {
  int nsm = 0;
  const int nba = cols_tma_blocks<0, CC, S>(&nsm), nbb = cols_tma_blocks<1, CC, S>(&nsm);
  CUtensorMap ta, tb;
  if (nba < 1 || nbb < 1 || nsm < 1 || !fa.status || !cols_tma_map(0, CC, fa, n_f, inter, &ta) ||
      !cols_tma_map(1, CC, fa, n_f, inter, &tb))
    return false;
  const int ncol = fa.nx / 2 + 1;
  const int n_tiles = (ncol + CC - 1) / CC * 64 * n_f;
  const int drop = (reinterpret_cast<uintptr_t>(inter) % 128 == 0 && fa.pitch % 16 == 0) ? 1 : 0;
  const size_t sm = cols_tma_smem<CC, S>();
  launch_pdl(k_cols4k_tma<0, CC, S>, dim3(std::min(n_tiles, nba * nsm)), dim3(8 * CC), sm, s, ta,
             fa, n_f, drop, (float2*)inter, (float2*)fhat);
  launch_pdl(k_cols4k_tma<1, CC, S>, dim3(std::min(n_tiles, nbb * nsm)), dim3(8 * CC), sm, s, tb,
             fa, n_f, drop, (float2*)inter, (float2*)fhat);
  return true;
}

constexpr int kTmaStages = 3;

static void cols4k_launch(const FftArgs& fa, int n_f, void* inter, void* fhat, cudaStream_t s) {
  if (fa.cols_tma) {
    const bool done = fa.cc4k == 32
                          ? cols4k_tma_launch_cc<32, kTmaStages>(fa, n_f, inter, fhat, s)
                          : cols4k_tma_launch_cc<16, kTmaStages>(fa, n_f, inter, fhat, s);
    if (done) return;
  }
  switch (fa.cc4k) {

    case 32: cols4k_launch_cc<32>(fa, n_f, inter, fhat, s); break;
    case 64: cols4k_launch_cc<64>(fa, n_f, inter, fhat, s); break;
    default: cols4k_launch_cc<16>(fa, n_f, inter, fhat, s); break;
  }
}

// ------------------------------------------------------------------------- //
// Inverse real row DFT (FP64) of rows whose half length NH = 2^LOGNH is a power of
// two: the inverse of the even/odd split gives Z_k = S_k + i conj(w^k) D_k from X_k and
// conj(X_{NH-k}), the length-NH transform runs as a forward transform of conj(Z) on the
// compile-time Stockham stages, and x_{2m} + i x_{2m+1} = conj of its result; plus the
// quadratic term c00[f] (x^2 + y^2)/4 when c00 is given.  One block per (row, function).
// ------------------------------------------------------------------------- //
template <int LOGNH>
__global__ void __launch_bounds__((1 << LOGNH) / 8)
    k_inverse_rows_p2(FftArgs fa, const double2* __restrict__ inter,
                      const double* __restrict__ c00, double a0, double b0, double h,
                      double* __restrict__ up) {
  using C = double2;
  constexpr int NH = 1 << LOGNH, E = 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int j = blockIdx.x, f = blockIdx.y, t = threadIdx.x;
  const C* row = inter + ((size_t)f * fa.ny + j) * fa.pitch;
  const C* rtw = reinterpret_cast<const C*>(fa.rtw);
  pdl_wait();
  pdl_trigger();
  for (int k = t; k < NH; k += blockDim.x) {
    const C bk = row[k];
    C bc = row[NH - k];
    bc.y = -bc.y;  // conj X_{NH-k}
    const C sm = {bk.x + bc.x, bk.y + bc.y}, d = {bk.x - bc.x, bk.y - bc.y};
    C w = __ldg(rtw + k);
    w.y = -w.y;  // conj(w^k)
    const C dw = {d.x * w.x - d.y * w.y, d.x * w.y + d.y * w.x};
    buf[pad<double>(k)] = C{sm.x - dw.y, -(sm.y + dw.x)};  // conj(s + i dw)
  }
  __syncthreads();
  block_fft<double, LOGNH, E>(buf, t, true, reinterpret_cast<const C*>(fa.tsx), 1);
  const double q = c00 ? c00[f] * 0.25 : 0.0;
  const double y = b0 + h * double(j);
  double* out = up + ((size_t)f * fa.ny + j) * (2 * NH);
  for (int m = t; m < NH; m += blockDim.x) {
    const C z = buf[pad<double>(m)];
    const double x0 = a0 + h * double(2 * m), x1 = a0 + h * double(2 * m + 1);
    out[2 * m] = z.x + q * (x0 * x0 + y * y);
    out[2 * m + 1] = -z.y + q * (x1 * x1 + y * y);
  }
}

template <int LOGNH>
static void inverse_rows_p2_launch(const FftArgs& fa, int n_f, const void* inter,
                                   const double* c00, double a0, double b0, double h,
                                   double* out, cudaStream_t s) {
  const size_t sm = (size_t)padded<double>(1 << LOGNH) * sizeof(double2);
  cudaFuncSetAttribute(k_inverse_rows_p2<LOGNH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sm);
  launch_pdl(k_inverse_rows_p2<LOGNH>, dim3(fa.ny, n_f), dim3((1 << LOGNH) / 8), sm, s, fa,
             (const double2*)inter, c00, a0, b0, h, out);
}

// ------------------------------------------------------------------------- //
// Fourier Forwarding modal advance on power-of-two columns (FP64; see wave.cu for the
// formulas): one block per (column, pair), both columns in place in padded shared
// memory, the compile-time Stockham stages of block_fft for the forward transforms, the
// advance, and the inverse transforms as forward transforms of the conjugates.
// ------------------------------------------------------------------------- //
template <int LOGNY>
__global__ void __launch_bounds__((1 << LOGNY) / 8, LOGNY == 11 ? 2 : 1)
    k_wave_cols_p2(FftArgs fa, int n_f, double2* __restrict__ inter, double c, double t,
                   double Lx, double Ly) {
  using C = double2;
  constexpr int N = 1 << LOGNY, E = 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* A = reinterpret_cast<C*>(smem_raw);
  C* Bv = A + padded<double>(N);
  const int kx = blockIdx.x, f = blockIdx.y, tid = threadIdx.x;
  C* colu = inter + (size_t)f * N * fa.pitch + kx;
  C* colt = inter + (size_t)(n_f + f) * N * fa.pitch + kx;
  const C* tw = reinterpret_cast<const C*>(fa.tsy);
  for (int y = tid; y < N; y += blockDim.x) {
    A[pad<double>(y)] = colu[(size_t)y * fa.pitch];
    Bv[pad<double>(y)] = colt[(size_t)y * fa.pitch];
  }
  __syncthreads();
#pragma unroll 1
  for (int h = 0; h < 2; ++h) block_fft<double, LOGNY, E>(h ? Bv : A, tid, true, tw, 1);
  const double two_pi = 6.283185307179586476925286766559;
  for (int ky = tid; ky < N; ky += blockDim.x) {
    const int m = ky <= N / 2 ? ky : ky - N;
    const double fl = kx / Lx, fm = m / Ly;
    const double w = two_pi * c * sqrt(fl * fl + fm * fm);
    const C a0 = A[pad<double>(ky)], b0 = Bv[pad<double>(ky)];
    const C F = C{a0.x * fa.scale, a0.y * fa.scale};
    const C G = C{b0.x * fa.scale, b0.y * fa.scale};
    C a, at;
    if (w == 0.0) {
      a = C{F.x + t * G.x, F.y + t * G.y};
      at = G;
    } else {
      double sn, co;
      sincos(w * t, &sn, &co);
      const double sw = sn / w;
      a = C{F.x * co + G.x * sw, F.y * co + G.y * sw};
      at = C{-F.x * w * sn + G.x * co, -F.y * w * sn + G.y * co};
    }
    A[pad<double>(ky)] = C{a.x, -a.y};  // conj: inverse by a forward transform
    Bv[pad<double>(ky)] = C{at.x, -at.y};
  }
  __syncthreads();
#pragma unroll 1
  for (int h = 0; h < 2; ++h) block_fft<double, LOGNY, E>(h ? Bv : A, tid, true, tw, 1);
  for (int y = tid; y < N; y += blockDim.x) {
    const C u = A[pad<double>(y)], v = Bv[pad<double>(y)];
    colu[(size_t)y * fa.pitch] = C{u.x, -u.y};
    colt[(size_t)y * fa.pitch] = C{v.x, -v.y};
  }
}

template <int LOGNY>
static void wave_cols_p2_launch(const FftArgs& fa, int n_f, void* inter, double c, double t,
                                double Lx, double Ly, cudaStream_t s) {
  const size_t sm = 2 * (size_t)padded<double>(1 << LOGNY) * sizeof(double2);
  cudaFuncSetAttribute(k_wave_cols_p2<LOGNY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_wave_cols_p2<LOGNY><<<dim3(fa.nx / 2 + 1, n_f), (1 << LOGNY) / 8, sm, s>>>(
      fa, n_f, (double2*)inter, c, t, Lx, Ly);
}

// ------------------------------------------------------------------------- //
// Fourier Forwarding solve, per small step (FP64, ff.cu): the modal advance of the
// normalised half spectra to time tau (a = F t0 + G t1 with (t0, t1) = (cos w tau,
// sin(w tau)/w), or for the time derivative (-w sin w tau, cos w tau); (1, tau) and
// (0, 1) at w = 0) and the inverse column DFT as a forward transform of the conjugate.
// One block per (column, output) loops over the n_f functions, so the 2 ny time
// factors of its column are computed once (in shared memory) for all of them; the
// transform runs on the compile-time Stockham stages in padded shared memory.
// ------------------------------------------------------------------------- //
template <int LOGNY>
__global__ void __launch_bounds__((1 << LOGNY) / 8)
    k_ff_cols_p2(FftArgs fa, int n_f, const double2* __restrict__ spec, double2* __restrict__ out,
                 double c, double tau, double Lx, double Ly) {
  using C = double2;
  constexpr int N = 1 << LOGNY, E = 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* tab = reinterpret_cast<double2*>(smem_raw);
  C* buf = tab + N;
  const int nxh = fa.nx / 2 + 1, kx = blockIdx.x, which = blockIdx.y, tid = threadIdx.x;
  const double two_pi = 6.283185307179586476925286766559;
  for (int ky = tid; ky < N; ky += blockDim.x) {
    const int m = ky <= N / 2 ? ky : ky - N;
    const double fl = kx / Lx, fm = m / Ly;
    const double w = two_pi * c * sqrt(fl * fl + fm * fm);
    double t0, t1;
    if (w == 0.0) {
      t0 = which ? 0.0 : 1.0;
      t1 = which ? 1.0 : tau;
    } else {
      double sn, co;
      sincos(w * tau, &sn, &co);
      t0 = which ? -w * sn : co;
      t1 = which ? co : sn / w;
    }
    tab[ky] = double2{t0, t1};
  }
  const C* tw = reinterpret_cast<const C*>(fa.tsy);
  for (int f = 0; f < n_f; ++f) {
    const C* colF = spec + (size_t)f * N * nxh + kx;
    const C* colG = spec + (size_t)(n_f + f) * N * nxh + kx;
    __syncthreads();  // the table is ready; the previous function's stores are done
    for (int ky = tid; ky < N; ky += blockDim.x) {
      const double2 t = tab[ky];
      const C F = colF[(size_t)ky * nxh], G = colG[(size_t)ky * nxh];
      buf[pad<double>(ky)] = C{F.x * t.x + G.x * t.y, -(F.y * t.x + G.y * t.y)};
    }
    __syncthreads();
    block_fft<double, LOGNY, E>(buf, tid, true, tw, 1);
    C* dst = out + ((size_t)which * n_f + f) * N * fa.pitch + kx;
    for (int y = tid; y < N; y += blockDim.x) {
      const C r = buf[pad<double>(y)];
      dst[(size_t)y * fa.pitch] = C{r.x, -r.y};
    }
  }
}

template <int LOGNY>
static void ff_cols_p2_launch(const FftArgs& fa, int n_f, int n_out, const void* spec, void* out,
                              double c, double tau, double Lx, double Ly, cudaStream_t s) {
  const size_t sm = ((size_t)(1 << LOGNY) + padded<double>(1 << LOGNY)) * sizeof(double2);
  cudaFuncSetAttribute(k_ff_cols_p2<LOGNY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_ff_cols_p2<LOGNY><<<dim3(fa.nx / 2 + 1, n_out), (1 << LOGNY) / 8, sm, s>>>(
      fa, n_f, (const double2*)spec, (double2*)out, c, tau, Lx, Ly);
}

template <typename T, typename TV, int L>
static void rows_launch(const FftArgs& fa, const RowArgs& ra, int n_f, int mode, const void* ext,
                        const double* fg, const void* vals, void* inter, cudaStream_t s) {
  constexpr int NT = row_threads<T, L>();
  const size_t sm = (size_t)padded<T>(1 << L) * sizeof(typename Cx<T>::type);
  auto k = k_fft_rows_p2<T, TV, L>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  launch_pdl(k, dim3(fa.ny, n_f), dim3(NT), sm, s, fa, ra, mode, (const T*)ext, fg,
             (const TV*)vals, (typename Cx<T>::type*)inter);
}

template <typename T, int L, int CB>
static void cols_launch(const FftArgs& fa, int n_f, const void* inter, void* fhat,
                        cudaStream_t s) {
  using C = typename Cx<T>::type;
  constexpr int NT = (1 << L) / elems<T>();
  const size_t sm = ((size_t)CB * padded<T>(1 << L) + col_lanes<T>()) * sizeof(C);
  auto k = k_fft_cols_p2<T, L, CB>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  const int ncol = fa.nx / 2 + 1;
  launch_pdl(k, dim3((ncol + CB - 1) / CB, n_f), dim3(CB * NT), sm, s, fa, (const C*)inter,
             (C*)fhat);
}

}  // namespace p2

static int ilog2_exact(int n) {
  if (n <= 0 || (n & (n - 1))) return -1;
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

// Power-of-two fast path.  Returns false (nothing launched) for other sizes.
bool launch_fft_rows_p2(const FftArgs& fa, const RowArgs& ra, int n_f, bool fp64, int mode,
                        const void* ext, const double* f_grid, const void* vals, void* inter,
                        cudaStream_t s) {
  const int L = ilog2_exact(fa.nx / 2);
#define FC2D_ROWS(LL)                                                                    \
  case LL:                                                                               \
    if (fp64)                                                                            \
      p2::rows_launch<double, double, LL>(fa, ra, n_f, mode, ext, f_grid, vals, inter, s); \
    else                                                                                 \
      p2::rows_launch<float, float, LL>(fa, ra, n_f, mode, ext, f_grid, vals, inter, s);   \
    return true;
  switch (L) {
    FC2D_ROWS(5)
    FC2D_ROWS(6)
    FC2D_ROWS(7)
    FC2D_ROWS(8)
    FC2D_ROWS(9)
    FC2D_ROWS(10)
    FC2D_ROWS(11)
    FC2D_ROWS(12)
    default: return false;
  }
#undef FC2D_ROWS
}

// FP32 rows of 2 x 64 N2 reals for N2 = 3, 5, 6, 10, 12.  Returns false (nothing launched)
// for other sizes.
bool launch_fft_rows_64n(const FftArgs& fa, const RowArgs& ra, int n_f, bool fp64, int mode,
                         const void* ext, const double* f_grid, const void* vals, void* inter,
                         cudaStream_t s) {
  if (fp64 || fa.nx % 128) return false;
  switch (fa.nx / 128) {
    case 3: p2::rows64n_launch<3>(fa, ra, n_f, mode, ext, f_grid, vals, inter, s); return true;
    case 5: p2::rows64n_launch<5>(fa, ra, n_f, mode, ext, f_grid, vals, inter, s); return true;
    case 6: p2::rows64n_launch<6>(fa, ra, n_f, mode, ext, f_grid, vals, inter, s); return true;
    case 10: p2::rows64n_launch<10>(fa, ra, n_f, mode, ext, f_grid, vals, inter, s); return true;
    case 12: p2::rows64n_launch<12>(fa, ra, n_f, mode, ext, f_grid, vals, inter, s); return true;
    default: return false;
  }
}

// FP32 columns of 64 N2 points for N2 = 6, 10, 12, 24 (two passes).  Returns false
// (nothing launched) for other sizes.
bool launch_fft_cols_64n(const FftArgs& fa, int n_f, bool fp64, void* inter, void* fhat,
                         cudaStream_t s) {
  if (fp64 || fa.ny % 64) return false;
  switch (fa.ny / 64) {
    case 6: p2::cols64_launch<2, 3>(fa, n_f, inter, fhat, s); return true;
    case 10: p2::cols64_launch<2, 5>(fa, n_f, inter, fhat, s); return true;
    case 12: p2::cols64_launch<4, 3>(fa, n_f, inter, fhat, s); return true;
    case 24: p2::cols64_launch<8, 3>(fa, n_f, inter, fhat, s); return true;
    default: return false;
  }
}

bool launch_fft_cols_p2(const FftArgs& fa, int n_f, bool fp64, void* inter, void* fhat,
                        cudaStream_t s) {
  const int L = ilog2_exact(fa.ny);
#define FC2D_COLS(LL, CB32, CB64)                                  \
  case LL:                                                         \
    if (fp64)                                                      \
      p2::cols_launch<double, LL, CB64>(fa, n_f, inter, fhat, s);  \
    else                                                           \
      p2::cols_launch<float, LL, CB32>(fa, n_f, inter, fhat, s);   \
    return true;
  switch (L) {
    FC2D_COLS(6, 8, 8)
    FC2D_COLS(7, 8, 8)
    FC2D_COLS(8, 8, 4)
    FC2D_COLS(9, 4, 4)
    FC2D_COLS(10, 4, 2)
    default: break;
  }
  // 2048- and 4096-point FP32 columns: two coalesced passes (64 x 32, 64 x 64)
  switch (L) {
    case 11:  // FP32: two passes of 64 x 32 (as the mixed-radix columns, N2 = 32)
      if (fp64) p2::cols_launch<double, 11, 2>(fa, n_f, inter, fhat, s);
      else p2::cols64_launch<4, 8>(fa, n_f, inter, fhat, s);
      return true;
    case 12:
      if (fp64) p2::cols_launch<double, 12, 1>(fa, n_f, inter, fhat, s);
      else p2::cols4k_launch(fa, n_f, inter, fhat, s);
      return true;
    default: return false;
  }
#undef FC2D_COLS
}

// FP64 inverse real rows with nx/2 = 2^8 .. 2^11; false (nothing launched) otherwise.
bool launch_inverse_rows_p2(const FftArgs& fa, int n_f, const void* inter, const double* c00,
                            double a0, double b0, double h, double* out, cudaStream_t s) {
  if (!fa.tsx || !fa.rtw) return false;  // needs the per-stage twiddle table
  switch (ilog2_exact(fa.nx / 2)) {
    case 8: p2::inverse_rows_p2_launch<8>(fa, n_f, inter, c00, a0, b0, h, out, s); return true;
    case 9: p2::inverse_rows_p2_launch<9>(fa, n_f, inter, c00, a0, b0, h, out, s); return true;
    case 10: p2::inverse_rows_p2_launch<10>(fa, n_f, inter, c00, a0, b0, h, out, s); return true;
    case 11: p2::inverse_rows_p2_launch<11>(fa, n_f, inter, c00, a0, b0, h, out, s); return true;
    default: return false;
  }
}

// Fourier Forwarding columns of 2048 or 4096 points; false (nothing launched) otherwise.
bool launch_wave_cols_p2(const FftArgs& fa, int n_f, void* inter, double c, double t,
                         double Lx, double Ly, cudaStream_t s) {
  if (!fa.tsy) return false;  // needs the per-stage twiddle table
  switch (ilog2_exact(fa.ny)) {
    case 11: p2::wave_cols_p2_launch<11>(fa, n_f, inter, c, t, Lx, Ly, s); return true;
    case 12: p2::wave_cols_p2_launch<12>(fa, n_f, inter, c, t, Lx, Ly, s); return true;
    default: return false;
  }
}

// One-time host setup of the 4096-point passes' TMA form on the current device (the
// shared-memory limit, the occupancy query, the tensor-map encoder), at plan time,
// outside any stream capture a later call may run under.
void cols4k_prepare() {
  int nsm = 0;
  using p2::kTmaStages;
  p2::cols_tma_blocks<0, 16, kTmaStages>(&nsm);
  p2::cols_tma_blocks<1, 16, kTmaStages>(&nsm);
  p2::cols_tma_blocks<0, 32, kTmaStages>(&nsm);
  p2::cols_tma_blocks<1, 32, kTmaStages>(&nsm);
  p2::encode_tiled();
}

// Whether the TMA form with cc columns per tile can run on the intermediate `inter` of
// n_f functions (its launch shape on this device and both tensor maps); where it cannot,
// a plan set to it runs the direct form with the same width.
bool cols4k_tma_usable(const FftArgs& fa, int cc, int n_f, void* inter) {
  if (fa.ny != 4096 || !fa.status || (cc != 16 && cc != 32)) return false;
  int nsm = 0;
  using p2::kTmaStages;
  const int nb = cc == 32 ? std::min(p2::cols_tma_blocks<0, 32, kTmaStages>(&nsm),
                                     p2::cols_tma_blocks<1, 32, kTmaStages>(&nsm))
                          : std::min(p2::cols_tma_blocks<0, 16, kTmaStages>(&nsm),
                                     p2::cols_tma_blocks<1, 16, kTmaStages>(&nsm));
  CUtensorMap t;
  return nb > 0 && nsm > 0 && p2::cols_tma_map(0, cc, fa, n_f, inter, &t) &&
         p2::cols_tma_map(1, cc, fa, n_f, inter, &t);
}

// Fourier Forwarding solve columns of 512 .. 4096 points; false (nothing launched)
// otherwise.
bool launch_ff_cols_p2(const FftArgs& fa, int n_f, int n_out, const void* spec, void* out,
                       double c, double tau, double Lx, double Ly, cudaStream_t s) {
  if (!fa.tsy) return false;  // needs the per-stage twiddle table
  switch (ilog2_exact(fa.ny)) {
    case 9: p2::ff_cols_p2_launch<9>(fa, n_f, n_out, spec, out, c, tau, Lx, Ly, s); return true;
    case 10: p2::ff_cols_p2_launch<10>(fa, n_f, n_out, spec, out, c, tau, Lx, Ly, s); return true;
    case 11: p2::ff_cols_p2_launch<11>(fa, n_f, n_out, spec, out, c, tau, Lx, Ly, s); return true;
    case 12: p2::ff_cols_p2_launch<12>(fa, n_f, n_out, spec, out, c, tau, Lx, Ly, s); return true;
    default: return false;
  }
}

}  // namespace fc2d
