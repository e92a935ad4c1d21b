// Generic mixed-radix (2, 3, 4, 5, 8) Stockham transform in shared memory, shared by
// the DFT kernels and the Poisson multiplier kernels.  Stockham autosort: butterfly j
// of a radix-R stage over sub-transforms of length Ns reads x[j + r N/R], multiplies
// by exp(-2 pi i r (j mod Ns)/(Ns R)) and writes y[(j/Ns) Ns R + (j mod Ns) + r Ns]
// (Govindaraju et al., SC 2008).
#pragma once
#include <cuda_runtime.h>

namespace fc2d {

template <typename T> struct Cx;
template <> struct Cx<double> { using type = double2; };
template <> struct Cx<float> { using type = float2; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return {a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return {a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C> __device__ __forceinline__ C mul_mi(C a) { return {a.y, -a.x}; }  // * (-i)
template <typename C> __device__ __forceinline__ C conj_(C a) { return {a.x, -a.y}; }

// forward DFT of length R in registers (R = 2, 3, 4, 5, 8)
template <typename T, typename C>
__device__ __forceinline__ void dft_small(C* v, int R) {
  if (R == 2) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if (R == 4) {
    C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    C t2 = cadd(v[1], v[3]), t3 = mul_mi(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  } else if (R == 8) {
    const T s = (T)0.70710678118654752440;
    C e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    dft_small<T, C>(e, 4);
    dft_small<T, C>(o, 4);
    // twiddles exp(-2 pi i k/8), k = 0..3
    C w1 = {s * (o[1].x + o[1].y), s * (o[1].y - o[1].x)};
    C w2 = mul_mi(o[2]);
    C w3 = {s * (o[3].y - o[3].x), -s * (o[3].x + o[3].y)};
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], w1);
    v[5] = csub(e[1], w1);
    v[2] = cadd(e[2], w2);
    v[6] = csub(e[2], w2);
    v[3] = cadd(e[3], w3);
    v[7] = csub(e[3], w3);
  } else if (R == 3) {
    const T c1 = (T)-0.5, s1 = (T)0.86602540378443864676;  // exp(-2 pi i/3) = c1 - i s1
    C a = v[0], b = v[1], c = v[2];
    C sbc = cadd(b, c), dbc = csub(b, c);
    v[0] = cadd(a, sbc);
    C m = {a.x + c1 * sbc.x, a.y + c1 * sbc.y};
    C r = {s1 * dbc.y, -s1 * dbc.x};  // -i s1 (b - c)
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
  } else if (R == 5) {
    const T c1 = (T)0.30901699437494742410, s1 = (T)0.95105651629515357212;
    const T c2 = (T)-0.80901699437494742410, s2 = (T)0.58778525229247312917;
    C a = v[0];
    C s14 = cadd(v[1], v[4]), d14 = csub(v[1], v[4]);
    C s23 = cadd(v[2], v[3]), d23 = csub(v[2], v[3]);
    v[0] = cadd(a, cadd(s14, s23));
    C m1 = {a.x + c1 * s14.x + c2 * s23.x, a.y + c1 * s14.y + c2 * s23.y};
    C m2 = {a.x + c2 * s14.x + c1 * s23.x, a.y + c2 * s14.y + c1 * s23.y};
    // -i (s1 d14 + s2 d23) and -i (s2 d14 - s1 d23)
    C r1 = {s1 * d14.y + s2 * d23.y, -(s1 * d14.x + s2 * d23.x)};
    C r2 = {s2 * d14.y - s1 * d23.y, -(s2 * d14.x - s1 * d23.x)};
    v[1] = cadd(m1, r1);
    v[4] = csub(m1, r1);
    v[2] = cadd(m2, r2);
    v[3] = csub(m2, r2);
  }
}

// nbatch transforms of length N stored contiguously (stride N) in a; b is scratch of
// the same size.  Returns the buffer holding the result.  tw: exp(-2 pi i t/Ntab),
// read at stride tws (Ntab = N tws).
template <typename T>
__device__ typename Cx<T>::type* stockham(typename Cx<T>::type* a, typename Cx<T>::type* b,
                                          int N, int nbatch, const int* radix, int nrad,
                                          const typename Cx<T>::type* __restrict__ tw,
                                          int tws) {
  using C = typename Cx<T>::type;
  int Ns = 1;
  for (int st = 0; st < nrad; ++st) {
    const int R = radix[st];
    const int NR = N / R;
    const int tstep = N / (Ns * R);
    // quotients by NR and Ns as (x + 1/2) * (1/d) truncated: exact for every x < 2^22
    // and every divisor 2^a 3^b 5^c <= 8192, far cheaper than integer division by a
    // runtime divisor
    const float inv_NR = 1.0f / (float)NR, inv_Ns = 1.0f / (float)Ns;
    for (int idx = threadIdx.x; idx < nbatch * NR; idx += blockDim.x) {
      const int c = (int)(((float)idx + 0.5f) * inv_NR), j = idx - c * NR;
      const int q = (int)(((float)j + 0.5f) * inv_Ns), k = j - q * Ns;
      const C* src = a + (size_t)c * N;
      C v[8];
#pragma unroll
      for (int r = 0; r < 8; ++r)
        if (r < R) {
          C x = src[j + r * NR];
          if (r > 0 && k > 0) x = cmul(x, __ldg(tw + (size_t)r * k * tstep * tws));
          v[r] = x;
        }
      dft_small<T, C>(v, R);
      C* dst = b + (size_t)c * N + q * Ns * R + k;
#pragma unroll
      for (int r = 0; r < 8; ++r)
        if (r < R) dst[r * Ns] = v[r];
    }
    __syncthreads();
    C* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

}  // namespace fc2d
