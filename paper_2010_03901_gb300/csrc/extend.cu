// 2D-FC Cartesian evaluation kernels (Section 3.5, steps 5-6) and the plan-time Newton
// foot search (step 4).
//
//   k_foot_newton     FP64 Newton on (q(t) - Q).q'(t) = 0 for every strip candidate.
//   k_gather_blend    one warp per (normal, function): the two-step interpolation of
//                     Section 3.2 gives the matching values f_{D_p}; then the Gram
//                     coefficients c = Q^T f_{D_p} and the strip values A_r c (eq. (2.6),
//                     Remark 2.2).  FP64; in the mixed form the warp stops at c.
//   k_interp          one thread per (strip point, function): the theta/eta Lagrange
//                     interpolation of Section 3.4 with FP64 weights.
//   k_assemble_rows   one block per (row, function): f on the inside intervals, the
//                     strip values, 0 elsewhere -> the extended grid.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "fc2d_kernels.cuh"
#include "interp.cuh"
#include "plan_internal.h"

namespace fc2d {

// ------------------------------------------------------------------------- //
// Newton foot search (plan time)
// ------------------------------------------------------------------------- //
constexpr int kMaxModes = 64;
__constant__ double c_curve[4 * kMaxModes];

__device__ void curve_eval(int nm, double t, double* x, double* y) {
  // x[0..2], y[0..2]: value, first and second derivative
  for (int d = 0; d < 3; ++d) x[d] = y[d] = 0.0;
  for (int k = 0; k < nm; ++k) {
    double s, c;
    sincos(double(k) * t, &s, &c);
    double ax = c_curve[k], bx = c_curve[kMaxModes + k];
    double ay = c_curve[2 * kMaxModes + k], by = c_curve[3 * kMaxModes + k];
    double kk = double(k);
    x[0] += ax * c + bx * s;
    y[0] += ay * c + by * s;
    x[1] += kk * (-ax * s + bx * c);
    y[1] += kk * (-ay * s + by * c);
    x[2] -= kk * kk * (ax * c + bx * s);
    y[2] -= kk * kk * (ay * c + by * s);
  }
}

// Seed: the closest of 2 kFootSamples + 1 curve samples within +-window of the given
// parameter; then Newton.
constexpr int kFootSamples = 24;

__global__ void k_foot_newton(int n, int nm, const double* __restrict__ qx,
                              const double* __restrict__ qy, double* __restrict__ th,
                              int* __restrict__ conv, double window) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double t = th[i], X = qx[i], Y = qy[i];
  {
    const double t0 = t;
    double best = 1e300;
    for (int k = -kFootSamples; k <= kFootSamples; ++k) {
      const double tk = t0 + window * double(k) / kFootSamples;
      double x[3], y[3];
      curve_eval(nm, tk, x, y);
      const double d2 = (x[0] - X) * (x[0] - X) + (y[0] - Y) * (y[0] - Y);
      if (d2 < best) {
        best = d2;
        t = tk;
      }
    }
  }
  int ok = 0;
  for (int it = 0; it < 60; ++it) {  // iteration cap: no unbounded loop
    double x[3], y[3];
    curve_eval(nm, t, x, y);
    double phi = (x[0] - X) * x[1] + (y[0] - Y) * y[1];
    double dphi = x[1] * x[1] + y[1] * y[1] + (x[0] - X) * x[2] + (y[0] - Y) * y[2];
    if (!(dphi > 0.0)) break;  // not a local minimum of the distance: give up
    double step = phi / dphi;
    t -= step;
    if (fabs(step) < 1e-12) {  // quadratic convergence: one more step reaches round-off
      curve_eval(nm, t, x, y);
      phi = (x[0] - X) * x[1] + (y[0] - Y) * y[1];
      dphi = x[1] * x[1] + y[1] * y[1] + (x[0] - X) * x[2] + (y[0] - Y) * y[2];
      if (dphi > 0.0) t -= phi / dphi;
      ok = 1;
      break;
    }
  }
  th[i] = t;
  conv[i] = ok;
}

fc2d_status foot_newton_gpu(const Curve& c, const std::vector<double>& qx,
                            const std::vector<double>& qy, std::vector<double>& theta,
                            std::vector<int>& conv, double window) {
  int nm = (int)c.cx.size();
  if (nm > kMaxModes) return set_error(FC2D_ERR_UNSUPPORTED, "boundary has too many modes");
  size_t n = qx.size();
  conv.assign(n, 0);
  if (n == 0) return FC2D_OK;
  std::vector<double> cc(4 * kMaxModes, 0.0);
  for (int k = 0; k < nm; ++k) {
    cc[k] = c.cx[k];
    cc[kMaxModes + k] = c.sx[k];
    cc[2 * kMaxModes + k] = c.cy[k];
    cc[3 * kMaxModes + k] = c.sy[k];
  }
  double *dqx = nullptr, *dqy = nullptr, *dth = nullptr;
  int* dconv = nullptr;
  fc2d_status st = FC2D_OK;
  if (cudaMalloc(&dqx, n * 8) || cudaMalloc(&dqy, n * 8) || cudaMalloc(&dth, n * 8) ||
      cudaMalloc(&dconv, n * 4)) {
    st = set_error(FC2D_ERR_NOMEM, "foot search: cudaMalloc failed");
  } else {
    cudaMemcpyToSymbol(c_curve, cc.data(), cc.size() * 8);
    cudaMemcpy(dqx, qx.data(), n * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(dqy, qy.data(), n * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(dth, theta.data(), n * 8, cudaMemcpyHostToDevice);
    k_foot_newton<<<(unsigned)((n + 127) / 128), 128>>>((int)n, nm, dqx, dqy, dth, dconv,
                                                         window);
    st = cuda_check(cudaGetLastError(), "foot search launch");
    if (st == FC2D_OK) st = cuda_check(cudaDeviceSynchronize(), "foot search");
    if (st == FC2D_OK) {
      cudaMemcpy(theta.data(), dth, n * 8, cudaMemcpyDeviceToHost);
      cudaMemcpy(conv.data(), dconv, n * 4, cudaMemcpyDeviceToHost);
    }
  }
  cudaFree(dqx);
  cudaFree(dqy);
  cudaFree(dth);
  cudaFree(dconv);
  return st;
}

// ------------------------------------------------------------------------- //
// Matching values + blending (Section 3.2, eq. (2.6))
// ------------------------------------------------------------------------- //
// A warp serves 32/GS normals, one group of GS lanes each.  In a group, lane s < M-1
// evaluates red star s (M taps), lane s < d-1 forms the matching value at r_{p,s}
// (lane d-1 holds the boundary datum), lane s < d the Gram coefficient
// c_s = sum_i Q[i][s] f_D[i]; then the group writes F[q] = (A_r c)_q (FP64 form) or the
// Gram coefficients (mixed form, consumed by the tensor-core contraction).
template <bool kFp64Blend, int GS>
__global__ void __launch_bounds__(256) k_gather_blend(GatherArgs a) {
  const int lane = threadIdx.x & 31;
  const int s = lane & (GS - 1), g0 = lane & ~(GS - 1);
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int f = blockIdx.y;
  const int p = warp * (32 / GS) + lane / GS;
  const bool live = p < a.B;
  const int pp = live ? p : 0;
  const int M = a.M, d = a.d, NS = M - 1;
  const double* fg = a.f_grid + (size_t)f * a.grid_stride;
  const double* fb = a.f_bdry ? a.f_bdry + (size_t)f * a.n_bdry : nullptr;
  const int nq = a.nq;
  pdl_wait();
  pdl_trigger();
  double star = 0.0;
  if (s < NS) {
    const int32_t* gi = a.gidx + ((size_t)pp * NS + s) * M;
    const double* gw = a.gw + ((size_t)pp * NS + s) * M;
    for (int e = 0; e < M; ++e) {
      int32_t id = __ldg(gi + e);
      double v = id >= 0 ? __ldg(fg + id) : __ldg(fb + (-1 - id));
      star = fma(__ldg(gw + e), v, star);
    }
  }
  const double fbp = fb ? __ldg(fb + pp) : 0.0;
  double fD;
  {
    const double* wn = a.wn + ((size_t)pp * nq + (s < nq ? s : 0)) * M;
    double acc = (s < nq) ? __ldg(wn) * fbp : 0.0;
    for (int e = 1; e < M; ++e) {
      const double st = __shfl_sync(0xffffffffu, star, g0 + e - 1);
      if (s < nq) acc = fma(__ldg(wn + e), st, acc);
    }
    fD = s < nq ? acc : (s == d - 1 ? fbp : 0.0);
  }
  // the value at the foot: the boundary datum, or its extrapolation (interior data)
  const double f0 = __shfl_sync(0xffffffffu, fD, g0 + d - 1);
  double cs = 0.0;  // Gram coefficient c_s (lanes s < d)
  for (int i = 0; i < d; ++i) {
    const double v = __shfl_sync(0xffffffffu, fD, g0 + i);
    if (s < d) cs = fma(__ldg(a.Q + i * d + s), v, cs);
  }
  if (kFp64Blend) {
    double c[GS];  // d <= GS: every Gram coefficient of the group
#pragma unroll
    for (int j = 0; j < GS; ++j) c[j] = __shfl_sync(0xffffffffu, cs, g0 + (j < d ? j : 0));
    if (!live) return;
    double* F = reinterpret_cast<double*>(a.F) + ((size_t)f * a.B + p) * (a.Cr + 1);
    if (s == 0) F[0] = f0;
    for (int q = s; q < a.Cr; q += GS) {
      const double* ar = a.Ar + (size_t)q * d;
      double v = 0.0;
#pragma unroll
      for (int j = 0; j < GS; ++j)
        if (j < d) v = fma(__ldg(ar + j), c[j], v);
      F[q + 1] = v;
    }
  } else {
    if (!live) return;
    if (s < d) a.coef[((size_t)f * a.B + p) * a.coef_ld + s] = cs;
    if (s == 0) a.bvals[(size_t)f * a.B + p] = f0;
  }
}

void launch_gather_blend(const GatherArgs& a, int n_f, bool fp64, cudaStream_t s) {
  // group size: the larger of M-1 red stars and d coefficients, rounded up to 8 or 16
  // (the plan keeps M <= 16 and d <= 12)
  const int GS = (a.M - 1 <= 8 && a.d <= 8) ? 8 : 16;
  const int per_warp = 32 / GS;
  const int warps = (a.B + per_warp - 1) / per_warp;
  dim3 grid((warps * 32 + 255) / 256, n_f);
  auto k = GS == 8 ? (fp64 ? k_gather_blend<true, 8> : k_gather_blend<false, 8>)
                    : (fp64 ? k_gather_blend<true, 16> : k_gather_blend<false, 16>);
  launch_pdl(k, grid, dim3(256), 0, s, a);
}

// ------------------------------------------------------------------------- //
// Interpolation onto the strip points (Section 3.4)
// ------------------------------------------------------------------------- //
// Lagrange weights at t for the nodes 0..M-1: prefix/suffix products of (t - m)
// times 1/prod_{m != k}(k - m).
__device__ __forceinline__ void lagrange_equispaced(int M, double t, double* w) {
  double pre[kMaxM], suf[kMaxM];
  pre[0] = 1.0;
  for (int k = 1; k < M; ++k) pre[k] = pre[k - 1] * (t - double(k - 1));
  suf[M - 1] = 1.0;
  for (int k = M - 2; k >= 0; --k) suf[k] = suf[k + 1] * (t - double(k + 1));
  // 1/prod_{m != k}(k - m) = (-1)^(M-1-k) / (k! (M-1-k)!)
  double fact[kMaxM];
  fact[0] = 1.0;
  for (int k = 1; k < M; ++k) fact[k] = fact[k - 1] * double(k);
  for (int k = 0; k < M; ++k) {
    double den = fact[k] * fact[M - 1 - k];
    double v = pre[k] * suf[k] / den;
    w[k] = ((M - 1 - k) & 1) ? -v : v;
  }
}

// Plan time, FP64: per strip point the theta and eta Lagrange weights (2 M values,
// stored [2M][n_strip], as double for the FP64 form and rounded to float for the mixed
// form), the first normal index p0 - K_l (may be negative: rows wrap mod B) and the
// first fine index s.
template <typename TW>
__global__ void k_interp_weights(int n_strip, int M, int Cr, double inv_k2, double nr_over_k1,
                                 const double* __restrict__ theta, const double* __restrict__ eta,
                                 TW* __restrict__ w, int32_t* __restrict__ pb,
                                 int32_t* __restrict__ sb) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_strip) return;
  const int Kl = (M + 1) / 2 - 1;
  double tt = theta[n] * inv_k2;
  double p0 = floor(tt);
  double wth[kMaxM], weta[kMaxM];
  lagrange_equispaced(M, tt - (p0 - Kl), wth);
  double u = eta[n] * nr_over_k1;
  int s = (int)floor(u) - Kl;
  s = s < 0 ? 0 : (s > Cr + 1 - M ? Cr + 1 - M : s);
  lagrange_equispaced(M, u - s, weta);
  for (int k = 0; k < M; ++k) {
    w[(size_t)k * n_strip + n] = (TW)wth[k];
    w[(size_t)(M + k) * n_strip + n] = (TW)weta[k];
  }
  pb[n] = (int32_t)p0 - Kl;
  sb[n] = s;
}

fc2d_status interp_weights_gpu(int n_strip, int M, int Cr, int B, double k1, int n_r,
                               const double* theta_dev, const double* eta_dev, bool fp64,
                               void* w_dev, int32_t* pb_dev, int32_t* sb_dev) {
  if (n_strip == 0) return FC2D_OK;
  const double inv_k2 = B / (2.0 * M_PI), nr_over_k1 = n_r / k1;
  const unsigned g = (unsigned)((n_strip + 255) / 256);
  if (fp64)
    k_interp_weights<double><<<g, 256>>>(n_strip, M, Cr, inv_k2, nr_over_k1, theta_dev, eta_dev,
                                         (double*)w_dev, pb_dev, sb_dev);
  else
    k_interp_weights<float><<<g, 256>>>(n_strip, M, Cr, inv_k2, nr_over_k1, theta_dev, eta_dev,
                                        (float*)w_dev, pb_dev, sb_dev);
  fc2d_status st = cuda_check(cudaGetLastError(), "interpolation weights launch");
  if (st == FC2D_OK) st = cuda_check(cudaDeviceSynchronize(), "interpolation weights");
  return st;
}

// One thread per (strip point, function); the arithmetic is interp_load/interp_apply
// (interp.cuh), accumulated in TA (double for the FP64 form, float for the mixed form).
// The weights are plan constants and are loaded before the wait on the blend kernel.
template <int MM, typename TF, typename TW, typename TA, typename TV, bool VEC>
__global__ void __launch_bounds__(256) k_interp(InterpArgs a, const TF* __restrict__ F,
                                                TV* __restrict__ vals) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int f = blockIdx.y;
  if (n >= a.n_strip) return;
  const InterpPoint<MM, TW> q = interp_load<MM, TW>(a, n);
  pdl_wait();
  pdl_trigger();
  const TF* Ff = F + (size_t)f * a.B * a.ldF;
  vals[(size_t)f * a.n_strip + n] = (TV)interp_apply<MM, TF, TW, TA, VEC>(a, Ff, q);
}

void launch_interp(const InterpArgs& a, int n_f, bool fp64, const void* F, void* vals,
                   cudaStream_t s) {
  if (a.n_strip == 0) return;
  dim3 grid((a.n_strip + 255) / 256, n_f);
  if (fp64) {
    auto k = a.M == 8 ? k_interp<8, double, double, double, double, false>
                      : k_interp<0, double, double, double, double, false>;
    launch_pdl(k, grid, dim3(256), 0, s, a, (const double*)F, (double*)vals);
  } else {
    const bool vec = a.ldF % 4 == 0 && a.ldF >= a.Cr + 12 &&
                     (reinterpret_cast<uintptr_t>(F) & 15) == 0;
    auto k = (a.M == 8 && vec) ? k_interp<8, float, float, float, float, true>
             : (a.M == 7 && vec) ? k_interp<7, float, float, float, float, true>
             : a.M == 8 ? k_interp<8, float, float, float, float, false>
                        : k_interp<0, float, float, float, float, false>;
    launch_pdl(k, grid, dim3(256), 0, s, a, (const float*)F, (float*)vals);
  }
}

// ------------------------------------------------------------------------- //
// Assemble the extended grid row by row (shared-memory row buffer)
// ------------------------------------------------------------------------- //
template <typename T>
__global__ void k_assemble_rows(RowArgs a, const double* __restrict__ f_grid,
                                const T* __restrict__ vals, T* __restrict__ ext) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* row = reinterpret_cast<T*>(smem_raw);
  const int j = blockIdx.x, f = blockIdx.y, nx = a.nx;
  load_row<T>(a, j, f, f_grid + (size_t)f * a.grid_stride, false, vals, row);
  __syncthreads();
  T* out = ext + (size_t)f * a.grid_stride + (size_t)j * nx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) out[i] = row[i];
}

void launch_assemble(const RowArgs& a, int n_f, bool fp64, const double* f_grid,
                     const void* vals, void* ext, cudaStream_t s) {
  dim3 grid(a.ny, n_f);
  size_t sm = (size_t)a.nx * (fp64 ? 8 : 4);
  if (fp64) {
    cudaFuncSetAttribute(k_assemble_rows<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sm);
    k_assemble_rows<double><<<grid, 256, sm, s>>>(a, f_grid, (const double*)vals,
                                                  (double*)ext);
  } else {
    cudaFuncSetAttribute(k_assemble_rows<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sm);
    k_assemble_rows<float><<<grid, 256, sm, s>>>(a, f_grid, (const float*)vals, (float*)ext);
  }
}

}  // namespace fc2d
