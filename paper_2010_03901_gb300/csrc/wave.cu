// Fourier Forwarding interior propagator (Section 4.2, eqs. (4.8)-(4.12)), FP64.
//
// For n_f pairs (u, u_t): the fused extension + row DFT of both, then k_wave_cols per
// column: forward column DFTs of the two spectra, the modal advance
//   a = hat f cos(w t) + hat g sin(w t)/w,  a' = -w hat f sin(w t) + hat g cos(w t)
//   (a_00 = hat f + t hat g, a'_00 = hat g), w = 2 pi c sqrt((l/L_x)^2 + (m/L_y)^2),
// and the inverse column DFTs; then the inverse real row DFTs give U_FC(., t) and its
// time derivative on the whole grid (the solution at distance >= c t from the curve).
#include <cuda_runtime.h>

#include <cstdint>

#include "fc2d_kernels.cuh"
#include "fft_generic.cuh"
#include "plan_internal.h"

namespace fc2d {

// one block per (column, pair); shared: three columns of ny complex values
__global__ void __launch_bounds__(256) k_wave_cols(FftArgs fa, int n_f, double2* inter, double c,
                                                   double t, double Lx, double Ly) {
  using C = double2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ny = fa.ny, kx = blockIdx.x, f = blockIdx.y;
  C* A = reinterpret_cast<C*>(smem_raw);
  C* Bv = A + ny;
  C* S = Bv + ny;
  C* colu = inter + (size_t)f * ny * fa.pitch + kx;
  C* colt = inter + (size_t)(n_f + f) * ny * fa.pitch + kx;
  const C* tw = reinterpret_cast<const C*>(fa.twy);
  for (int y = threadIdx.x; y < ny; y += blockDim.x) A[y] = colu[(size_t)y * fa.pitch];
  __syncthreads();
  C* r = stockham<double>(A, S, ny, 1, fa.ry, fa.nry, tw, 1);
  if (r != A) {
    for (int y = threadIdx.x; y < ny; y += blockDim.x) A[y] = r[y];
    __syncthreads();
  }
  for (int y = threadIdx.x; y < ny; y += blockDim.x) Bv[y] = colt[(size_t)y * fa.pitch];
  __syncthreads();
  r = stockham<double>(Bv, S, ny, 1, fa.ry, fa.nry, tw, 1);
  if (r != Bv) {
    for (int y = threadIdx.x; y < ny; y += blockDim.x) Bv[y] = r[y];
    __syncthreads();
  }
  const double two_pi = 6.283185307179586476925286766559;
  for (int ky = threadIdx.x; ky < ny; ky += blockDim.x) {
    const int m = ky <= ny / 2 ? ky : ky - ny;
    const double fl = kx / Lx, fm = m / Ly;
    const double w = two_pi * c * sqrt(fl * fl + fm * fm);
    const C F = C{A[ky].x * fa.scale, A[ky].y * fa.scale};
    const C G = C{Bv[ky].x * fa.scale, Bv[ky].y * fa.scale};
    C a, at;
    if (w == 0.0) {
      a = C{F.x + t * G.x, F.y + t * G.y};
      at = G;
    } else {
      double s, co;
      sincos(w * t, &s, &co);
      const double sw = s / w;
      a = C{F.x * co + G.x * sw, F.y * co + G.y * sw};
      at = C{-F.x * w * s + G.x * co, -F.y * w * s + G.y * co};
    }
    A[ky] = C{a.x, -a.y};     // conj: inverse by a forward transform
    Bv[ky] = C{at.x, -at.y};
  }
  __syncthreads();
  r = stockham<double>(A, S, ny, 1, fa.ry, fa.nry, tw, 1);
  for (int y = threadIdx.x; y < ny; y += blockDim.x) colu[(size_t)y * fa.pitch] = C{r[y].x, -r[y].y};
  __syncthreads();
  r = stockham<double>(Bv, S, ny, 1, fa.ry, fa.nry, tw, 1);
  for (int y = threadIdx.x; y < ny; y += blockDim.x) colt[(size_t)y * fa.pitch] = C{r[y].x, -r[y].y};
}

bool launch_wave_cols_p2(const FftArgs& fa, int n_f, void* inter, double c, double t,
                         double Lx, double Ly, cudaStream_t s);

void launch_wave_cols(const FftArgs& fa, int n_f, void* inter, double c, double t, double Lx,
                      double Ly, cudaStream_t s) {
  if (launch_wave_cols_p2(fa, n_f, inter, c, t, Lx, Ly, s)) return;
  const size_t sm = 3 * (size_t)fa.ny * sizeof(double2);
  cudaFuncSetAttribute(k_wave_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_wave_cols<<<dim3(fa.nx / 2 + 1, n_f), 256, sm, s>>>(fa, n_f, (double2*)inter, c, t, Lx, Ly);
}

}  // namespace fc2d
