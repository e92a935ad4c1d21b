// Hand-written 2D real-to-complex DFT of the extended grid (eq. (3.1), Section 3.5
// step 7) for sizes 2^a 3^b 5^c.
//
// Pass 1 (k_fft_rows): one block per (row, function).  The row of nx reals is loaded
// into shared memory as nx/2 complex pairs z_n = x_{2n} + i x_{2n+1} -- either from an
// extended grid or assembled on the fly from f inside the domain and the strip values
// (fused extension: exterior points are never read).  A mixed-radix Stockham FFT of
// length nx/2 runs in shared memory, then the standard even/odd split gives X_k,
// k = 0..nx/2, written to an intermediate [ny][pitch] array.
// Pass 2 (k_fft_cols): one block per (group of columns, function): the column
// transforms of length ny, scaled by 1/(nx ny), written to fhat [ny][nx/2+1].
//
// Stockham autosort (stage with radix R over sub-transforms of length Ns): butterfly
// j reads x[j + r N/R], multiplies by exp(-2 pi i r (j mod Ns)/(Ns R)) and writes
// y[(j/Ns) Ns R + (j mod Ns) + r Ns] (Govindaraju et al., SC 2008).
#include <cuda_runtime.h>

#include "fc2d_kernels.cuh"
#include "fft_generic.cuh"

namespace fc2d {

template <typename T, typename TV>
__global__ void __launch_bounds__(256) k_fft_rows(FftArgs fa, RowArgs ra, int mode,
                                                  const T* __restrict__ ext,
                                                  const double* __restrict__ f_grid,
                                                  const TV* __restrict__ vals,
                                                  typename Cx<T>::type* __restrict__ inter) {
  using C = typename Cx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nx = fa.nx, Nh = nx / 2;
  C* A = reinterpret_cast<C*>(smem_raw);
  C* Bf = A + Nh;
  const int j = blockIdx.x, f = blockIdx.y;
  T* rowr = reinterpret_cast<T*>(A);
  if (mode == 0) {
    const T* src = ext + (size_t)f * ra.grid_stride + (size_t)j * nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) rowr[i] = src[i];
  } else {
    load_row<T>(ra, j, f, f_grid + (size_t)f * ra.grid_stride, mode == 2, vals, rowr);
  }
  __syncthreads();
  const C* tw = reinterpret_cast<const C*>(fa.twx);
  C* Z = stockham<T>(A, Bf, Nh, 1, fa.rx, fa.nrx, tw, 1);
  // even/odd split: X_k = (Z_k + conj Z_{Nh-k})/2 - i w^k (Z_k - conj Z_{Nh-k})/2
  const C* rtw = reinterpret_cast<const C*>(fa.rtw);
  C* out = inter + ((size_t)f * fa.ny + j) * fa.pitch;
  for (int k = threadIdx.x; k <= Nh; k += blockDim.x) {
    C zk = Z[k == Nh ? 0 : k];
    C zc = conj_(Z[k == 0 ? 0 : Nh - k]);
    C e = {(T)0.5 * (zk.x + zc.x), (T)0.5 * (zk.y + zc.y)};
    C o = {(T)0.5 * (zk.x - zc.x), (T)0.5 * (zk.y - zc.y)};
    C w = __ldg(rtw + k);
    C wo = cmul(w, o);
    out[k] = {e.x + wo.y, e.y - wo.x};  // e - i (w o)
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_fft_cols(FftArgs fa, int cb,
                                                  const typename Cx<T>::type* __restrict__ inter,
                                                  typename Cx<T>::type* __restrict__ fhat) {
  using C = typename Cx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ny = fa.ny, ncol = fa.nx / 2 + 1;
  const int c0 = blockIdx.x * cb, f = blockIdx.y;
  const int nc = min(cb, ncol - c0);
  C* A = reinterpret_cast<C*>(smem_raw);
  C* Bf = A + (size_t)cb * ny;
  const C* src = inter + (size_t)f * ny * fa.pitch + c0;
  for (int idx = threadIdx.x; idx < ny * cb; idx += blockDim.x) {
    int y = idx / cb, c = idx - y * cb;
    A[(size_t)c * ny + y] = c < nc ? src[(size_t)y * fa.pitch + c] : C{0, 0};
  }
  __syncthreads();
  const C* tw = reinterpret_cast<const C*>(fa.twy);
  C* Y = stockham<T>(A, Bf, ny, cb, fa.ry, fa.nry, tw, 1);
  C* dst = fhat + (size_t)f * ny * ncol + c0;
  const T sc = (T)fa.scale;
  for (int idx = threadIdx.x; idx < ny * cb; idx += blockDim.x) {
    int y = idx / cb, c = idx - y * cb;
    if (c < nc) {
      C v = Y[(size_t)c * ny + y];
      dst[(size_t)y * ncol + c] = {v.x * sc, v.y * sc};
    }
  }
}

bool launch_fft_rows_p2(const FftArgs& fa, const RowArgs& ra, int n_f, bool fp64, int mode,
                        const void* ext, const double* f_grid, const void* vals, void* inter,
                        cudaStream_t s);
bool launch_fft_rows_64n(const FftArgs& fa, const RowArgs& ra, int n_f, bool fp64, int mode,
                         const void* ext, const double* f_grid, const void* vals, void* inter,
                         cudaStream_t s);
bool launch_fft_cols_p2(const FftArgs& fa, int n_f, bool fp64, void* inter, void* fhat,
                        cudaStream_t s);
bool launch_fft_cols_64n(const FftArgs& fa, int n_f, bool fp64, void* inter, void* fhat,
                         cudaStream_t s);

void launch_fft_rows(const FftArgs& fa, const RowArgs& ra, int n_f, bool fp64, int mode,
                     const void* ext, const double* f_grid, const void* vals, void* inter,
                     cudaStream_t s) {
  if (launch_fft_rows_p2(fa, ra, n_f, fp64, mode, ext, f_grid, vals, inter, s)) return;
  if (launch_fft_rows_64n(fa, ra, n_f, fp64, mode, ext, f_grid, vals, inter, s)) return;
  dim3 grid(fa.ny, n_f);
  if (fp64) {
    size_t sm = (size_t)fa.nx * sizeof(double2);  // two buffers of nx/2 complex
    auto k = k_fft_rows<double, double>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k<<<grid, 256, sm, s>>>(fa, ra, mode, (const double*)ext, f_grid, (const double*)vals,
                            (double2*)inter);
  } else {
    size_t sm = (size_t)fa.nx * sizeof(float2);
    auto k = k_fft_rows<float, float>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k<<<grid, 256, sm, s>>>(fa, ra, mode, (const float*)ext, f_grid, (const float*)vals,
                            (float2*)inter);
  }
}

static int pick_cb(int ny, size_t csize) {
  const size_t budget = 200 * 1024;
  int cb = 1;
  while (cb < 8 && 2 * (size_t)(2 * cb) * ny * csize <= budget) cb *= 2;
  return cb;
}

void launch_fft_cols(const FftArgs& fa, int n_f, bool fp64, void* inter, void* fhat,
                     cudaStream_t s) {
  if (launch_fft_cols_p2(fa, n_f, fp64, inter, fhat, s)) return;
  if (launch_fft_cols_64n(fa, n_f, fp64, inter, fhat, s)) return;
  const int ncol = fa.nx / 2 + 1;
  if (fp64) {
    int cb = pick_cb(fa.ny, sizeof(double2));
    size_t sm = 2 * (size_t)cb * fa.ny * sizeof(double2);
    auto k = k_fft_cols<double>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k<<<dim3((ncol + cb - 1) / cb, n_f), 256, sm, s>>>(fa, cb, (const double2*)inter,
                                                       (double2*)fhat);
  } else {
    int cb = pick_cb(fa.ny, sizeof(float2));
    size_t sm = 2 * (size_t)cb * fa.ny * sizeof(float2);
    auto k = k_fft_cols<float>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k<<<dim3((ncol + cb - 1) / cb, n_f), 256, sm, s>>>(fa, cb, (const float2*)inter,
                                                       (float2*)fhat);
  }
}

// Full spectrum of a complex function u + i v from the half spectra A of u and B of v
// ([2 n_f][ny][nx/2+1], u and v of function f at 2f and 2f + 1): X[m][l] = A[m][l] +
// i B[m][l] for l <= nx/2, and above, from the Hermitian symmetry of a real function's
// spectrum, X[m][l] = conj(A[-m][nx-l]) + i conj(B[-m][nx-l]).  One block row per (m, f).
template <typename C>
__global__ void __launch_bounds__(256) k_complex_spectrum(int nx, int ny, const C* __restrict__ half,
                                                          C* __restrict__ out) {
  const int m = blockIdx.y, f = blockIdx.z, nh = nx / 2 + 1;
  const C* A = half + (size_t)2 * f * ny * nh;
  const C* B = A + (size_t)ny * nh;
  C* o = out + ((size_t)f * ny + m) * nx;
  const int mc = m ? ny - m : 0;
  pdl_wait();
  pdl_trigger();
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nx; l += gridDim.x * blockDim.x) {
    C a, b;
    if (l < nh) {
      a = A[(size_t)m * nh + l];
      b = B[(size_t)m * nh + l];
    } else {
      a = A[(size_t)mc * nh + (nx - l)];
      b = B[(size_t)mc * nh + (nx - l)];
      a.y = -a.y;
      b.y = -b.y;
    }
    o[l] = C{a.x - b.y, a.y + b.x};
  }
}

void launch_complex_spectrum(int nx, int ny, int n_f, bool fp64, const void* half, void* out,
                             cudaStream_t s) {
  const dim3 grid((nx + 255) / 256, ny, n_f);
  if (fp64)
    launch_pdl(k_complex_spectrum<double2>, grid, dim3(256), 0, s, nx, ny,
               static_cast<const double2*>(half), static_cast<double2*>(out));
  else
    launch_pdl(k_complex_spectrum<float2>, grid, dim3(256), 0, s, nx, ny,
               static_cast<const float2*>(half), static_cast<float2*>(out));
}

}  // namespace fc2d
