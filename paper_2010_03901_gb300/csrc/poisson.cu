// 2D-FC Poisson solver (Section 4.1, eqs. (4.1)-(4.6)), FP64 data; the double-layer
// sums on the grid in double-float arithmetic (about 48 bits, see below).
//
//   u = u_p + v.  u_p: the spectrum of the extension of f times the inverse Laplacian
//   symbol -1/((2 pi l/L_x)^2 + (2 pi m/L_y)^2) (0 at the origin), inverse DFT, plus
//   hat f_00 (x^2 + y^2)/4 (sign taken so that Delta u_p = f^c).
//   v: double-layer potential, -phi/2 + K phi = g - u_p on the curve, trapezoidal
//   Nystrom on N_b equispaced parameters, solved by GMRES (host-driven, device
//   mat-vec and orthogonalisation kernels).  v on the grid points inside: the
//   trapezoidal sum; within 5 s of the curve (s = (2 pi/N_b) max|q'|) the density is
//   refined R = 8 times by trigonometric interpolation and, closer than 5 s/R, v is
//   the degree M_P - 1 Lagrange interpolant along the normal through the boundary
//   value (trigonometric interpolation of g - u_p) and refined sums at 5s/R..(M_P+3)s/R.
//
// Kernels: k_poisson_cols (forward column DFT, multiplier, inverse column DFT in
// shared memory), k_poisson_rows (inverse real row DFT + quadratic term), k_up_nodes,
// GMRES kernels, k_density_dft / k_density_refine, k_dlp (trapezoidal sums over a point
// list), k_dlp_close (one block per close point), k_zero_outside.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "dd.h"
#include "fc2d_kernels.cuh"
#include "fft_generic.cuh"
#include "plan_internal.h"

namespace fc2d {

constexpr int kGmresMax = 200;
constexpr int kRefine = 8;

struct PoissonState {
  int Nb = 0, R = kRefine, MP = 8;
  double s = 0, delta = 0;
  double *bx = nullptr, *by = nullptr, *bx1 = nullptr, *by1 = nullptr;  // nodes [Nb]
  double* A = nullptr;                                                  // [Nb][Nb]
  double *rx = nullptr, *ry = nullptr, *rx1 = nullptr, *ry1 = nullptr;  // refined [R Nb]
  double* twb = nullptr;                                                // e^{-2 pi i t/Nb}
  double* twr = nullptr;                                                // e^{+2 pi i t/(R Nb)}
  int32_t *ui0 = nullptr, *uj0 = nullptr;                               // [Nb]
  double *uwx = nullptr, *uwy = nullptr;                                // [Nb][MP]
  int64_t n_far = 0, n_mid = 0, n_close = 0;
  int n_sm = 0;                 // SMs of the plan's device
  int s_far = 1, s_mid = 1;     // node splits of the far and mid point sums (dlp_splits)
  double* part = nullptr;       // [S][n] partial sums of a split launch
  int32_t *far_lin = nullptr, *mid_lin = nullptr, *close_lin = nullptr;
  double* close_geo = nullptr;  // [n_close][5]: foot x, y, normal x, y, theta
  double* close_w = nullptr;    // [n_close][MP]
  std::vector<double> close_nodes;  // [MP] distances along the normal
  double* dnodes = nullptr;         // device copy
  // per-solve workspace
  double *V = nullptr, *w = nullptr, *h = nullptr, *g = nullptr, *phi = nullptr;
  struct GmresDev* gm = nullptr;  // GMRES's Hessenberg part and state (device)
  double *ghat = nullptr, *phiR = nullptr, *c00 = nullptr;
  float4 *ab = nullptr, *abR = nullptr;        // double-float node coefficients [Nb], [R Nb]
  float4 *posB = nullptr, *posR = nullptr;     // nodes in grid units [Nb][2], [R Nb][2]
  std::vector<double> xy_host;  // node coordinates [Nb][2]
  int last_iters = 0;
  double last_resid = 0;
  std::vector<void*> allocs;
};

static void poisson_free(PoissonState* P) {
  if (!P) return;
  for (void* q : P->allocs) cudaFree(q);
  delete P;
}

void poisson_destroy(fc2d_plan_s* p) {
  poisson_free(static_cast<PoissonState*>(p->poisson));
  p->poisson = nullptr;
}

// ------------------------------------------------------------------------- //
// Kernels
// ------------------------------------------------------------------------- //
// Forward column DFT, hat f = scale * DFT, record hat f_00, multiply by the inverse
// Laplacian symbol, inverse (unnormalised) column DFT by conj(DFT(conj)), in place.
__global__ void __launch_bounds__(256) k_poisson_cols(FftArgs fa, int cb, double2* inter,
                                                      double* c00, double Lx, double Ly) {
  using C = double2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ny = fa.ny, ncol = fa.nx / 2 + 1;
  const int c0 = blockIdx.x * cb, f = blockIdx.y;
  const int nc = min(cb, ncol - c0);
  C* A = reinterpret_cast<C*>(smem_raw);
  C* Bf = A + (size_t)cb * ny;
  C* col = inter + (size_t)f * ny * fa.pitch + c0;
  for (int idx = threadIdx.x; idx < ny * cb; idx += blockDim.x) {
    int y = idx / cb, c = idx - y * cb;
    A[(size_t)c * ny + y] = c < nc ? col[(size_t)y * fa.pitch + c] : C{0, 0};
  }
  __syncthreads();
  const C* tw = reinterpret_cast<const C*>(fa.twy);
  C* Y = stockham<double>(A, Bf, ny, cb, fa.ry, fa.nry, tw, 1);
  C* other = (Y == A) ? Bf : A;
  const double two_pi = 6.283185307179586476925286766559;
  for (int idx = threadIdx.x; idx < ny * cb; idx += blockDim.x) {
    int c = idx / ny, ky = idx - c * ny;
    int kx = c0 + c;
    C v = Y[idx];
    v.x *= fa.scale;
    v.y *= fa.scale;
    int m = ky <= ny / 2 ? ky : ky - ny;
    double kxx = two_pi * kx / Lx, kyy = two_pi * m / Ly;
    double k2 = kxx * kxx + kyy * kyy;
    C b;
    if (kx == 0 && ky == 0) {
      c00[f] = v.x;
      b = C{0, 0};
    } else {
      b = C{-v.x / k2, -v.y / k2};
    }
    Y[idx] = C{b.x, -b.y};  // conj for the inverse
  }
  __syncthreads();
  C* Z = stockham<double>(Y, other, ny, cb, fa.ry, fa.nry, tw, 1);
  for (int idx = threadIdx.x; idx < ny * cb; idx += blockDim.x) {
    int y = idx / cb, c = idx - y * cb;
    if (c < nc) {
      C v = Z[(size_t)c * ny + y];
      col[(size_t)y * fa.pitch + c] = C{v.x, -v.y};
    }
  }
}

// Inverse real row DFT: from B_k (k = 0..nx/2) the real row x_n = sum B_k e^{2 pi i k n/nx}
// (full Hermitian sum), via z = length-nx/2 inverse DFT of
// Z'_k = (B_k + conj B_{nx/2-k}) + i (B_k - conj B_{nx/2-k}) conj(w^k), w = e^{-2 pi i/nx},
// x_{2m} = Re z_m, x_{2m+1} = Im z_m; plus c00 (x^2 + y^2)/4.
__global__ void __launch_bounds__(256) k_poisson_rows(FftArgs fa, const double2* inter,
                                                      const double* c00, double a0, double b0,
                                                      double h, double* up) {
  using C = double2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nx = fa.nx, Nh = nx / 2, j = blockIdx.x, f = blockIdx.y;
  C* A = reinterpret_cast<C*>(smem_raw);
  C* Bf = A + Nh;
  const C* row = inter + ((size_t)f * fa.ny + j) * fa.pitch;
  const C* rtw = reinterpret_cast<const C*>(fa.rtw);
  for (int k = threadIdx.x; k < Nh; k += blockDim.x) {
    C bk = row[k];
    C bc = row[Nh - k];
    bc.y = -bc.y;  // conj B_{Nh-k}
    C s = C{bk.x + bc.x, bk.y + bc.y};
    C d = C{bk.x - bc.x, bk.y - bc.y};
    C w = rtw[k];
    w.y = -w.y;  // conj(w^k)
    C dw = C{d.x * w.x - d.y * w.y, d.x * w.y + d.y * w.x};
    C z = C{s.x - dw.y, s.y + dw.x};  // s + i dw
    A[k] = C{z.x, -z.y};              // conj for the inverse
  }
  __syncthreads();
  const C* tw = reinterpret_cast<const C*>(fa.twx);
  C* Z = stockham<double>(A, Bf, Nh, 1, fa.rx, fa.nrx, tw, 1);
  const double q = c00 ? c00[f] * 0.25 : 0.0;
  const double y = b0 + h * double(j);
  double* out = up + ((size_t)f * fa.ny + j) * nx;
  for (int m = threadIdx.x; m < Nh; m += blockDim.x) {
    C z = Z[m];
    double x0 = a0 + h * double(2 * m), x1 = a0 + h * double(2 * m + 1);
    out[2 * m] = z.x + q * (x0 * x0 + y * y);
    out[2 * m + 1] = -z.y + q * (x1 * x1 + y * y);
  }
}

// u_p at the BIE nodes: iterated 1D interpolation (x on MP rows, then y).
__global__ void k_up_nodes(int Nb, int MP, int nx, const int32_t* i0, const int32_t* j0,
                           const double* wx, const double* wy, const double* up,
                           const double* g, double* ghom) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Nb) return;
  double acc = 0.0;
  for (int a = 0; a < MP; ++a) {
    const double* r = up + (size_t)(j0[k] + a) * nx + i0[k];
    double v = 0.0;
    for (int b = 0; b < MP; ++b) v = fma(wx[k * MP + b], r[b], v);
    acc = fma(wy[k * MP + a], v, acc);
  }
  ghom[k] = g[k] - acc;
}

__global__ void k_bie_matrix(int Nb, const double* x, const double* y, const double* x1,
                             const double* y1, const double* diag, double* A) {
  int i = blockIdx.y, k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Nb) return;
  const double w = 1.0 / Nb;  // (2 pi/Nb) * 1/(2 pi)
  double v;
  if (i == k) {
    v = -0.5 + diag[i];
  } else {
    double dx = x[i] - x[k], dy = y[i] - y[k];
    v = w * (y1[k] * dx - x1[k] * dy) / (dx * dx + dy * dy);
  }
  A[(size_t)i * Nb + k] = v;
}

// y = A x, one warp per row
// The GMRES vector kernels return at once when *stop is set (a batch of iterations
// launched ahead of the host's convergence check ran past the converged one).
__global__ void k_gemv(int n, const double* A, const double* x, double* y, const int* stop) {
  if (*stop) return;
  int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (row >= n) return;
  const double* a = A + (size_t)row * n;
  double s = 0.0;
  for (int k = lane; k < n; k += 32) s = fma(a[k], x[k], s);
  for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = s;
}

// h[i] = <V_i, w>, i < m (one block per i)
__global__ void k_dots(int n, int m, const double* V, const double* w, double* h, const int* stop) {
  __shared__ double red[256];
  int i = blockIdx.x;
  if (i >= m || *stop) return;
  double s = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) s = fma(V[(size_t)i * n + k], w[k], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) h[i] = red[0];
}

// w -= sum_{i<m} h[i] V_i
__global__ void k_sub_proj(int n, int m, const double* V, const double* h, double* w,
                           const int* stop) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n || *stop) return;
  double s = w[k];
  for (int i = 0; i < m; ++i) s = fma(-h[i], V[(size_t)i * n + k], s);
  w[k] = s;
}

__global__ void k_scale_to(int n, const double* w, const double* nrm, double* v, const int* stop) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n && !*stop) v[k] = w[k] / *nrm;
}

// x = sum_{i<m} y[i] V_i
__global__ void k_combine(int n, int m, const double* V, const double* y, double* x) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double s = 0.0;
  for (int i = 0; i < m; ++i) s = fma(y[i], V[(size_t)i * n + k], s);
  x[k] = s;
}

// GMRES's small dense part on the device (one thread): the Hessenberg matrix H, the
// Givens rotations (cs, sn), the rotated right-hand side e and the state, so that the
// host reads the state once per batch of iterations instead of after every dot product.
struct GmresDev {
  double H[(kGmresMax + 1) * kGmresMax];  // H[i][j] at i kGmresMax + j
  double cs[kGmresMax], sn[kGmresMax], e[kGmresMax + 1], y[kGmresMax];
  double h1[kGmresMax + 1], h2[kGmresMax + 1];  // the two Gram-Schmidt passes' projections
  double nn, hn, beta, resid;                   // ||w||^2, ||w||, ||g||, |e_m| / beta
  int stop, done, m, pad;                       // stop: no further vector work
};

// beta = ||g|| (nn holds <g, g>); V_0 = g / beta follows with hn = beta
__global__ void k_gmres_init(GmresDev* G) {
  const double beta = sqrt(G->nn);
  G->beta = beta;
  G->hn = beta;
  G->e[0] = beta;
  G->m = 0;
  G->resid = 0.0;
  G->done = beta == 0.0 ? 1 : 0;
  G->stop = G->done;
}

// Iteration j after the two projections (h1, h2) and <w, w> (nn): column j of H, the
// earlier rotations applied to it, its own rotation, the residual estimate |e_{j+1}|.
__global__ void k_gmres_step(GmresDev* G, int j, double tol) {
  if (G->done) return;
  double* H = G->H;
  for (int i = 0; i <= j; ++i) H[i * kGmresMax + j] = G->h1[i] + G->h2[i];
  const double hn = sqrt(G->nn);
  G->hn = hn;
  H[(j + 1) * kGmresMax + j] = hn;
  for (int i = 0; i < j; ++i) {
    const double a = H[i * kGmresMax + j], b = H[(i + 1) * kGmresMax + j];
    H[i * kGmresMax + j] = G->cs[i] * a + G->sn[i] * b;
    H[(i + 1) * kGmresMax + j] = -G->sn[i] * a + G->cs[i] * b;
  }
  const double a = H[j * kGmresMax + j], b = H[(j + 1) * kGmresMax + j];
  const double r = hypot(a, b);
  G->cs[j] = r == 0 ? 1.0 : a / r;
  G->sn[j] = r == 0 ? 0.0 : b / r;
  H[j * kGmresMax + j] = r;
  H[(j + 1) * kGmresMax + j] = 0.0;
  G->e[j + 1] = -G->sn[j] * G->e[j];
  G->e[j] = G->cs[j] * G->e[j];
  G->m = j + 1;
  G->resid = fabs(G->e[j + 1]) / G->beta;
  if (fabs(G->e[j + 1]) <= tol * G->beta || hn == 0.0 || j + 1 == kGmresMax) {
    G->done = 1;
    G->stop = 1;
  }
}

// y from the triangular system R y = e over the first m columns
__global__ void k_gmres_solve(GmresDev* G) {
  const int m = G->m;
  for (int i = m - 1; i >= 0; --i) {
    double sacc = G->e[i];
    for (int k = i + 1; k < m; ++k) sacc -= G->H[i * kGmresMax + k] * G->y[k];
    G->y[i] = sacc / G->H[i * kGmresMax + i];
  }
}

// hat phi_k = (1/Nb) sum_j phi_j e^{-2 pi i jk/Nb}, k = 0..Nb/2
__global__ void k_density_dft(int Nb, const double* phi, const double2* twb, double2* ghat) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > Nb / 2) return;
  double re = 0.0, im = 0.0;
  for (int j = 0; j < Nb; ++j) {
    double2 w = twb[(int)(((int64_t)j * k) % Nb)];
    re = fma(phi[j], w.x, re);
    im = fma(phi[j], w.y, im);
  }
  ghat[k] = double2{re / Nb, im / Nb};
}

// trigonometric interpolant of the density at the R Nb refined parameters
__global__ void k_density_refine(int Nb, int NR, const double2* ghat, const double2* twr,
                                 double* out) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= NR) return;
  const int half = Nb / 2;
  double s = ghat[0].x;
  for (int k = 1; k <= half; ++k) {
    double2 e = twr[(int)(((int64_t)k * m) % NR)];  // e^{+2 pi i k m/NR}
    double re = ghat[k].x * e.x - ghat[k].y * e.y;
    double fac = (2 * k == Nb) ? 1.0 : 2.0;
    s = fma(fac, re, s);
  }
  out[m] = s;
}

// node coefficients of the trapezoidal sum: a_k = y'_k phi_k / N, b_k = x'_k phi_k / N
// ------------------------------------------------------------------------- //
// Double-layer sums in double-float arithmetic on the FP32 units.  A value is the
// unevaluated sum hi + lo of two floats (about 48 significant bits), built from Knuth's
// TwoSum, the FMA form of Dekker's TwoProduct and the sums and products of Dekker
// (1971).  The narrow FP64 pipe would need ~12 operations per (point, node) term.
// Coordinates are in grid units: a grid point is an exact integer pair, a node or an
// off-grid point an integer cell index plus a double-float fraction, so every
// coordinate difference is an integer minus a fraction, accurate to ~2^-48 of a cell.
// With d' = d/h, r2' = r2/h^2 the term (a dx - b dy)/r2 = (a dx' - b dy')/(h r2').
// ------------------------------------------------------------------------- //
struct dfl {
  float hi, lo;
};
__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
  dfl s = two_sum(x.hi, y.hi);
  const dfl t = two_sum(x.lo, y.lo);
  s = fast_two_sum(s.hi, s.lo + t.hi);
  return fast_two_sum(s.hi, s.lo + t.lo);
}
__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
  const float p = __fmul_rn(x.hi, y.hi);  // never fused into the sum below
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}
// integer n minus the fraction (fh, fl)
__device__ __forceinline__ dfl int_minus(float n, float fh, float fl) {
  const dfl s = two_sum(n, -fh);
  return fast_two_sum(s.hi, s.lo - fl);
}
// (a dx - b dy) / (dx^2 + dy^2) with a = (ah, al), b = (bh, bl)
__device__ __forceinline__ dfl dl_term(dfl dx, dfl dy, float ah, float al, float bh, float bl) {
  const dfl xx = df_mul(dx, dx), yy = df_mul(dy, dy);
  const dfl r2 = df_add(xx, yy);
  const dfl num = df_add(df_mul({ah, al}, dx), df_mul({-bh, -bl}, dy));
  // 1/r2: the correctly rounded float reciprocal and one Newton step (relative error
  // about the square of the seed's, 2^-46)
  const float y0 = __frcp_rn(r2.hi);
  float t = fmaf(-r2.hi, y0, 1.0f);
  t = fmaf(-r2.lo, y0, t);
  return df_mul(num, fast_two_sum(y0, y0 * t));
}
__device__ __forceinline__ void split_df(double v, float& hi, float& lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

// per-solve node coefficients (y' phi/N, x' phi/N) as double-float pairs (ah, al, bh, bl)
__global__ void k_node_coef(int N, const double* x1, const double* y1, const double* phi,
                            float4* ab) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  float4 c;
  split_df(y1[k] * phi[k] / N, c.x, c.y);
  split_df(x1[k] * phi[k] / N, c.z, c.w);
  ab[k] = c;
}

// v at listed grid points by the trapezoidal sum over N nodes; u = u_p + v there.
// Blocks of 256 points, tiles of 256 nodes.  SPLIT: blockIdx.y picks one of gridDim.y
// node ranges and the partial sums go to part[blockIdx.y][n] (k_dlp_combine adds them).
// pos: per node (ix, iy, fx_hi, fx_lo), (fy_hi, fy_lo, -, -) in grid units.
template <bool SPLIT>
__global__ void __launch_bounds__(256) k_dlp(int n_pts, const int32_t* lin, int nx, double inv_h,
                                             int N, const float4* pos, const float4* ab,
                                             double* u, double* part) {
  __shared__ float4 s0[256], s1[256], sc[256];
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  bool act = n < n_pts;
  int l = act ? lin[n] : 0;
  const float pi = (float)(l % nx), pj = (float)(l / nx);
  // node range of this block row (the whole set when the launch is not split)
  const int k0 = SPLIT ? (int)((int64_t)N * blockIdx.y / gridDim.y) : 0;
  const int k1 = SPLIT ? (int)((int64_t)N * (blockIdx.y + 1) / gridDim.y) : N;
  dfl acc = {0.f, 0.f};
  for (int t0 = k0; t0 < k1; t0 += 256) {
    __syncthreads();
    for (int q = threadIdx.x; q < 256 && t0 + q < k1; q += blockDim.x) {
      s0[q] = pos[2 * (t0 + q)];
      s1[q] = pos[2 * (t0 + q) + 1];
      sc[q] = ab[t0 + q];
    }
    __syncthreads();
    const int cnt = min(256, k1 - t0);
    for (int k = 0; k < cnt; ++k) {
      const float4 a = s0[k], b = s1[k], c = sc[k];
      const dfl dx = int_minus(pi - a.x, a.z, a.w), dy = int_minus(pj - a.y, b.x, b.y);
      const dfl term = dl_term(dx, dy, c.x, c.y, c.z, c.w);
      const dfl s = two_sum(acc.hi, term.hi);
      acc = fast_two_sum(s.hi, s.lo + (acc.lo + term.lo));
    }
  }
  if (!act) return;
  const double v = (double)acc.hi + (double)acc.lo;
  if (SPLIT) part[(size_t)blockIdx.y * n_pts + n] = v;
  else u[l] += v * inv_h;
}

// A split k_dlp launch's S partial sums per point, added in node-range order: u += sum / h.
__global__ void __launch_bounds__(256) k_dlp_combine(int n_pts, const int32_t* lin, int S,
                                                     const double* part, double inv_h, double* u) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_pts) return;
  double v = 0.0;
  for (int y = 0; y < S; ++y) v += part[(size_t)y * n_pts + n];
  u[lin[n]] += v * inv_h;
}

// close points: one block per point; the MP - 1 refined sums along the normal (each
// thread takes a node once for all of them), the boundary value by trigonometric
// interpolation of g - u_p, and the Lagrange combination.
template <int KMP>  // compile-time M_P (0: any M_P <= kMaxM)
__global__ void __launch_bounds__(256) k_dlp_close(int n_close, const int32_t* lin,
                                                   const double* cgeo, const double* cw,
                                                   const double* nodes, int MP, int NR,
                                                   double a0, double b0, double h,
                                                   const float4* posR, const float4* abR,
                                                   int Nb, const double2* ghat_g, double* u) {
  constexpr int NP = KMP > 0 ? KMP : kMaxM;
  if (KMP > 0) MP = KMP;
  __shared__ double red[256];
  __shared__ float pt[NP][6];  // per point: ix, iy, fx_hi, fx_lo, fy_hi, fy_lo
  const int n = blockIdx.x;
  if (n >= n_close) return;
  const double fx = cgeo[5 * n], fy = cgeo[5 * n + 1], nxv = cgeo[5 * n + 2],
               nyv = cgeo[5 * n + 3], th = cgeo[5 * n + 4];
  const double inv_h = 1.0 / h;
  if (threadIdx.x < MP - 1) {
    const int j = threadIdx.x + 1;
    const double ux = (fx - nodes[j] * nxv - a0) * inv_h, uy = (fy - nodes[j] * nyv - b0) * inv_h;
    const double ix = floor(ux), iy = floor(uy);
    pt[j][0] = (float)ix;
    pt[j][1] = (float)iy;
    split_df(ux - ix, pt[j][2], pt[j][3]);
    split_df(uy - iy, pt[j][4], pt[j][5]);
  }
  __syncthreads();
  dfl acc[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) acc[j] = {0.f, 0.f};
  for (int k = threadIdx.x; k < NR; k += blockDim.x) {
    const float4 a = posR[2 * k], b = posR[2 * k + 1], c = abR[k];
#pragma unroll
    for (int j = 1; j < NP; ++j) {
      if (KMP == 0 && j >= MP) break;
      // (point - node) = (i_p - i_n) + (f_p - f_n)
      const dfl dx = df_add(int_minus(pt[j][0] - a.x, a.z, a.w), {pt[j][2], pt[j][3]});
      const dfl dy = df_add(int_minus(pt[j][1] - a.y, b.x, b.y), {pt[j][4], pt[j][5]});
      const dfl term = dl_term(dx, dy, c.x, c.y, c.z, c.w);
      const dfl s = two_sum(acc[j].hi, term.hi);
      acc[j] = fast_two_sum(s.hi, s.lo + (acc[j].lo + term.lo));
    }
  }
  double vals[NP];
#pragma unroll
  for (int j = 1; j < NP; ++j) {
    if (KMP == 0 && j >= MP) break;
    red[threadIdx.x] = (double)acc[j].hi + (double)acc[j].lo;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    vals[j] = red[0] * inv_h;
    __syncthreads();
  }
  // boundary value: sum_k c_k e^{i k theta} over the Hermitian half (Nyquist halved)
  {
    double acc0 = 0.0;
    const int half = Nb / 2;
    // e^{i k theta} for k = tid, tid + blockDim, ...: one sincos each for the first k and
    // the stride, then complex products (at most a few steps: Nb/2 <= a few blockDim)
    double s, c, ss, cs;
    sincos(double(threadIdx.x) * th, &s, &c);
    sincos(double(blockDim.x) * th, &ss, &cs);
    for (int k = threadIdx.x; k <= half; k += blockDim.x) {
      double re = ghat_g[k].x * c - ghat_g[k].y * s;
      double fac = (k == 0 || 2 * k == Nb) ? 1.0 : 2.0;
      acc0 = fma(fac, re, acc0);
      const double c2 = c * cs - s * ss, s2 = s * cs + c * ss;
      c = c2;
      s = s2;
    }
    red[threadIdx.x] = acc0;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    vals[0] = red[0];
  }
  if (threadIdx.x == 0) {
    double v = 0.0;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      if (KMP == 0 && j >= MP) break;
      v = fma(cw[(size_t)n * MP + j], vals[j], v);
    }
    u[lin[n]] += v;
  }
}

__global__ void k_zero_outside(int nx, const int32_t* row_iv_off, const int32_t* row_iv,
                               double* u) {
  const int j = blockIdx.x;
  double* r = u + (size_t)j * nx;
  const int iv0 = row_iv_off[j], iv1 = row_iv_off[j + 1];
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    bool in = false;
    for (int k = iv0; k < iv1; ++k) in |= (i >= row_iv[2 * k] && i <= row_iv[2 * k + 1]);
    if (!in) r[i] = 0.0;
  }
}

// ------------------------------------------------------------------------- //
// Setup
// ------------------------------------------------------------------------- //
template <typename T>
static fc2d_status up(PoissonState* P, T** dst, const std::vector<T>& src) {
  size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
  if (cudaMalloc((void**)dst, bytes) != cudaSuccess)
    return set_error(FC2D_ERR_NOMEM, "Poisson setup: cudaMalloc failed");
  P->allocs.push_back(*dst);
  if (!src.empty() &&
      cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return set_error(FC2D_ERR_CUDA, "Poisson setup: cudaMemcpy failed");
  return FC2D_OK;
}

template <typename T>
static fc2d_status alloc(PoissonState* P, T** dst, size_t n) {
  if (cudaMalloc((void**)dst, std::max<size_t>(1, n) * sizeof(T)) != cudaSuccess)
    return set_error(FC2D_ERR_NOMEM, "Poisson setup: cudaMalloc failed");
  P->allocs.push_back(*dst);
  return FC2D_OK;
}

// Node positions in grid units for the double-float sums: per node (ix, iy, fx_hi,
// fx_lo), (fy_hi, fy_lo, 0, 0), with (x - a0)/h = ix + fx, 0 <= fx < 1 (the same in y).
static std::vector<float4> grid_units(const std::vector<double>& x, const std::vector<double>& y,
                                      double a0, double b0, double h) {
  std::vector<float4> out(2 * x.size());
  for (size_t k = 0; k < x.size(); ++k) {
    const double ux = (x[k] - a0) / h, uy = (y[k] - b0) / h;
    const double ix = std::floor(ux), iy = std::floor(uy), fx = ux - ix, fy = uy - iy;
    const float fxh = (float)fx, fyh = (float)fy;
    out[2 * k] = make_float4((float)ix, (float)iy, fxh, (float)(fx - (double)fxh));
    out[2 * k + 1] = make_float4(fyh, (float)(fy - (double)fyh), 0.f, 0.f);
  }
  return out;
}

static void lagr(const double* nodes, int n, double t, double* w) {
  for (int k = 0; k < n; ++k) {
    double v = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != k) v *= (t - nodes[m]) / (nodes[k] - nodes[m]);
    w[k] = v;
  }
}

// Node splits of a k_dlp launch over n points and N nodes: each point's sum over the
// nodes is cut into S consecutive node ranges, one row of blocks each (partial sums
// combined by k_dlp_combine in range order), so that a launch over few points still
// has about 48 warps per SM; below that the sums are bound by each warp's dependent
// double-float chain rather than by issue.  At most 8 ranges of at least 1024 nodes.
static int dlp_splits(int64_t n, int N, int n_sm) {
  if (n_sm <= 0 || n <= 0) return 1;
  const int64_t warps = (n + 255) / 256 * 8;
  int64_t S = (48LL * n_sm + warps - 1) / warps;
  S = std::min<int64_t>(S, 8);
  S = std::min<int64_t>(S, std::max(1, N / 1024));
  return (int)std::max<int64_t>(S, 1);
}

fc2d_status poisson_setup(fc2d_plan_s* p, int Nb) {
  if (p->prm.precision != FC2D_FP64)
    return set_error(FC2D_ERR_UNSUPPORTED, "fc2d_poisson_plan: the Poisson solver needs an FP64 plan");
  const int nx = p->grid.nx, ny = p->grid.ny, MP = p->prm.M;
  if (Nb <= 0) Nb = nx;
  if (Nb < 16 || Nb > 65536) return set_error(FC2D_ERR_ARG, "fc2d_poisson_plan: bad n_b");
  poisson_destroy(p);
  auto* P = new PoissonState();
  P->Nb = Nb;
  P->MP = MP;
  if (cudaDeviceGetAttribute(&P->n_sm, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess)
    P->n_sm = 0;
  const Curve& cv = p->curve;
  const double a0 = p->grid.a0, b0 = p->grid.b0, h = p->grid.h;
  const double two_pi = 2.0 * M_PI;
  auto fail = [&](fc2d_status s) {
    poisson_free(P);
    return s;
  };
  // nodes
  std::vector<double> x(Nb), y(Nb), x1(Nb), y1(Nb), diag(Nb);
  P->xy_host.assign(2 * (size_t)Nb, 0.0);
  for (int k = 0; k < Nb; ++k) {
    double t = two_pi * k / Nb, xx, yy, xd, yd, x2, y2;
    cv.eval(t, xx, yy);
    cv.eval_d(t, 1, xd, yd);
    cv.eval_d(t, 2, x2, y2);
    x[k] = xx;
    y[k] = yy;
    x1[k] = xd;
    y1[k] = yd;
    diag[k] = (x2 * yd - xd * y2) / (4.0 * M_PI * (xd * xd + yd * yd)) * (two_pi / Nb);
    P->xy_host[2 * k] = xx;
    P->xy_host[2 * k + 1] = yy;
  }
  // largest node spacing and the near bands
  double smax = 0.0;
  for (int k = 0; k < 4096; ++k) {
    double xd, yd;
    cv.eval_d(two_pi * k / 4096, 1, xd, yd);
    smax = std::max(smax, std::hypot(xd, yd));
  }
  P->s = two_pi / Nb * smax;
  P->delta = 5.0 * P->s;
  const int R = P->R, NR = R * Nb;
  std::vector<double> rx(NR), ry(NR), rx1(NR), ry1(NR);
  for (int m = 0; m < NR; ++m) {
    double t = two_pi * m / NR;
    cv.eval(t, rx[m], ry[m]);
    cv.eval_d(t, 1, rx1[m], ry1[m]);
  }
  std::vector<double> twb(2 * (size_t)Nb), twr(2 * (size_t)NR);
  for (int t = 0; t < Nb; ++t) {
    double ang = two_pi * t / Nb;
    twb[2 * t] = std::cos(ang);
    twb[2 * t + 1] = -std::sin(ang);
  }
  for (int t = 0; t < NR; ++t) {
    double ang = two_pi * t / NR;
    twr[2 * t] = std::cos(ang);
    twr[2 * t + 1] = std::sin(ang);
  }
  // u_p interpolation stencils at the nodes
  std::vector<int32_t> ui0(Nb), uj0(Nb);
  std::vector<double> uwx((size_t)Nb * MP), uwy((size_t)Nb * MP);
  const int off = (MP + 1) / 2 - 1;
  for (int k = 0; k < Nb; ++k) {
    int i0 = (int)std::floor((x[k] - a0) / h) - off;
    int j0 = (int)std::floor((y[k] - b0) / h) - off;
    i0 = std::min(std::max(i0, 0), nx - MP);
    j0 = std::min(std::max(j0, 0), ny - MP);
    ui0[k] = i0;
    uj0[k] = j0;
    double nxs[kMaxM], nys[kMaxM];
    for (int e = 0; e < MP; ++e) {
      nxs[e] = a0 + h * double(i0 + e);
      nys[e] = b0 + h * double(j0 + e);
    }
    lagr(nxs, MP, x[k], &uwx[(size_t)k * MP]);
    lagr(nys, MP, y[k], &uwy[(size_t)k * MP]);
  }
  // near points: inside points closer than delta; seeds from the nearest node of a
  // fine sampling of the curve (boxes around each sample)
  std::vector<uint8_t> inside((size_t)nx * ny, 0);
  for (int j = 0; j < ny; ++j)
    for (int k = p->row_iv_off[j]; k < p->row_iv_off[j + 1]; ++k)
      for (int i = p->row_iv[2 * k]; i <= p->row_iv[2 * k + 1]; ++i) inside[(size_t)j * nx + i] = 1;
  const int ns = std::max(p->prm.B, 4 * Nb);
  std::vector<double> seed((size_t)nx * ny, -1.0), best((size_t)nx * ny, 1e300);
  const double reach = P->delta + 2.0 * h;
  for (int q = 0; q < ns; ++q) {
    double t = two_pi * q / ns, cx, cy;
    cv.eval(t, cx, cy);
    int i0 = std::max(0, (int)std::floor((cx - reach - a0) / h));
    int i1 = std::min(nx - 1, (int)std::ceil((cx + reach - a0) / h));
    int j0 = std::max(0, (int)std::floor((cy - reach - b0) / h));
    int j1 = std::min(ny - 1, (int)std::ceil((cy + reach - b0) / h));
    for (int j = j0; j <= j1; ++j)
      for (int i = i0; i <= i1; ++i) {
        size_t l = (size_t)j * nx + i;
        if (!inside[l]) continue;
        double dx = a0 + h * double(i) - cx, dy = b0 + h * double(j) - cy;
        double d2 = dx * dx + dy * dy;
        if (d2 < best[l] && d2 <= reach * reach) {
          best[l] = d2;
          seed[l] = t;
        }
      }
  }
  std::vector<int32_t> cl;
  std::vector<double> qx, qy, tq;
  for (size_t l = 0; l < seed.size(); ++l)
    if (seed[l] >= 0) {
      cl.push_back((int32_t)l);
      qx.push_back(a0 + h * double(l % nx));
      qy.push_back(b0 + h * double(l / nx));
      tq.push_back(seed[l]);
    }
  std::vector<int> conv;
  fc2d_status st = foot_newton_gpu(cv, qx, qy, tq, conv, two_pi / ns);
  if (st) return fail(st);
  std::vector<uint8_t> near((size_t)nx * ny, 0);
  std::vector<int32_t> mid, close;
  std::vector<double> cgeo, cw;
  P->close_nodes.assign(MP, 0.0);
  for (int j = 1; j < MP; ++j) P->close_nodes[j] = (P->delta + P->s * (j - 1)) / R;
  for (size_t n = 0; n < cl.size(); ++n) {
    double fx, fy;
    cv.eval(tq[n], fx, fy);
    double eta = std::hypot(qx[n] - fx, qy[n] - fy);
    if (!(eta < P->delta)) continue;
    if (!conv[n]) return fail(set_error(FC2D_ERR_NOT_CONVERGED, "Poisson setup: foot search"));
    near[cl[n]] = 1;
    if (eta >= P->delta / R) {
      mid.push_back(cl[n]);
    } else {
      double t = std::fmod(tq[n], two_pi);
      if (t < 0) t += two_pi;
      double xd, yd;
      cv.eval_d(t, 1, xd, yd);
      double sp = std::hypot(xd, yd);
      close.push_back(cl[n]);
      cgeo.insert(cgeo.end(), {fx, fy, yd / sp, -xd / sp, t});
      double w[kMaxM];
      lagr(P->close_nodes.data(), MP, eta, w);
      cw.insert(cw.end(), w, w + MP);
    }
  }
  std::vector<int32_t> far;
  for (size_t l = 0; l < inside.size(); ++l)
    if (inside[l] && !near[l]) far.push_back((int32_t)l);
  P->n_far = (int64_t)far.size();
  P->n_mid = (int64_t)mid.size();
  P->n_close = (int64_t)close.size();
  if ((st = up(P, &P->bx, x)) || (st = up(P, &P->by, y)) || (st = up(P, &P->bx1, x1)) ||
      (st = up(P, &P->by1, y1)) || (st = up(P, &P->rx, rx)) || (st = up(P, &P->ry, ry)) ||
      (st = up(P, &P->rx1, rx1)) || (st = up(P, &P->ry1, ry1)) || (st = up(P, &P->twb, twb)) ||
      (st = up(P, &P->twr, twr)) || (st = up(P, &P->ui0, ui0)) || (st = up(P, &P->uj0, uj0)) ||
      (st = up(P, &P->uwx, uwx)) || (st = up(P, &P->uwy, uwy)) ||
      (st = up(P, &P->far_lin, far)) || (st = up(P, &P->mid_lin, mid)) ||
      (st = up(P, &P->close_lin, close)) || (st = up(P, &P->close_geo, cgeo)) ||
      (st = up(P, &P->close_w, cw)) || (st = up(P, &P->dnodes, P->close_nodes)) ||
      (st = up(P, &P->posB, grid_units(x, y, a0, b0, h))) ||
      (st = up(P, &P->posR, grid_units(rx, ry, a0, b0, h))))
    return fail(st);
  double* ddiag = nullptr;
  if ((st = up(P, &ddiag, diag)) || (st = alloc(P, &P->A, (size_t)Nb * Nb)) ||
      (st = alloc(P, &P->V, (size_t)(kGmresMax + 1) * Nb)) || (st = alloc(P, &P->w, Nb)) ||
      (st = alloc(P, &P->h, kGmresMax + 2)) || (st = alloc(P, &P->gm, 1)) ||
      (st = alloc(P, &P->g, Nb)) ||
      (st = alloc(P, &P->phi, Nb)) || (st = alloc(P, &P->ghat, 2 * (Nb / 2 + 1))) ||
      (st = alloc(P, &P->phiR, NR)) || (st = alloc(P, &P->ab, (size_t)Nb)) ||
      (st = alloc(P, &P->abR, (size_t)NR)) || (st = alloc(P, &P->c00, 1024)))
    return fail(st);
  P->s_far = dlp_splits(P->n_far, Nb, P->n_sm);
  P->s_mid = dlp_splits(P->n_mid, NR, P->n_sm);
  const size_t n_part = std::max(P->s_far > 1 ? (size_t)P->s_far * P->n_far : 0,
                                 P->s_mid > 1 ? (size_t)P->s_mid * P->n_mid : 0);
  if (n_part && (st = alloc(P, &P->part, n_part))) return fail(st);
  k_bie_matrix<<<dim3((Nb + 255) / 256, Nb), 256>>>(Nb, P->bx, P->by, P->bx1, P->by1, ddiag,
                                                    P->A);
  if ((st = cuda_check(cudaDeviceSynchronize(), "BIE matrix"))) return fail(st);
  p->poisson = P;
  return FC2D_OK;
}

// GMRES (no restart) for A phi = g: Arnoldi with classical Gram-Schmidt twice on device
// vectors, the Hessenberg least squares by Givens rotations on the device
// (k_gmres_step); iterations are launched in batches of kGmresBatch and the host reads
// the state once per batch (the vector kernels of iterations past convergence return
// at once).
constexpr int kGmresBatch = 8;
static fc2d_status gmres(PoissonState* P, cudaStream_t s, double tol) {
  const int n = P->Nb;
  const unsigned gb = (unsigned)((n + 255) / 256);
  GmresDev* G = P->gm;
  int* stop = &G->stop;
  cudaMemsetAsync(stop, 0, sizeof(int), s);
  // beta = ||g||, V_0 = g / beta
  k_dots<<<1, 256, 0, s>>>(n, 1, P->g, P->g, &G->nn, stop);
  k_gmres_init<<<1, 1, 0, s>>>(G);
  k_scale_to<<<gb, 256, 0, s>>>(n, P->g, &G->hn, P->V, stop);
  int state[4] = {0, 0, 0, 0};  // stop, done, m, pad
  for (int j0 = 0; j0 < kGmresMax && !state[1]; j0 += kGmresBatch) {
    for (int j = j0; j < std::min(j0 + kGmresBatch, kGmresMax); ++j) {
      const double* vj = P->V + (size_t)j * n;
      k_gemv<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(n, P->A, vj, P->w, stop);
      k_dots<<<j + 1, 256, 0, s>>>(n, j + 1, P->V, P->w, G->h1, stop);
      k_sub_proj<<<gb, 256, 0, s>>>(n, j + 1, P->V, G->h1, P->w, stop);
      k_dots<<<j + 1, 256, 0, s>>>(n, j + 1, P->V, P->w, G->h2, stop);
      k_sub_proj<<<gb, 256, 0, s>>>(n, j + 1, P->V, G->h2, P->w, stop);
      k_dots<<<1, 256, 0, s>>>(n, 1, P->w, P->w, &G->nn, stop);
      k_gmres_step<<<1, 1, 0, s>>>(G, j, tol);
      k_scale_to<<<gb, 256, 0, s>>>(n, P->w, &G->hn, P->V + (size_t)(j + 1) * n, stop);
    }
    cudaMemcpyAsync(state, stop, sizeof(state), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(cudaGetLastError(), "GMRES");
  }
  const int m = state[2];
  double resid = 0.0;
  cudaMemcpyAsync(&resid, &G->resid, sizeof(double), cudaMemcpyDeviceToHost, s);
  k_gmres_solve<<<1, 1, 0, s>>>(G);
  k_combine<<<gb, 256, 0, s>>>(n, m, P->V, G->y, P->phi);
  if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(cudaGetLastError(), "GMRES");
  P->last_iters = m;
  P->last_resid = resid;
  if (resid > 1e3 * tol)
    return set_error(FC2D_ERR_NOT_CONVERGED, "GMRES did not reach its tolerance");
  return cuda_check(cudaGetLastError(), "GMRES");
}

fc2d_status poisson_solve(fc2d_plan_s* p, int n_f, const double* fg, const double* fb,
                          const double* gn, double* u, double* phi_out, void* inter,
                          cudaStream_t s) {
  auto* P = static_cast<PoissonState*>(p->poisson);
  const int nx = p->grid.nx, ny = p->grid.ny, Nb = P->Nb, MP = P->MP, NR = P->R * Nb;
  const double a0 = p->grid.a0, b0 = p->grid.b0, h = p->grid.h;
  if (n_f > 1024) return set_error(FC2D_ERR_ARG, "fc2d_poisson: n_f <= 1024");
  // u_p (forward rows already in `inter` from the caller): multiplier + inverse
  FftArgs fa{};
  fa.nx = nx;
  fa.ny = ny;
  fa.pitch = (int)row_pitch(p);
  fa.nrx = p->fx.n_radix;
  fa.nry = p->fy.n_radix;
  for (int i = 0; i < fa.nrx; ++i) fa.rx[i] = p->fx.radix[i];
  for (int i = 0; i < fa.nry; ++i) fa.ry[i] = p->fy.radix[i];
  fa.twx = p->fx.tw64;
  fa.twy = p->fy.tw64;
  fa.tsx = p->fx.tws64;  // per-stage tables of the power-of-two inverse rows
  fa.tsy = p->fy.tws64;
  fa.rtw = p->rtw64;
  fa.scale = 1.0 / ((double)nx * ny);
  {
    ProfScope ps(p, "poisson_cols", s);
    const int ncol = nx / 2 + 1;
    int cb = 1;
    while (cb < 8 && 2 * (size_t)(2 * cb) * ny * sizeof(double2) <= 200 * 1024) cb *= 2;
    size_t sm = 2 * (size_t)cb * ny * sizeof(double2);
    cudaFuncSetAttribute(k_poisson_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_poisson_cols<<<dim3((ncol + cb - 1) / cb, n_f), 256, sm, s>>>(
        fa, cb, (double2*)inter, P->c00, nx * h, ny * h);
  }
  {
    ProfScope ps(p, "poisson_rows", s);
    launch_inverse_rows(fa, n_f, inter, P->c00, a0, b0, h, u, s);
  }
  fc2d_status st = cuda_check(cudaGetLastError(), "Poisson particular solution");
  if (st) return st;
  const unsigned gb = (unsigned)((Nb + 255) / 256);
  for (int f = 0; f < n_f; ++f) {
    double* uf = u + (size_t)f * nx * ny;
    k_up_nodes<<<gb, 256, 0, s>>>(Nb, MP, nx, P->ui0, P->uj0, P->uwx, P->uwy, uf,
                                  gn + (size_t)f * Nb, P->g);
    {
      ProfScope ps(p, "bie_gmres", s);
      if ((st = gmres(P, s, 1e-14))) return st;
    }
    if (phi_out) cudaMemcpyAsync(phi_out + (size_t)f * Nb, P->phi, Nb * 8, cudaMemcpyDeviceToDevice, s);
    // density refinement and node coefficients
    k_density_dft<<<(unsigned)((Nb / 2 + 1 + 127) / 128), 128, 0, s>>>(Nb, P->phi,
                                                                     (const double2*)P->twb,
                                                                     (double2*)P->ghat);
    k_density_refine<<<(unsigned)((NR + 255) / 256), 256, 0, s>>>(Nb, NR, (const double2*)P->ghat,
                                                                 (const double2*)P->twr, P->phiR);
    k_node_coef<<<gb, 256, 0, s>>>(Nb, P->bx1, P->by1, P->phi, P->ab);
    k_node_coef<<<(unsigned)((NR + 255) / 256), 256, 0, s>>>(NR, P->rx1, P->ry1, P->phiR,
                                                            P->abR);
    // the trapezoidal sums at n listed points over N nodes, split into S node ranges
    auto dlp = [&](int64_t n, const int32_t* lin, int N, int S, const float4* pos,
                   const float4* ab) {
      const unsigned nb = (unsigned)((n + 255) / 256);
      if (S == 1) {
        k_dlp<false><<<nb, 256, 0, s>>>((int)n, lin, nx, 1.0 / h, N, pos, ab, uf, nullptr);
        return;
      }
      k_dlp<true><<<dim3(nb, (unsigned)S), 256, 0, s>>>((int)n, lin, nx, 1.0 / h, N, pos, ab, uf,
                                                       P->part);
      k_dlp_combine<<<nb, 256, 0, s>>>((int)n, lin, S, P->part, 1.0 / h, uf);
    };
    {
      ProfScope ps(p, "dlp_far", s);
      if (P->n_far) dlp(P->n_far, P->far_lin, Nb, P->s_far, P->posB, P->ab);
    }
    {
      ProfScope ps(p, "dlp_near", s);
      if (P->n_mid) dlp(P->n_mid, P->mid_lin, NR, P->s_mid, P->posR, P->abR);
      if (P->n_close) {
        // boundary values g - u_p: reuse ghat for their coefficients
        k_density_dft<<<(unsigned)((Nb / 2 + 1 + 127) / 128), 128, 0, s>>>(
            Nb, P->g, (const double2*)P->twb, (double2*)P->ghat);
        auto kc = MP == 8    ? k_dlp_close<8>
                  : MP == 13 ? k_dlp_close<13>
                  : MP == 15 ? k_dlp_close<15>
                             : k_dlp_close<0>;
        kc<<<(unsigned)P->n_close, 256, 0, s>>>(
            (int)P->n_close, P->close_lin, P->close_geo, P->close_w, P->dnodes, MP, NR, a0, b0,
            h, P->posR, P->abR, Nb, (const double2*)P->ghat, uf);
      }
    }
    k_zero_outside<<<ny, 256, 0, s>>>(nx, p->dev.row_iv_off, p->dev.row_iv, uf);
  }
  return cuda_check(cudaGetLastError(), "Poisson solve");
}

// inverse real 2D-DFT rows (after an inverse column pass) for callers outside this file
bool launch_inverse_rows_p2(const FftArgs& fa, int n_f, const void* inter, const double* c00,
                            double a0, double b0, double h, double* out, cudaStream_t s);

void launch_inverse_rows(const FftArgs& fa, int n_f, const void* inter, const double* c00,
                         double a0, double b0, double h, double* out, cudaStream_t s) {
  if (launch_inverse_rows_p2(fa, n_f, inter, c00, a0, b0, h, out, s)) return;
  size_t sm = (size_t)fa.nx * sizeof(double2);
  cudaFuncSetAttribute(k_poisson_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_poisson_rows<<<dim3(fa.ny, n_f), 256, sm, s>>>(fa, (const double2*)inter, c00, a0, b0, h, out);
}

int poisson_nb(const fc2d_plan_s* p) {
  return p->poisson ? static_cast<const PoissonState*>(p->poisson)->Nb : 0;
}

const double* poisson_nodes(const fc2d_plan_s* p) {
  return p->poisson ? static_cast<const PoissonState*>(p->poisson)->xy_host.data() : nullptr;
}

void poisson_stats(const fc2d_plan_s* p, int* iters, double* resid, int64_t* n_near) {
  auto* P = static_cast<const PoissonState*>(p->poisson);
  if (iters) *iters = P ? P->last_iters : 0;
  if (resid) *resid = P ? P->last_resid : 0.0;
  if (n_near) *n_near = P ? P->n_mid + P->n_close : 0;
}

}  // namespace fc2d
