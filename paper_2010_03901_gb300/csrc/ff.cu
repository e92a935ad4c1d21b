// Fourier Forwarding (Section 4.2): the interior propagator U_FC combined with the
// near-boundary solver U_B by eq. (4.9), large step after large step (FP64).
//
// Large step j (T_j = j Delta T, Delta T = n_c h / c, S = 8 n_c small steps of
// Delta t = Delta T / S, i.e. c Delta t = h/8, CFL 0.125 as in Section 4.2.1):
//   1. the 2D-FC spectra of u(T_j) and u_t(T_j) (eq. (4.10)) with the Dirichlet data
//      g(T_j) and its time derivative (capi.cu wave_spectra);
//   2. for each small step s: the modal solution a(s Delta t) (eq. (4.12), w the square
//      root of the paper's alpha) and its inverse DFT (k_ff_cols + inverse rows): U_FC on
//      the grid, whose values at U_B's interface points feed the step;
//   3. the U_B small step (k_ub_step): u^{n+1} = 2u^n - u^{n-1} + (h/8)^2 L(u^n)
//      - 0.3 D(u^n - u^{n-1}), the first step of the solve by the Taylor start
//      u^1 = u^0 + dt u_t^0 + (h/8)^2/2 L(u^0); L and D are the plan-time operators of
//      wave_band.cpp (rows per unknown, columns keyed unknown / interface grid point /
//      boundary point);
//   4. U_FC(T_{j+1}) and dU_FC/dt on the grid, one further U_B step for the time
//      derivative (u^{N+1} - u^{N-1})/(2 dt), and the merge: at the band points nearer
//      than delta = n_c h to the curve the grid takes U_B's values (slaved points by their
//      boundary polynomial).
// The U_B state is function-minor ([unknown][n_f]), so that a warp reads one operator
// row for 32 functions with coalesced loads.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <string>

#include "fc2d_kernels.cuh"
#include "fft_generic.cuh"
#include "plan_internal.h"
#include "wave_band.h"

namespace fc2d {

fc2d_status wave_spectra(fc2d_plan_s* p, int n_f, const double* u, const double* ub,
                         const double* ut, const double* utb, void* spec, cudaStream_t s);
bool launch_ff_cols_p2(const FftArgs& fa, int n_f, int n_out, const void* spec, void* out,
                       double c, double tau, double Lx, double Ly, cudaStream_t s);

namespace {

struct DevCsr {
  int32_t* off = nullptr;
  uint32_t* col = nullptr;
  double* w = nullptr;
  int64_t rows = 0, nnz = 0;
};

struct DevBand {
  WaveBand host;
  DevCsr L, D, S;
  int32_t* unknown_lin = nullptr;
  int32_t* near_lin = nullptr;
  int32_t* near_src = nullptr;
};

struct Scratch {
  int n_f = 0;
  size_t bytes = 0;
  void* base = nullptr;
};

struct WaveState {
  std::map<int, std::unique_ptr<DevBand>> bands;  // by n_c
  Scratch scr;
};

template <typename T>
fc2d_status upload(T** dst, const std::vector<T>& src) {
  *dst = nullptr;
  const size_t n = std::max<size_t>(1, src.size());
  if (cudaMalloc(dst, n * sizeof(T)) != cudaSuccess)
    return set_error(FC2D_ERR_NOMEM, "wave band: cudaMalloc failed");
  if (!src.empty() && cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return set_error(FC2D_ERR_CUDA, "wave band: upload failed");
  return FC2D_OK;
}

fc2d_status upload_csr(DevCsr& d, const Csr& h) {
  d.rows = (int64_t)h.off.size() - 1;
  d.nnz = (int64_t)h.w.size();
  fc2d_status st;
  if ((st = upload(&d.off, h.off)) || (st = upload(&d.col, h.col)) || (st = upload(&d.w, h.w)))
    return st;
  return FC2D_OK;
}

void free_csr(DevCsr& d) {
  cudaFree(d.off);
  cudaFree(d.col);
  cudaFree(d.w);
}

WaveState* state(fc2d_plan_s* p) {
  if (!p->wave) p->wave = new WaveState();
  return static_cast<WaveState*>(p->wave);
}

fc2d_status get_band(fc2d_plan_s* p, int n_c, DevBand** out) {
  WaveState* W = state(p);
  auto it = W->bands.find(n_c);
  if (it != W->bands.end()) {
    *out = it->second.get();
    return FC2D_OK;
  }
  auto b = std::make_unique<DevBand>();
  fc2d_status st = build_wave_band(p, n_c, b->host);
  if (st) return st;
  // operator entries of a grid kind must index the grid (30 bits), boundary data too
  if ((int64_t)p->grid.nx * p->grid.ny > (int64_t)kKeyIndex || p->n_bdry > (int64_t)kKeyIndex)
    return set_error(FC2D_ERR_UNSUPPORTED, "wave band: grid too large for the operator keys");
  if ((st = upload_csr(b->L, b->host.L)) || (st = upload_csr(b->D, b->host.D)) ||
      (st = upload_csr(b->S, b->host.S)) || (st = upload(&b->unknown_lin, b->host.unknown_lin)) ||
      (st = upload(&b->near_lin, b->host.near_lin)) || (st = upload(&b->near_src, b->host.near_src)))
    return st;
  *out = b.get();
  W->bands[n_c] = std::move(b);
  return FC2D_OK;
}

// ------------------------------------------------------------------------- //
// Kernels
// ------------------------------------------------------------------------- //

// U_B state from grids: out[r][f] = grid[f][lin[r]]
__global__ void k_ub_gather(int64_t n, int n_f, int64_t grid_stride, const int32_t* __restrict__ lin,
                            const double* __restrict__ grid, double* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n_f) return;
  const int64_t r = t / n_f;
  const int f = (int)(t - r * n_f);
  out[t] = grid[(size_t)f * grid_stride + lin[r]];
}

// value of an operator column for function f
__device__ __forceinline__ double ub_value(uint32_t key, int f, int n_f, int64_t grid_stride,
                                           int64_t n_b, const double* __restrict__ u,
                                           const double* __restrict__ grid,
                                           const double* __restrict__ g) {
  const uint32_t kind = key & kKeyKind, idx = key & kKeyIndex;
  if (kind == kKeyUnknown) return u[(size_t)idx * n_f + f];
  if (kind == kKeyGrid) return grid[(size_t)f * grid_stride + idx];
  return g ? g[(size_t)f * n_b + idx] : 0.0;
}

// One U_B small step for every (unknown r, function f), thread t = r n_f + f.
//   mode 0: out = u + dt ut + cdt2/2 L(u)                (Taylor start; ut: [N][n_f])
//   mode 1: out = 2u - up + cdt2 L(u) - sigma D(u - up)
//   mode 2: the mode-1 value v, stored as (v - up)/(2 dt)  (the time derivative at u's time)
// L's interface columns read `grid` (U_FC at u's time), D's the difference grid - grid_prev;
// g: Dirichlet data [n_f][n_b] at u's time (NULL: zero).
__global__ void __launch_bounds__(256) k_ub_step(int mode, int64_t n, int n_f, int64_t grid_stride,
                                                 int64_t n_b, const int32_t* __restrict__ Loff,
                                                 const uint32_t* __restrict__ Lcol,
                                                 const double* __restrict__ Lw,
                                                 const int32_t* __restrict__ Doff,
                                                 const uint32_t* __restrict__ Dcol,
                                                 const double* __restrict__ Dw,
                                                 const double* __restrict__ u,
                                                 const double* __restrict__ up,
                                                 const double* __restrict__ ut,
                                                 const double* __restrict__ grid,
                                                 const double* __restrict__ grid_prev,
                                                 const double* __restrict__ g, double cdt2,
                                                 double dt, double sigma, double* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n_f) return;
  const int64_t r = t / n_f;
  const int f = (int)(t - r * n_f);
  double lap = 0.0;
  for (int k = Loff[r]; k < Loff[r + 1]; ++k)
    lap += Lw[k] * ub_value(Lcol[k], f, n_f, grid_stride, n_b, u, grid, g);
  const double u0 = u[t];
  if (mode == 0) {
    out[t] = u0 + dt * ut[t] + 0.5 * cdt2 * lap;
    return;
  }
  double dis = 0.0;
  for (int k = Doff[r]; k < Doff[r + 1]; ++k) {
    const uint32_t key = Dcol[k], idx = key & kKeyIndex;
    double d;
    if ((key & kKeyKind) == kKeyUnknown) {
      d = u[(size_t)idx * n_f + f] - up[(size_t)idx * n_f + f];
    } else {
      const size_t o = (size_t)f * grid_stride + idx;
      d = grid[o] - grid_prev[o];
    }
    dis += Dw[k] * d;
  }
  const double v = 2.0 * u0 - up[t] + cdt2 * lap - sigma * dis;
  out[t] = mode == 1 ? v : (v - up[t]) / (2.0 * dt);
}

// The merge of eq. (4.9) at the band points nearer than delta to the curve: unknowns
// copy U_B's value and time derivative, slaved points evaluate their boundary
// polynomial on (U_B values, the grid's U_FC values at interface points, Dirichlet data)
// and on the time derivatives of the same.
__global__ void k_ff_merge(int64_t n_near, int n_f, int64_t grid_stride, int64_t n_b,
                           const int32_t* __restrict__ near_lin, const int32_t* __restrict__ near_src,
                           const int32_t* __restrict__ Soff, const uint32_t* __restrict__ Scol,
                           const double* __restrict__ Sw, const double* __restrict__ uB,
                           const double* __restrict__ utB, const double* __restrict__ g,
                           const double* __restrict__ gt, double* __restrict__ u,
                           double* __restrict__ ut) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_near * n_f) return;
  const int64_t q = t / n_f;
  const int f = (int)(t - q * n_f);
  const int32_t src = near_src[q];
  double v, vt;
  if (src >= 0) {
    v = uB[(size_t)src * n_f + f];
    vt = utB[(size_t)src * n_f + f];
  } else {
    const int s = -1 - src;
    v = 0.0;
    vt = 0.0;
    for (int k = Soff[s]; k < Soff[s + 1]; ++k) {
      v += Sw[k] * ub_value(Scol[k], f, n_f, grid_stride, n_b, uB, u, g);
      vt += Sw[k] * ub_value(Scol[k], f, n_f, grid_stride, n_b, utB, ut, gt);
    }
  }
  const size_t o = (size_t)f * grid_stride + near_lin[q];
  u[o] = v;
  ut[o] = vt;
}

// Zero the grid points outside the domain (row intervals of the inside points).
__global__ void k_zero_outside(int nx, int ny, int n_f, const int32_t* __restrict__ iv_off,
                               const int32_t* __restrict__ iv, double* __restrict__ a,
                               double* __restrict__ b) {
  const int j = blockIdx.x, f = blockIdx.y;
  double* ra = a + ((size_t)f * ny + j) * nx;
  double* rb = b + ((size_t)f * ny + j) * nx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    bool in = false;
    for (int k = iv_off[j]; k < iv_off[j + 1]; ++k) in |= (i >= iv[2 * k] && i <= iv[2 * k + 1]);
    if (!in) {
      ra[i] = 0.0;
      rb[i] = 0.0;
    }
  }
}

// Modal advance of the normalised half spectra (F: spec[f], G: spec[n_f + f]) to time
// tau and the inverse column DFT (a forward transform of the conjugate), into the
// row-pass layout [n_out][ny][pitch] for the inverse real row DFT: blockIdx.y = 0: a(tau)
// into out[f]; 1: a'(tau) into out[n_f + f].  One block per (column, output) loops over
// the functions, so the column's time factors (t0, t1) are computed once: a = F t0 + G t1
// with (cos w tau, sin(w tau)/w), or (-w sin w tau, cos w tau) for a'; (1, tau) and (0, 1)
// at w = 0.  Mixed-radix sizes; power-of-two columns take k_ff_cols_p2 (fft_pow2.cu).
__global__ void __launch_bounds__(256) k_ff_cols(FftArgs fa, int n_f, const double2* __restrict__ spec,
                                                 double2* __restrict__ out, double c, double tau,
                                                 double Lx, double Ly) {
  using C = double2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ny = fa.ny, nxh = fa.nx / 2 + 1, kx = blockIdx.x, which = blockIdx.y;
  double2* tab = reinterpret_cast<double2*>(smem_raw);
  C* A = tab + ny;
  C* S = A + ny;
  const double two_pi = 6.283185307179586476925286766559;
  for (int ky = threadIdx.x; ky < ny; ky += blockDim.x) {
    const int m = ky <= ny / 2 ? ky : ky - ny;
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
  for (int f = 0; f < n_f; ++f) {
    const C* colF = spec + (size_t)f * ny * nxh + kx;
    const C* colG = spec + (size_t)(n_f + f) * ny * nxh + kx;
    __syncthreads();
    for (int ky = threadIdx.x; ky < ny; ky += blockDim.x) {
      const double2 t = tab[ky];
      const C F = colF[(size_t)ky * nxh], G = colG[(size_t)ky * nxh];
      A[ky] = C{F.x * t.x + G.x * t.y, -(F.y * t.x + G.y * t.y)};
    }
    __syncthreads();
    const C* r = stockham<double>(A, S, ny, 1, fa.ry, fa.nry, reinterpret_cast<const C*>(fa.twy), 1);
    C* dst = out + ((size_t)which * n_f + f) * ny * fa.pitch + kx;
    for (int y = threadIdx.x; y < ny; y += blockDim.x) dst[(size_t)y * fa.pitch] = C{r[y].x, -r[y].y};
  }
}

unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void wave_destroy(fc2d_plan_s* p) {
  if (!p->wave) return;
  auto* W = static_cast<WaveState*>(p->wave);
  for (auto& kv : W->bands) {
    DevBand& b = *kv.second;
    free_csr(b.L);
    free_csr(b.D);
    free_csr(b.S);
    cudaFree(b.unknown_lin);
    cudaFree(b.near_lin);
    cudaFree(b.near_src);
  }
  cudaFree(W->scr.base);
  delete W;
  p->wave = nullptr;
}

}  // namespace fc2d

using namespace fc2d;

namespace {

fc2d_status wave_checks(fc2d_plan_t p, int n_c, const char* who) {
  if (!p) return set_error(FC2D_ERR_ARG, std::string(who) + ": null plan");
  if (n_c < 1 || n_c > 256) return set_error(FC2D_ERR_ARG, std::string(who) + ": n_c in 1..256");
  if (p->prm.precision != FC2D_FP64)
    return set_error(FC2D_ERR_UNSUPPORTED, std::string(who) + ": FP64 plans only");
  return FC2D_OK;
}

}  // namespace

extern "C" fc2d_status fc2d_wave_band_info(fc2d_plan_t p, int n_c, int64_t* counts) {
  fc2d_status st = wave_checks(p, n_c, "fc2d_wave_band_info");
  if (st) return st;
  if (!counts) return set_error(FC2D_ERR_ARG, "fc2d_wave_band_info: null argument");
  cudaSetDevice(p->device);
  DevBand* b;
  if ((st = get_band(p, n_c, &b))) return st;
  counts[0] = (int64_t)b->host.unknown_lin.size();
  counts[1] = (int64_t)b->host.slaved_lin.size();
  counts[2] = (int64_t)b->host.iface_lin.size();
  counts[3] = (int64_t)b->host.near_lin.size();
  return FC2D_OK;
}

extern "C" fc2d_status fc2d_wave_band_points(fc2d_plan_t p, int n_c, int32_t* unknown_lin,
                                             int32_t* slaved_lin, int32_t* iface_lin,
                                             int32_t* near_lin) {
  fc2d_status st = wave_checks(p, n_c, "fc2d_wave_band_points");
  if (st) return st;
  cudaSetDevice(p->device);
  DevBand* b;
  if ((st = get_band(p, n_c, &b))) return st;
  const WaveBand& w = b->host;
  auto cp = [](int32_t* dst, const std::vector<int32_t>& v) {
    if (dst && !v.empty()) std::memcpy(dst, v.data(), v.size() * sizeof(int32_t));
  };
  cp(unknown_lin, w.unknown_lin);
  cp(slaved_lin, w.slaved_lin);
  cp(iface_lin, w.iface_lin);
  cp(near_lin, w.near_lin);
  return FC2D_OK;
}

extern "C" fc2d_status fc2d_wave_ub_step(fc2d_plan_t p, int n_c, int n_f, int mode, double c,
                                         const double* u, const double* u_prev, const double* ut,
                                         const double* grid, const double* grid_prev,
                                         const double* g, double* out, void* stream) {
  fc2d_status st = wave_checks(p, n_c, "fc2d_wave_ub_step");
  if (st) return st;
  if ((st = check_nf(p, n_f))) return st;
  if (mode < 0 || mode > 2 || !u || !grid || !out || (mode == 0 && !ut) ||
      (mode > 0 && (!u_prev || !grid_prev)) || !(c > 0))
    return set_error(FC2D_ERR_ARG, "fc2d_wave_ub_step: bad mode, c or null pointer");
  cudaSetDevice(p->device);
  DevBand* b;
  if ((st = get_band(p, n_c, &b))) return st;
  const double h = p->grid.h, cdt2 = (kUbCfl * h) * (kUbCfl * h);
  const double dt = kUbCfl * h / c;
  const int64_t n = b->L.rows;
  if (n > 0)
    k_ub_step<<<blocks(n * n_f, 256), 256, 0, (cudaStream_t)stream>>>(
        mode, n, n_f, (int64_t)p->grid.nx * p->grid.ny, p->n_bdry, b->L.off, b->L.col, b->L.w,
        b->D.off, b->D.col, b->D.w, u, u_prev, ut, grid, grid_prev, g, cdt2, dt, kUbSigma, out);
  return cuda_check(cudaGetLastError(), "fc2d_wave_ub_step");
}

extern "C" fc2d_status fc2d_forward_wave(fc2d_plan_t p, int n_f, double c, int n_c, int n_large,
                                         double* u, double* ut, const double* g_dir,
                                         const double* gt_dir, void* stream) {
  fc2d_status st = wave_checks(p, n_c, "fc2d_forward_wave");
  if (st) return st;
  if ((st = check_nf(p, n_f))) return st;
  if (!u || !ut) return set_error(FC2D_ERR_ARG, "fc2d_forward_wave: null pointer");
  if (!(c > 0) || n_large < 0)
    return set_error(FC2D_ERR_ARG, "fc2d_forward_wave: c > 0 and n_large >= 0 required");
  if (3 * (size_t)p->grid.ny * sizeof(double2) > 227 * 1024)
    return set_error(FC2D_ERR_UNSUPPORTED, "fc2d_forward_wave: ny <= 4842");
  if (n_large == 0) return FC2D_OK;
  cudaSetDevice(p->device);
  cudaStream_t s = (cudaStream_t)stream;
  DevBand* b;
  if ((st = get_band(p, n_c, &b))) return st;
  const int nx = p->grid.nx, ny = p->grid.ny, nxh = nx / 2 + 1;
  const int64_t NN = (int64_t)nx * ny, nb = p->n_bdry, Nu = b->L.rows;
  const size_t pitch = row_pitch(p);
  const int S = 8 * n_c;
  const double h = p->grid.h, dT = n_c * h / c, dt = dT / S, cdt2 = (c * dt) * (c * dt);
  // scratch: spectra [2 n_f][ny][nxh], row-pass layout [2 n_f][ny][pitch], two U_FC grids,
  // four U_B arrays, zero boundary data
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t b_spec = al((size_t)2 * n_f * ny * nxh * 16), b_inter = al((size_t)2 * n_f * ny * pitch * 16),
               b_grid = al((size_t)n_f * NN * 8), b_ub = al((size_t)std::max<int64_t>(1, Nu) * n_f * 8),
               b_zero = al((size_t)n_f * nb * 8);
  const size_t need = b_spec + b_inter + 2 * b_grid + 4 * b_ub + b_zero;
  WaveState* W = state(p);
  if (W->scr.bytes < need) {
    cudaDeviceSynchronize();
    cudaFree(W->scr.base);
    W->scr = Scratch();
    if (cudaMalloc(&W->scr.base, need) != cudaSuccess)
      return set_error(FC2D_ERR_NOMEM, "fc2d_forward_wave: scratch cudaMalloc failed");
    W->scr.bytes = need;
  }
  char* base = static_cast<char*>(W->scr.base);
  double2* spec = reinterpret_cast<double2*>(base);
  double2* inter = reinterpret_cast<double2*>(base + b_spec);
  double* ufc[2] = {reinterpret_cast<double*>(base + b_spec + b_inter),
                    reinterpret_cast<double*>(base + b_spec + b_inter + b_grid)};
  double* ub[4];
  for (int k = 0; k < 4; ++k)
    ub[k] = reinterpret_cast<double*>(base + b_spec + b_inter + 2 * b_grid + k * b_ub);
  double* zero = reinterpret_cast<double*>(base + b_spec + b_inter + 2 * b_grid + 4 * b_ub);
  cudaMemsetAsync(zero, 0, (size_t)n_f * nb * 8, s);
  auto gat = [&](int64_t m) { return g_dir ? g_dir + (size_t)m * n_f * nb : nullptr; };
  auto gtat = [&](int64_t j) { return gt_dir ? gt_dir + (size_t)j * n_f * nb : nullptr; };
  FftArgs fa = fft_args(p);
  const double Lx = nx * h, Ly = ny * h;
  const size_t smc = 3 * (size_t)ny * sizeof(double2);
  cudaFuncSetAttribute(k_ff_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc);
  auto eval_ufc = [&](double tau, int n_out, double* out_u, double* out_ut) {
    {
      ProfScope ps(p, "ff_cols", s);
      if (!launch_ff_cols_p2(fa, n_f, n_out, spec, inter, c, tau, Lx, Ly, s))
        k_ff_cols<<<dim3(nxh, n_out), 256, smc, s>>>(fa, n_f, spec, inter, c, tau, Lx, Ly);
    }
    ProfScope ps(p, "inverse_rows", s);
    launch_inverse_rows(fa, n_f, inter, nullptr, p->grid.a0, p->grid.b0, h, out_u, s);
    if (n_out == 2)
      launch_inverse_rows(fa, n_f, inter + (size_t)n_f * ny * pitch, nullptr, p->grid.a0,
                          p->grid.b0, h, out_ut, s);
  };
  auto ub_step = [&](int mode, const double* uc, const double* upv, const double* utv,
                     const double* grid, const double* grid_prev, const double* g, double* out) {
    if (Nu == 0) return;
    ProfScope ps(p, "ub_step", s);
    k_ub_step<<<blocks(Nu * n_f, 256), 256, 0, s>>>(mode, Nu, n_f, NN, nb, b->L.off, b->L.col,
                                                    b->L.w, b->D.off, b->D.col, b->D.w, uc, upv,
                                                    utv, grid, grid_prev, g, cdt2, dt, kUbSigma, out);
  };
  // U_B at t = 0: u^0 and u_t^0 at the unknowns
  int i_prev = 0, i_cur = 1, i_next = 2;
  const int i_ut = 3;
  if (Nu > 0) {
    k_ub_gather<<<blocks(Nu * n_f, 256), 256, 0, s>>>(Nu, n_f, NN, b->unknown_lin, u, ub[i_cur]);
    k_ub_gather<<<blocks(Nu * n_f, 256), 256, 0, s>>>(Nu, n_f, NN, b->unknown_lin, ut, ub[i_ut]);
  }
  int f_cur = 0;  // U_FC grid of the current small step; the other holds the previous one
  for (int j = 0; j < n_large; ++j) {
    const int64_t m0 = (int64_t)j * S;
    if ((st = wave_spectra(p, n_f, u, g_dir ? gat(m0) : zero, ut, gt_dir ? gtat(j) : zero, spec, s)))
      return st;
    for (int sidx = 0; sidx < S; ++sidx) {
      const int64_t m = m0 + sidx;
      eval_ufc(sidx * dt, 1, ufc[f_cur], nullptr);
      if (m == 0) {
        ub_step(0, ub[i_cur], nullptr, ub[i_ut], ufc[f_cur], nullptr, gat(m), ub[i_next]);
      } else {
        ub_step(1, ub[i_cur], ub[i_prev], nullptr, ufc[f_cur], ufc[1 - f_cur], gat(m), ub[i_next]);
      }
      const int t0 = i_prev;
      i_prev = i_cur;
      i_cur = i_next;
      i_next = t0;
      f_cur = 1 - f_cur;
    }
    // T_{j+1}: U_FC and its time derivative on the grid (into u, ut), then U_B's time
    // derivative from one further step and the merge of eq. (4.9)
    eval_ufc(dT, 2, u, ut);
    const int64_t mN = m0 + S;
    ub_step(2, ub[i_cur], ub[i_prev], nullptr, u, ufc[1 - f_cur], gat(mN), ub[i_ut]);
    const int64_t n_near = (int64_t)b->host.near_lin.size();
    if (n_near > 0) {
      ProfScope ps(p, "ff_merge", s);
      k_ff_merge<<<blocks(n_near * n_f, 256), 256, 0, s>>>(
          n_near, n_f, NN, nb, b->near_lin, b->near_src, b->S.off, b->S.col, b->S.w, ub[i_cur],
          ub[i_ut], g_dir ? gat(mN) : zero, gt_dir ? gtat(j + 1) : zero, u, ut);
    }
  }
  k_zero_outside<<<dim3(ny, n_f), 256, 0, s>>>(nx, ny, n_f, p->dev.row_iv_off, p->dev.row_iv, u, ut);
  return cuda_check(cudaGetLastError(), "fc2d_forward_wave");
}
