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

struct DevSquares {
  SquareSet host;
  int32_t* origin = nullptr;        // [n_sq][2] (row, column) of the first grid point
  int32_t* served_off = nullptr;    // [n_sq + 1]
  int32_t* served_lin = nullptr;
  int32_t* served_local = nullptr;
  double* A = nullptr;              // [C][d]
  double* Q = nullptr;              // [d][d]
  double2* tw = nullptr;            // exp(-2 pi i t / P), t < P
  float4* tw_df = nullptr;          // the same as double-float pairs (re hi, lo, im hi, lo)
  int32_t* rows = nullptr;          // [n_sq][2]: first and last box row holding served points
  int n = 0;
};

struct DevBand {
  WaveBand host;
  DevCsr L, D, S;
  int32_t* unknown_lin = nullptr;
  int32_t* near_lin = nullptr;
  int32_t* near_src = nullptr;
  std::unique_ptr<DevSquares> sq;   // the small-square procedure's squares (mode 1)
};

struct Scratch {
  int n_f = 0;
  size_t bytes = 0;
  void* base = nullptr;
};

struct WaveState {
  std::map<std::pair<int, int>, std::unique_ptr<DevBand>> bands;  // by (n_c, interface mode)
  Scratch scr;
  // double-float twiddles for U_FC in interface mode 2 (built on first use):
  // w_ny^t (t < ny), w_{nx/2}^t (t < nx/2), w_nx^k (k <= nx/2), as (re hi, lo, im hi, lo)
  float4 *df_twy = nullptr, *df_twx = nullptr, *df_rtw = nullptr;
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

// The band reach (grid units) for an interface mode: 0 full U_FC at every small step,
// 1 the small squares (whose service needs interface points at sqrt(2) n_c h or more).
int reach_cells(int n_c, int mode) {
  return mode ? (int)std::ceil(std::sqrt(2.0) * n_c) + 2 : n_c + kUbBandExtra;
}

fc2d_status upload_squares(const fc2d_plan_s* p, DevBand& b, int n_c) {
  auto q = std::make_unique<DevSquares>();
  fc2d_status st = build_wave_squares(p, b.host, n_c, q->host);
  if (st) return st;
  const SquareSet& h = q->host;
  q->n = (int)h.origin_j.size();
  std::vector<int32_t> origin(2 * (size_t)q->n);
  for (int k = 0; k < q->n; ++k) {
    origin[2 * k] = h.origin_j[k];
    origin[2 * k + 1] = h.origin_i[k];
  }
  std::vector<int32_t> rows(2 * (size_t)q->n);
  for (int k = 0; k < q->n; ++k) {
    int lo = h.P, hi = -1;
    for (int i = h.served_off[k]; i < h.served_off[k + 1]; ++i) {
      lo = std::min(lo, h.served_local[i] / h.P);
      hi = std::max(hi, h.served_local[i] / h.P);
    }
    rows[2 * k] = lo;
    rows[2 * k + 1] = hi;
  }
  std::vector<double2> tw(h.P);
  std::vector<float4> tw_df(h.P);
  for (int t = 0; t < h.P; ++t) {
    const double ang = -2.0 * M_PI * double(t) / double(h.P);
    tw[t] = double2{std::cos(ang), std::sin(ang)};
    const float ch = (float)tw[t].x, sh = (float)tw[t].y;
    tw_df[t] = float4{ch, (float)(tw[t].x - (double)ch), sh, (float)(tw[t].y - (double)sh)};
  }
  if ((st = upload(&q->origin, origin)) || (st = upload(&q->served_off, h.served_off)) ||
      (st = upload(&q->served_lin, h.served_lin)) || (st = upload(&q->served_local, h.served_local)) ||
      (st = upload(&q->A, h.A)) || (st = upload(&q->Q, h.Q)) || (st = upload(&q->tw, tw)) ||
      (st = upload(&q->tw_df, tw_df)) || (st = upload(&q->rows, rows)))
    return st;
  b.sq = std::move(q);
  return FC2D_OK;
}

// The double-float twiddle tables of interface mode 2, from the plan's FP64 tables
// (interleaved re, im): hi = RN(v), lo = RN(v - hi).
fc2d_status df_tables(fc2d_plan_s* p, WaveState* W) {
  if (W->df_twy) return FC2D_OK;
  auto split = [](const std::vector<double>& v, size_t n) {
    std::vector<float4> out(n);
    for (size_t t = 0; t < n; ++t) {
      const double re = v[2 * t], im = v[2 * t + 1];
      const float rh = (float)re, ih = (float)im;
      out[t] = float4{rh, (float)(re - (double)rh), ih, (float)(im - (double)ih)};
    }
    return out;
  };
  fc2d_status st;
  if ((st = upload(&W->df_twy, split(p->fy.tw_host, (size_t)p->grid.ny))) ||
      (st = upload(&W->df_twx, split(p->fx.tw_host, (size_t)p->grid.nx / 2))) ||
      (st = upload(&W->df_rtw, split(p->rtw_host, (size_t)p->grid.nx / 2 + 1))))
    return st;
  return FC2D_OK;
}

fc2d_status get_band(fc2d_plan_s* p, int n_c, int mode, DevBand** out) {
  WaveState* W = state(p);
  auto it = W->bands.find({n_c, mode});
  if (it != W->bands.end()) {
    *out = it->second.get();
    return FC2D_OK;
  }
  auto b = std::make_unique<DevBand>();
  fc2d_status st = build_wave_band(p, n_c, reach_cells(n_c, mode), b->host);
  if (st) return st;
  if (mode && (st = upload_squares(p, *b, n_c))) return st;
  // operator entries of a grid kind must index the grid (30 bits), boundary data too
  if ((int64_t)p->grid.nx * p->grid.ny > (int64_t)kKeyIndex || p->n_bdry > (int64_t)kKeyIndex)
    return set_error(FC2D_ERR_UNSUPPORTED, "wave band: grid too large for the operator keys");
  if ((st = upload_csr(b->L, b->host.L)) || (st = upload_csr(b->D, b->host.D)) ||
      (st = upload_csr(b->S, b->host.S)) || (st = upload(&b->unknown_lin, b->host.unknown_lin)) ||
      (st = upload(&b->near_lin, b->host.near_lin)) || (st = upload(&b->near_src, b->host.near_src)))
    return st;
  *out = b.get();
  W->bands[{n_c, mode}] = std::move(b);
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

// ------------------------------------------------------------------------- //
// The small-square procedure (Section 4.2; wave_band.cpp builds the squares)
// ------------------------------------------------------------------------- //
constexpr int kSqThreads = 256;

// 1D-FC continuation (eq. (2.7)) of the length-n sequence x[at(0)], ..., x[at(n-1)]
// (complex values: two real functions at once) into x[at(n)] .. x[at(n + C - 1)]:
// the C values (A Q^T r)_k + (A Q^T l)_{C-1-k}, r the last d values, l the first d in
// reverse order.  One thread per continuation point.
template <typename At>
__device__ __forceinline__ void fc1d_continue(double2* x, At at, int n, int C, int d,
                                              const double* __restrict__ A,
                                              const double* __restrict__ Q, int k) {
  double2 cr[kMaxD], cl[kMaxD];
  for (int i = 0; i < d; ++i) {  // Gram coefficients c = Q^T f
    double2 r = {0.0, 0.0}, l = {0.0, 0.0};
    for (int m = 0; m < d; ++m) {
      const double qm = __ldg(Q + m * d + i);
      const double2 fr = x[at(n - d + m)], fl = x[at(d - 1 - m)];
      r.x += qm * fr.x;
      r.y += qm * fr.y;
      l.x += qm * fl.x;
      l.y += qm * fl.y;
    }
    cr[i] = r;
    cl[i] = l;
  }
  double2 vr = {0.0, 0.0}, vl = {0.0, 0.0};
  for (int i = 0; i < d; ++i) {
    const double ar = __ldg(A + k * d + i), al = __ldg(A + (C - 1 - k) * d + i);
    vr.x += ar * cr[i].x;
    vr.y += ar * cr[i].y;
    vl.x += al * cl[i].x;
    vl.y += al * cl[i].y;
  }
  x[at(n + k)] = double2{vl.x + vr.x, vl.y + vr.y};
}

// 64-point DFT of the padded sequence x[pad(e) ST], e < 64 (pad(e) = e + e/8), by the 8
// threads q = 0..7 of a group, as 8 x 8: X[k1 + 8 k2] = sum_q w8^(q k2) w64^(q k1)
// sum_r x[q + 8 r] w8^(r k1); the result replaces x in natural order.  Every thread of
// the block calls it (three barriers, the last after the result is stored); `active`
// false: a group with nothing to transform.
__device__ __forceinline__ int sq_pad(int e) { return e + (e >> 3); }

// Forward 8-point DFT in registers (radix 2 x 4: two 4-point DFTs of the even and odd
// entries, the twiddles exp(-2 pi i k/8), one butterfly).
__device__ __forceinline__ void dft8_regs(double2 (&v)[8]) {
  const double s = 0.70710678118654752440;
  auto d4 = [](double2& a0, double2& a1, double2& a2, double2& a3) {
    const double2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3);
    const double2 t3 = mul_mi(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
  };
  double2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  d4(e0, e1, e2, e3);
  d4(o0, o1, o2, o3);
  const double2 w1 = {s * (o1.x + o1.y), s * (o1.y - o1.x)};
  const double2 w2 = mul_mi(o2);
  const double2 w3 = {s * (o3.y - o3.x), -s * (o3.x + o3.y)};
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, w1);
  v[5] = csub(e1, w1);
  v[2] = cadd(e2, w2);
  v[6] = csub(e2, w2);
  v[3] = cadd(e3, w3);
  v[7] = csub(e3, w3);
}

template <int ST = 1>
__device__ __forceinline__ void fft64(double2* x, int q, bool active,
                                      const double2* __restrict__ tw) {
  double2 v[8];
  if (active) {
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = x[sq_pad(q + 8 * r) * ST];
    dft8_regs(v);
#pragma unroll
    for (int k = 1; k < 8; ++k) v[k] = cmul(v[k], __ldg(tw + q * k));  // w64^(q k1)
#pragma unroll
    for (int k = 0; k < 8; ++k) x[sq_pad(q + 8 * k) * ST] = v[k];
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = x[sq_pad(8 * q + r) * ST];  // thread q is k1 here
    dft8_regs(v);
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[sq_pad(q + 8 * k) * ST] = v[k];
  }
  __syncthreads();
}

// A complex double as double-float pairs: hi = RN(x), lo = RN(x - hi).
__device__ __forceinline__ float4 split_df(double2 v) {
  const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
  return float4{rh, __double2float_rn(v.x - (double)rh), ih, __double2float_rn(v.y - (double)ih)};
}

// Once per large step: each square's expansion.  Block (square, function): the square's
// u and u_t as one complex field z = u + i u_t, continued along rows, then columns, to
// P x P; its 2D DFT, normalised, stored transposed: Z[l][m] (l: x frequency).
// DF: Z as double-float pairs (float4 re hi, re lo, im hi, im lo) for k_sq_eval_df.
// One padded buffer holds the field and both transforms in place: value (y, x) at
// sq_pad(y) kSqRow + sq_pad(x).  The 64-point DFTs (fft64, 8 threads each) run along x at
// unit stride and along y at stride kSqRow; kSqRow is odd in 16-byte units, so both
// access patterns of fft64 (consecutive and every 8th element) spread over all banks in
// either direction.  83 KB of shared memory allow two blocks per SM.
constexpr int kSqRow = 73;                       // row stride (complex values)
constexpr int kSqRows = 64 + 64 / 8 - 1;         // sq_pad(63) + 1 rows
constexpr size_t kSqForwardSmem = (size_t)kSqRows * kSqRow * sizeof(double2);

template <bool DF>
__global__ void __launch_bounds__(kSqThreads, 2) k_sq_forward(
    int n_side, int C, int d, int nx, int64_t grid_stride, int n_f,
    const int32_t* __restrict__ origin, const double* __restrict__ A,
    const double* __restrict__ Q, const double2* __restrict__ tw, const double* __restrict__ u,
    const double* __restrict__ ut, double2* __restrict__ Z) {
  constexpr int P = kSqP;  // n_side + C = P (the host checks)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* buf = reinterpret_cast<double2*>(smem_raw);
  const int sq = blockIdx.x, f = blockIdx.y;
  const int j0 = __ldg(origin + 2 * sq), i0 = __ldg(origin + 2 * sq + 1);
  const double* uf = u + (size_t)f * grid_stride;
  const double* tf = ut + (size_t)f * grid_stride;
  for (int t = threadIdx.x; t < n_side * n_side; t += blockDim.x) {
    const int y = t / n_side, x = t - y * n_side;
    const size_t g = (size_t)(j0 + y) * nx + (i0 + x);
    buf[sq_pad(y) * kSqRow + sq_pad(x)] = double2{uf[g], tf[g]};
  }
  __syncthreads();
  const auto along_x = [](int i) { return sq_pad(i); };
  const auto along_y = [](int i) { return sq_pad(i) * kSqRow; };
  for (int t = threadIdx.x; t < n_side * C; t += blockDim.x) {  // rows
    const int y = t / C, k = t - y * C;
    fc1d_continue(buf + sq_pad(y) * kSqRow, along_x, n_side, C, d, A, Q, k);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < P * C; t += blockDim.x) {  // columns
    const int x = t / C, k = t - x * C;
    fc1d_continue(buf + sq_pad(x), along_y, n_side, C, d, A, Q, k);
  }
  __syncthreads();
  const int g = threadIdx.x >> 3, q = threadIdx.x & 7;
  constexpr int G = kSqThreads / 8;  // transforms per call
#pragma unroll 1
  for (int y0 = 0; y0 < P; y0 += G)  // along x: (y, l)
    fft64<1>(buf + sq_pad(y0 + g) * kSqRow, q, y0 + g < P, tw);
#pragma unroll 1
  for (int l0 = 0; l0 < P; l0 += G)  // along y: (m, l)
    fft64<kSqRow>(buf + sq_pad(l0 + g), q, l0 + g < P, tw);
  const double sc = 1.0 / ((double)P * P);
  double2* dst = Z + ((size_t)sq * n_f + f) * P * P;
  for (int t = threadIdx.x; t < P * P; t += blockDim.x) {
    const int l = t / P, m = t - l * P;
    const double2 w = buf[sq_pad(m) * kSqRow + sq_pad(l)];
    const double2 v = double2{w.x * sc, w.y * sc};
    if constexpr (DF) reinterpret_cast<float4*>(dst)[t] = split_df(v);
    else dst[t] = v;
  }
}

constexpr int kSqPad = 72;        // padded length of a 64-point sequence
constexpr int kSqEvalThreads = 512;

// Every small step: U at the served interface points at time tau = s dt after the
// expansion.  Block (square, function pair) of 512 threads (64 groups of 8): for functions
// f0 = 2 blockIdx.y and f0 + 1 the spectra of u and u_t are separated from Z (hat f =
// (Z_k + conj Z_-k)/2, hat g = (Z_k - conj Z_-k)/(2i)), advanced with the time factors
// (cos w tau, sin(w tau)/w) of the P-periodic box (table tab[l][m]) and packed as
// conj(a_f0 + i a_f1); the inverse 2D DFT runs as forward 64-point DFTs along m for every
// l, a transpose of the rows the served points need (rows r0..r1 of the square), and
// forward DFTs along l for those rows; the real part of the conjugated result is f0's
// field, the imaginary part with its sign changed f1's.
__global__ void __launch_bounds__(kSqEvalThreads, 2) k_sq_eval(
    int n_f, const double2* __restrict__ Z, const double2* __restrict__ tab,
    const double2* __restrict__ tw, const int32_t* __restrict__ served_off,
    const int32_t* __restrict__ served_lin, const int32_t* __restrict__ served_local,
    const int32_t* __restrict__ rows, int64_t grid_stride, double* __restrict__ out) {
  constexpr int P = kSqP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* T1 = reinterpret_cast<double2*>(smem_raw);  // [64][72]: transform l along m
  double2* T2 = T1 + P * kSqPad;                        // [rows][72]: transform y along l
  const int sq = blockIdx.x, f0 = 2 * blockIdx.y;
  const bool two = f0 + 1 < n_f;
  const double2* Z0 = Z + ((size_t)sq * n_f + f0) * P * P;
  const double2* Z1 = Z0 + (size_t)P * P;
  const int g = threadIdx.x >> 3, q = threadIdx.x & 7;
  for (int t = threadIdx.x; t < P * P; t += blockDim.x) {
    const int l = t / P, m = t - l * P;
    const int tn = ((P - l) & (P - 1)) * P + ((P - m) & (P - 1));  // the index of -k
    const double2 tt = __ldg(tab + t);
    auto adv = [&](const double2* Zf) {
      const double2 zk = Zf[t], zn = Zf[tn];
      const double2 F = {0.5 * (zk.x + zn.x), 0.5 * (zk.y - zn.y)};   // (Z_k + conj Z_-k)/2
      const double2 G = {0.5 * (zk.y + zn.y), -0.5 * (zk.x - zn.x)};  // (Z_k - conj Z_-k)/(2i)
      return double2{F.x * tt.x + G.x * tt.y, F.y * tt.x + G.y * tt.y};
    };
    const double2 a0 = adv(Z0);
    const double2 a1 = two ? adv(Z1) : double2{0.0, 0.0};
    T1[l * kSqPad + sq_pad(m)] = double2{a0.x - a1.y, -(a0.y + a1.x)};  // conj(a0 + i a1)
  }
  __syncthreads();
  fft64(T1 + g * kSqPad, q, true, tw);  // T1[l][y]
  const int r0 = __ldg(rows + 2 * sq), nr = __ldg(rows + 2 * sq + 1) - r0 + 1;
  for (int t = threadIdx.x; t < nr * P; t += blockDim.x) {
    const int yr = t / P, l = t - yr * P;
    T2[yr * kSqPad + sq_pad(l)] = T1[l * kSqPad + sq_pad(r0 + yr)];
  }
  __syncthreads();
  fft64(T2 + g * kSqPad, q, g < nr, tw);  // T2[y - r0][x]
  const int s0 = __ldg(served_off + sq), s1 = __ldg(served_off + sq + 1);
  for (int k = s0 + threadIdx.x; k < s1; k += blockDim.x) {
    const int loc = __ldg(served_local + k), y = loc / P, x = loc - y * P;
    const double2 v = T2[(y - r0) * kSqPad + sq_pad(x)];
    const int32_t lin = __ldg(served_lin + k);
    out[(size_t)f0 * grid_stride + lin] = v.x;
    if (two) out[(size_t)(f0 + 1) * grid_stride + lin] = -v.y;
  }
}

// ------------------------------------------------------------------------- //
// The same evaluation in double-float arithmetic (interface mode 2).  A real number is
// the unevaluated sum hi + lo of two floats; sums use Knuth's TwoSum with the low parts
// added after it and Dekker's FastTwoSum to renormalise, products the FMA form of
// Dekker's TwoProduct (Dekker 1971; Knuth, TAOCP vol. 2, 4.2.2).  Each operation is
// accurate to about 2^-44 of its operands' size, on the FP32 pipe, which on this part
// issues 64 times as many operations as the FP64 pipe.
// ------------------------------------------------------------------------- //
struct df2 {
  float hi, lo;
};
struct dfc {
  df2 re, im;
};
__device__ __forceinline__ df2 df_fast(float a, float b) {  // |a| >= |b| or a = 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df2 df_add(df2 a, df2 b) {
  const float s = __fadd_rn(a.hi, b.hi), bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return df_fast(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df2 df_neg(df2 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df2 df_sub(df2 a, df2 b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df2 df_mul(df2 a, df2 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast(p, e);
}
__device__ __forceinline__ df2 df_half(df2 a) { return {0.5f * a.hi, 0.5f * a.lo}; }
__device__ __forceinline__ dfc dfc_load(float4 v) { return {{v.x, v.y}, {v.z, v.w}}; }
__device__ __forceinline__ float4 dfc_store(dfc a) { return float4{a.re.hi, a.re.lo, a.im.hi, a.im.lo}; }
__device__ __forceinline__ dfc dfc_add(dfc a, dfc b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ dfc dfc_sub(dfc a, dfc b) { return {df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
__device__ __forceinline__ dfc dfc_mul_mi(dfc a) { return {a.im, df_neg(a.re)}; }  // -i a
__device__ __forceinline__ dfc dfc_mul(dfc a, dfc b) {
  return {df_sub(df_mul(a.re, b.re), df_mul(a.im, b.im)),
          df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
__device__ __forceinline__ double df_to_double(df2 a) { return (double)a.hi + (double)a.lo; }

// Forward 8-point DFT in registers (as dft8_regs)
__device__ __forceinline__ void dft8_df(dfc (&v)[8]) {
  constexpr double kS = 0.70710678118654752440;
  const df2 s = {(float)kS, (float)(kS - (double)(float)kS)};
  auto d4 = [](dfc& a0, dfc& a1, dfc& a2, dfc& a3) {
    const dfc t0 = dfc_add(a0, a2), t1 = dfc_sub(a0, a2), t2 = dfc_add(a1, a3);
    const dfc t3 = dfc_mul_mi(dfc_sub(a1, a3));
    a0 = dfc_add(t0, t2);
    a2 = dfc_sub(t0, t2);
    a1 = dfc_add(t1, t3);
    a3 = dfc_sub(t1, t3);
  };
  dfc e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  d4(e0, e1, e2, e3);
  d4(o0, o1, o2, o3);
  const dfc w1 = {df_mul(s, df_add(o1.re, o1.im)), df_mul(s, df_sub(o1.im, o1.re))};
  const dfc w2 = dfc_mul_mi(o2);
  const dfc w3 = {df_mul(s, df_sub(o3.im, o3.re)), df_neg(df_mul(s, df_add(o3.re, o3.im)))};
  v[0] = dfc_add(e0, o0);
  v[4] = dfc_sub(e0, o0);
  v[1] = dfc_add(e1, w1);
  v[5] = dfc_sub(e1, w1);
  v[2] = dfc_add(e2, w2);
  v[6] = dfc_sub(e2, w2);
  v[3] = dfc_add(e3, w3);
  v[7] = dfc_sub(e3, w3);
}

// 64-point DFT of the padded sequence x[pad(e)] (as fft64)
__device__ __forceinline__ void fft64_df(float4* x, int q, bool active,
                                         const float4* __restrict__ tw) {
  dfc v[8];
  if (active) {
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = dfc_load(x[sq_pad(q + 8 * r)]);
    dft8_df(v);
#pragma unroll
    for (int k = 1; k < 8; ++k) v[k] = dfc_mul(v[k], dfc_load(__ldg(tw + q * k)));
#pragma unroll
    for (int k = 0; k < 8; ++k) x[sq_pad(q + 8 * k)] = dfc_store(v[k]);
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = dfc_load(x[sq_pad(8 * q + r)]);
    dft8_df(v);
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[sq_pad(q + 8 * k)] = dfc_store(v[k]);
  }
  __syncthreads();
}

// k_sq_eval in double-float: Z and tab hold double-float pairs (float4), tw_df the box's
// twiddles; the served values are converted to double on output.
__global__ void __launch_bounds__(kSqEvalThreads, 2) k_sq_eval_df(
    int n_f, const float4* __restrict__ Z, const float4* __restrict__ tab,
    const float4* __restrict__ tw, const int32_t* __restrict__ served_off,
    const int32_t* __restrict__ served_lin, const int32_t* __restrict__ served_local,
    const int32_t* __restrict__ rows, int64_t grid_stride, double* __restrict__ out) {
  constexpr int P = kSqP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* T1 = reinterpret_cast<float4*>(smem_raw);  // [64][72]: transform l along m
  float4* T2 = T1 + P * kSqPad;                       // [rows][72]: transform y along l
  const int sq = blockIdx.x, f0 = 2 * blockIdx.y;
  const bool two = f0 + 1 < n_f;
  const float4* Z0 = Z + ((size_t)sq * n_f + f0) * P * P;
  const float4* Z1 = Z0 + (size_t)P * P;
  const int g = threadIdx.x >> 3, q = threadIdx.x & 7;
  for (int t = threadIdx.x; t < P * P; t += blockDim.x) {
    const int l = t / P, m = t - l * P;
    const int tn = ((P - l) & (P - 1)) * P + ((P - m) & (P - 1));  // the index of -k
    const dfc tt = dfc_load(__ldg(tab + t));                        // (cos w tau, sin(w tau)/w)
    auto adv = [&](const float4* Zf) {
      const dfc zk = dfc_load(Zf[t]), zn = dfc_load(Zf[tn]);
      const dfc F = {df_half(df_add(zk.re, zn.re)), df_half(df_sub(zk.im, zn.im))};
      const dfc G = {df_half(df_add(zk.im, zn.im)), df_neg(df_half(df_sub(zk.re, zn.re)))};
      return dfc{df_add(df_mul(F.re, tt.re), df_mul(G.re, tt.im)),
                 df_add(df_mul(F.im, tt.re), df_mul(G.im, tt.im))};
    };
    const dfc a0 = adv(Z0);
    const dfc a1 = two ? adv(Z1) : dfc{{0.f, 0.f}, {0.f, 0.f}};
    T1[l * kSqPad + sq_pad(m)] = dfc_store(dfc{df_sub(a0.re, a1.im), df_neg(df_add(a0.im, a1.re))});
  }
  __syncthreads();
  fft64_df(T1 + g * kSqPad, q, true, tw);  // T1[l][y]
  const int r0 = __ldg(rows + 2 * sq), nr = __ldg(rows + 2 * sq + 1) - r0 + 1;
  for (int t = threadIdx.x; t < nr * P; t += blockDim.x) {
    const int yr = t / P, l = t - yr * P;
    T2[yr * kSqPad + sq_pad(l)] = T1[l * kSqPad + sq_pad(r0 + yr)];
  }
  __syncthreads();
  fft64_df(T2 + g * kSqPad, q, g < nr, tw);  // T2[y - r0][x]
  const int s0 = __ldg(served_off + sq), s1 = __ldg(served_off + sq + 1);
  for (int k = s0 + threadIdx.x; k < s1; k += blockDim.x) {
    const int loc = __ldg(served_local + k), y = loc / P, x = loc - y * P;
    const dfc v = dfc_load(T2[(y - r0) * kSqPad + sq_pad(x)]);
    const int32_t lin = __ldg(served_lin + k);
    out[(size_t)f0 * grid_stride + lin] = df_to_double(v.re);
    if (two) out[(size_t)(f0 + 1) * grid_stride + lin] = -df_to_double(v.im);
  }
}

// ------------------------------------------------------------------------- //
// U_FC at T_{j+1} in double-float (interface mode 2): the modal advance and the inverse
// column DFT (k_ff_cols_df), then the inverse real rows (k_inverse_rows_df), on a
// power-of-two Stockham transform in double-float.  Doubles enter through split_fast and
// leave through df_to_double_fast, both on the integer and FP32 pipes.
// ------------------------------------------------------------------------- //

// x as hi + lo, hi = RN(x) and lo = RN(x - hi), for |x| in [2^-74, 2^125] (exponent e in
// [949, 1148]) on the integer pipe: hi by rounding the 64-bit pattern at bit 29 (as
// d2f_rn), x - hi as the integer difference of the patterns of x and of hi (in units of
// x's ulp 2^(e-1075), |d| <= 2^28; a carry into hi's exponent keeps the difference
// exact), converted to float and scaled by that ulp.  Zero gives (0, 0); other values
// take the FP64 conversions.
__device__ __forceinline__ df2 split_fast(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned h32 = (unsigned)(b >> 32), e = (h32 >> 20) & 0x7FFu;
  if (e - 949u > 1148u - 949u) {
    if ((b << 1) == 0ull) return {__uint_as_float(h32 & 0x80000000u), 0.f};
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
  }
  const unsigned long long u = b + 0x0FFFFFFFull + ((b >> 29) & 1ull);
  const unsigned sign = h32 & 0x80000000u;
  const float hi = __uint_as_float(((unsigned)(u >> 29) - (896u << 23)) | sign);
  const long long d = (long long)(b - (u & ~0x1FFFFFFFull));  // |x| - |hi| in ulps
  const float ulp = __uint_as_float((e - 948u) << 23);        // 2^(e - 1075)
  const float lo = __int2float_rn((int)d) * ulp;
  return {hi, __uint_as_float(__float_as_uint(lo) ^ sign)};
}

// hi + lo as a double: the two floats widened on the integer pipe (normal floats; zero
// and others through the hardware conversion), one FP64 addition.
__device__ __forceinline__ double f2d_fast(float v) {
  const unsigned a = __float_as_uint(v), ex = (a >> 23) & 0xFFu;
  if (ex - 1u > 253u) return (double)v;  // zero, subnormal, inf, NaN
  const unsigned long long bits = ((unsigned long long)(a & 0x80000000u) << 32) |
                                  ((unsigned long long)(ex + 896u) << 52) |
                                  ((unsigned long long)(a & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ double df_to_double_fast(df2 a) { return f2d_fast(a.hi) + f2d_fast(a.lo); }

// length-R DFT in registers for the Stockham stages (R = 8, 4, 2)
template <int R> __device__ __forceinline__ void dft_df(dfc* v) {
  if constexpr (R == 8) {
    dfc w[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) w[i] = v[i];
    dft8_df(w);
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = w[i];
  } else if constexpr (R == 4) {
    const dfc t0 = dfc_add(v[0], v[2]), t1 = dfc_sub(v[0], v[2]), t2 = dfc_add(v[1], v[3]);
    const dfc t3 = dfc_mul_mi(dfc_sub(v[1], v[3]));
    v[0] = dfc_add(t0, t2);
    v[2] = dfc_sub(t0, t2);
    v[1] = dfc_add(t1, t3);
    v[3] = dfc_sub(t1, t3);
  } else {
    const dfc a = v[0], b = v[1];
    v[0] = dfc_add(a, b);
    v[1] = dfc_sub(a, b);
  }
}

// One Stockham stage of radix R over N = 2^LOGN values in padded shared memory (index
// sq_pad), NS the product of the earlier radices: the N/R butterflies j go to the N/8
// threads, 8/R each; inputs x[j + r N/R], twiddles w_N^(r k N/(NS R)) with k = j mod NS
// (tw[t] = w_N^t), outputs at (j/NS) NS R + k + r NS.  Reads, barrier, writes, barrier.
template <int LOGN, int R, int NS>
__device__ __forceinline__ void stage_df(float4* buf, int t, const float4* __restrict__ tw) {
  constexpr int N = 1 << LOGN, NT = N / 8, M = 8 / R, NR = N / R;
  dfc v[8];
#pragma unroll
  for (int mm = 0; mm < M; ++mm) {
    const int j = t + mm * NT;
#pragma unroll
    for (int r = 0; r < R; ++r) v[mm * R + r] = dfc_load(buf[sq_pad(j + r * NR)]);
  }
  __syncthreads();
#pragma unroll
  for (int mm = 0; mm < M; ++mm) {
    const int j = t + mm * NT;
    const int k = j & (NS - 1);
    if constexpr (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r)
        v[mm * R + r] = dfc_mul(v[mm * R + r], dfc_load(__ldg(tw + r * k * (N / (NS * R)))));
    }
    dft_df<R>(v + mm * R);
    const int base = (j / NS) * NS * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) buf[sq_pad(base + r * NS)] = dfc_store(v[mm * R + r]);
  }
  __syncthreads();
}

// Forward DFT of N = 2^LOGN padded values by N/8 threads (radix 8, the last stage 4 or 2)
template <int LOGN, int NS = 1>
__device__ __forceinline__ void fft_df(float4* buf, int t, const float4* __restrict__ tw) {
  constexpr int N = 1 << LOGN;
  if constexpr (NS < N) {
    constexpr int R = N / NS >= 8 ? 8 : N / NS;
    stage_df<LOGN, R, NS>(buf, t, tw);
    fft_df<LOGN, NS * R>(buf, t, tw);
  }
}

// k_ff_cols_p2 in double-float: the time factors (FP64, split), the FP64 half spectra
// split on load, the advance a = F t0 + G t1 conjugated into shared memory, the forward
// transform (the inverse of the conjugate), the conjugate of the result to the
// intermediate as double-float pairs (float4).  Block (column, output) of N/8 threads.
template <int LOGNY>
__global__ void __launch_bounds__((1 << LOGNY) / 8)
    k_ff_cols_df(FftArgs fa, int n_f, const double2* __restrict__ spec, float4* __restrict__ out,
                 double c, double tau, double Lx, double Ly, const float4* __restrict__ tw) {
  constexpr int N = 1 << LOGNY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* tab = reinterpret_cast<float4*>(smem_raw);
  float4* buf = tab + N;
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
    tab[ky] = split_df(double2{t0, t1});
  }
  for (int f = 0; f < n_f; ++f) {
    const double2* colF = spec + (size_t)f * N * nxh + kx;
    const double2* colG = spec + (size_t)(n_f + f) * N * nxh + kx;
    __syncthreads();  // the table is ready; the previous function's stores are done
    for (int ky = tid; ky < N; ky += blockDim.x) {
      const dfc t = dfc_load(tab[ky]);  // re: t0, im: t1
      const double2 F = colF[(size_t)ky * nxh], G = colG[(size_t)ky * nxh];
      const df2 fr = split_fast(F.x), fi = split_fast(F.y);
      const df2 gr = split_fast(G.x), gi = split_fast(G.y);
      const df2 ar = df_add(df_mul(fr, t.re), df_mul(gr, t.im));
      const df2 ai = df_add(df_mul(fi, t.re), df_mul(gi, t.im));
      buf[sq_pad(ky)] = dfc_store(dfc{ar, df_neg(ai)});
    }
    __syncthreads();
    fft_df<LOGNY>(buf, tid, tw);
    float4* dst = out + ((size_t)which * n_f + f) * N * fa.pitch + kx;
    for (int y = tid; y < N; y += blockDim.x) {
      const dfc r = dfc_load(buf[sq_pad(y)]);
      dst[(size_t)y * fa.pitch] = dfc_store(dfc{r.re, df_neg(r.im)});
    }
  }
}

// k_inverse_rows_p2 in double-float (no quadratic term): Z_k = S_k + i conj(w^k) D_k from
// X_k and conj(X_{NH-k}) (double-float intermediate rows), the forward transform of
// conj(Z), x_{2m} + i x_{2m+1} = conj of its result, written as doubles.
template <int LOGNH>
__global__ void __launch_bounds__((1 << LOGNH) / 8)
    k_inverse_rows_df(FftArgs fa, const float4* __restrict__ inter, double* __restrict__ up,
                      const float4* __restrict__ rtw, const float4* __restrict__ tw) {
  constexpr int NH = 1 << LOGNH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* buf = reinterpret_cast<float4*>(smem_raw);
  const int j = blockIdx.x, f = blockIdx.y, t = threadIdx.x;
  const float4* row = inter + ((size_t)f * fa.ny + j) * fa.pitch;
  for (int k = t; k < NH; k += blockDim.x) {
    const dfc bk = dfc_load(row[k]);
    dfc bc = dfc_load(row[NH - k]);
    bc.im = df_neg(bc.im);  // conj X_{NH-k}
    const dfc sm = dfc_add(bk, bc), d = dfc_sub(bk, bc);
    dfc w = dfc_load(__ldg(rtw + k));
    w.im = df_neg(w.im);    // conj(w^k)
    const dfc dw = dfc_mul(d, w);
    buf[sq_pad(k)] = dfc_store(dfc{df_sub(sm.re, dw.im), df_neg(df_add(sm.im, dw.re))});
  }
  __syncthreads();
  fft_df<LOGNH>(buf, t, tw);
  double* o = up + ((size_t)f * fa.ny + j) * (2 * NH);
  for (int m = t; m < NH; m += blockDim.x) {
    const dfc z = dfc_load(buf[sq_pad(m)]);
    o[2 * m] = df_to_double_fast(z.re);
    o[2 * m + 1] = -df_to_double_fast(z.im);
  }
}

// The U_FC evaluation at tau in double-float for power-of-two grids (ny = 2^9..2^12,
// nx = 2^9..2^12); false (nothing launched) otherwise.
template <int LOGNY>
static void ff_cols_df_launch(const FftArgs& fa, int n_f, int n_out, const double2* spec,
                              float4* out, double c, double tau, double Lx, double Ly,
                              const float4* tw, cudaStream_t s) {
  const size_t sm = ((size_t)(1 << LOGNY) + (1 << LOGNY) + (1 << LOGNY) / 8) * sizeof(float4);
  cudaFuncSetAttribute(k_ff_cols_df<LOGNY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_ff_cols_df<LOGNY><<<dim3(fa.nx / 2 + 1, n_out), (1 << LOGNY) / 8, sm, s>>>(
      fa, n_f, spec, out, c, tau, Lx, Ly, tw);
}
template <int LOGNH>
static void inverse_rows_df_launch(const FftArgs& fa, int n_f, const float4* inter, double* up,
                                   const float4* rtw, const float4* tw, cudaStream_t s) {
  const size_t sm = ((size_t)(1 << LOGNH) + (1 << LOGNH) / 8) * sizeof(float4);
  cudaFuncSetAttribute(k_inverse_rows_df<LOGNH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_inverse_rows_df<LOGNH><<<dim3(fa.ny, n_f), (1 << LOGNH) / 8, sm, s>>>(fa, inter, up, rtw, tw);
}
bool df_sizes_ok(int nx, int ny) {
  auto p2 = [](int v, int lo, int hi) {
    for (int l = lo; l <= hi; ++l)
      if (v == (1 << l)) return true;
    return false;
  };
  return p2(ny, 9, 12) && p2(nx / 2, 8, 11) && nx % 2 == 0;
}
bool ff_cols_df(const FftArgs& fa, int n_f, int n_out, const double2* spec, float4* out, double c,
                double tau, double Lx, double Ly, const float4* tw, cudaStream_t s) {
  switch (fa.ny) {
    case 512: ff_cols_df_launch<9>(fa, n_f, n_out, spec, out, c, tau, Lx, Ly, tw, s); return true;
    case 1024: ff_cols_df_launch<10>(fa, n_f, n_out, spec, out, c, tau, Lx, Ly, tw, s); return true;
    case 2048: ff_cols_df_launch<11>(fa, n_f, n_out, spec, out, c, tau, Lx, Ly, tw, s); return true;
    case 4096: ff_cols_df_launch<12>(fa, n_f, n_out, spec, out, c, tau, Lx, Ly, tw, s); return true;
    default: return false;
  }
}
bool inverse_rows_df(const FftArgs& fa, int n_f, const float4* inter, double* up, const float4* rtw,
                     const float4* tw, cudaStream_t s) {
  switch (fa.nx / 2) {
    case 256: inverse_rows_df_launch<8>(fa, n_f, inter, up, rtw, tw, s); return true;
    case 512: inverse_rows_df_launch<9>(fa, n_f, inter, up, rtw, tw, s); return true;
    case 1024: inverse_rows_df_launch<10>(fa, n_f, inter, up, rtw, tw, s); return true;
    case 2048: inverse_rows_df_launch<11>(fa, n_f, inter, up, rtw, tw, s); return true;
    default: return false;
  }
}

// The box's time factors for the small steps s = 0..S-1: tab[s][l][m] =
// (cos w tau, sin(w tau)/w) at tau = s dt ((1, tau) at w = 0), w = 2 pi c |k| / (P h).
template <bool DF>
__global__ void k_sq_table(int P, int S, double c, double h, double dt, double2* __restrict__ tab) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)S * P * P) return;
  const int s = (int)(t / (P * P)), lm = (int)(t - (int64_t)s * P * P);
  const int l = lm / P, m = lm - l * P;
  const int ls = l <= P / 2 ? l : l - P, ms = m <= P / 2 ? m : m - P;
  const double L = P * h, tau = s * dt;
  const double fl = ls / L, fm = ms / L;
  const double w = 6.283185307179586476925286766559 * c * sqrt(fl * fl + fm * fm);
  double2 v;
  if (w == 0.0) {
    v = double2{1.0, tau};
  } else {
    double sn, co;
    sincos(w * tau, &sn, &co);
    v = double2{co, sn / w};
  }
  if constexpr (DF) reinterpret_cast<float4*>(tab)[t] = split_df(v);
  else tab[t] = v;
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
    if (b.sq) {
      DevSquares& q = *b.sq;
      for (void* ptr : {(void*)q.origin, (void*)q.served_off, (void*)q.served_lin,
                        (void*)q.served_local, (void*)q.A, (void*)q.Q, (void*)q.tw, (void*)q.tw_df,
                        (void*)q.rows})
        cudaFree(ptr);
    }
  }
  cudaFree(W->scr.base);
  cudaFree(W->df_twy);
  cudaFree(W->df_twx);
  cudaFree(W->df_rtw);
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

extern "C" fc2d_status fc2d_wave_band_info(fc2d_plan_t p, int n_c, int interface_mode,
                                           int64_t* counts) {
  fc2d_status st = wave_checks(p, n_c, "fc2d_wave_band_info");
  if (st) return st;
  if (!counts) return set_error(FC2D_ERR_ARG, "fc2d_wave_band_info: null argument");
  if (interface_mode < 0 || interface_mode > 1)
    return set_error(FC2D_ERR_ARG, "fc2d_wave_band_info: interface_mode 0 or 1");
  cudaSetDevice(p->device);
  DevBand* b;
  if ((st = get_band(p, n_c, interface_mode, &b))) return st;
  counts[0] = (int64_t)b->host.unknown_lin.size();
  counts[1] = (int64_t)b->host.slaved_lin.size();
  counts[2] = (int64_t)b->host.iface_lin.size();
  counts[3] = (int64_t)b->host.near_lin.size();
  counts[4] = b->sq ? (int64_t)b->sq->n : 0;
  return FC2D_OK;
}

extern "C" fc2d_status fc2d_wave_band_points(fc2d_plan_t p, int n_c, int interface_mode,
                                             int32_t* unknown_lin,
                                             int32_t* slaved_lin, int32_t* iface_lin,
                                             int32_t* near_lin) {
  fc2d_status st = wave_checks(p, n_c, "fc2d_wave_band_points");
  if (st) return st;
  if (interface_mode < 0 || interface_mode > 1)
    return set_error(FC2D_ERR_ARG, "fc2d_wave_band_points: interface_mode 0 or 1");
  cudaSetDevice(p->device);
  DevBand* b;
  if ((st = get_band(p, n_c, interface_mode, &b))) return st;
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
  if ((st = get_band(p, n_c, 0, &b))) return st;
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
                                         int interface_mode, double* u, double* ut,
                                         const double* g_dir, const double* gt_dir,
                                         void* stream) {
  fc2d_status st = wave_checks(p, n_c, "fc2d_forward_wave");
  if (st) return st;
  if ((st = check_nf(p, n_f))) return st;
  if (!u || !ut) return set_error(FC2D_ERR_ARG, "fc2d_forward_wave: null pointer");
  if (!(c > 0) || n_large < 0)
    return set_error(FC2D_ERR_ARG, "fc2d_forward_wave: c > 0 and n_large >= 0 required");
  if (interface_mode < 0 || interface_mode > 2)
    return set_error(FC2D_ERR_ARG, "fc2d_forward_wave: interface_mode 0, 1 or 2");
  if (3 * (size_t)p->grid.ny * sizeof(double2) > 227 * 1024)
    return set_error(FC2D_ERR_UNSUPPORTED, "fc2d_forward_wave: ny <= 4842");
  if (n_large == 0) return FC2D_OK;
  cudaSetDevice(p->device);
  cudaStream_t s = (cudaStream_t)stream;
  DevBand* b;
  // mode 2: the squares of mode 1, evaluated in double-float arithmetic
  const bool df = interface_mode == 2;
  if ((st = get_band(p, n_c, interface_mode ? 1 : 0, &b))) return st;
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
  const DevSquares* sq = b->sq.get();
  const int P = sq ? sq->host.P : 0, n_sq = sq ? sq->n : 0;
  const size_t b_sqz = al((size_t)n_sq * n_f * P * P * 16), b_sqt = al((size_t)S * P * P * 16);
  const size_t need = b_spec + b_inter + 2 * b_grid + 4 * b_ub + b_zero + b_sqz + b_sqt;
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
  double2* sqZ = reinterpret_cast<double2*>(base + b_spec + b_inter + 2 * b_grid + 4 * b_ub + b_zero);
  double2* sqT = reinterpret_cast<double2*>(base + b_spec + b_inter + 2 * b_grid + 4 * b_ub + b_zero + b_sqz);
  cudaMemsetAsync(zero, 0, (size_t)n_f * nb * 8, s);
  const size_t sm_sq = kSqForwardSmem;
  int max_rows = 0;
  if (sq)
    for (int k = 0; k < n_sq; ++k) {
      int lo = P, hi = -1;
      for (int i = sq->host.served_off[k]; i < sq->host.served_off[k + 1]; ++i) {
        lo = std::min(lo, sq->host.served_local[i] / P);
        hi = std::max(hi, sq->host.served_local[i] / P);
      }
      max_rows = std::max(max_rows, hi - lo + 1);
    }
  const size_t sm_ev = (size_t)(P + max_rows) * kSqPad * sizeof(double2);
  if (sq) {
    cudaFuncSetAttribute(k_sq_forward<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_sq);
    cudaFuncSetAttribute(k_sq_forward<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_sq);
    cudaFuncSetAttribute(k_sq_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_ev);
    cudaFuncSetAttribute(k_sq_eval_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_ev);
    if (df) k_sq_table<true><<<blocks((int64_t)S * P * P, 256), 256, 0, s>>>(P, S, c, h, dt, sqT);
    else k_sq_table<false><<<blocks((int64_t)S * P * P, 256), 256, 0, s>>>(P, S, c, h, dt, sqT);
  }
  auto gat = [&](int64_t m) { return g_dir ? g_dir + (size_t)m * n_f * nb : nullptr; };
  auto gtat = [&](int64_t j) { return gt_dir ? gt_dir + (size_t)j * n_f * nb : nullptr; };
  FftArgs fa = fft_args(p);
  const double Lx = nx * h, Ly = ny * h;
  const size_t smc = 3 * (size_t)ny * sizeof(double2);
  cudaFuncSetAttribute(k_ff_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc);
  // interface mode 2 on power-of-two grids: U_FC at T_{j+1} in double-float too
  const bool df_ufc = df && df_sizes_ok(nx, ny);
  if (df_ufc && (st = df_tables(p, W))) return st;
  auto eval_ufc_df = [&](double tau, double* out_u, double* out_ut) {
    float4* interf = reinterpret_cast<float4*>(inter);
    {
      ProfScope ps(p, "ff_cols", s);
      ff_cols_df(fa, n_f, 2, spec, interf, c, tau, Lx, Ly, W->df_twy, s);
    }
    ProfScope ps(p, "inverse_rows", s);
    inverse_rows_df(fa, n_f, interf, out_u, W->df_rtw, W->df_twx, s);
    inverse_rows_df(fa, n_f, interf + (size_t)n_f * ny * pitch, out_ut, W->df_rtw, W->df_twx, s);
  };
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
    if (sq) {  // the squares' expansions of u(T_j), u_t(T_j), before u and ut change
      ProfScope ps(p, "sq_forward", s);
      const SquareSet& H = sq->host;
      auto kf = df ? k_sq_forward<true> : k_sq_forward<false>;
      kf<<<dim3(n_sq, n_f), kSqThreads, sm_sq, s>>>(2 * H.a + 1, H.C, H.d, nx, NN, n_f,
                                                     sq->origin, sq->A, sq->Q, sq->tw, u, ut, sqZ);
    }
    if ((st = wave_spectra(p, n_f, u, g_dir ? gat(m0) : zero, ut, gt_dir ? gtat(j) : zero, spec, s)))
      return st;
    for (int sidx = 0; sidx < S; ++sidx) {
      const int64_t m = m0 + sidx;
      if (sq) {
        ProfScope ps(p, "sq_eval", s);
        if (df)
          k_sq_eval_df<<<dim3(n_sq, (n_f + 1) / 2), kSqEvalThreads, sm_ev, s>>>(
              n_f, reinterpret_cast<const float4*>(sqZ),
              reinterpret_cast<const float4*>(sqT) + (size_t)sidx * P * P, sq->tw_df,
              sq->served_off, sq->served_lin, sq->served_local, sq->rows, NN, ufc[f_cur]);
        else
          k_sq_eval<<<dim3(n_sq, (n_f + 1) / 2), kSqEvalThreads, sm_ev, s>>>(
              n_f, sqZ, sqT + (size_t)sidx * P * P, sq->tw, sq->served_off, sq->served_lin,
              sq->served_local, sq->rows, NN, ufc[f_cur]);
      } else {
        eval_ufc(sidx * dt, 1, ufc[f_cur], nullptr);
      }
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
    if (df_ufc) eval_ufc_df(dT, u, ut);
    else eval_ufc(dT, 2, u, ut);
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
