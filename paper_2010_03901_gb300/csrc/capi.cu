// C-ABI entry points that launch the 2D-FC kernels (declared in include/fc2d.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fc2d_kernels.cuh"
#include "plan_internal.h"

using namespace fc2d;

namespace fc2d {

fc2d_status ensure_workspace(fc2d_plan_s* p, size_t bytes) {
  if (p->ws.bytes >= bytes) return FC2D_OK;
  if (p->ws.base) {
    cudaDeviceSynchronize();
    cudaFree(p->ws.base);
    p->ws.base = nullptr;
    p->ws.bytes = 0;
  }
  if (cudaMalloc(&p->ws.base, bytes) != cudaSuccess)
    return set_error(FC2D_ERR_NOMEM, "workspace cudaMalloc failed");
  p->ws.bytes = bytes;
  return FC2D_OK;
}

}  // namespace fc2d

namespace {

size_t al(size_t b) { return (b + 255) / 256 * 256; }

struct Layout {
  size_t F, vals, inter, coef, bvals, total;
  size_t oF, ovals, ointer, ocoef, obvals;
};

// Row length of the strip values F in workspace: Cr + 1 for FP64; for the mixed form
// a multiple of 4 floats with room for the interpolation's aligned float4 windows.
int ws_ldF(const fc2d_plan_s* p) {
  return p->prm.precision == FC2D_MIXED ? (p->Cr + 12 + 3) / 4 * 4 : p->Cr + 1;
}

Layout layout(const fc2d_plan_s* p, int n_f) {
  Layout L{};
  const size_t esz = p->prm.precision == FC2D_MIXED ? 4 : 8;
  const size_t pitch = row_pitch(p);
  L.F = al((size_t)n_f * p->prm.B * ws_ldF(p) * esz);
  L.vals = al((size_t)n_f * std::max<size_t>(1, p->strip_lin.size()) * esz);
  L.inter = al((size_t)n_f * p->grid.ny * pitch * 2 * esz);
  L.coef = al((size_t)n_f * p->prm.B * kMaxD * 8);
  L.bvals = al((size_t)n_f * p->prm.B * 8);
  L.oF = 0;
  L.ovals = L.oF + L.F;
  L.ointer = L.ovals + L.vals;
  L.ocoef = L.ointer + L.inter;
  L.obvals = L.ocoef + L.coef;
  L.total = L.obvals + L.bvals;
  return L;
}

char* ws(fc2d_plan_s* p, size_t off) { return static_cast<char*>(p->ws.base) + off; }

// compact: f given at the inside points only ([n_f][n_inside], row by row)
GatherArgs gather_args(fc2d_plan_s* p, const double* fg, const double* fb, void* F,
                       double* coef, double* bvals, bool compact = false) {
  GatherArgs a{};
  a.B = p->prm.B;
  a.M = p->prm.M;
  a.d = p->prm.d;
  a.Cr = p->Cr;
  a.n_bdry = p->n_bdry;
  a.grid_stride = compact ? p->n_inside : (int64_t)p->grid.nx * p->grid.ny;
  a.f_grid = fg;
  a.f_bdry = fb;
  if (fb) {
    a.nq = p->prm.d - 1;
    a.gidx = compact ? p->dev.gidx_c : p->dev.gidx;
    a.gw = p->dev.gw;
    a.wn = p->dev.wn;
  } else {  // interior data only (Remark 3.2 II)
    a.nq = p->prm.d;
    a.gidx = compact ? p->dev.gidx_ic : p->dev.gidx_i;
    a.gw = p->dev.gw_i;
    a.wn = p->dev.wn_i;
  }
  a.Q = p->dev.Q;
  a.Ar = p->dev.Ar;
  a.F = F;
  a.coef = coef;
  a.coef_ld = kMaxD;
  a.bvals = bvals;
  return a;
}

InterpArgs interp_args(fc2d_plan_s* p, int ldF) {
  InterpArgs a{};
  a.n_strip = (int)p->strip_lin.size();
  a.M = p->prm.M;
  a.B = p->prm.B;
  a.Cr = p->Cr;
  a.ldF = ldF;
  a.w = p->dev.s_w;
  a.pb = p->dev.s_pb;
  a.sb = p->dev.s_sb;
  return a;
}

}  // namespace

// Argument blocks shared with the allocation-free entry point (static_scratch.cu).
namespace fc2d {

RowArgs row_args(fc2d_plan_s* p, bool compact) {
  RowArgs a{};
  a.nx = p->grid.nx;
  a.ny = p->grid.ny;
  a.grid_stride = compact ? p->n_inside : (int64_t)p->grid.nx * p->grid.ny;
  a.row_iv_coff = p->dev.row_iv_coff;
  a.n_strip = (int64_t)p->strip_lin.size();
  a.row_iv_off = p->dev.row_iv_off;
  a.row_iv = p->dev.row_iv;
  a.row_strip_off = p->dev.row_strip_off;
  a.s_lin = p->dev.s_lin;
  return a;
}

FftArgs fft_args(fc2d_plan_s* p) {
  FftArgs a{};
  const bool f64 = p->prm.precision == FC2D_FP64;
  a.nx = p->grid.nx;
  a.ny = p->grid.ny;
  a.pitch = (int)row_pitch(p);
  a.nrx = p->fx.n_radix;
  a.nry = p->fy.n_radix;
  for (int i = 0; i < a.nrx; ++i) a.rx[i] = p->fx.radix[i];
  for (int i = 0; i < a.nry; ++i) a.ry[i] = p->fy.radix[i];
  a.twx = f64 ? (const void*)p->fx.tw64 : (const void*)p->fx.tw32;
  a.twy = f64 ? (const void*)p->fy.tw64 : (const void*)p->fy.tw32;
  a.rtw = f64 ? (const void*)p->rtw64 : (const void*)p->rtw32;
  a.tsx = f64 ? (const void*)p->fx.tws64 : (const void*)p->fx.tws32;
  a.tsy = f64 ? (const void*)p->fy.tws64 : (const void*)p->fy.tws32;
  a.scale = 1.0 / ((double)p->grid.nx * p->grid.ny);
  a.cc4k = p->tune_cc4k;
  a.cols_tma = p->tune_tma;
  a.status = p->dev.status;
  return a;
}

fc2d_status check_nf(fc2d_plan_s* p, int n_f) {
  if (!p) return set_error(FC2D_ERR_ARG, "null plan");
  if (n_f < 1) return set_error(FC2D_ERR_ARG, "n_f must be >= 1");
  if ((int64_t)n_f * p->grid.nx * p->grid.ny > INT64_C(1) << 40)
    return set_error(FC2D_ERR_ARG, "n_f too large");
  return FC2D_OK;
}

}  // namespace fc2d

namespace {

fc2d_status launched(const char* what) { return cuda_check(cudaGetLastError(), what); }

// Mixed form of step 5: matching values and Gram coefficients in FP64, then the
// contraction with A_r on the tensor cores into float strip values F.
fc2d_status mixed_blend(fc2d_plan_s* p, int n_f, const double* fg, const double* fb, void* F,
                        int ldF, const Layout& L, cudaStream_t s, bool compact = false) {
  if (p->prm.M - 1 <= 8 && p->prm.d <= 8) {
    ProfScope ps(p, "gather_blend_tc", s);
    return launch_gather_blend_tc(gather_args(p, fg, fb, nullptr, nullptr, nullptr, compact), n_f,
                                  ldF, p->dev.Ar_hi, p->dev.Ar_lo, static_cast<float*>(F),
                                  p->dev.status, s);
  }
  double* coef = reinterpret_cast<double*>(ws(p, L.ocoef));
  double* bvals = reinterpret_cast<double*>(ws(p, L.obvals));
  {
    ProfScope ps(p, "gather_coef", s);
    launch_gather_blend(gather_args(p, fg, fb, nullptr, coef, bvals, compact), n_f, false, s);
  }
  ProfScope ps(p, "blend_tc", s);
  return launch_blend_tc(n_f * p->prm.B, p->Cr, p->prm.d, ldF, coef, kMaxD, bvals,
                         p->dev.Ar_hi, p->dev.Ar_lo, static_cast<float*>(F), p->dev.status, s);
}

// The fused blend + interpolation call (mixed form, M = 8) for n_f functions: one
// function on CTAs of 512 threads, one per SM (own[0]); several on CTAs of 256 threads,
// two per SM, one function each, over the balanced ranges while the call's CTAs fit in
// about one wave, else over the fewest CTAs (own[1]).
GiPlanArgs gi_call(fc2d_plan_s* p, int n_f, const double* fg, const double* fb,
                   const Layout& L, bool compact, int* nt, const DeviceTables::Owners** own) {
  const auto& o = (n_f > 1 && p->dev.own[1].n && n_f * (int64_t)p->dev.own[0].n > 3 * (int64_t)p->n_sm)
                      ? p->dev.own[1]
                      : p->dev.own[0];
  GiPlanArgs a{};
  a.g = gather_args(p, fg, fb, nullptr, nullptr, nullptr, compact);
  a.n_f = n_f;
  a.ldS = ws_ldF(p);
  a.Ar_hi = p->dev.Ar_hi;
  a.Ar_lo = p->dev.Ar_lo;
  a.own_off = o.off;
  a.own_k = o.k;
  a.own_pack = o.pack;
  a.own_start = o.start;
  a.own_w = o.w;
  a.n_own = o.n;
  a.n_strip = (int)p->strip_lin.size();
  a.vals = reinterpret_cast<float*>(ws(p, L.ovals));
  a.status = p->dev.status;
  *nt = n_f == 1 ? 512 : 256;
  if (own) *own = &o;
  return a;
}

// Steps 5 and 6 into workspace: strip values F, then the strip-point values.
fc2d_status strip_values(fc2d_plan_s* p, int n_f, const double* fg, const double* fb,
                         const Layout& L, cudaStream_t s, bool compact = false) {
  const bool f64 = p->prm.precision == FC2D_FP64;
  void* F = ws(p, L.oF);
  if (!f64 && p->dev.own[0].off) {
    // mixed form, M = 8: blend and interpolation in one kernel, F stays on chip
    int nt = 0;
    const GiPlanArgs a = gi_call(p, n_f, fg, fb, L, compact, &nt, nullptr);
    ProfScope ps(p, "gather_blend_interp_tc", s);
    return launch_gather_interp_tc(a, nt, s);
  }
  if (f64) {
    ProfScope ps(p, "gather_blend", s);
    launch_gather_blend(gather_args(p, fg, fb, F, nullptr, nullptr, compact), n_f, true, s);
  } else {
    fc2d_status st = mixed_blend(p, n_f, fg, fb, F, ws_ldF(p), L, s, compact);
    if (st) return st;
  }
  {
    ProfScope ps(p, "interp", s);
    launch_interp(interp_args(p, ws_ldF(p)), n_f, f64, F, ws(p, L.ovals), s);
  }
  return launched("strip values");
}

}  // namespace

// fb == null selects the interior-data-only stencils; they exist unless a red star's
// chord held no grid node
static fc2d_status check_interior(fc2d_plan_t p, const double* fb, const char* who) {
  if (!fb && !p->interior_ok)
    return set_error(FC2D_ERR_UNSUPPORTED, std::string(who) +
                                               ": no interior-only stencils (a red star's chord "
                                               "holds no grid node); pass boundary values");
  return FC2D_OK;
}

namespace fc2d {
// the plan workspace for an n_f-function call (plan groups allocate it before capturing)
fc2d_status ensure_plan_workspace(fc2d_plan_s* p, int n_f) {
  fc2d_status st = check_nf(p, n_f);
  if (st) return st;
  cudaSetDevice(p->device);
  return ensure_workspace(p, layout(p, n_f).total);
}
}  // namespace fc2d

extern "C" fc2d_status fc2d_blend(fc2d_plan_t p, int n_f, const double* fg, const double* fb,
                                  void* F, void* stream) {
  fc2d_status st = check_nf(p, n_f);
  if (st) return st;
  if (!fg || !F) return set_error(FC2D_ERR_ARG, "fc2d_blend: null pointer");
  if ((st = check_interior(p, fb, "fc2d_blend"))) return st;
  cudaSetDevice(p->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (p->prm.precision == FC2D_FP64) {
    launch_gather_blend(gather_args(p, fg, fb, F, nullptr, nullptr), n_f, true, s);
    return launched("fc2d_blend");
  }
  Layout L = layout(p, n_f);
  if ((st = ensure_workspace(p, L.total))) return st;
  if ((st = mixed_blend(p, n_f, fg, fb, F, p->Cr + 1, L, s))) return st;
  return launched("fc2d_blend");
}

extern "C" fc2d_status fc2d_interp(fc2d_plan_t p, int n_f, const void* F, void* vals,
                                   void* stream) {
  fc2d_status st = check_nf(p, n_f);
  if (st) return st;
  if (!F || !vals) return set_error(FC2D_ERR_ARG, "fc2d_interp: null pointer");
  cudaSetDevice(p->device);
  launch_interp(interp_args(p, p->Cr + 1), n_f, p->prm.precision == FC2D_FP64, F, vals,
                (cudaStream_t)stream);
  return launched("fc2d_interp");
}

extern "C" fc2d_status fc2d_extend(fc2d_plan_t p, int n_f, const double* fg, const double* fb,
                                   void* ext, void* stream) {
  fc2d_status st = check_nf(p, n_f);
  if (st) return st;
  if (!fg || !ext) return set_error(FC2D_ERR_ARG, "fc2d_extend: null pointer");
  if ((st = check_interior(p, fb, "fc2d_extend"))) return st;
  cudaSetDevice(p->device);
  Layout L = layout(p, n_f);
  if ((st = ensure_workspace(p, L.total))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = strip_values(p, n_f, fg, fb, L, s))) return st;
  {
    ProfScope ps(p, "assemble_rows", s);
    launch_assemble(row_args(p), n_f, p->prm.precision == FC2D_FP64, fg, ws(p, L.ovals), ext, s);
  }
  return launched("fc2d_extend");
}

extern "C" fc2d_status fc2d_coeffs(fc2d_plan_t p, int n_f, const void* ext, void* fhat,
                                   void* stream) {
  fc2d_status st = check_nf(p, n_f);
  if (st) return st;
  if (!ext || !fhat) return set_error(FC2D_ERR_ARG, "fc2d_coeffs: null pointer");
  cudaSetDevice(p->device);
  Layout L = layout(p, n_f);
  if ((st = ensure_workspace(p, L.total))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const bool f64 = p->prm.precision == FC2D_FP64;
  FftArgs fa = fft_args(p);
  {
    ProfScope ps(p, "fft_rows", s);
    launch_fft_rows(fa, row_args(p), n_f, f64, 0, ext, nullptr, nullptr, ws(p, L.ointer), s);
  }
  {
    ProfScope ps(p, "fft_cols", s);
    launch_fft_cols(fa, n_f, f64, ws(p, L.ointer), fhat, s);
  }
  return launched("fc2d_coeffs");
}

namespace fc2d {

// The argument checks of fc2d_extend_coeffs.
fc2d_status extend_coeffs_check(fc2d_plan_s* p, int n_f, const double* fg, const double* fb,
                                const void* fhat) {
  fc2d_status st = check_nf(p, n_f);
  if (st) return st;
  if (!fg || !fhat) return set_error(FC2D_ERR_ARG, "fc2d_extend_coeffs: null pointer");
  return check_interior(p, fb, "fc2d_extend_coeffs");
}

// Steps 6-7 of fc2d_extend_coeffs after the strip-point values are in the workspace:
// the fused row DFT (f and the strip values) and the column DFT.
fc2d_status extend_coeffs_dft(fc2d_plan_s* p, int n_f, const double* fg, void* fhat,
                              cudaStream_t s) {
  const bool f64 = p->prm.precision == FC2D_FP64;
  const Layout L = layout(p, n_f);
  FftArgs fa = fft_args(p);
  {
    ProfScope ps(p, "fft_rows_fused", s);
    launch_fft_rows(fa, row_args(p), n_f, f64, 1, nullptr, fg, ws(p, L.ovals),
                    ws(p, L.ointer), s);
  }
  {
    ProfScope ps(p, "fft_cols", s);
    launch_fft_cols(fa, n_f, f64, ws(p, L.ointer), fhat, s);
  }
  return launched("fc2d_extend_coeffs");
}

// A group member whose strip values the group's persistent kernel computes: mixed form
// with the fused kernel's tables.  Its call description and each range's strip-point
// count (the cost of a work item).
bool group_fused(const fc2d_plan_s* p) {
  return p->prm.precision == FC2D_MIXED && p->dev.own[0].off;
}
GiPlanArgs group_fused_args(fc2d_plan_s* p, int n_f, const double* fg, const double* fb,
                            std::vector<int32_t>* points) {
  int nt = 0;
  const DeviceTables::Owners* o = nullptr;
  const GiPlanArgs a = gi_call(p, n_f, fg, fb, layout(p, n_f), false, &nt, &o);
  points->resize(o->n);
  for (int c = 0; c < o->n; ++c) (*points)[c] = o->off_host[c + 1] - o->off_host[c];
  return a;
}

}  // namespace fc2d

extern "C" fc2d_status fc2d_extend_coeffs(fc2d_plan_t p, int n_f, const double* fg,
                                          const double* fb, void* fhat, void* stream) {
  fc2d_status st = extend_coeffs_check(p, n_f, fg, fb, fhat);
  if (st) return st;
  cudaSetDevice(p->device);
  Layout L = layout(p, n_f);
  if ((st = ensure_workspace(p, L.total))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = strip_values(p, n_f, fg, fb, L, s))) return st;
  return extend_coeffs_dft(p, n_f, fg, fhat, s);
}

extern "C" fc2d_status fc2d_extend_coeffs_complex(fc2d_plan_t p, int n_f, const double* fg,
                                                  const double* fb, void* fhat, void* stream) {
  fc2d_status st = check_nf(p, n_f);
  if (st) return st;
  if (n_f > (1 << 29)) return set_error(FC2D_ERR_ARG, "fc2d_extend_coeffs_complex: n_f too large");
  if (!fg || !fhat) return set_error(FC2D_ERR_ARG, "fc2d_extend_coeffs_complex: null pointer");
  if ((st = check_interior(p, fb, "fc2d_extend_coeffs_complex"))) return st;
  cudaSetDevice(p->device);
  const int n2 = 2 * n_f;  // the real and imaginary parts as functions 2f and 2f + 1
  Layout L = layout(p, n2);
  const bool f64 = p->prm.precision == FC2D_FP64;
  const size_t esz = f64 ? 8 : 4;
  const size_t ohalf = L.total;
  const size_t half = al((size_t)n2 * p->grid.ny * (p->grid.nx / 2 + 1) * 2 * esz);
  if ((st = ensure_workspace(p, ohalf + half))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  FftArgs fa = fft_args(p);
  if ((st = strip_values(p, n2, fg, fb, L, s))) return st;
  {
    ProfScope ps(p, "fft_rows_fused", s);
    launch_fft_rows(fa, row_args(p), n2, f64, 1, nullptr, fg, ws(p, L.ovals), ws(p, L.ointer),
                    s);
  }
  {
    ProfScope ps(p, "fft_cols", s);
    launch_fft_cols(fa, n2, f64, ws(p, L.ointer), ws(p, ohalf), s);
  }
  {
    ProfScope ps(p, "complex_spectrum", s);
    launch_complex_spectrum(p->grid.nx, p->grid.ny, n_f, f64, ws(p, ohalf), fhat, s);
  }
  return launched("fc2d_extend_coeffs_complex");
}

extern "C" fc2d_status fc2d_inside_points(fc2d_plan_t p, int64_t* lin_host) {
  if (!p || !lin_host) return set_error(FC2D_ERR_ARG, "fc2d_inside_points: null argument");
  const int nx = p->grid.nx, ny = p->grid.ny;
  int64_t n = 0;
  for (int j = 0; j < ny; ++j)
    for (int k = p->row_iv_off[j]; k < p->row_iv_off[j + 1]; ++k)
      for (int i = p->row_iv[2 * k]; i <= p->row_iv[2 * k + 1]; ++i) lin_host[n++] = (int64_t)j * nx + i;
  return FC2D_OK;
}

extern "C" fc2d_status fc2d_extend_coeffs_compact(fc2d_plan_t p, int n_f, const double* f_inside,
                                                  const double* fb, void* fhat, void* stream) {
  fc2d_status st = check_nf(p, n_f);
  if (st) return st;
  if (!f_inside || !fhat)
    return set_error(FC2D_ERR_ARG, "fc2d_extend_coeffs_compact: null pointer");
  if ((st = check_interior(p, fb, "fc2d_extend_coeffs_compact"))) return st;
  if (!p->dev.row_iv_coff || !p->dev.gidx_c)
    return set_error(FC2D_ERR_UNSUPPORTED,
                     "fc2d_extend_coeffs_compact: more than 2^31 - 1 inside points");
  cudaSetDevice(p->device);
  Layout L = layout(p, n_f);
  if ((st = ensure_workspace(p, L.total))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const bool f64 = p->prm.precision == FC2D_FP64;
  FftArgs fa = fft_args(p);
  if ((st = strip_values(p, n_f, f_inside, fb, L, s, true))) return st;
  {
    ProfScope ps(p, "fft_rows_fused", s);
    launch_fft_rows(fa, row_args(p, true), n_f, f64, 2, nullptr, f_inside, ws(p, L.ovals),
                    ws(p, L.ointer), s);
  }
  {
    ProfScope ps(p, "fft_cols", s);
    launch_fft_cols(fa, n_f, f64, ws(p, L.ointer), fhat, s);
  }
  return launched("fc2d_extend_coeffs_compact");
}

extern "C" fc2d_status fc2d_sync_status(fc2d_plan_t p, void* stream) {
  if (!p) return set_error(FC2D_ERR_ARG, "null plan");
  cudaSetDevice(p->device);
  fc2d_status st = cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "stream sync");
  if (st) return st;
  int h = 0;
  st = cuda_check(cudaMemcpy(&h, p->dev.status, sizeof(int), cudaMemcpyDeviceToHost),
                  "status read");
  if (st) return st;
  if (!h) return FC2D_OK;
  // report once: clear the word, so that the plan's next calls start from FC2D_OK
  st = cuda_check(cudaMemset(p->dev.status, 0, sizeof(int)), "status clear");
  if (st) return st;
  return set_error((fc2d_status)h, "device status latched");
}

extern "C" fc2d_status fc2d_wait_selftest(fc2d_plan_t p, uint32_t polls, void* stream) {
  if (!p) return set_error(FC2D_ERR_ARG, "null plan");
  if (polls < 1 || polls > (1u << 22)) return set_error(FC2D_ERR_ARG, "polls must be in 1 .. 2^22");
  cudaSetDevice(p->device);
  return fc2d::launch_wait_probe(p->dev.status, polls, (cudaStream_t)stream);
}

// ------------------------------------------------------------------------- //
// Kernel timing
// ------------------------------------------------------------------------- //
namespace fc2d {

static void* take_event(fc2d_plan_s* p) {
  if (!p->event_pool.empty()) {
    void* e = p->event_pool.back();
    p->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return (void*)e;
}

ProfScope::ProfScope(fc2d_plan_s* p_, const char* name_, void* stream_)
    : p(p_), name(name_), stream(stream_) {
  if (!p->profiling) return;
  ev0 = take_event(p);
  cudaEventRecord((cudaEvent_t)ev0, (cudaStream_t)stream);
}

ProfScope::~ProfScope() {
  if (!p->profiling || !ev0) return;
  void* ev1 = take_event(p);
  cudaEventRecord((cudaEvent_t)ev1, (cudaStream_t)stream);
  p->prof.push_back({name, ev0, ev1});
}

}  // namespace fc2d

extern "C" fc2d_status fc2d_profile(fc2d_plan_t p, int enable) {
  if (!p) return set_error(FC2D_ERR_ARG, "null plan");
  p->profiling = enable != 0;
  return FC2D_OK;
}

extern "C" fc2d_status fc2d_profile_read(fc2d_plan_t p, int max_kernels, char* names,
                                         int64_t* launches, double* ms, int* n_out) {
  if (!p || !n_out || (max_kernels > 0 && (!names || !launches || !ms)))
    return set_error(FC2D_ERR_ARG, "fc2d_profile_read: null argument");
  std::vector<std::string> nm;
  std::vector<int64_t> cnt;
  std::vector<double> tot;
  for (auto& r : p->prof) {
    cudaEventSynchronize((cudaEvent_t)r.stop);
    float t = 0.f;
    cudaEventElapsedTime(&t, (cudaEvent_t)r.start, (cudaEvent_t)r.stop);
    size_t k = 0;
    while (k < nm.size() && nm[k] != r.name) ++k;
    if (k == nm.size()) {
      nm.push_back(r.name);
      cnt.push_back(0);
      tot.push_back(0.0);
    }
    cnt[k] += 1;
    tot[k] += t;
    p->event_pool.push_back(r.start);
    p->event_pool.push_back(r.stop);
  }
  p->prof.clear();
  *n_out = (int)nm.size();
  for (int k = 0; k < (int)nm.size() && k < max_kernels; ++k) {
    std::snprintf(names + 64 * k, 64, "%s", nm[k].c_str());
    launches[k] = cnt[k];
    ms[k] = tot[k];
  }
  return FC2D_OK;
}

// ------------------------------------------------------------------------- //
// Poisson solver (Section 4.1)
// ------------------------------------------------------------------------- //
extern "C" fc2d_status fc2d_poisson_plan(fc2d_plan_t p, int n_b) {
  if (!p) return set_error(FC2D_ERR_ARG, "null plan");
  cudaSetDevice(p->device);
  return poisson_setup(p, n_b);
}

extern "C" fc2d_status fc2d_poisson_nodes(fc2d_plan_t p, double* xy_host, int* n_b) {
  if (!p || !n_b) return set_error(FC2D_ERR_ARG, "fc2d_poisson_nodes: null argument");
  *n_b = poisson_nb(p);
  if (!*n_b) return set_error(FC2D_ERR_ARG, "fc2d_poisson_nodes: call fc2d_poisson_plan first");
  if (xy_host) std::memcpy(xy_host, poisson_nodes(p), sizeof(double) * 2 * (size_t)*n_b);
  return FC2D_OK;
}

extern "C" fc2d_status fc2d_poisson_info(fc2d_plan_t p, int* gmres_iters, double* gmres_resid,
                                         int64_t* n_near) {
  if (!p) return set_error(FC2D_ERR_ARG, "null plan");
  poisson_stats(p, gmres_iters, gmres_resid, n_near);
  return FC2D_OK;
}

extern "C" fc2d_status fc2d_poisson(fc2d_plan_t p, int n_f, const double* fg, const double* fb,
                                    const double* g_nodes, double* u, double* phi,
                                    void* stream) {
  fc2d_status st = check_nf(p, n_f);
  if (st) return st;
  if (!fg || !fb || !g_nodes || !u) return set_error(FC2D_ERR_ARG, "fc2d_poisson: null pointer");
  if (!p->poisson) return set_error(FC2D_ERR_ARG, "fc2d_poisson: call fc2d_poisson_plan first");
  if (p->prm.precision != FC2D_FP64)
    return set_error(FC2D_ERR_UNSUPPORTED, "fc2d_poisson: FP64 plans only");
  cudaSetDevice(p->device);
  Layout L = layout(p, n_f);
  if ((st = ensure_workspace(p, L.total))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = strip_values(p, n_f, fg, fb, L, s))) return st;
  {
    ProfScope ps(p, "fft_rows_fused", s);
    launch_fft_rows(fft_args(p), row_args(p), n_f, true, 1, nullptr, fg, ws(p, L.ovals),
                    ws(p, L.ointer), s);
  }
  return poisson_solve(p, n_f, fg, fb, g_nodes, u, phi, ws(p, L.ointer), s);
}

// ------------------------------------------------------------------------- //
// Fourier Forwarding interior propagator (Section 4.2)
// ------------------------------------------------------------------------- //
namespace fc2d {
void cols4k_prepare();
bool cols4k_tma_usable(const FftArgs& fa, int cc, int n_f, void* inter);

// Plan-time autotuning of the mixed form's 4096-point column passes.  Every candidate
// (the direct form with 16, 32 or 64 columns per block, the TMA-pipelined form with 16
// or 32) runs inside this plan's own extension step: fc2d_extend_coeffs of one function
// on two alternating synthetic inputs and outputs (each byte 0x3F, so every value is a
// normal double and the FP64 to FP32 conversions take their usual path; two grids of
// f exceed the L2 together), 3 warm-up steps, then 10 timed back to back with events
// on a private stream.  The fastest step is kept.  The passes timed on their own do not
// predict the step, where their blocks also overlap the previous and the next kernel.
// Without the memory for the inputs the plan keeps the untuned shape {16, direct}.
fc2d_status tune_plan(fc2d_plan_s* p) {
  if (p->prm.precision != FC2D_MIXED || p->grid.ny != 4096) return FC2D_OK;
  cols4k_prepare();
  const size_t ng = (size_t)p->grid.nx * p->grid.ny;
  const size_t nh = (size_t)p->grid.ny * (p->grid.nx / 2 + 1) * 2 * sizeof(float);
  const size_t nb = (size_t)std::max<int64_t>(1, p->n_bdry) * sizeof(double);
  void *fg[2] = {nullptr, nullptr}, *fh[2] = {nullptr, nullptr}, *fb = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  fc2d_status st = FC2D_OK;
  bool have = cudaMalloc(&fb, nb) == cudaSuccess;
  for (int i = 0; i < 2; ++i)
    have = have && cudaMalloc(&fg[i], ng * sizeof(double)) == cudaSuccess &&
           cudaMalloc(&fh[i], nh) == cudaSuccess;
  have = have && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  if (!have) {
    cudaGetLastError();  // not enough memory to time: the untuned shape stays
  } else {
    for (int i = 0; i < 2; ++i) cudaMemsetAsync(fg[i], 0x3F, ng * sizeof(double), s);
    cudaMemsetAsync(fb, 0x3F, nb, s);
    const int cand[5] = {16, 32, 64, 16, 32}, form[5] = {0, 0, 0, 1, 1};
    float best_us = 0.f;
    int best = -1;
    for (int k = 0; k < 5 && !st; ++k) {
      p->tune_cc4k = cand[k];
      p->tune_tma = form[k];
      p->tune_us[k] = 0.f;
      const double* fb_arg = p->n_bdry > 0 ? (const double*)fb : nullptr;
      int n = 0;
      for (; n < 3 && !st; ++n)
        st = fc2d_extend_coeffs(p, 1, (const double*)fg[n & 1], fb_arg, fh[n & 1], s);
      // a TMA candidate that cannot run on this plan's intermediate is not timed
      if (st || (form[k] && !cols4k_tma_usable(fft_args(p), cand[k], 1,
                                                 ws(p, layout(p, 1).ointer))))
        continue;
      cudaEventRecord(e0, s);
      for (int r = 0; r < 10 && !st; ++r, ++n)
        st = fc2d_extend_coeffs(p, 1, (const double*)fg[n & 1], fb_arg, fh[n & 1], s);
      cudaEventRecord(e1, s);
      if (!st) st = cuda_check(cudaEventSynchronize(e1), "column tuner");
      float ms = 0.f;
      if (!st) st = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "column tuner");
      if (st) break;
      p->tune_us[k] = ms * 100.f;  // microseconds per step (10 steps)
      if (best < 0 || p->tune_us[k] < best_us) {
        best_us = p->tune_us[k];
        best = k;
      }
    }
    if (!st) st = fc2d_sync_status(p, s);
    p->tune_cc4k = best >= 0 ? cand[best] : 16;
    p->tune_tma = best >= 0 ? form[best] : 0;
  }
  if (s) cudaStreamSynchronize(s);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  for (int i = 0; i < 2; ++i) {
    cudaFree(fg[i]);
    cudaFree(fh[i]);
  }
  cudaFree(fb);
  return st;
}
}  // namespace fc2d

extern "C" fc2d_status fc2d_tuning_set(fc2d_plan_t p, const int32_t* choice) {
  if (!p || !choice) return set_error(FC2D_ERR_ARG, "fc2d_tuning_set: null argument");
  if (choice[1] != 0 && choice[1] != 1)
    return set_error(FC2D_ERR_ARG, "fc2d_tuning_set: form 0 (direct) or 1 (TMA-pipelined)");
  if (choice[0] != 16 && choice[0] != 32 && (choice[0] != 64 || choice[1] == 1))
    return set_error(FC2D_ERR_ARG,
                     "fc2d_tuning_set: columns per block 16, 32 or 64 (direct), 16 or 32 (TMA)");
  p->tune_cc4k = choice[0];
  p->tune_tma = choice[1];
  return FC2D_OK;
}

extern "C" fc2d_status fc2d_tuning(fc2d_plan_t p, int32_t* choice, float* us) {
  if (!p || !choice) return set_error(FC2D_ERR_ARG, "fc2d_tuning: null argument");
  choice[0] = p->tune_cc4k;
  choice[1] = p->tune_tma;
  if (us)
    for (int k = 0; k < 5; ++k) us[k] = p->tune_us[k];
  return FC2D_OK;
}

namespace fc2d {
// The 2D-FC spectra (eq. (3.1), normalised) of n_f functions u and n_f functions ut
// (grid values + boundary data, as fc2d_extend takes them) into spec
// [2 n_f][ny][nx/2+1] complex: u's first, then ut's.  FP64 plans; uses the plan
// workspace for 2 n_f functions.
fc2d_status wave_spectra(fc2d_plan_s* p, int n_f, const double* u, const double* ub,
                         const double* ut, const double* utb, void* spec, cudaStream_t s) {
  Layout L = layout(p, 2 * n_f);
  fc2d_status st = ensure_workspace(p, L.total);
  if (st) return st;
  const size_t pitch = row_pitch(p);
  FftArgs fa = fft_args(p);
  for (int half = 0; half < 2; ++half) {
    const double* fg = half ? ut : u;
    const double* fb = half ? utb : ub;
    double* F = reinterpret_cast<double*>(ws(p, L.oF)) + (size_t)half * n_f * p->prm.B * (p->Cr + 1);
    double* vals = reinterpret_cast<double*>(ws(p, L.ovals)) + (size_t)half * n_f * p->strip_lin.size();
    double2* inter = reinterpret_cast<double2*>(ws(p, L.ointer)) + (size_t)half * n_f * p->grid.ny * pitch;
    {
      ProfScope ps(p, "gather_blend", s);
      launch_gather_blend(gather_args(p, fg, fb, F, nullptr, nullptr), n_f, true, s);
    }
    {
      ProfScope ps(p, "interp", s);
      launch_interp(interp_args(p, p->Cr + 1), n_f, true, F, vals, s);
    }
    {
      ProfScope ps(p, "fft_rows_fused", s);
      launch_fft_rows(fa, row_args(p), n_f, true, 1, nullptr, fg, vals, inter, s);
    }
  }
  {
    ProfScope ps(p, "fft_cols", s);
    launch_fft_cols(fa, 2 * n_f, true, ws(p, L.ointer), spec, s);
  }
  return launched("wave spectra");
}
}  // namespace fc2d

extern "C" fc2d_status fc2d_wave_interior(fc2d_plan_t p, int n_f, double c, double t,
                                          const double* u0, const double* u0_bdry,
                                          const double* ut0, const double* ut0_bdry,
                                          double* u_out, double* ut_out, void* stream) {
  fc2d_status st = check_nf(p, n_f);
  if (st) return st;
  if (!u0 || !ut0 || !u_out || !ut_out)
    return set_error(FC2D_ERR_ARG, "fc2d_wave_interior: null pointer");
  if ((st = check_interior(p, u0_bdry, "fc2d_wave_interior")) ||
      (st = check_interior(p, ut0_bdry, "fc2d_wave_interior")))
    return st;
  if (!(c > 0) || !(t >= 0)) return set_error(FC2D_ERR_ARG, "fc2d_wave_interior: c > 0, t >= 0");
  if (p->prm.precision != FC2D_FP64)
    return set_error(FC2D_ERR_UNSUPPORTED, "fc2d_wave_interior: FP64 plans only");
  if (3 * (size_t)p->grid.ny * sizeof(double2) > 227 * 1024)
    return set_error(FC2D_ERR_UNSUPPORTED, "fc2d_wave_interior: ny <= 4736");
  cudaSetDevice(p->device);
  Layout L = layout(p, 2 * n_f);
  if ((st = ensure_workspace(p, L.total))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t pitch = row_pitch(p);
  FftArgs fa = fft_args(p);
  for (int half = 0; half < 2; ++half) {
    const double* fg = half ? ut0 : u0;
    const double* fb = half ? ut0_bdry : u0_bdry;
    double* F = reinterpret_cast<double*>(ws(p, L.oF)) + (size_t)half * n_f * p->prm.B * (p->Cr + 1);
    double* vals = reinterpret_cast<double*>(ws(p, L.ovals)) + (size_t)half * n_f * p->strip_lin.size();
    double2* inter = reinterpret_cast<double2*>(ws(p, L.ointer)) + (size_t)half * n_f * p->grid.ny * pitch;
    {
      ProfScope ps(p, "gather_blend", s);
      launch_gather_blend(gather_args(p, fg, fb, F, nullptr, nullptr), n_f, true, s);
    }
    {
      ProfScope ps(p, "interp", s);
      launch_interp(interp_args(p, p->Cr + 1), n_f, true, F, vals, s);
    }
    {
      ProfScope ps(p, "fft_rows_fused", s);
      launch_fft_rows(fa, row_args(p), n_f, true, 1, nullptr, fg, vals, inter, s);
    }
  }
  {
    ProfScope ps(p, "wave_cols", s);
    launch_wave_cols(fa, n_f, ws(p, L.ointer), c, t, p->grid.nx * p->grid.h,
                     p->grid.ny * p->grid.h, s);
  }
  {
    ProfScope ps(p, "inverse_rows", s);
    double2* inter = reinterpret_cast<double2*>(ws(p, L.ointer));
    launch_inverse_rows(fa, n_f, inter, nullptr, p->grid.a0, p->grid.b0, p->grid.h, u_out, s);
    launch_inverse_rows(fa, n_f, inter + (size_t)n_f * p->grid.ny * pitch, nullptr, p->grid.a0,
                        p->grid.b0, p->grid.h, ut_out, s);
  }
  return launched("fc2d_wave_interior");
}
