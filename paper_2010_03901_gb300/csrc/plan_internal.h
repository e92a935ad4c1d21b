// Internal state of an fc2d plan (host tables + device tables + workspace).
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fc2d.h"

namespace fc2d {

constexpr int kMaxRadices = 24;
constexpr int kMaxM = 16;
// Mixed form, M = 8: a blend CTA computes kTcComputed consecutive normals (mod B) and
// interpolates the strip points whose first normal lies in its first kTcOwned, whose
// M-normal stencils then lie within the CTA's normals.
constexpr int kTcComputed = 64;
constexpr int kTcOwned = 57;

// One 1D FFT length: its radix sequence and twiddle tables exp(-2 pi i t/N), t < N.
struct FftAxis {
  int n = 0;
  int n_radix = 0;
  int radix[kMaxRadices] = {0};
  std::vector<double> tw_host;   // interleaved re, im (2N doubles)
  double* tw64 = nullptr;        // device, 2N doubles
  float* tw32 = nullptr;         // device, 2N floats
  // power-of-two lengths: per-stage twiddles [stage][r][k] for the radix-8 (double) and
  // radix-16 (float) Stockham sequences (see stage_twiddles in plan.cpp)
  double* tws64 = nullptr;
  float* tws32 = nullptr;
};

struct Curve {
  std::vector<double> cx, sx, cy, sy;
  void eval(double t, double& x, double& y) const;
  void eval_d(double t, int der, double& x, double& y) const;
};

struct DeviceTables {
  // FC matrices
  double* Q = nullptr;       // [d][d]
  double* Ar = nullptr;      // [Cr][d]
  float* Ar_hi = nullptr;    // [Cr][d] TF32-representable high part of A_r
  float* Ar_lo = nullptr;    // [Cr][d] remainder
  // matching stencils
  int32_t* gidx = nullptr;   // [B][M-1][M]  >= 0 grid index, < 0 boundary index -1-k
  double* gw = nullptr;      // [B][M-1][M]
  double* wn = nullptr;      // [B][d-1][M]
  // strip points
  int32_t* s_lin = nullptr;  // [n_strip]
  double* s_theta = nullptr; // [n_strip]
  double* s_eta = nullptr;   // [n_strip]
  void* s_w = nullptr;       // [2M][n_strip] interpolation weights (double or float)
  int32_t* s_pb = nullptr;   // [n_strip] first normal index
  int32_t* s_sb = nullptr;   // [n_strip] first fine index
  // strip points grouped by owning blend CTA (mixed form, M = 8; else null)
  // ownership of the strip points by the blend + interpolation CTAs (mixed, M = 8):
  // own[0] one CTA per SM (balanced ranges), own[1] the fewest CTAs (n = 0: same as 0)
  struct Owners {
    int32_t* off = nullptr;    // [n + 1] offsets of each CTA's points
    int32_t* k = nullptr;      // [n_strip] strip index of each grouped point
    int32_t* pack = nullptr;   // [n_strip] (first normal - CTA's first normal) | s << 8
    float* w = nullptr;        // [2M][n_strip] interpolation weights, grouped order
    int32_t* start = nullptr;  // [n + 1] first normal owned by each CTA, then B
    int n = 0;                 // CTAs per function (ownership ranges)
    std::vector<int32_t> off_host;  // host copy of off (work costs of plan groups)
  } own[2];
  // per-row tables
  int32_t* row_iv_off = nullptr;    // [ny+1] offsets into row_iv
  int32_t* row_iv = nullptr;        // pairs (i_lo, i_hi), inclusive
  int32_t* row_strip_off = nullptr; // [ny+1] offsets into the strip list
  // compact input (f at the inside points only, row by row): the compact index of each
  // inside interval's first point, and the stencil taps as compact indices
  int32_t* row_iv_coff = nullptr;   // [n_iv]
  int32_t* gidx_c = nullptr;        // [B][M-1][M] as gidx, >= 0 entries compact
  // interior data only (no boundary values): stencils from grid nodes alone
  int32_t* gidx_i = nullptr;        // [B][M-1][M] grid indices
  int32_t* gidx_ic = nullptr;       // [B][M-1][M] the same as compact indices
  double* gw_i = nullptr;           // [B][M-1][M]
  double* wn_i = nullptr;           // [B][d][M] (slot 0, the boundary datum, is zero)
  int* status = nullptr;            // latched device status word
};

struct ProfileRecord {
  const char* name;
  void* start;  // cudaEvent_t
  void* stop;
};

struct Workspace {
  void* base = nullptr;
  size_t bytes = 0;
};

}  // namespace fc2d

struct fc2d_plan_s {
  fc2d_grid grid;
  fc2d_params prm;
  int Cr = 0;
  int device = 0;
  fc2d::Curve curve;
  // host copies
  std::vector<double> Q, Ar;                 // d*d, Cr*d
  std::vector<double> bdry_xy;               // 2*n_bdry
  // boundary points of column i's crossings: col_off[i] .. col_off[i+1] (y ascending),
  // of row j's: row_off[j] .. row_off[j+1] (x ascending)
  std::vector<int64_t> col_off, row_off;
  std::vector<int32_t> strip_lin;
  std::vector<double> strip_theta, strip_eta;
  std::vector<int32_t> row_iv_off, row_iv, row_strip_off;
  std::vector<int32_t> row_iv_coff;         // compact offset of each inside interval
  int64_t n_inside = 0;
  int64_t n_bdry = 0;
  bool interior_ok = true;  // every red star has a grid node (interior-only form usable)
  int n_sm = 0;             // SMs of the plan's device
  fc2d::FftAxis fx, fy;                      // nx/2 (complex) and ny
  std::vector<double> rtw_host;              // exp(-2 pi i k/nx), k <= nx/2 (R2C post-process)
  double* rtw64 = nullptr;
  float* rtw32 = nullptr;   // [2][nx/2 + 1] complex: exp(-2 pi i k/nx), then halved
  fc2d::DeviceTables dev;
  fc2d::Workspace ws;
  int host_status = 0;
  bool profiling = false;
  std::vector<fc2d::ProfileRecord> prof;       // events of the current record
  std::vector<void*> event_pool;               // reusable cudaEvent_t
  void* poisson = nullptr;                     // Poisson tables (poisson.cu)
  void* wave = nullptr;                        // Fourier Forwarding state (ff.cu)
  // autotuned launch shapes (tune_plan): columns per block of the 4096-point FP32
  // column passes, their form (0 a block per tile, direct loads; 1 persistent blocks,
  // TMA-pipelined loads) and the candidates' times (microseconds per call, direct 16,
  // 32, 64 then TMA 16, 32; 0: not tuned)
  int tune_cc4k = 16;
  int tune_tma = 0;
  float tune_us[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
};

namespace fc2d {
// Row length (complex values) of the row-DFT intermediate: nx/2 + 1 rounded up to 16,
// so that every row starts on a 128-byte line (16 FP32 complex values).
inline size_t row_pitch(const fc2d_plan_s* p) { return ((size_t)p->grid.nx / 2 + 1 + 15) / 16 * 16; }
}  // namespace fc2d

namespace fc2d {
// error reporting (thread-local message)
fc2d_status set_error(fc2d_status s, const std::string& msg);
fc2d_status cuda_check(int err, const char* what);

// plan-time GPU kernel: foot of the normal through each point (nearest curve point):
// the best of 49 samples within +-window of theta[i], then Newton's method.
fc2d_status foot_newton_gpu(const Curve& c, const std::vector<double>& qx,
                            const std::vector<double>& qy, std::vector<double>& theta,
                            std::vector<int>& conv, double window);

// workspace of at least `bytes` bytes (grows, synchronously, when needed)
fc2d_status ensure_workspace(fc2d_plan_s* p, size_t bytes);

// Poisson solver (poisson.cu)
fc2d_status poisson_setup(fc2d_plan_s* p, int n_b);
fc2d_status poisson_solve(fc2d_plan_s* p, int n_f, const double* f_grid, const double* f_bdry,
                          const double* g_nodes, double* u, double* phi_out, void* inter,
                          cudaStream_t s);
void poisson_destroy(fc2d_plan_s* p);
int poisson_nb(const fc2d_plan_s* p);
const double* poisson_nodes(const fc2d_plan_s* p);
void poisson_stats(const fc2d_plan_s* p, int* iters, double* resid, int64_t* n_near);

// Fourier Forwarding state (ff.cu)
void wave_destroy(fc2d_plan_s* p);

// Plan-time autotuning of launch shapes that change no result (capi.cu).
fc2d_status tune_plan(fc2d_plan_s* p);

// kernel timing: bracket one launch with events when the plan is profiling
struct ProfScope {
  fc2d_plan_s* p;
  const char* name;
  void* stream;
  void* ev0 = nullptr;
  ProfScope(fc2d_plan_s* p, const char* name, void* stream);
  ~ProfScope();
};
}  // namespace fc2d
