// Kernel argument blocks and shared device helpers of the 2D-FC kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/fc2d.h"

struct fc2d_plan_s;

namespace fc2d {

constexpr int kMaxD = 8;

struct GatherArgs {
  int B, M, d, Cr;
  int nq;                 // rows of wn: d-1 (boundary data given) or d (interior data only)
  int64_t n_bdry, grid_stride;
  const double* f_grid;   // [n_f][ny][nx]
  const double* f_bdry;   // [n_f][n_bdry], or null: interior data only
  const int32_t* gidx;    // [B][M-1][M]
  const double* gw;       // [B][M-1][M]
  const double* wn;       // [B][nq][M]: weights of (boundary datum, red stars)
  const double* Q;        // [d][d]
  const double* Ar;       // [Cr][d]
  void* F;                // FP64 form: [n_f][B][Cr+1]
  double* coef;           // mixed form: Gram coefficients [n_f][B][coef_ld]
  int coef_ld;
  double* bvals;          // mixed form: boundary datum per normal [n_f][B]
};

struct InterpArgs {
  int n_strip, M, B, Cr;
  int ldF;               // row length of F (>= Cr + 1)
  const void* w;         // [2M][n_strip] theta then eta weights (double or float)
  const int32_t* pb;     // first normal index (mod B)
  const int32_t* sb;     // first fine index along the normal
};

fc2d_status interp_weights_gpu(int n_strip, int M, int Cr, int B, double k1, int n_r,
                               const double* theta_dev, const double* eta_dev, bool fp64,
                               void* w_dev, int32_t* pb_dev, int32_t* sb_dev);

struct RowArgs {
  int nx, ny;
  int64_t grid_stride, n_strip;
  const int32_t* row_iv_off;
  const int32_t* row_iv;
  const int32_t* row_strip_off;
  const int32_t* s_lin;
  const int32_t* row_iv_coff;  // mode 2 (compact input): compact offset of each interval
};

#if defined(__CUDACC__)
// Programmatic dependent launch.  A kernel started by launch_pdl may begin while the
// previous kernel on its stream is still finishing.  It calls pdl_wait() before it reads
// anything written by earlier work on the stream and before its first global write;
// pdl_wait() returns once the previous grid has completed and its writes are visible
// (immediately when the kernel was launched without the attribute).  Plan constants
// (tables written at plan time) may be read before it.  pdl_trigger() lets the next
// kernel on the stream be launched early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t stream, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Fill a shared-memory row with the extension: 0, then f on the inside intervals,
// then the strip values.  Ends with the row complete (after a __syncthreads()).
// fg: the function's grid values ([ny][nx], compact == false) or its inside values
// ([n_inside] row by row, compact == true).
template <typename T, typename TV>
__device__ __forceinline__ void load_row(const RowArgs& a, int j, int f,
                                         const double* __restrict__ fg, bool compact,
                                         const TV* __restrict__ vals, T* row) {
  const int nx = a.nx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) row[i] = T(0);
  __syncthreads();
  const int iv0 = __ldg(a.row_iv_off + j), iv1 = __ldg(a.row_iv_off + j + 1);
  for (int k = iv0; k < iv1; ++k) {
    const int lo = __ldg(a.row_iv + 2 * k), hi = __ldg(a.row_iv + 2 * k + 1);
    const double* src = compact ? fg + ((int64_t)__ldg(a.row_iv_coff + k) - lo)
                                : fg + (size_t)j * nx;
    for (int i = lo + threadIdx.x; i <= hi; i += blockDim.x) row[i] = (T)__ldg(src + i);
  }
  const int s0 = __ldg(a.row_strip_off + j), s1 = __ldg(a.row_strip_off + j + 1);
  const TV* v = vals + (size_t)f * a.n_strip;
  const int base = j * nx;
  for (int k = s0 + threadIdx.x; k < s1; k += blockDim.x)
    row[__ldg(a.s_lin + k) - base] = (T)__ldg(v + k);
}
#endif

void launch_gather_blend(const GatherArgs& a, int n_f, bool fp64, cudaStream_t s);
// mixed form of the blend: F[n][0] = bvals[n], F[n][1+q] = (A_r c_n)_q on the tensor
// cores (TF32 hi/lo, FP32 accumulate); n over n_cols = n_f * B normals, row stride ldF.
fc2d_status launch_blend_tc(int n_cols, int Cr, int d, int ldF, const double* coef,
                            int coef_ld, const double* bvals, const float* Ar_hi,
                            const float* Ar_lo, float* F, int* status, cudaStream_t s);
// fused mixed form: matching values + Gram coefficients + tensor-core contraction in one
// kernel (M <= 9, d <= 8); F [n_f*B][ldF] float.
fc2d_status launch_gather_blend_tc(const GatherArgs& g, int n_f, int ldF, const float* Ar_hi,
                                   const float* Ar_lo, float* F, int* status, cudaStream_t s);
// Mixed form, M = 8: matching values, blend and interpolation in one kernel; writes the
// strip-point values (the plan's owner tables group the strip points by CTA, each CTA
// owning the points of a balanced range of at most kTcOwned normals).
struct GiPlanArgs {
  GatherArgs g;
  int n_f, ldS;                 // functions; staging row length (workspace ldF)
  const float *Ar_hi, *Ar_lo;   // split A_r
  const int32_t *own_off, *own_k, *own_pack, *own_start;  // the chosen owner set
  const float* own_w;
  int n_own, n_strip;
  float* vals;                  // [n_f][n_strip] strip-point values out
  int* status;                  // the plan's device status word
};
// nt: threads per CTA, 512 (one CTA per SM) or 256 (two per SM)
fc2d_status launch_gather_interp_tc(const GiPlanArgs& in, int nt, cudaStream_t s);
// Persistent form for plan groups: work items (plan, range, function) as int4
// {plan, range, function, 0}, taken in order through *counter (zero at launch) by n_cta
// CTAs of nt threads.  work: one record per plan (gi_work_bytes() each, written by
// gi_work_fill, which also returns the plan's staging row length); max_ldS: the largest.
size_t gi_work_bytes();
fc2d_status gi_work_fill(const GiPlanArgs& in, void* out, int* ldS);
fc2d_status launch_gather_interp_queue(const void* work, const int4* items, int n_items,
                                       int* counter, int nt, int max_ldS, int n_cta,
                                       cudaStream_t s);
// The tensor-core kernels' bounded mbarrier wait on a barrier nothing arrives on: after
// 2 x limit polls FC2D_ERR_TIMEOUT is latched in *status and the kernel returns.
fc2d_status launch_wait_probe(int* status, uint32_t limit, cudaStream_t s);
void launch_interp(const InterpArgs& a, int n_f, bool fp64, const void* F, void* vals,
                   cudaStream_t s);
void launch_assemble(const RowArgs& a, int n_f, bool fp64, const double* f_grid,
                     const void* vals, void* ext, cudaStream_t s);

struct FftArgs {
  int nx, ny, pitch;          // pitch: complex elements per intermediate row
  int nrx, nry;               // number of radices
  int rx[24], ry[24];
  const void* twx;            // exp(-2 pi i t/(nx/2)) table for the row transform
  const void* twy;            // exp(-2 pi i t/ny)
  const void* rtw;            // exp(-2 pi i k/nx), k <= nx/2
  const void* tsx;            // per-stage twiddles of the row transform (power-of-two sizes)
  const void* tsy;            // per-stage twiddles of the column transform
  double scale;               // 1/(nx ny)
  int cc4k;                   // columns per block of the 4096-point FP32 column passes
  int cols_tma;               // 1: those passes in the TMA-pipelined persistent form
  int* status;                // device status word (bounded waits record a timeout)
};

// rows: mode 0 reads an extended grid (ext, type T); mode 1 assembles the extension
// on the fly from f_grid + strip values; mode 2 likewise from f given at the inside
// points only (f_grid = [n_f][n_inside], row by row; ra.grid_stride = n_inside).
void launch_fft_rows(const FftArgs& fa, const RowArgs& ra, int n_f, bool fp64, int mode,
                     const void* ext, const double* f_grid, const void* vals, void* inter,
                     cudaStream_t s);
// cols: the length-ny column DFTs of the row-pass intermediate into the half spectrum;
// the intermediate is scratch and may be overwritten (the 4096-point FP32 form works
// in place in two passes).
void launch_fft_cols(const FftArgs& fa, int n_f, bool fp64, void* inter, void* fhat,
                     cudaStream_t s);
// complex f: the full spectrum [n_f][ny][nx] from the half spectra of the real and
// imaginary parts, stored as functions 2f and 2f + 1 of `half`
void launch_complex_spectrum(int nx, int ny, int n_f, bool fp64, const void* half, void* out,
                             cudaStream_t s);
// Fourier Forwarding: modal advance of [2 n_f] row spectra (u's then u_t's), in place.
void launch_wave_cols(const FftArgs& fa, int n_f, void* inter, double c, double t, double Lx,
                      double Ly, cudaStream_t s);
// FP64 inverse real row DFT of an [n_f][ny][pitch] half spectrum already inverted along
// the columns; c00 (NULL allowed) adds c00[f] (x^2 + y^2)/4.
void launch_inverse_rows(const FftArgs& fa, int n_f, const void* inter, const double* c00,
                         double a0, double b0, double h, double* out, cudaStream_t s);

// Argument blocks of a plan (capi.cu): the row pass (compact: f given at the inside
// points only) and the DFT of both axes; check_nf validates a function count.
RowArgs row_args(fc2d_plan_s* p, bool compact = false);
FftArgs fft_args(fc2d_plan_s* p);
fc2d_status check_nf(fc2d_plan_s* p, int n_f);

}  // namespace fc2d
