// Mixed-precision blending to zero (eq. (2.6), Remark 2.2) on the 5th-generation
// tensor cores: F[n][1+q] = sum_j A_r[q][j] c[n][j] for every normal n, with the
// Gram coefficients c = Q^T f_{D_n} formed in FP64 by k_gather_blend<false>.
//
// One CTA of 128 threads handles 128 normals (the MMA's M = 128 rows):
//   D[n][q] = C[n][:] . A_r[q][:]  (M = 128 normals, N = Cr rounded up to 16, K = 8)
// Both operands are split into TF32-exact high parts and float low parts,
//   D = C_hi A_hi^T + C_hi A_lo^T + C_lo A_hi^T,
// three tcgen05.mma kind::tf32 issued by one thread, accumulating in FP32 in tensor
// memory (TMEM).  The blending matrix has entries up to ~4e3, but the Gram
// coefficients that multiply the large entries are small for smooth data, so the
// split keeps the strip values to ~2^-22 relative.  The epilogue reads TMEM with
// tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = normals) and writes F rows.
//
// Operands sit in shared memory in the K-major, no-swizzle canonical layout: core
// matrices of 8 rows x 16 bytes (4 TF32 values), K = 8 is two core matrices wide:
//   byte(row r, k) = (r/8)*256 + (k/4)*128 + (r%8)*16 + (k%4)*4,
// so the leading-dimension byte offset (next 16-byte K chunk) is 128 and the
// stride-dimension byte offset (next 8-row group) is 256.
//
// The single wait (an mbarrier the MMAs arrive on) is bounded: after kSpinLimit polls
// the kernel latches FC2D_ERR_TIMEOUT in the plan's status word, waits (bounded)
// again, frees its TMEM and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "fc2d_kernels.cuh"
#include "interp.cuh"
#include "plan_internal.h"

namespace fc2d {

constexpr int kTileN = 128;           // normals per CTA (MMA M)
constexpr int kMaxCrPad = 256;        // MMA N limit
constexpr int kTmemCols = 256;        // power of two >= N
constexpr uint32_t kSpinLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Bounded wait for the phase of parity `parity` (0 for the first use) of the mbarrier at
// shared address mbar (the MMAs' commit arrives on it): at most `limit` polls.  If they run out, thread 0 latches
// FC2D_ERR_TIMEOUT in *status and the wait is given `limit` polls once more, since
// MMAs still in flight must end before their TMEM is freed.  True once the phase
// completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, int* status, uint32_t limit,
                                                  uint32_t parity = 0) {
  uint32_t done = 0;
  auto poll = [&] {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
  };
  for (uint32_t it = 0; it < limit && !done; ++it) poll();
  if (!done) {
    if (threadIdx.x == 0) atomicExch(status, (int)FC2D_ERR_TIMEOUT);
    for (uint32_t it = 0; it < limit && !done; ++it) poll();
  }
  return done != 0;
}

// K-major, no-swizzle shared-memory matrix descriptor (tcgen05 format).
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for this architecture
  // base offset 0, no swizzle (bits 61-63 = 0)
  return d;
}

// Instruction descriptor: D = F32, A = B = TF32, both K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4)                       // D format F32
         | (2u << 7)                     // A format TF32
         | (2u << 10)                    // B format TF32
         | ((uint32_t)(N >> 3) << 17)    // N / 8
         | ((uint32_t)(M >> 4) << 24);   // M / 16
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ int kmaj_off(int r, int k) {
  return (r >> 3) * 256 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

struct TcArgs {
  int n_cols;         // n_f * B normals in total
  int Cr, d, ldF, ncr_pad;
  const double* coef; // [n_cols][coef_ld] Gram coefficients
  int coef_ld;
  const double* bvals;  // [n_cols] boundary datum
  const float* Ar_hi;   // [Cr][d]
  const float* Ar_lo;
  float* F;             // [n_cols][ldF]
  int* status;
};

__global__ void __launch_bounds__(128, 1) k_blend_tc(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  // layout: C_hi, C_lo (128 x 8 tf32 = 4 KB each), A_hi, A_lo (ncr_pad x 8 = up to 8 KB
  // each), mbarrier (8 B), TMEM address (4 B)
  unsigned char* c_hi = smem;
  unsigned char* c_lo = smem + 4096;
  unsigned char* a_hi = smem + 8192;
  unsigned char* a_lo = a_hi + kMaxCrPad * 32;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(a_lo + kMaxCrPad * 32);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n0 = blockIdx.x * kTileN;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tmem_slot)), "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // operand C: row tid = normal n0 + tid, k = 0..7 (zero beyond d)
  {
    const int n = n0 + tid;
    for (int k = 0; k < 8; ++k) {
      double v = (n < a.n_cols && k < a.d) ? a.coef[(size_t)n * a.coef_ld + k] : 0.0;
      float hi = to_tf32((float)v);
      float lo = (float)(v - (double)hi);
      *reinterpret_cast<float*>(c_hi + kmaj_off(tid, k)) = hi;
      *reinterpret_cast<float*>(c_lo + kmaj_off(tid, k)) = lo;
    }
  }
  // operand A_r: rows q < ncr_pad (zero beyond Cr), k = 0..7 (zero beyond d)
  for (int idx = tid; idx < a.ncr_pad * 8; idx += blockDim.x) {
    const int q = idx >> 3, k = idx & 7;
    float hi = 0.f, lo = 0.f;
    if (q < a.Cr && k < a.d) {
      hi = a.Ar_hi[q * a.d + k];
      lo = a.Ar_lo[q * a.d + k];
    }
    *reinterpret_cast<float*>(a_hi + kmaj_off(q, k)) = hi;
    *reinterpret_cast<float*>(a_lo + kmaj_off(q, k)) = lo;
  }
  // generic-proxy shared stores -> visible to the tensor core (async proxy)
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (tid == 0) {
    const uint32_t idesc = idesc_tf32(kTileN, a.ncr_pad);
    const uint64_t dch = umma_desc(smem_u32(c_hi), 128, 256);
    const uint64_t dcl = umma_desc(smem_u32(c_lo), 128, 256);
    const uint64_t dah = umma_desc(smem_u32(a_hi), 128, 256);
    const uint64_t dal = umma_desc(smem_u32(a_lo), 128, 256);
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(tmem), "l"(dch), "l"(dah), "r"(idesc), "r"(0));
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(tmem), "l"(dch), "l"(dal), "r"(idesc), "r"(1));
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(tmem), "l"(dcl), "l"(dah), "r"(idesc), "r"(1));
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
        ::"r"(smem_u32(mbar)) : "memory");
  }
  // bounded wait for the MMAs (phase 0 of the mbarrier)
  uint32_t done = mbar_wait_bounded(smem_u32(mbar), a.status, kSpinLimit) ? 1u : 0u;
  // the epilogue's tcgen05.ld is warp-collective: run it only if every lane saw the
  // MMAs complete
  done = __all_sync(0xffffffffu, done != 0) ? 1u : 0u;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (done) {
    // epilogue: warp w reads TMEM lanes 32w..32w+31 (normals), 8 columns at a time
    const int n = n0 + warp * 32 + lane;
    float* Frow = a.F + (size_t)n * a.ldF;
    for (int c0 = 0; c0 < a.ncr_pad; c0 += 8) {
      uint32_t r[8];
      const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
            "=r"(r[6]), "=r"(r[7])
          : "r"(addr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (n < a.n_cols) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int q = c0 + e;
          if (q < a.Cr) Frow[1 + q] = __uint_as_float(r[e]);
        }
      }
    }
    if (n < a.n_cols) {
      Frow[0] = (float)a.bvals[n];
      for (int q = a.Cr + 1; q < a.ldF; ++q) Frow[q] = 0.f;  // row padding
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols));
  }
}

size_t blend_tc_smem_bytes() { return 8192 + 2 * kMaxCrPad * 32 + 64 + 1024; }

fc2d_status launch_blend_tc(int n_cols, int Cr, int d, int ldF, const double* coef,
                            int coef_ld, const double* bvals, const float* Ar_hi,
                            const float* Ar_lo, float* F, int* status, cudaStream_t s) {
  if (Cr > kMaxCrPad || d > 8)
    return set_error(FC2D_ERR_UNSUPPORTED, "tensor-core blend: C n_r must be <= 256, d <= 8");
  TcArgs a;
  a.n_cols = n_cols;
  a.Cr = Cr;
  a.d = d;
  a.ldF = ldF;
  a.ncr_pad = (Cr + 15) / 16 * 16;
  a.coef = coef;
  a.coef_ld = coef_ld;
  a.bvals = bvals;
  a.Ar_hi = Ar_hi;
  a.Ar_lo = Ar_lo;
  a.F = F;
  a.status = status;
  // at most two CTAs per SM (each holds 256 TMEM columns of the SM's 512)
  size_t sm = 96 * 1024;
  cudaFuncSetAttribute(k_blend_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_blend_tc<<<(n_cols + kTileN - 1) / kTileN, 128, sm, s>>>(a);
  return cuda_check(cudaGetLastError(), "tensor-core blend launch");
}


// ------------------------------------------------------------------------- //
// Fused form, one CTA per 32 normals.  The roles of the operands are swapped so
// that a small group of normals fills an MMA: the fine points are the M side,
//   D_t[q][n] = A_r[128 t + q][:] . C[n][:]   (M = 128 fine points per tile t,
//                                             N = 32 normals, K = 8),
// with ceil(Cr/128) tiles, three split MMAs each (A_hi C_hi, A_hi C_lo, A_lo C_hi).
// The 8 warps first compute the matching values and Gram coefficients of the 32
// normals (groups of 8 lanes, as in k_gather_blend) into the C tiles; the stencil
// indices and weights are plan constants and are loaded before the dependent-launch
// wait, the grid values after it.  Epilogue: warp w reads TMEM lanes 32(w%4).. of
// tile w/4 (fine points) for the 32 normals (columns), writes them transposed into a
// [32][Cr+1] staging tile (column 0 = the boundary datum) and the CTA stores the 32
// contiguous rows of F.  Requires M - 1 <= 8, d <= 8, Cr <= 256.
// ------------------------------------------------------------------------- //
constexpr int kTcNormals = 32;      // normals per CTA (MMA N)
constexpr int kTcQTile = 128;       // fine points per MMA (MMA M)
constexpr int kTcTmemCols = 64;     // two tiles of 32 columns
constexpr int kTcStageOff = 2 * kMaxCrPad * 32 + 2 * kTcNormals * 32;  // after A and C tiles
constexpr int kTcMaxLd = kMaxCrPad + 16;  // staging row length limit (ldF)
constexpr int kTcBarOff = kTcStageOff + kTcNormals * kTcMaxLd * 4;
constexpr int kTcSmem = kTcBarOff + 16;

template <int MM>
__global__ void __launch_bounds__(256, 2) k_gather_blend_tc(GatherArgs g, TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* a_hi = smem;                                 // [256 q][8 k] K-major
  unsigned char* a_lo = smem + kMaxCrPad * 32;
  unsigned char* c_hi = smem + 2 * kMaxCrPad * 32;            // [32 n][8 k] K-major
  unsigned char* c_lo = c_hi + kTcNormals * 32;
  float* stage = reinterpret_cast<float*>(smem + kTcStageOff);  // [32][ldF]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + kTcBarOff);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n0 = blockIdx.x * kTcNormals;
  const int ldS = a.ldF;  // staging rows as in F: Cr + 1 values, then zeros
  const int nqt = (a.Cr + kTcQTile - 1) / kTcQTile;
  for (int idx = tid; idx < kTcNormals * (ldS - a.Cr - 1); idx += blockDim.x) {
    const int r = idx / (ldS - a.Cr - 1);
    stage[r * ldS + a.Cr + 1 + (idx - r * (ldS - a.Cr - 1))] = 0.f;
  }

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tmem_slot)), "r"(kTcTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // A_r tiles (plan constants): all loads of a thread in flight, then the stores
  {
    constexpr int kPer = kMaxCrPad * 8 / 256;
    float hi[kPer], lo[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int idx = tid + u * 256, q = idx >> 3, k = idx & 7;
      const bool on = q < a.Cr && k < a.d;
      hi[u] = on ? __ldg(a.Ar_hi + q * a.d + k) : 0.f;
      lo[u] = on ? __ldg(a.Ar_lo + q * a.d + k) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int idx = tid + u * 256, q = idx >> 3, k = idx & 7;
      *reinterpret_cast<float*>(a_hi + kmaj_off(q, k)) = hi[u];
      *reinterpret_cast<float*>(a_lo + kmaj_off(q, k)) = lo[u];
    }
  }
  // matching values and Gram coefficients (Section 3.2, eq. (2.6)) into the C tiles
  constexpr int kTaps = MM > 0 ? MM : 9;
  const int s = lane & 7, g0 = lane & ~7;
  const int ln = warp * 4 + (lane >> 3);  // local normal = C tile row
  {
    const int M = MM > 0 ? MM : g.M, d = g.d, NS = M - 1;
    const bool star_lane = s < NS;
    const int n = n0 + ln;
    const bool live = n < a.n_cols;
    const int nn = live ? n : 0;
    const int ff = nn / g.B, pp = nn - ff * g.B;
    const size_t base = ((size_t)pp * NS + (star_lane ? s : 0)) * M;
    int32_t id[kTaps];
    double wv[kTaps];
#pragma unroll
    for (int e = 0; e < kTaps; ++e) {
      const bool on = star_lane && e < M;
      id[e] = on ? __ldg(g.gidx + base + e) : 0;
      wv[e] = on ? __ldg(g.gw + base + e) : 0.0;
    }
    const int nq = g.nq;
    const double* wn = g.wn + ((size_t)pp * nq + (s < nq ? s : 0)) * M;
    double wnv[kTaps];
#pragma unroll
    for (int e = 0; e < kTaps; ++e) wnv[e] = (s < nq && e < M) ? __ldg(wn + e) : 0.0;
    double qv[kMaxD];
#pragma unroll
    for (int i = 0; i < kMaxD; ++i) qv[i] = (s < d && i < d) ? __ldg(g.Q + i * d + s) : 0.0;
    pdl_wait();
    pdl_trigger();
    const double* fg = g.f_grid + (size_t)ff * g.grid_stride;
    const double* fb = g.f_bdry ? g.f_bdry + (size_t)ff * g.n_bdry : nullptr;
    double val[kTaps];
#pragma unroll
    for (int e = 0; e < kTaps; ++e) {
      const int32_t k = id[e];
      val[e] = (star_lane && e < M) ? __ldg(k >= 0 ? fg + k : fb + (-1 - k)) : 0.0;
    }
    const double fbp = fb ? __ldg(fb + pp) : 0.0;
    double star = 0.0;
#pragma unroll
    for (int e = 0; e < kTaps; ++e) star = fma(wv[e], val[e], star);
    double acc = wnv[0] * fbp;
#pragma unroll
    for (int e = 1; e < kTaps; ++e) {
      const double st = __shfl_sync(0xffffffffu, star, g0 + (e - 1 < 8 ? e - 1 : 0));
      if (e < M) acc = fma(wnv[e], st, acc);
    }
    const double fD = s < nq ? acc : (s == d - 1 ? fbp : 0.0);
    // the value at the foot: the boundary datum, or its extrapolation (interior data)
    const double f0 = __shfl_sync(0xffffffffu, fD, g0 + d - 1);
    double cs = 0.0;
#pragma unroll
    for (int i = 0; i < kMaxD; ++i) {
      const double v = __shfl_sync(0xffffffffu, fD, g0 + i);
      if (i < d) cs = fma(qv[i], v, cs);
    }
    const double v = (live && s < d) ? cs : 0.0;
    const float hi = to_tf32((float)v);
    *reinterpret_cast<float*>(c_hi + kmaj_off(ln, s)) = hi;
    *reinterpret_cast<float*>(c_lo + kmaj_off(ln, s)) = (float)(v - (double)hi);
    if (s == 0) stage[ln * ldS] = (float)f0;  // column 0: the boundary datum
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  if (tid == 0) {
    const uint32_t idesc = idesc_tf32(kTcQTile, kTcNormals);
    const uint64_t dch = umma_desc(smem_u32(c_hi), 128, 256);
    const uint64_t dcl = umma_desc(smem_u32(c_lo), 128, 256);
    for (int t = 0; t < nqt; ++t) {
      const uint32_t dt = tmem + (uint32_t)(t * kTcNormals);
      const uint64_t dah = umma_desc(smem_u32(a_hi) + t * kTcQTile * 32, 128, 256);
      const uint64_t dal = umma_desc(smem_u32(a_lo) + t * kTcQTile * 32, 128, 256);
      asm volatile(
          "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
          "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
          ::"r"(dt), "l"(dah), "l"(dch), "r"(idesc), "r"(0));
      asm volatile(
          "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
          "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
          ::"r"(dt), "l"(dah), "l"(dcl), "r"(idesc), "r"(1));
      asm volatile(
          "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
          "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
          ::"r"(dt), "l"(dal), "l"(dch), "r"(idesc), "r"(1));
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
        ::"r"(smem_u32(mbar)) : "memory");
  }
  uint32_t done = mbar_wait_bounded(smem_u32(mbar), a.status, kSpinLimit) ? 1u : 0u;
  done = __all_sync(0xffffffffu, done != 0) ? 1u : 0u;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int quarter = warp & 3, t = warp >> 2;
  if (done && t < nqt) {
    // TMEM lanes = fine points 128 t + 32 quarter + lane, columns = the 32 normals
    uint32_t r[32];
    const uint32_t addr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(t * kTcNormals);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
          "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
          "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]),
          "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
          "=r"(r[30]), "=r"(r[31])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int q = t * kTcQTile + quarter * 32 + lane;
    if (q < a.Cr) {
#pragma unroll
      for (int nl = 0; nl < kTcNormals; ++nl) stage[nl * ldS + 1 + q] = __uint_as_float(r[nl]);
    }
  }
  __syncthreads();
  if (done) {
    // rows n0.. of F are contiguous and laid out as the staging tile
    const int rows = min(kTcNormals, a.n_cols - n0);
    float* dst = a.F + (size_t)n0 * ldS;
    const int total = rows * ldS;
    if ((ldS & 3) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
      const float4* src4 = reinterpret_cast<const float4*>(stage);
      float4* dst4 = reinterpret_cast<float4*>(dst);
      for (int idx = tid; idx < total / 4; idx += blockDim.x) dst4[idx] = src4[idx];
    } else {
      for (int idx = tid; idx < total; idx += blockDim.x) dst[idx] = stage[idx];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTcTmemCols));
  }
}

// ------------------------------------------------------------------------- //
// Blend and interpolation in one kernel (mixed form, M = 8).  CTA (c, fb) of NT threads
// computes the kTcComputed = 64 normals start_c + i (mod B) of NF functions fb NF ..
// fb NF + NF - 1 as above (MMA N = 64 per function; the gather takes NT / 8 normals per
// pass, groups of 8 lanes, and skips the warps whose normals lie past the last one its
// points use, start_{c+1} - start_c + M - 1, leaving their C columns zero), keeps their
// strip values in shared [64][ldS] tiles (zero padded; ldS a multiple of 4, >= Cr + 12,
// and not 16 mod 32 words so that neighbouring rows fall in different banks) and
// interpolates the strip points it owns (Section 3.4) from those tiles, two per thread
// in flight, writing the strip-point values; F is not written.  With NF = 2 the stencil
// tables, the TMEM allocation, the A_r tiles and each point's interpolation weights
// would serve two functions; the launcher uses NF = 1.  NT = 512 runs one CTA per SM
// (calls of one function), NT = 256 two, whose serial phases (tables, gather, MMAs,
// interpolation) then overlap (calls of several functions: 3% faster on the eight-star
// workload than two functions per 512-thread CTA).
// ------------------------------------------------------------------------- //
template <int NF> __host__ __device__ constexpr int gi_tmem_cols() { return 128 * NF; }  // 2 tiles of 64 per function
template <int NF> __host__ __device__ constexpr int gi_stage_off() {
  return 2 * kMaxCrPad * 32 + 2 * NF * kTcComputed * 32;
}
// the mbarrier and the TMEM address after the NF staging tiles of [64][ldS] floats
template <int NF> __host__ __device__ inline int gi_bar_off(int ldS) {
  return gi_stage_off<NF>() + NF * kTcComputed * ldS * 4;
}
template <int NF> __host__ __device__ inline int gi_smem(int ldS) { return gi_bar_off<NF>(ldS) + 16; }

struct OwnArgs {
  const int32_t* off;    // [n_own + 1]
  const int32_t* k;      // [n_strip] strip index
  const int32_t* pack;   // [n_strip] local first normal | first fine node << 8
  const float* w;        // [16][n_strip] theta weights then eta weights
  const int32_t* start;  // [n_own + 1] first normal of each CTA's range
  int n_own, n_strip;
  float* vals;           // [n_f][n_strip]
};

// TMEM columns for the CTA (warp 0) and the MMA mbarrier (thread 0); both become
// visible to the CTA at the item's first barrier.
template <int NF>
__device__ __forceinline__ void gi_setup(uint64_t* mbar, uint32_t* tmem_slot) {
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tmem_slot)), "r"(gi_tmem_cols<NF>()));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
}

template <int NF>
__device__ __forceinline__ void gi_release(uint32_t tmem) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(gi_tmem_cols<NF>()));
  }
}

// One work item: range c of the owner set, function block fblk (functions fblk NF ..).
// The CTA holds gi_tmem_cols<NF>() TMEM columns (address in *tmem_slot) and the
// mbarrier, whose phase this item's MMAs complete has parity `parity`.  Returns, to
// every thread, false when that wait timed out (the status is set; the caller stops).
template <int NF, int NT>
__device__ __forceinline__ bool gi_item(const GatherArgs& g, const TcArgs& a, const OwnArgs& o,
                                        int n_f, int c, int fblk, unsigned char* smem,
                                        uint64_t* mbar, const uint32_t* tmem_slot,
                                        uint32_t parity) {
  constexpr int MM = 8;
  unsigned char* a_hi = smem;
  unsigned char* a_lo = smem + kMaxCrPad * 32;
  // function ff's C tiles at c_hi/c_lo + ff * kTcComputed * 32 (c_lo after all c_hi)
  unsigned char* c_hi = smem + 2 * kMaxCrPad * 32;
  unsigned char* c_lo = c_hi + NF * kTcComputed * 32;
  float* stage0 = reinterpret_cast<float*>(smem + gi_stage_off<NF>());  // NF x [64][ldS]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int f0 = fblk * NF;
  const int nfl = min(NF, n_f - f0);  // functions of this item (the last may have fewer)
  const int ldS = a.ldF;  // staging row length (see the launcher)
  const int nqt = (a.Cr + kTcQTile - 1) / kTcQTile;
  const int o0 = __ldg(o.off + c), o1 = __ldg(o.off + c + 1);

  for (int idx = tid; idx < NF * kTcComputed * (ldS - a.Cr - 1); idx += blockDim.x) {
    const int r = idx / (ldS - a.Cr - 1);  // row of the NF stacked tiles
    stage0[r * ldS + a.Cr + 1 + (idx - r * (ldS - a.Cr - 1))] = 0.f;
  }
  {
    constexpr int kPer = (kMaxCrPad * 8 + NT - 1) / NT;
    float hi[kPer], lo[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int idx = tid + u * NT, q = idx >> 3, k = idx & 7;
      const bool on = idx < kMaxCrPad * 8 && q < a.Cr && k < a.d;
      hi[u] = on ? __ldg(a.Ar_hi + q * a.d + k) : 0.f;
      lo[u] = on ? __ldg(a.Ar_lo + q * a.d + k) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int idx = tid + u * NT, q = idx >> 3, k = idx & 7;
      if (idx < kMaxCrPad * 8) {
        *reinterpret_cast<float*>(a_hi + kmaj_off(q, k)) = hi[u];
        *reinterpret_cast<float*>(a_lo + kmaj_off(q, k)) = lo[u];
      }
    }
  }
  // matching values and Gram coefficients of the 64 normals into the C tiles, NT / 8
  // normals per pass; a warp whose four normals all lie past `need` writes zero columns
  const int s = lane & 7, g0 = lane & ~7;
  const int need = min(kTcComputed, __ldg(o.start + c + 1) - __ldg(o.start + c) + MM - 1);
#pragma unroll 1
  for (int pass = 0; pass < kTcComputed * 8 / NT; ++pass) {
    const int ln = pass * (NT / 8) + warp * 4 + (lane >> 3);
    if (pass * (NT / 8) + warp * 4 >= need) {  // warp-uniform
      if (pass == 0) {
        pdl_wait();
        pdl_trigger();
      }
      for (int ff = 0; ff < nfl; ++ff) {
        *reinterpret_cast<float*>(c_hi + ff * kTcComputed * 32 + kmaj_off(ln, s)) = 0.f;
        *reinterpret_cast<float*>(c_lo + ff * kTcComputed * 32 + kmaj_off(ln, s)) = 0.f;
        if (s == 0) stage0[(size_t)ff * kTcComputed * ldS + ln * ldS] = 0.f;
      }
      continue;
    }
    const int M = MM, d = g.d, NS = M - 1;
    const bool star_lane = s < NS;
    const int pp = (__ldg(o.start + c) + ln) % g.B;
    const size_t base = ((size_t)pp * NS + (star_lane ? s : 0)) * M;
    int32_t id[MM];
    double wv[MM], wnv[MM], qv[kMaxD];
#pragma unroll
    for (int e = 0; e < MM; ++e) {
      id[e] = star_lane ? __ldg(g.gidx + base + e) : 0;
      wv[e] = star_lane ? __ldg(g.gw + base + e) : 0.0;
    }
    const int nq = g.nq;
    const double* wn = g.wn + ((size_t)pp * nq + (s < nq ? s : 0)) * M;
#pragma unroll
    for (int e = 0; e < MM; ++e) wnv[e] = s < nq ? __ldg(wn + e) : 0.0;
#pragma unroll
    for (int i = 0; i < kMaxD; ++i) qv[i] = (s < d && i < d) ? __ldg(g.Q + i * d + s) : 0.0;
    if (pass == 0) {
      pdl_wait();
      pdl_trigger();
    }
    for (int ff = 0; ff < nfl; ++ff) {
    const int f = f0 + ff;
    float* stage = stage0 + (size_t)ff * kTcComputed * ldS;
    const double* fg = g.f_grid + (size_t)f * g.grid_stride;
    const double* fb = g.f_bdry ? g.f_bdry + (size_t)f * g.n_bdry : nullptr;
    double val[MM];
#pragma unroll
    for (int e = 0; e < MM; ++e) {
      const int32_t k = id[e];
      val[e] = star_lane ? __ldg(k >= 0 ? fg + k : fb + (-1 - k)) : 0.0;
    }
    const double fbp = fb ? __ldg(fb + pp) : 0.0;
    double star = 0.0;
#pragma unroll
    for (int e = 0; e < MM; ++e) star = fma(wv[e], val[e], star);
    double acc = wnv[0] * fbp;
#pragma unroll
    for (int e = 1; e < MM; ++e) acc = fma(wnv[e], __shfl_sync(0xffffffffu, star, g0 + e - 1), acc);
    const double fD = s < nq ? acc : (s == d - 1 ? fbp : 0.0);
    // the value at the foot: the boundary datum, or its extrapolation (interior data)
    const double fv0 = __shfl_sync(0xffffffffu, fD, g0 + d - 1);
    double cs = 0.0;
#pragma unroll
    for (int i = 0; i < kMaxD; ++i) {
      const double v = __shfl_sync(0xffffffffu, fD, g0 + i);
      if (i < d) cs = fma(qv[i], v, cs);
    }
    const double v = s < d ? cs : 0.0;
    const float hi = to_tf32((float)v);
    *reinterpret_cast<float*>(c_hi + ff * kTcComputed * 32 + kmaj_off(ln, s)) = hi;
    *reinterpret_cast<float*>(c_lo + ff * kTcComputed * 32 + kmaj_off(ln, s)) =
        (float)(v - (double)hi);
    if (s == 0) stage[ln * ldS] = (float)fv0;
    }  // functions of the CTA
  }
  // the interpolation's plan records of this CTA's points (16 weight rows, packed
  // indices, strip indices) into L2 while the MMAs and the epilogue run
  {
    const int nl = ((o1 - o0) * 4 + 127) / 128 + 1;  // 128-byte lines per record row
    for (int idx = tid; idx < 18 * nl; idx += NT) {
      const int rowi = idx / nl, line = idx - rowi * nl;
      const char* base = rowi < 16 ? reinterpret_cast<const char*>(o.w + (size_t)rowi * o.n_strip + o0)
                         : rowi == 16 ? reinterpret_cast<const char*>(o.pack + o0)
                                      : reinterpret_cast<const char*>(o.k + o0);
      const char* a = base + (size_t)line * 128;
      // stay inside the record row: the last line starts before its end
      if (a < base + (size_t)(o1 - o0) * 4) asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  if (tid == 0) {
    const uint32_t idesc = idesc_tf32(kTcQTile, kTcComputed);
    for (int ff = 0; ff < nfl; ++ff)
    for (int t = 0; t < nqt; ++t) {
      const uint64_t dch = umma_desc(smem_u32(c_hi + ff * kTcComputed * 32), 128, 256);
      const uint64_t dcl = umma_desc(smem_u32(c_lo + ff * kTcComputed * 32), 128, 256);
      const uint32_t dt = tmem + (uint32_t)((ff * 2 + t) * kTcComputed);
      const uint64_t dah = umma_desc(smem_u32(a_hi) + t * kTcQTile * 32, 128, 256);
      const uint64_t dal = umma_desc(smem_u32(a_lo) + t * kTcQTile * 32, 128, 256);
      asm volatile(
          "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
          "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
          ::"r"(dt), "l"(dah), "l"(dch), "r"(idesc), "r"(0));
      asm volatile(
          "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
          "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
          ::"r"(dt), "l"(dah), "l"(dcl), "r"(idesc), "r"(1));
      asm volatile(
          "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
          "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
          ::"r"(dt), "l"(dal), "l"(dch), "r"(idesc), "r"(1));
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
        ::"r"(smem_u32(mbar)) : "memory");
  }
  uint32_t done = mbar_wait_bounded(smem_u32(mbar), a.status, kSpinLimit, parity) ? 1u : 0u;
  done = __all_sync(0xffffffffu, done != 0) ? 1u : 0u;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int quarter = warp & 3, t = warp >> 2;
  for (int ff = 0; ff < nfl; ++ff)
  if (done && t < nqt) {
    float* stage = stage0 + (size_t)ff * kTcComputed * ldS;
    // lanes = fine points 128 t + 32 quarter + lane; columns = the 64 normals
    uint32_t r[kTcComputed];
    const uint32_t addr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((ff * 2 + t) * kTcComputed);
#pragma unroll
    for (int h = 0; h < kTcComputed / 32; ++h) {
      uint32_t* rr = r + 32 * h;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
          "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]),
            "=r"(rr[6]), "=r"(rr[7]), "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]),
            "=r"(rr[12]), "=r"(rr[13]), "=r"(rr[14]), "=r"(rr[15]), "=r"(rr[16]),
            "=r"(rr[17]), "=r"(rr[18]), "=r"(rr[19]), "=r"(rr[20]), "=r"(rr[21]),
            "=r"(rr[22]), "=r"(rr[23]), "=r"(rr[24]), "=r"(rr[25]), "=r"(rr[26]),
            "=r"(rr[27]), "=r"(rr[28]), "=r"(rr[29]), "=r"(rr[30]), "=r"(rr[31])
          : "r"(addr + 32u * h));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int q = t * kTcQTile + quarter * 32 + lane;
    if (q < a.Cr) {
#pragma unroll
      for (int nl = 0; nl < kTcComputed; ++nl) stage[nl * ldS + 1 + q] = __uint_as_float(r[nl]);
    }
  }
  __syncthreads();
  if (done) {
    // the strip points owned by this CTA (Section 3.4), from the shared tile
    InterpArgs ia{};
    ia.M = MM;
    ia.B = kTcComputed;  // local rows: no wrap inside the tile
    ia.ldF = ldS;
    auto load = [&](int idx, InterpPoint<MM, float>& q) {
      const int pk = __ldg(o.pack + idx);
      q.pb = pk & 0xFF;
      q.s = pk >> 8;
#pragma unroll
      for (int b = 0; b < MM; ++b) {
        q.th[b] = __ldg(o.w + (size_t)b * o.n_strip + idx);
        q.eta[b] = __ldg(o.w + (size_t)(MM + b) * o.n_strip + idx);
      }
    };
    const int step = blockDim.x;
    for (int idx = o0 + tid; idx < o1; idx += 2 * step) {
      const int idx2 = idx + step;
      InterpPoint<MM, float> q0, q1;
      load(idx, q0);
      const int k0 = __ldg(o.k + idx);
      int k1 = -1;
      if (idx2 < o1) {
        load(idx2, q1);
        k1 = __ldg(o.k + idx2);
      }
#pragma unroll
      for (int ff = 0; ff < NF; ++ff) {
        if (ff >= nfl) break;
        const float* stage = stage0 + (size_t)ff * kTcComputed * ldS;
        float* out = o.vals + (size_t)(f0 + ff) * o.n_strip;
        out[k0] = interp_apply<MM, float, float, float, true, false>(ia, stage, q0);
        if (k1 >= 0) out[k1] = interp_apply<MM, float, float, float, true, false>(ia, stage, q1);
      }
    }
  }
  // the next item rewrites the staging tiles and TMEM: every thread is past its reads
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  return __syncthreads_and(done != 0) != 0;
}

template <int NF, int NT>
__global__ void __launch_bounds__(NT, 512 / NT) k_gather_interp_tc(GatherArgs g, TcArgs a,
                                                                    OwnArgs o, int n_f) {
  static_assert(NT == 256 || NT == 512, "k_gather_interp_tc: 256 or 512 threads");
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + gi_bar_off<NF>(a.ldF));
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);
  gi_setup<NF>(mbar, tmem_slot);
  gi_item<NF, NT>(g, a, o, n_f, blockIdx.x, blockIdx.y, smem, mbar, tmem_slot, 0);
  gi_release<NF>(*tmem_slot);
}

// Persistent form for a plan group: each CTA takes work items (plan, range, function)
// from `items` in order, one at a time, through the atomic counter (zeroed before the
// launch), and runs them with its one TMEM allocation and mbarrier.  The items are
// sorted by decreasing cost on the host, so the longest start first and the uneven
// domains' work ends together.  A timed-out wait ends the CTA's loop.
struct GiWork {
  GatherArgs g;
  TcArgs a;
  OwnArgs o;
  int n_f;
};

template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT) k_gather_interp_queue(const GiWork* __restrict__ work,
                                                                       const int4* __restrict__ items,
                                                                       int n_items, int* counter) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int next;
  gi_setup<1>(&mbar, &tmem_slot);
  uint32_t parity = 0;
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(counter, 1);
    __syncthreads();
    const int it = next;
    if (it >= n_items) break;  // the same value in every thread
    const int4 w = items[it];
    const GiWork& W = work[w.x];
    if (!gi_item<1, NT>(W.g, W.a, W.o, W.n_f, w.y, w.z, smem, &mbar, &tmem_slot, parity)) break;
    parity ^= 1u;
  }
  gi_release<1>(tmem_slot);
}

template <int NF, int NT>
static cudaError_t gi_launch(int n_own, int n_f, const GatherArgs& g, const TcArgs& a,
                             const OwnArgs& o, cudaStream_t s) {
  const int sm = gi_smem<NF>(a.ldF);
  cudaFuncSetAttribute(k_gather_interp_tc<NF, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  return launch_pdl(k_gather_interp_tc<NF, NT>, dim3(n_own, (n_f + NF - 1) / NF), dim3(NT),
                    (size_t)sm, s, g, a, o, n_f);
}

// The fused kernel's argument blocks from a call's description.
static fc2d_status gi_args(const GiPlanArgs& in, TcArgs* a, OwnArgs* o) {
  const GatherArgs& g = in.g;
  const int ldS = in.ldS;
  if (g.Cr > kMaxCrPad || g.d > 8 || g.M != 8 || ldS % 4 || ldS < g.Cr + 12 ||
      ldS + 4 > kTcMaxLd || !in.own_off)
    return set_error(FC2D_ERR_UNSUPPORTED, "blend + interpolation kernel: M = 8, d <= 8");
  *a = TcArgs{};
  a->n_cols = in.n_f * g.B;
  a->Cr = g.Cr;
  a->d = g.d;
  a->ldF = (ldS % 32 == 16) ? ldS + 4 : ldS;  // staging rows: avoid a 16-word stride
  a->ncr_pad = (g.Cr + 15) / 16 * 16;
  a->Ar_hi = in.Ar_hi;
  a->Ar_lo = in.Ar_lo;
  a->status = in.status;
  *o = OwnArgs{in.own_off, in.own_k, in.own_pack, in.own_w, in.own_start, in.n_own, in.n_strip,
               in.vals};
  return FC2D_OK;
}

fc2d_status launch_gather_interp_tc(const GiPlanArgs& in, int nt, cudaStream_t s) {
  TcArgs a;
  OwnArgs o;
  fc2d_status st = gi_args(in, &a, &o);
  if (st) return st;
  if (nt != 256 && nt != 512)
    return set_error(FC2D_ERR_UNSUPPORTED, "blend + interpolation kernel: 256 or 512 threads");
  const cudaError_t e = nt == 256 ? gi_launch<1, 256>(in.n_own, in.n_f, in.g, a, o, s)
                                  : gi_launch<1, 512>(in.n_own, in.n_f, in.g, a, o, s);
  return cuda_check(e, "blend + interpolation launch");
}

size_t gi_work_bytes() { return sizeof(GiWork); }

fc2d_status gi_work_fill(const GiPlanArgs& in, void* out, int* ldS) {
  GiWork w{};
  fc2d_status st = gi_args(in, &w.a, &w.o);
  if (st) return st;
  w.g = in.g;
  w.n_f = in.n_f;
  std::memcpy(out, &w, sizeof(w));
  *ldS = w.a.ldF;
  return FC2D_OK;
}

fc2d_status launch_gather_interp_queue(const void* work, const int4* items, int n_items,
                                       int* counter, int nt, int max_ldS, int n_cta,
                                       cudaStream_t s) {
  if (nt != 256 && nt != 512)
    return set_error(FC2D_ERR_UNSUPPORTED, "blend + interpolation queue: 256 or 512 threads");
  const int sm = gi_stage_off<1>() + kTcComputed * max_ldS * 4;
  auto k = nt == 256 ? k_gather_interp_queue<256> : k_gather_interp_queue<512>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  k<<<n_cta, nt, sm, s>>>(static_cast<const GiWork*>(work), items, n_items, counter);
  return cuda_check(cudaGetLastError(), "blend + interpolation queue launch");
}

fc2d_status launch_gather_blend_tc(const GatherArgs& g, int n_f, int ldF, const float* Ar_hi,
                                   const float* Ar_lo, float* F, int* status, cudaStream_t s) {
  if (g.Cr > kMaxCrPad || g.d > 8 || g.M - 1 > 8 || ldF < g.Cr + 1 || ldF > kTcMaxLd)
    return set_error(FC2D_ERR_UNSUPPORTED, "fused tensor-core blend: C n_r <= 256, d <= 8, M <= 9");
  TcArgs a{};
  a.n_cols = n_f * g.B;
  a.Cr = g.Cr;
  a.d = g.d;
  a.ldF = ldF;
  a.ncr_pad = (g.Cr + 15) / 16 * 16;
  a.Ar_hi = Ar_hi;
  a.Ar_lo = Ar_lo;
  a.F = F;
  a.status = status;
  const size_t sm = kTcSmem;
  auto k = g.M == 8 ? k_gather_blend_tc<8> : (g.M == 7 ? k_gather_blend_tc<7> : k_gather_blend_tc<0>);
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  return cuda_check(
      launch_pdl(k, dim3((a.n_cols + kTcNormals - 1) / kTcNormals), dim3(256), sm, s, g, a),
      "fused tensor-core blend launch");
}

// A wait that nothing ends: mbar_wait_bounded, exactly as the tensor-core kernels call
// it, on a fresh mbarrier that no thread or MMA arrives on, so that the timeout path
// (FC2D_ERR_TIMEOUT latched, the kernel returns) can be run on purpose.  One warp.
__global__ void __launch_bounds__(32) k_wait_probe(int* status, uint32_t limit) {
  __shared__ __align__(8) uint64_t mbar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  mbar_wait_bounded(smem_u32(&mbar), status, limit);
}

fc2d_status launch_wait_probe(int* status, uint32_t limit, cudaStream_t s) {
  k_wait_probe<<<1, 32, 0, s>>>(status, limit);
  return cuda_check(cudaGetLastError(), "wait probe launch");
}

}  // namespace fc2d
