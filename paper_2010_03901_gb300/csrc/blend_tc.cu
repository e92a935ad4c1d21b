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

#include "fc2d_kernels.cuh"
#include "plan_internal.h"

namespace fc2d {

constexpr int kTileN = 128;           // normals per CTA (MMA M)
constexpr int kMaxCrPad = 256;        // MMA N limit
constexpr int kTmemCols = 256;        // power of two >= N
constexpr uint32_t kSpinLimit = 1u << 22;
constexpr int kStageBytes = kTileN * (kMaxCrPad + 1) * 4;  // fused kernel's output staging

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
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
  float* F;             // [n_cols][ldF], or [Cr+1][n_cols] when q_major
  int* status;
  int q_major;          // 1: F[q * n_cols + n] (coalesced epilogue stores)
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
  uint32_t done = 0;
  for (uint32_t it = 0; it < kSpinLimit && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done) : "r"(smem_u32(mbar)), "r"(0) : "memory");
  }
  if (!done) {
    if (tid == 0) atomicExch(a.status, (int)FC2D_ERR_TIMEOUT);
    for (uint32_t it = 0; it < kSpinLimit && !done; ++it) {
      asm volatile(
          "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}\n"
          : "=r"(done) : "r"(smem_u32(mbar)), "r"(0) : "memory");
    }
  }
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
    if (n < a.n_cols) Frow[0] = (float)a.bvals[n];
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
// Fused form: the matching values and Gram coefficients of the CTA's 128 normals are
// computed by its 8 warps (4 normals per warp and pass, groups of 8 lanes, as in
// k_gather_blend) straight into the MMA operand tiles; then the three MMAs and the
// epilogue, warps w and w+4 reading the two halves of the TMEM columns of lanes
// 32(w%4)..32(w%4)+31.  Requires M - 1 <= 8 and d <= 8.
// ------------------------------------------------------------------------- //
__global__ void __launch_bounds__(256, 1) k_gather_blend_tc(GatherArgs g, TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* c_hi = smem;
  unsigned char* c_lo = smem + 4096;
  unsigned char* a_hi = smem + 8192;
  unsigned char* a_lo = a_hi + kMaxCrPad * 32;
  // after the MMAs the operand tiles are dead: the output tile is staged over them
  float* stage = reinterpret_cast<float*>(smem);            // [128][Cr+1]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + kStageBytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n0 = blockIdx.x * kTileN;
  const int ldS = a.Cr + 1;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tmem_slot)), "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
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
  // matching values and Gram coefficients (Section 3.2, eq. (2.6)) into the C tiles
  float bd_row[kTileN / 32];
  {
    const int s = lane & 7, g0 = lane & ~7;
    const int M = g.M, d = g.d, NS = M - 1;
    for (int pass = 0; pass < kTileN / 32; ++pass) {
      const int ln = pass * 32 + warp * 4 + (lane >> 3);  // local normal (tile row)
      const int n = n0 + ln;
      const bool live = n < a.n_cols;
      const int nn = live ? n : 0;
      const int f = nn / g.B, pp = nn - f * g.B;
      const double* fg = g.f_grid + (size_t)f * g.grid_stride;
      const double* fb = g.f_bdry + (size_t)f * g.n_bdry;
      double star = 0.0;
      if (s < NS) {
        const int32_t* gi = g.gidx + ((size_t)pp * NS + s) * M;
        const double* gw = g.gw + ((size_t)pp * NS + s) * M;
        for (int e = 0; e < M; ++e) {
          const int32_t id = __ldg(gi + e);
          const double v = id >= 0 ? __ldg(fg + id) : __ldg(fb + (-1 - id));
          star = fma(__ldg(gw + e), v, star);
        }
      }
      const double fbp = __ldg(fb + pp);
      double fD;
      {
        const double* wn = g.wn + ((size_t)pp * (d - 1) + (s < d - 1 ? s : 0)) * M;
        double acc = (s < d - 1) ? __ldg(wn) * fbp : 0.0;
        for (int e = 1; e < M; ++e) {
          const double st = __shfl_sync(0xffffffffu, star, g0 + e - 1);
          if (s < d - 1) acc = fma(__ldg(wn + e), st, acc);
        }
        fD = s < d - 1 ? acc : (s == d - 1 ? fbp : 0.0);
      }
      double cs = 0.0;
      for (int i = 0; i < d; ++i) {
        const double v = __shfl_sync(0xffffffffu, fD, g0 + i);
        if (s < d) cs = fma(__ldg(g.Q + i * d + s), v, cs);
      }
      const double v = (live && s < d) ? cs : 0.0;
      const float hi = to_tf32((float)v);
      *reinterpret_cast<float*>(c_hi + kmaj_off(ln, s)) = hi;
      *reinterpret_cast<float*>(c_lo + kmaj_off(ln, s)) = (float)(v - (double)hi);
      // boundary datum of row ln, kept in a register until the staging area is free
      if (s == 0) bd_row[pass] = (float)fbp;
    }
  }
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
  uint32_t done = 0;
  for (uint32_t it = 0; it < kSpinLimit && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done) : "r"(smem_u32(mbar)), "r"(0) : "memory");
  }
  if (!done) {
    if (tid == 0) atomicExch(a.status, (int)FC2D_ERR_TIMEOUT);
    for (uint32_t it = 0; it < kSpinLimit && !done; ++it) {
      asm volatile(
          "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}\n"
          : "=r"(done) : "r"(smem_u32(mbar)), "r"(0) : "memory");
    }
  }
  done = __all_sync(0xffffffffu, done != 0) ? 1u : 0u;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (done) {
    // TMEM -> staging [local normal][q] (rows of the tile), then one contiguous store
    const int quarter = warp & 3;
    const int half = ((a.ncr_pad / 2) + 7) / 8 * 8;
    const int cbeg = warp < 4 ? 0 : half, cend = warp < 4 ? half : a.ncr_pad;
    const int ln = quarter * 32 + lane;
    for (int c0 = cbeg; c0 < cend; c0 += 8) {
      uint32_t r[8];
      const uint32_t addr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
            "=r"(r[6]), "=r"(r[7])
          : "r"(addr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int q = c0 + e;
        if (q < a.Cr) stage[ln * ldS + 1 + q] = __uint_as_float(r[e]);
      }
    }
  }
  // boundary data: group lane s == 0 of (warp, group) served rows pass*32 + warp*4 + group
  if ((lane & 7) == 0) {
#pragma unroll
    for (int pass = 0; pass < kTileN / 32; ++pass)
      stage[(pass * 32 + warp * 4 + (lane >> 3)) * ldS] = bd_row[pass];
  }
  __syncthreads();
  if (done) {
    const int rows = min(kTileN, a.n_cols - n0);
    float* dst = a.F + (size_t)n0 * a.ldF;  // rows n0.. are contiguous (ldF = Cr + 1)
    for (int idx = tid; idx < rows * ldS; idx += blockDim.x) dst[idx] = stage[idx];
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols));
  }
}

fc2d_status launch_gather_blend_tc(const GatherArgs& g, int n_f, int ldF, const float* Ar_hi,
                                   const float* Ar_lo, float* F, int* status, cudaStream_t s,
                                   bool q_major) {
  if (g.Cr > kMaxCrPad || g.d > 8 || g.M - 1 > 8 || q_major)
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
  a.q_major = q_major ? 1 : 0;
  // staging + barrier; at most two CTAs per SM (256 TMEM columns each)
  size_t sm = std::max<size_t>(96 * 1024, kStageBytes + 64);
  cudaFuncSetAttribute(k_gather_blend_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_gather_blend_tc<<<(a.n_cols + kTileN - 1) / kTileN, 256, sm, s>>>(g, a);
  return cuda_check(cudaGetLastError(), "fused tensor-core blend launch");
}

}  // namespace fc2d
