// Contribution-based vector quantisation of SH (Sec. 3.3; Appendix C gives
// a codebook of 8192 entries and a quantisation ratio of 0.4).
//
// The surfels whose contribution lies at or below the ratio's percentile get
// their SH vector (all 3 (deg+1)^2 coefficients, rounded to binary16) replaced
// by the nearest entry of a codebook fitted with Lloyd's K-means; every other
// SH vector, and rotation, scale and opacity, are kept in binary16.
//
// K-means here:
//   - assignment, argmin_j ||x - c_j||^2 = argmin_j (||c_j||^2 - 2 x . c_j):
//     a dense contraction of the vectors [m x C] with the codebook [C x K],
//     run on the tensor cores (tcgen05.mma kind::f16, binary16 operands,
//     FP32 accumulation in TMEM) with the argmin fused into the epilogue.
//     The operands are augmented so that one product gives the score:
//     x' = (x, 1, 1, 0...), c' = (-2 c, h, l, 0...), h + l = ||c||^2 split into
//     two binary16 values (h = rn(||c||^2), l = rn(||c||^2 - h)).  The
//     epilogue takes the minimum of each group of 16 scores with three-input
//     mins, keeps the scores of the best group so far (selects, skipped by
//     warps where no lane improved) and finds the position once per tile.
//     The m x K score matrix is never stored.  A CUDA-core FP32 kernel
//     computes the same scores for checking and for codebooks whose size is
//     not a multiple of 256.
//   - update: exact.  Binary16 values are integer multiples of 2^-24, so each
//     coordinate is summed as a 64-bit integer (order-independent atomics),
//     and the centroid is rn16((double(sum) * 2^-24) / count); an entry with
//     no vector keeps its value.
#include <cuda_fp16.h>
#include <stdint.h>

#include "gs2d_internal.cuh"

namespace gs2d {
namespace {

constexpr int kBM = 128;      // vectors per tile (the MMA's M)
constexpr int kBN = 256;      // codebook entries per chunk (the MMA's N)
constexpr int kStages = 4;    // codebook chunks in flight
constexpr int kEpiWarps = 8;  // two per TMEM lane quarter, one per half of the chunk's columns
constexpr int kTcThreads = 32 * (2 + kEpiWarps);
constexpr int kTmemCols = 2 * kBN;  // double-buffered FP32 accumulator
constexpr uint32_t kSpinLimit = 1u << 26;
constexpr uint64_t kWaitNs = 1000000000ull;  // no single wait of a healthy pipeline comes near a second

// ---- PTX wrappers -----------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for the phase with the given parity to complete.  Gives up
// (returns false) after kWaitNs nanoseconds, after kSpinLimit polls, or when
// another role has aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 1; i < kSpinLimit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 0u && (*abort_flag || global_ns() - t0 > kWaitNs)) return false;
  }
  return false;
}
// Contiguous global -> shared copy by the TMA engine; completes `bytes` on bar.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Arrives once on bar when every tcgen05.mma issued so far by this thread has completed.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T, M = 128, N = 256, K = 16, binary16 in, FP32 out.
__device__ __forceinline__ void tc_mma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                           uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// 32 consecutive FP32 columns of this thread's TMEM lane (the registers are
// valid after tc_wait_ld()).
__device__ __forceinline__ void tc_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor, no swizzle, K-major: the operand is stored
// as 8-row x 16-byte core matrices (each 128 contiguous bytes); lbo = byte
// distance between core matrices adjacent along K, sbo = between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this MMA generation; base offset 0, no swizzle
  return d;
}
// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1),
// A and B binary16 (bits 7-9, 10-12 = 0), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kBN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);

// Element offset of (row r, column k) in the core-matrix layout of a block of
// `rows` rows and D columns (D a multiple of 16): row groups of 8 rows, each
// holding D/8 core matrices of 8 x 8 binary16.
__host__ __device__ __forceinline__ size_t core_offset(int r, int k, int D) {
  return (size_t)(r >> 3) * (8 * D) + (size_t)(k >> 3) * 64 + (size_t)(r & 7) * 8 + (k & 7);
}

// Order-preserving key of (score, index): the smaller score, then the
// smaller index, gives the smaller key.
__device__ __forceinline__ unsigned long long score_key(float s, int idx) {
  const uint32_t b = __float_as_uint(s);
  const uint32_t o = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
  return ((unsigned long long)o << 32) | (uint32_t)idx;
}

__device__ __forceinline__ float fmin3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
// Smallest of the 16 scores v[o..o+15] with three-input mins (8 instructions).
__device__ __forceinline__ float min16(const float (&v)[32], int o) {
  const float a0 = fmin3(v[o], v[o + 1], v[o + 2]), a1 = fmin3(v[o + 3], v[o + 4], v[o + 5]);
  const float a2 = fmin3(v[o + 6], v[o + 7], v[o + 8]), a3 = fmin3(v[o + 9], v[o + 10], v[o + 11]);
  const float a4 = fmin3(v[o + 12], v[o + 13], v[o + 14]);
  return fminf(fmin3(a0, a1, a2), fmin3(a3, a4, v[o + 15]));
}

template <int D>
struct TcSmem {
  uint16_t A[2][kBM * D];        // vector tiles (double-buffered)
  uint16_t B[kStages][kBN * D];  // codebook chunks
  uint64_t a_full[2], a_empty[2], b_full[kStages], b_empty[kStages], t_full[2], t_empty[2], done;
  uint32_t tmem_base;
  int abort_flag;
};

// Persistent: CTA b takes vector tiles b, b + grid, ...; for each tile it
// streams all K / 256 codebook chunks.  Warp 0 (one lane) issues the bulk
// copies, warp 1 (one lane) the MMAs into one of two TMEM accumulators, and
// warps 2..9 read the accumulators (warp w may read TMEM lanes 32 (w % 4) ..
// + 31, i.e. those vectors; warps 2-5 take the chunk's first 128 columns,
// warps 6-9 the rest) and keep each vector's best (score, index).  The two
// halves meet in a 64-bit atomicMin on best64[row] (initialised to ~0).
// Every wait is bounded: on a timeout the kernel records err = 1, the other
// roles stop at their next wait, the producer waits (bounded) for its copies
// in flight and the MMA lane for its MMAs, and TMEM is freed.
template <int D>
__global__ void __launch_bounds__(kTcThreads, 1)
    vq_assign_tc_kernel(const uint16_t* __restrict__ xt, int m, const uint16_t* __restrict__ ct, int K,
                        unsigned long long* __restrict__ best64, int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  TcSmem<D>& S = *reinterpret_cast<TcSmem<D>*>(smem_raw);
  constexpr uint32_t kBytesA = kBM * D * 2, kBytesB = kBN * D * 2;
  constexpr uint32_t kLBO = 128, kSBO = 16 * D;  // core matrix along K; 8-row group
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = (m + kBM - 1) / kBM;
  const int nch = K / kBN;
  volatile int* abort_flag = &S.abort_flag;

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&S.a_full[i], 1);
      mbar_init(&S.a_empty[i], 1);
      mbar_init(&S.t_full[i], 1);
      mbar_init(&S.t_empty[i], kEpiWarps);
    }
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&S.b_full[i], 1);
      mbar_init(&S.b_empty[i], 1);
    }
    mbar_init(&S.done, 1);
    S.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&S.tmem_base)),
                 "r"((uint32_t)kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;

  if (warp == 0) {
    if (lane == 0) {  // producer
      uint32_t g = 0, lt = 0, a_n[2] = {0u, 0u}, b_n[kStages] = {};
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++lt) {
        const int ab = lt & 1;
        if (lt >= 2 && !mbar_wait(&S.a_empty[ab], ((lt >> 1) - 1) & 1, abort_flag)) {
          ok = false;
          break;
        }
        mbar_expect_tx(&S.a_full[ab], kBytesA);
        bulk_g2s(S.A[ab], xt + (size_t)t * kBM * D, kBytesA, &S.a_full[ab]);
        ++a_n[ab];
        for (int c = 0; c < nch; ++c, ++g) {
          const int st = g % kStages;
          if (g >= kStages && !mbar_wait(&S.b_empty[st], ((g / kStages) - 1) & 1, abort_flag)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&S.b_full[st], kBytesB);
          bulk_g2s(S.B[st], ct + (size_t)c * kBN * D, kBytesB, &S.b_full[st]);
          ++b_n[st];
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(err, 1);
      }
      // the copies this lane started must land before the CTA exits, whichever
      // role stopped the pipeline (without an abort they have all landed)
      volatile int never = 0;
      for (int i = 0; i < 2; ++i)
        if (a_n[i] && !mbar_wait(&S.a_full[i], (a_n[i] - 1) & 1, &never)) atomicExch(err, 1);
      for (int i = 0; i < kStages; ++i)
        if (b_n[i] && !mbar_wait(&S.b_full[i], (b_n[i] - 1) & 1, &never)) atomicExch(err, 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      uint32_t g = 0, lt = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++lt) {
        const int ab = lt & 1;
        if (!mbar_wait(&S.a_full[ab], (lt >> 1) & 1, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a_base = smem_addr(S.A[ab]);
        for (int c = 0; c < nch; ++c, ++g) {
          const int st = g % kStages, tb = g & 1;
          if (!mbar_wait(&S.b_full[st], (g / kStages) & 1, abort_flag) ||
              (g >= 2 && !mbar_wait(&S.t_empty[tb], ((g >> 1) - 1) & 1, abort_flag))) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t b_base = smem_addr(S.B[st]);
#pragma unroll
          for (int ks = 0; ks < D / 16; ++ks)
            tc_mma_f16(tmem + (uint32_t)(tb * kBN), smem_desc(a_base + ks * 256, kLBO, kSBO),
                       smem_desc(b_base + ks * 256, kLBO, kSBO), kIdesc, ks > 0 ? 1u : 0u);
          tc_commit(&S.b_empty[st]);
          tc_commit(&S.t_full[tb]);
        }
        if (ok) tc_commit(&S.a_empty[ab]);
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(err, 1);
      }
      // no MMA may be in flight when TMEM is freed
      tc_commit(&S.done);
      volatile int never = 0;
      if (!mbar_wait(&S.done, 0, &never)) atomicExch(err, 1);
    }
  } else {  // epilogue
    const int q = warp & 3;          // TMEM lane quarter this warp may read
    const int half = (warp - 2) >> 2;  // columns [0, 128) or [128, 256) of each chunk
    uint32_t g = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      // per group of 32 scores only its minimum is compared; the scores of
      // the best group are kept to find the position at the end of the tile
      float best = __int_as_float(0x7f800000);
      int grp = 0;
      float keep[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) keep[i] = best;
      for (int c = 0; c < nch; ++c, ++g) {
        const int tb = g & 1;
        const bool w = __all_sync(0xffffffffu, mbar_wait(&S.t_full[tb], (g >> 1) & 1, abort_flag));
        if (!w) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(tb * kBN + half * 128);
#pragma unroll 1
        for (int p = 0; p < 4; p += 2) {  // two groups per wait
          uint32_t r[2][32];
          tc_ld32_async(base + (uint32_t)(p * 32), r[0]);
          tc_ld32_async(base + (uint32_t)(p * 32 + 32), r[1]);
          tc_wait_ld();
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            float v[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[h][i]);
#pragma unroll
            for (int o = 0; o < 32; o += 16) {  // groups of 16 scores
              const float m = min16(v, o);
              const bool take = m < best;  // an equal minimum of a later group never wins
              best = take ? m : best;
              grp = take ? c * kBN + half * 128 + (p + h) * 32 + o : grp;
              if (__any_sync(0xffffffffu, take)) {  // improvements grow rare along the tile
#pragma unroll
                for (int i = 0; i < 16; ++i) keep[i] = take ? v[o + i] : keep[i];
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.t_empty[tb]);
      }
      if (!ok) break;
      int pos = 0;  // the first position of the minimum in its group
#pragma unroll
      for (int i = 15; i >= 0; --i) pos = keep[i] == best ? i : pos;
      atomicMin(best64 + (size_t)t * kBM + q * 32 + lane, score_key(best, grp + pos));
    }
    if (!ok) {
      *abort_flag = 1;
      if (lane == 0) atomicExch(err, 1);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)kTmemCols)
                 : "memory");
  }
}

// ---- operand packing ----------------------------------------------------------

__device__ __forceinline__ uint16_t rn16(float v) { return __half_as_ushort(__float2half_rn(v)); }
__device__ __forceinline__ float f16(uint16_t b) { return __half2float(__ushort_as_half(b)); }
__device__ __forceinline__ bool finite16(uint16_t b) { return (b & 0x7C00u) != 0x7C00u; }

// flags[i] = (keep[i] != 0) == want
__global__ void vq_flags_kernel(const uint8_t* __restrict__ keep, int n, int want, uint32_t* __restrict__ flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flags[i] = ((keep[i] != 0) == (want != 0)) ? 1u : 0u;
}
// rows[offs[i]] = i for the listed surfels ((keep[i] != 0) == want)
__global__ void vq_list_kernel(const uint8_t* __restrict__ keep, const uint32_t* __restrict__ offs, int n, int want,
                               uint32_t* __restrict__ rows) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && (keep[i] != 0) == (want != 0)) rows[offs[i]] = (uint32_t)i;
}

// xr[r][k] = rn16(sh[rows[r]][k]) (row-major) and xt = the augmented operand
// (x, 1, 1, 0...) in the core-matrix layout, rows m..m_pad-1 all zero.
__global__ void vq_pack_x_kernel(const float* __restrict__ sh, const uint32_t* __restrict__ rows, int m, int m_pad,
                                 int C, int D, uint16_t* __restrict__ xr, uint16_t* __restrict__ xt,
                                 int* __restrict__ err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)m_pad * D) return;
  const int r = (int)(i / D), k = (int)(i % D);
  uint16_t v = 0;
  if (r < m) {
    if (k < C) {
      v = rn16(sh[(size_t)rows[r] * C + k]);
      if (!finite16(v)) atomicExch(err, 2);
      xr[(size_t)r * C + k] = v;
    } else if (k < C + 2) {
      v = 0x3C00u;  // 1.0
    }
  }
  xt[core_offset(r, k, D)] = v;
}

// Per entry: hl[j] = (h, l), h = rn16(||c_j||^2) and l = rn16(||c_j||^2 - h),
// the squared norm taken in FP64 (exact up to one rounding for binary16 inputs).
__global__ void vq_norms_kernel(const uint16_t* __restrict__ cb, int K, int C, float2* __restrict__ hl,
                                int* __restrict__ err) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= K) return;
  double n2 = 0.0;
  for (int k = 0; k < C; ++k) {
    const double c = (double)f16(cb[(size_t)j * C + k]);
    n2 = fma(c, c, n2);
  }
  const __half h = __double2half(n2);
  const __half l = __double2half(n2 - (double)__half2float(h));
  if (!finite16(__half_as_ushort(h))) atomicExch(err, 2);
  hl[j] = make_float2(__half2float(h), __half2float(l));
}

// ct = the augmented codebook (-2 c, h, l, 0...) in the core-matrix layout.
__global__ void vq_pack_c_kernel(const uint16_t* __restrict__ cb, const float2* __restrict__ hl, int K, int C, int D,
                                 uint16_t* __restrict__ ct, int* __restrict__ err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)K * D) return;
  const int j = (int)(i / D), k = (int)(i % D);
  uint16_t v = 0;
  if (k < C) {
    v = rn16(-2.f * f16(cb[(size_t)j * C + k]));  // exact unless it overflows
    if (!finite16(v)) atomicExch(err, 2);
  } else if (k == C) {
    v = rn16(hl[j].x);
  } else if (k == C + 1) {
    v = rn16(hl[j].y);
  }
  ct[core_offset(j, k, D)] = v;
}

// ---- CUDA-core assignment (FP32 scores, same formula) --------------------------

constexpr int kSimtCodes = 64;

template <int C>
__global__ void __launch_bounds__(256) vq_assign_simt_kernel(const uint16_t* __restrict__ xr, int m,
                                                             const uint16_t* __restrict__ cb,
                                                             const float2* __restrict__ hl, int K,
                                                             unsigned long long* __restrict__ best64) {
  __shared__ float cs[kSimtCodes][C];
  __shared__ float2 hs[kSimtCodes];
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  float x[C];
#pragma unroll
  for (int k = 0; k < C; ++k) x[k] = r < m ? f16(xr[(size_t)r * C + k]) : 0.f;
  float best = __int_as_float(0x7f800000);
  int bi = 0;
  for (int j0 = 0; j0 < K; j0 += kSimtCodes) {
    const int nj = min(kSimtCodes, K - j0);
    __syncthreads();
    for (int e = threadIdx.x; e < nj * C; e += blockDim.x)
      cs[e / C][e % C] = -2.f * f16(cb[(size_t)j0 * C + e]);
    if (threadIdx.x < nj) hs[threadIdx.x] = hl[j0 + threadIdx.x];
    __syncthreads();
    for (int jj = 0; jj < nj; ++jj) {
      float acc = hs[jj].x + hs[jj].y;
#pragma unroll
      for (int k = 0; k < C; ++k) acc = fmaf(x[k], cs[jj][k], acc);
      if (acc < best) {
        best = acc;
        bi = j0 + jj;
      }
    }
  }
  if (r < m) best64[r] = score_key(best, bi);
}

// ---- update ------------------------------------------------------------------

// a = the entry of vector r; optionally adds the vector to its entry's exact
// sum (int64, units of 2^-24) and count; adds ||x_r - c_a||^2 (FP64) to *objective.
__global__ void __launch_bounds__(256) vq_accum_kernel(const uint16_t* __restrict__ xr, int m, int C,
                                                       const unsigned long long* __restrict__ best64,
                                                       const uint16_t* __restrict__ cb, int K,
                                                       int32_t* __restrict__ best_idx,
                                                       unsigned long long* __restrict__ sums,
                                                       unsigned int* __restrict__ cnt, double* __restrict__ objective) {
  __shared__ double part[8];
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  double d = 0.0;
  if (r < m) {
    int a = (int)(uint32_t)(best64[r] & 0xffffffffull);
    if (a < 0 || a >= K) a = 0;  // only reachable through a failed kernel (err is set there)
    best_idx[r] = a;
    for (int k = 0; k < C; ++k) {
      const float xv = f16(xr[(size_t)r * C + k]);
      const double e = (double)xv - (double)f16(cb[(size_t)a * C + k]);
      d = fma(e, e, d);
      if (sums) atomicAdd(sums + (size_t)a * C + k, (unsigned long long)__float2ll_rn(xv * 16777216.f));
    }
    if (cnt) atomicAdd(cnt + a, 1u);
  }
  if (objective) {
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
      atomicAdd(objective, s);
    }
  }
}

// c = rn16((double(sum) * 2^-24) / count) where count > 0; else unchanged.
__global__ void vq_update_kernel(const unsigned long long* __restrict__ sums, const unsigned int* __restrict__ cnt,
                                 int K, int C, uint16_t* __restrict__ cb) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)K * C) return;
  const unsigned int n = cnt[i / C];
  if (n == 0) return;
  const double mean = ((double)(long long)sums[i] * 0x1p-24) / (double)n;
  cb[i] = __half_as_ushort(__double2half(mean));
}

// Entry j starts as vector floor(u_j m) (clamped to [0, m - 1]).
__global__ void vq_init_kernel(const uint16_t* __restrict__ xr, int m, int C, const float* __restrict__ u, int K,
                               uint16_t* __restrict__ cb) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)K * C) return;
  const int j = (int)(i / C), k = (int)(i % C);
  double f = floor((double)u[j] * (double)m);
  if (!(f >= 0.0)) f = 0.0;
  if (f > (double)(m - 1)) f = (double)(m - 1);
  cb[i] = xr[(size_t)f * C + k];
}

__global__ void vq_scatter_kernel(const uint32_t* __restrict__ rows, const int32_t* __restrict__ best_idx, int m,
                                  int32_t* __restrict__ assign) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < m) assign[rows[r]] = best_idx[r];
}

// ---- compressed render layout ---------------------------------------------------

__global__ void vq_pack_scene_kernel(int n, int C, int K, const float* __restrict__ quat, const float* __restrict__ scale,
                                     const float* __restrict__ opacity, const uint8_t* __restrict__ keep,
                                     const int32_t* __restrict__ assign, const uint32_t* __restrict__ kept_offs,
                                     uint16_t* __restrict__ q16, uint16_t* __restrict__ s16,
                                     uint16_t* __restrict__ o16, uint32_t* __restrict__ sh_row, int* __restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int k = 0; k < 4; ++k) q16[4 * i + k] = rn16(quat[4 * i + k]);
  for (int k = 0; k < 2; ++k) s16[2 * i + k] = rn16(scale[2 * i + k]);
  o16[i] = rn16(opacity[i]);
  if (!finite16(s16[2 * i]) || !finite16(s16[2 * i + 1])) atomicExch(err, 2);
  if (!keep[i]) {
    int a = assign[i];
    if (a < 0 || a >= K) {
      atomicExch(err, 3);
      a = 0;
    }
    sh_row[i] = (uint32_t)a;
  } else {
    sh_row[i] = (uint32_t)K + kept_offs[i];
  }
}
__global__ void vq_pack_table_kernel(int n, int C, int K, const float* __restrict__ sh, const uint8_t* __restrict__ keep,
                                     const uint32_t* __restrict__ kept_offs, uint16_t* __restrict__ table,
                                     int* __restrict__ err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * C) return;
  const int s = (int)(i / C), k = (int)(i % C);
  if (!keep[s]) return;
  const uint16_t v = rn16(sh[i]);
  if (!finite16(v)) atomicExch(err, 2);
  table[((size_t)K + kept_offs[s]) * C + k] = v;
}
// err = 1 when a row index is outside [0, rows)
__global__ void vq_check_rows_kernel(const uint32_t* __restrict__ sh_row, int n, uint32_t rows, int* __restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && sh_row[i] >= rows) atomicExch(err, 1);
}

}  // namespace
}  // namespace gs2d

// ---- launchers -------------------------------------------------------------------

namespace gs2d {
namespace {

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <int D>
cudaError_t launch_tc(const VqBufs& b, int m, int K, int num_sms, cudaStream_t st) {
  // at least 120 KB so that one CTA holds an SM (and its 512 TMEM columns) alone
  const size_t smem = sizeof(TcSmem<D>) > 122880 ? sizeof(TcSmem<D>) : 122880;
  static bool attr = false;
  if (!attr) {
    const cudaError_t e =
        cudaFuncSetAttribute(vq_assign_tc_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int ntiles = (m + kBM - 1) / kBM;
  const int grid = ntiles < num_sms ? ntiles : num_sms;
  vq_assign_tc_kernel<D><<<grid, kTcThreads, smem, st>>>(b.xt, m, b.ct, K, b.best64, b.err);
  count_launch();
  return cudaGetLastError();
}

template <int C>
cudaError_t launch_simt(const VqBufs& b, int m, const uint16_t* cb, int K, cudaStream_t st) {
  vq_assign_simt_kernel<C><<<blocks_for(m, 256), 256, 0, st>>>(b.xr, m, cb, b.hl, K, b.best64);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

int vq_width(int sh_degree, int* C) {
  *C = 3 * (sh_degree + 1) * (sh_degree + 1);
  return 16 * ((*C + 2 + 15) / 16);
}

cudaError_t launch_vq_list(const uint8_t* keep, int n, int want, uint32_t* flags, uint32_t* offs, uint32_t* total,
                           uint32_t* scan_tmp, uint32_t* rows, cudaStream_t st) {
  if (n <= 0) return cudaMemsetAsync(total, 0, sizeof(uint32_t), st);
  vq_flags_kernel<<<blocks_for(n, 256), 256, 0, st>>>(keep, n, want, flags);
  count_launch();
  cudaError_t e = launch_scan(flags, offs, n, total, scan_tmp, st);
  if (e != cudaSuccess || !rows) return e;
  vq_list_kernel<<<blocks_for(n, 256), 256, 0, st>>>(keep, offs, n, want, rows);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_vq_pack_x(const float* sh, const VqBufs& b, int m, int C, int D, cudaStream_t st) {
  const int m_pad = (m + kBM - 1) / kBM * kBM;
  if (m_pad == 0) return cudaSuccess;
  vq_pack_x_kernel<<<blocks_for((int64_t)m_pad * D, 256), 256, 0, st>>>(sh, b.rows, m, m_pad, C, D, b.xr, b.xt, b.err);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_vq_init(const VqBufs& b, int m, int C, const float* u, int K, uint16_t* cb, cudaStream_t st) {
  if (m == 0) return cudaMemsetAsync(cb, 0, sizeof(uint16_t) * (size_t)K * C, st);
  vq_init_kernel<<<blocks_for((int64_t)K * C, 256), 256, 0, st>>>(b.xr, m, C, u, K, cb);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_vq_assign(const VqBufs& b, int m, int C, int D, const uint16_t* cb, int K, bool tensor, int num_sms,
                             cudaStream_t st) {
  if (m == 0) return cudaSuccess;
  const int m_pad = (m + kBM - 1) / kBM * kBM;
  vq_norms_kernel<<<blocks_for(K, 256), 256, 0, st>>>(cb, K, C, b.hl, b.err);
  count_launch();
  cudaError_t e = cudaMemsetAsync(b.best64, 0xFF, sizeof(unsigned long long) * (size_t)m_pad, st);
  if (e != cudaSuccess) return e;
  if (tensor) {
    vq_pack_c_kernel<<<blocks_for((int64_t)K * D, 256), 256, 0, st>>>(cb, b.hl, K, C, D, b.ct, b.err);
    count_launch();
    ProfScope prof(kProfVqAssign, st);
    switch (D) {
      case 16: return launch_tc<16>(b, m, K, num_sms, st);
      case 32: return launch_tc<32>(b, m, K, num_sms, st);
      case 64: return launch_tc<64>(b, m, K, num_sms, st);
      default: return cudaErrorInvalidValue;
    }
  }
  ProfScope prof(kProfVqAssign, st);
  switch (C) {
    case 3: return launch_simt<3>(b, m, cb, K, st);
    case 12: return launch_simt<12>(b, m, cb, K, st);
    case 27: return launch_simt<27>(b, m, cb, K, st);
    case 48: return launch_simt<48>(b, m, cb, K, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_vq_accum(const VqBufs& b, int m, int C, const uint16_t* cb, int K, bool with_sums, double* objective,
                            cudaStream_t st) {
  if (with_sums) {
    cudaError_t e = cudaMemsetAsync(b.sums, 0, sizeof(unsigned long long) * (size_t)K * C, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.cnt, 0, sizeof(unsigned int) * (size_t)K, st);
    if (e != cudaSuccess) return e;
  }
  if (m == 0) return cudaSuccess;
  vq_accum_kernel<<<blocks_for(m, 256), 256, 0, st>>>(b.xr, m, C, b.best64, cb, K, b.best_idx,
                                                       with_sums ? b.sums : nullptr, with_sums ? b.cnt : nullptr,
                                                       objective);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_vq_update(const VqBufs& b, int C, uint16_t* cb, int K, cudaStream_t st) {
  vq_update_kernel<<<blocks_for((int64_t)K * C, 256), 256, 0, st>>>(b.sums, b.cnt, K, C, cb);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_vq_scatter(const VqBufs& b, int m, int32_t* assign, cudaStream_t st) {
  if (m == 0) return cudaSuccess;
  vq_scatter_kernel<<<blocks_for(m, 256), 256, 0, st>>>(b.rows, b.best_idx, m, assign);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_vq_pack_scene(int n, int C, int K, const float* quat, const float* scale, const float* opacity,
                                 const float* sh, const uint8_t* keep, const int32_t* assign,
                                 const uint32_t* kept_offs, const uint16_t* codebook, uint16_t* q16, uint16_t* s16,
                                 uint16_t* o16, uint32_t* sh_row, uint16_t* table, int* err, cudaStream_t st) {
  if (K > 0) {
    const cudaError_t e =
        cudaMemcpyAsync(table, codebook, sizeof(uint16_t) * (size_t)K * C, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
  }
  if (n == 0) return cudaSuccess;
  vq_pack_scene_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, C, K, quat, scale, opacity, keep, assign, kept_offs,
                                                           q16, s16, o16, sh_row, err);
  count_launch();
  vq_pack_table_kernel<<<blocks_for((int64_t)n * C, 256), 256, 0, st>>>(n, C, K, sh, keep, kept_offs, table, err);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_vq_check_rows(const uint32_t* sh_row, int n, uint32_t rows, int* err, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  vq_check_rows_kernel<<<blocks_for(n, 256), 256, 0, st>>>(sh_row, n, rows, err);
  count_launch();
  return cudaGetLastError();
}

}  // namespace gs2d
