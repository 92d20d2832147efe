// Trim contribution (Sec. 3.3, Eq. 3-4) bookkeeping and percentile pruning.
//
// The per-view contribution C_{n,k} = sum / |P_k| comes from the
// contribution blend (blend.cu); here the candidates' accumulators are
// cleared before it and weight * C_{n,k} is added to the caller's running
// average after it (Eq. 4 with weight = 1 / |V_m|).  Pruning removes the
// surfels whose contribution is at or below the bound at the given ratio
// (Sec. 3.3), found by a four-pass radix select on order-preserving keys.
#include <math.h>

#include "gs2d_internal.cuh"

namespace gs2d {
namespace {

constexpr int kThreads = 256;

__global__ void contrib_zero_kernel(const uint32_t* __restrict__ cand, const uint32_t* __restrict__ ncand,
                                    float* __restrict__ csum, uint32_t* __restrict__ ccnt) {
  const uint32_t nc = *ncand;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    const uint32_t n = cand[i];
    csum[n] = 0.f;
    ccnt[n] = 0u;
  }
}

__global__ void contrib_finalize_kernel(const uint32_t* __restrict__ cand, const uint32_t* __restrict__ ncand,
                                        const float* __restrict__ csum, const uint32_t* __restrict__ ccnt,
                                        float weight, float* __restrict__ contrib) {
  const uint32_t nc = *ncand;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    const uint32_t n = cand[i];
    const uint32_t c = ccnt[n];
    if (c != 0u) contrib[n] += weight * (csum[n] / (float)c);
  }
}

// Order-preserving 32-bit key of a float (both zeros map to the same key).
__device__ __forceinline__ uint32_t float_key(float x) {
  const uint32_t b = x == 0.f ? 0u : __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_float(uint32_t k) {
  const uint32_t b = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
  return __uint_as_float(b);
}

// Selection state: [0] key prefix, [1] prefix mask, [2] rank still to skip
// within the prefix, then the 256-bin histogram of the current digit.
constexpr int kSelState = 4;
constexpr int kSelWords = kSelState + 256;

__global__ void select_init_kernel(uint32_t* __restrict__ st, uint32_t rank) {
  const int t = threadIdx.x;
  if (t == 0) { st[0] = 0u; st[1] = 0u; st[2] = rank; }
  st[kSelState + t] = 0u;
}

// Histogram of the digit at `shift` over the keys that match the prefix.
__global__ void __launch_bounds__(kThreads) select_hist_kernel(const float* __restrict__ v, int64_t n, int shift,
                                                               uint32_t* __restrict__ st) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0u;
  __syncthreads();
  const uint32_t prefix = st[0], mask = st[1];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = float_key(v[i]);
    if ((k & mask) == prefix) atomicAdd(&h[(k >> shift) & 255u], 1u);
  }
  __syncthreads();
  if (h[threadIdx.x] != 0u) atomicAdd(&st[kSelState + threadIdx.x], h[threadIdx.x]);
}

// One block of 256 threads: the digit holding the remaining rank; extends the
// prefix, lowers the rank, clears the histogram for the next digit.
__global__ void __launch_bounds__(256) select_pick_kernel(int shift, uint32_t* __restrict__ st) {
  __shared__ uint32_t ws[8];
  __shared__ uint32_t pick_d, pick_below;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const uint32_t c = st[kSelState + t];
  uint32_t v = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  if (lane == 31) ws[w] = v;
  __syncthreads();
  uint32_t before = 0u;
  for (int i = 0; i < w; ++i) before += ws[i];
  const uint32_t incl = before + v, excl = incl - c;
  const uint32_t rank = st[2];
  if (c != 0u && excl <= rank && rank < incl) {
    pick_d = (uint32_t)t;
    pick_below = excl;
  }
  __syncthreads();
  if (t == 0) {
    st[0] |= pick_d << shift;
    st[1] |= 255u << shift;
    st[2] = rank - pick_below;
  }
  st[kSelState + t] = 0u;
}

__global__ void prune_keep_kernel(const float* __restrict__ v, int64_t n, const uint32_t* __restrict__ st,
                                  uint8_t* __restrict__ keep, float* __restrict__ bound) {
  const uint32_t bk = st[0];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    keep[i] = float_key(v[i]) > bk ? 1u : 0u;
  if (bound && blockIdx.x == 0 && threadIdx.x == 0) *bound = key_float(bk);
}

__global__ void prune_keep_all_kernel(int64_t n, uint8_t* __restrict__ keep, float* __restrict__ bound) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    keep[i] = 1u;
  if (bound && blockIdx.x == 0 && threadIdx.x == 0) *bound = -INFINITY;
}

unsigned grid_for(int64_t n) {
  const int64_t b = (n + kThreads - 1) / kThreads;
  return (unsigned)(b < 1 ? 1 : (b > 1216 ? 1216 : b));
}

}  // namespace

cudaError_t launch_contribution(const CamDev& cam, const SetDev& set, float gamma, float weight,
                                const uint32_t* order, const float4* rec, const RowGeom* geom,
                                const uint32_t* vals, const int2* ranges, const uint32_t* cand,
                                const uint32_t* ncand, int64_t n, bool zero_cand, float* csum, uint32_t* ccnt,
                                float* contrib, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  {
    ProfScope ps(kProfContrib, st);
    if (zero_cand) {
      count_launch();
      contrib_zero_kernel<<<grid_for(n), kThreads, 0, st>>>(cand, ncand, csum, ccnt);
    }
  }
  cudaError_t e = launch_blend_contrib(cam, set, gamma, order, rec, geom, vals, ranges, csum, ccnt, st);
  if (e != cudaSuccess || !contrib) return e;
  ProfScope ps(kProfContrib, st);
  count_launch();
  contrib_finalize_kernel<<<grid_for(n), kThreads, 0, st>>>(cand, ncand, csum, ccnt, weight, contrib);
  return cudaGetLastError();
}

size_t select_tmp_words() { return kSelWords; }

cudaError_t launch_prune(int64_t n, const float* contrib, int64_t k, uint8_t* keep, float* bound, uint32_t* tmp,
                         cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  ProfScope ps(kProfContrib, st);
  if (k <= 0) {
    count_launch();
    prune_keep_all_kernel<<<grid_for(n), kThreads, 0, st>>>(n, keep, bound);
    return cudaGetLastError();
  }
  // rank k - 1 (0-based) of the ascending order
  count_launch(10);
  select_init_kernel<<<1, 256, 0, st>>>(tmp, (uint32_t)(k - 1));
  for (int shift = 24; shift >= 0; shift -= 8) {
    select_hist_kernel<<<grid_for(n), kThreads, 0, st>>>(contrib, n, shift, tmp);
    select_pick_kernel<<<1, 256, 0, st>>>(shift, tmp);
  }
  prune_keep_kernel<<<grid_for(n), kThreads, 0, st>>>(contrib, n, tmp, keep, bound);
  return cudaGetLastError();
}

}  // namespace gs2d
