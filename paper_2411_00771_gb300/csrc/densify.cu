// Decomposed-gradient densification statistics and selection (Sec. 3.2,
// Eq. 2) and the elongation filter (Sec. 3.2, eta = min(s) / max(s)).
#include "gs2d_internal.cuh"

namespace gs2d {
namespace {

// Visible = non-empty tile rectangle in this view.  kVec: stats rows are
// 16-byte and screen pairs 8-byte aligned (vector reads and writes).
template <bool kVec>
__global__ void densify_acc_kernel(const uint2* __restrict__ rect, const float* __restrict__ screen,
                                   int n, int n_sets, float* __restrict__ stats) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint2 r = rect[i];
  if ((r.y & 0xFFFF) <= (r.x & 0xFFFF)) return;
  float g[3] = {0.f, 0.f, 0.f};
  for (int k = 0; k < n_sets && k < 3; ++k) {
    const size_t j = (size_t)k * n + i;
    const float2 v = kVec ? reinterpret_cast<const float2*>(screen)[j] : make_float2(screen[2 * j], screen[2 * j + 1]);
    g[k] = sqrtf(v.x * v.x + v.y * v.y);
  }
  if constexpr (kVec) {
    float4* s = reinterpret_cast<float4*>(stats) + i;
    float4 t = *s;
    t.x += g[0];
    if (n_sets > 1) t.y += g[1];
    if (n_sets > 2) t.z += g[2];
    t.w += 1.f;
    *s = t;
  } else {
    float* s = stats + 4 * (size_t)i;
    for (int k = 0; k < n_sets && k < 3; ++k) s[k] += g[k];
    s[3] += 1.f;
  }
}

__device__ __forceinline__ float4 load_stats(const float* stats, int64_t i, bool vec) {
  if (vec) return reinterpret_cast<const float4*>(stats)[i];
  const float* s = stats + 4 * i;
  return make_float4(s[0], s[1], s[2], s[3]);
}

// Per-block sums (double) of S_tot/cnt, S_ssim/cnt and of cnt > 0; the
// block that finishes last adds the blocks' sums in block order and writes
// k = max(omega * avg_tot / avg_ssim, 1) to part[0] (as double) and k_out.
// part[3 * nb ..] holds the arrival counter (zeroed before the launch).
constexpr int kAvgUnroll = 4;
__global__ void __launch_bounds__(256) densify_avg_kernel(const float* __restrict__ stats, int64_t n, bool vec,
                                                          float omega, double* __restrict__ part,
                                                          float* __restrict__ k_out) {
  __shared__ double red[3][256];
  double a = 0.0, b = 0.0, c = 0.0;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += kAvgUnroll * step) {
    float4 v[kAvgUnroll];
#pragma unroll
    for (int u = 0; u < kAvgUnroll; ++u) {
      const int64_t i = i0 + u * step;
      v[u] = i < n ? load_stats(stats, i, vec) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kAvgUnroll; ++u) {
      if (v[u].w > 0.f) {
        a += (double)(v[u].x / v[u].w);
        b += (double)(v[u].y / v[u].w);
        c += 1.0;
      }
    }
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  red[2][threadIdx.x] = c;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) {
      red[0][threadIdx.x] += red[0][threadIdx.x + k];
      red[1][threadIdx.x] += red[1][threadIdx.x + k];
      red[2][threadIdx.x] += red[2][threadIdx.x + k];
    }
    __syncthreads();
  }
  __shared__ bool last;
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = red[0][0];
    part[3 * blockIdx.x + 1] = red[1][0];
    part[3 * blockIdx.x + 2] = red[2][0];
    __threadfence();
    unsigned* done = reinterpret_cast<unsigned*>(part + 3 * gridDim.x);
    last = atomicAdd(done, 1u) == gridDim.x - 1u;
    if (last) __threadfence();
  }
  __syncthreads();
  if (!last) return;
  a = b = c = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    a += __ldcg(part + 3 * i);
    b += __ldcg(part + 3 * i + 1);
    c += __ldcg(part + 3 * i + 2);
  }
  __syncthreads();
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  red[2][threadIdx.x] = c;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) {
      red[0][threadIdx.x] += red[0][threadIdx.x + k];
      red[1][threadIdx.x] += red[1][threadIdx.x + k];
      red[2][threadIdx.x] += red[2][threadIdx.x + k];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  a = red[0][0];
  b = red[1][0];
  c = red[2][0];
  double k = 1.0;
  if (c > 0.0 && b > 0.0) {
    const double r = (double)omega * (a / c) / (b / c);
    k = r > 1.0 ? r : 1.0;
  }
  part[0] = k;
  if (k_out) *k_out = (float)k;
}

__global__ void densify_select_kernel(const float* __restrict__ stats, const float* __restrict__ scale,
                                      int64_t n, bool vec, const double* __restrict__ kdev, float grad_thr,
                                      float eta_thr, uint8_t* __restrict__ mask, float* __restrict__ g_out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 s = load_stats(stats, i, vec);
  const float2 sc = vec ? reinterpret_cast<const float2*>(scale)[i] : make_float2(scale[2 * i], scale[2 * i + 1]);
  const float k = (float)kdev[0];
  const float g = s.w > 0.f ? k * (s.y / s.w) : 0.f;
  const float eta = fminf(sc.x, sc.y) / fmaxf(sc.x, sc.y);
  if (g_out) g_out[i] = g;
  mask[i] = (uint8_t)(s.w > 0.f && g >= grad_thr && eta >= eta_thr);
}

__global__ void elongation_kernel(int64_t n, const float* __restrict__ scale, float eta_thr,
                                  uint8_t* __restrict__ keep) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float su = scale[2 * i], sv = scale[2 * i + 1];
  keep[i] = (uint8_t)(fminf(su, sv) / fmaxf(su, sv) >= eta_thr);
}

constexpr int kAvgBlocks = 304;  // two CTAs per SM on 152 SMs

bool aligned(const void* p, size_t b) { return ((uintptr_t)p % b) == 0; }

}  // namespace

// block sums, then the arrival counter
size_t densify_tmp_doubles(int64_t) { return 3 * kAvgBlocks + 8; }

cudaError_t launch_densify_accumulate(const uint2* rect, const float* screen, int n,
                                      int n_sets, float* stats, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  ProfScope ps(kProfDensify, st);
  count_launch();
  if (aligned(stats, 16) && aligned(screen, 8))
    densify_acc_kernel<true><<<div_up(n, 256), 256, 0, st>>>(rect, screen, n, n_sets, stats);
  else
    densify_acc_kernel<false><<<div_up(n, 256), 256, 0, st>>>(rect, screen, n, n_sets, stats);
  return cudaGetLastError();
}

cudaError_t launch_densify_select(int64_t n, const float* stats, const float* scale, float omega,
                                  float grad_thr, float eta_thr, uint8_t* mask, float* g_out,
                                  float* k_out, double* tmp, cudaStream_t st) {
  ProfScope ps(kProfDensify, st);
  const bool vec = aligned(stats, 16) && aligned(scale, 8);
  cudaError_t e = cudaMemsetAsync(tmp + 3 * kAvgBlocks, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  count_launch(n > 0 ? 2 : 1);
  densify_avg_kernel<<<kAvgBlocks, 256, 0, st>>>(stats, n, vec, omega, tmp, k_out);
  if (n > 0)
    densify_select_kernel<<<div_up(n, 256), 256, 0, st>>>(stats, scale, n, vec, tmp, grad_thr, eta_thr, mask,
                                                          g_out);
  return cudaGetLastError();
}

cudaError_t launch_elongation(int64_t n, const float* scale, float eta_thr, uint8_t* keep,
                              cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  ProfScope ps(kProfDensify, st);
  count_launch();
  elongation_kernel<<<div_up(n, 256), 256, 0, st>>>(n, scale, eta_thr, keep);
  return cudaGetLastError();
}

}  // namespace gs2d
