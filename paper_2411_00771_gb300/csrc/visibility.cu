// Visible frequency of points over many views (Sec. 4, crop volume
// estimation): each ground-truth point is an isotropic 3D Gaussian of
// standard deviation sigma, and its count is the number of views in which
// the rasterizer would keep it: in front of the near plane, with the
// 3-sigma square of its EWA-projected footprint (sigma^2 J J^T plus a low-pass
// of `lowpass` px^2, J the Jacobian of the perspective projection)
// overlapping the image.  Occlusion plays no part (the rasterizer's
// per-primitive visible mask).
//
// One thread per point, the views staged through shared memory in chunks;
// per (point, view) about 40 FP32 operations, no memory traffic beyond the
// point itself, so the count over N points and V views is bound by FP32
// issue.  The kept points' height range is a block reduction.
#include <math.h>

#include "gs2d_internal.cuh"

namespace gs2d {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 128;  // views per shared-memory chunk

__global__ void __launch_bounds__(kThreads) vis_count_kernel(const float* __restrict__ pts, int64_t n,
                                                             float sigma2, float lowpass, float near_plane,
                                                             const VisCam* __restrict__ cams, int nviews,
                                                             uint32_t* __restrict__ counts) {
  __shared__ VisCam sc[kChunk];
  const int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const bool live = j < n;
  const float x = live ? pts[3 * j] : 0.f, y = live ? pts[3 * j + 1] : 0.f, z = live ? pts[3 * j + 2] : 0.f;
  uint32_t c = 0;
  for (int v0 = 0; v0 < nviews; v0 += kChunk) {
    const int nv = min(kChunk, nviews - v0);
    __syncthreads();
    for (int i = threadIdx.x; i < nv; i += kThreads) sc[i] = cams[v0 + i];
    __syncthreads();
    if (!live) continue;
    for (int v = 0; v < nv; ++v) {
      const VisCam& k = sc[v];
      const float pz = fmaf(k.R[6], x, fmaf(k.R[7], y, fmaf(k.R[8], z, k.t[2])));
      if (!(pz > near_plane)) continue;
      const float px = fmaf(k.R[0], x, fmaf(k.R[1], y, fmaf(k.R[2], z, k.t[0])));
      const float py = fmaf(k.R[3], x, fmaf(k.R[4], y, fmaf(k.R[5], z, k.t[1])));
      const float iz = 1.f / pz;
      const float ux = px * iz, uy = py * iz;  // x/z, y/z
      const float gx = k.fx * iz, gy = k.fy * iz;
      // sigma^2 J J^T with J = [[gx, 0, -gx ux], [0, gy, -gy uy]]
      const float sxx = fmaf(sigma2 * gx * gx, fmaf(ux, ux, 1.f), lowpass);
      const float syy = fmaf(sigma2 * gy * gy, fmaf(uy, uy, 1.f), lowpass);
      const float sxy = sigma2 * gx * gy * ux * uy;
      const float mid = 0.5f * (sxx + syy), half = 0.5f * (sxx - syy);
      const float r = 3.f * sqrtf(mid + sqrtf(fmaf(half, half, sxy * sxy)));
      const float cx = fmaf(k.fx, ux, k.cx), cy = fmaf(k.fy, uy, k.cy);
      c += (cx + r > 0.f && cx - r < k.W && cy + r > 0.f && cy - r < k.H) ? 1u : 0u;
    }
  }
  if (live) counts[j] += c;
}

// Points seen in at least min_count views: keep mask, and the lowest and
// highest world z among them (ordered-int atomics on the float bits).
__device__ __forceinline__ int ord(float f) {
  const int b = __float_as_int(f);
  return b >= 0 ? b : b ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float unord(int b) { return __int_as_float(b >= 0 ? b : b ^ 0x7FFFFFFF); }

__global__ void vis_init_kernel(int* __restrict__ zr) {
  zr[0] = 0x7FFFFFFF;         // min (as an ordered int)
  zr[1] = (int)0x80000000;    // max
}

__global__ void __launch_bounds__(kThreads) vis_keep_kernel(const float* __restrict__ pts, int64_t n,
                                                            const uint32_t* __restrict__ counts, uint32_t min_count,
                                                            uint8_t* __restrict__ keep, int* __restrict__ zr) {
  int lo = 0x7FFFFFFF, hi = (int)0x80000000;
  for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j < n; j += (int64_t)gridDim.x * kThreads) {
    const bool k = counts[j] >= min_count;
    keep[j] = k ? 1u : 0u;
    if (k) {
      const int o = ord(pts[3 * j + 2]);
      lo = min(lo, o);
      hi = max(hi, o);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&zr[0], lo);
    atomicMax(&zr[1], hi);
  }
}

__global__ void vis_range_kernel(const int* __restrict__ zr, float* __restrict__ zrange) {
  const bool any = zr[0] != 0x7FFFFFFF;
  zrange[0] = any ? unord(zr[0]) : NAN;
  zrange[1] = any ? unord(zr[1]) : NAN;
}

}  // namespace

cudaError_t launch_visibility_count(const float* pts, int64_t n, float sigma, float lowpass, float near_plane,
                                    const VisCam* cams, int nviews, uint32_t* counts, cudaStream_t st) {
  if (n <= 0 || nviews <= 0) return cudaSuccess;
  ProfScope ps(kProfContrib, st);
  count_launch();
  vis_count_kernel<<<div_up(n, kThreads), kThreads, 0, st>>>(pts, n, sigma * sigma, lowpass, near_plane, cams,
                                                             nviews, counts);
  return cudaGetLastError();
}

cudaError_t launch_visibility_keep(const float* pts, int64_t n, const uint32_t* counts, uint32_t min_count,
                                   uint8_t* keep, float* zrange, int* tmp, cudaStream_t st) {
  ProfScope ps(kProfContrib, st);
  count_launch(3);
  vis_init_kernel<<<1, 1, 0, st>>>(tmp);
  if (n > 0) {
    const unsigned g = div_up(n, kThreads) < 1216u ? div_up(n, kThreads) : 1216u;
    vis_keep_kernel<<<g, kThreads, 0, st>>>(pts, n, counts, min_count, keep, tmp);
  }
  vis_range_kernel<<<1, 1, 0, st>>>(tmp, zrange);
  return cudaGetLastError();
}

}  // namespace gs2d
