// Decomposed-gradient densification statistics and selection (Sec. 3.2,
// Eq. 2) and the elongation filter (Sec. 3.2, eta = min(s) / max(s)).
#include "gs2d_internal.cuh"

namespace gs2d {
namespace {

// Visible = non-empty tile rectangle in this view.
__global__ void densify_acc_kernel(const uint2* __restrict__ rect, const float* __restrict__ screen,
                                   int n, int n_sets, float* __restrict__ stats) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint2 r = rect[i];
  if ((r.y & 0xFFFF) <= (r.x & 0xFFFF)) return;
  float* s = stats + 4 * (size_t)i;
  for (int k = 0; k < n_sets && k < 3; ++k) {
    const float gx = screen[((size_t)k * n + i) * 2], gy = screen[((size_t)k * n + i) * 2 + 1];
    s[k] += sqrtf(gx * gx + gy * gy);
  }
  s[3] += 1.f;
}

// Per-block sums (double) of S_tot/cnt, S_ssim/cnt and of cnt > 0.
__global__ void densify_avg_kernel(const float* __restrict__ stats, int64_t n, double* __restrict__ part) {
  __shared__ double red[3][256];
  double a = 0.0, b = 0.0, c = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float* s = stats + 4 * i;
    if (s[3] > 0.f) {
      a += (double)(s[0] / s[3]);
      b += (double)(s[1] / s[3]);
      c += 1.0;
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
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = red[0][0];
    part[3 * blockIdx.x + 1] = red[1][0];
    part[3 * blockIdx.x + 2] = red[2][0];
  }
}

// k = max(omega * avg_tot / avg_ssim, 1); written to part[0] (as double)
__global__ void densify_scale_kernel(double* __restrict__ part, int nb, float omega, float* k_out) {
  __shared__ double red[3][256];
  double a = 0.0, b = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    a += part[3 * i];
    b += part[3 * i + 1];
    c += part[3 * i + 2];
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
                                      int64_t n, const double* __restrict__ kdev, float grad_thr,
                                      float eta_thr, uint8_t* __restrict__ mask, float* __restrict__ g_out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float k = (float)kdev[0];
  const float* s = stats + 4 * i;
  const float g = s[3] > 0.f ? k * (s[1] / s[3]) : 0.f;
  const float su = scale[2 * i], sv = scale[2 * i + 1];
  const float eta = fminf(su, sv) / fmaxf(su, sv);
  if (g_out) g_out[i] = g;
  mask[i] = (uint8_t)(s[3] > 0.f && g >= grad_thr && eta >= eta_thr);
}

__global__ void elongation_kernel(int64_t n, const float* __restrict__ scale, float eta_thr,
                                  uint8_t* __restrict__ keep) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float su = scale[2 * i], sv = scale[2 * i + 1];
  keep[i] = (uint8_t)(fminf(su, sv) / fmaxf(su, sv) >= eta_thr);
}

constexpr int kAvgBlocks = 304;  // two CTAs per SM on 152 SMs

}  // namespace

size_t densify_tmp_doubles(int64_t) { return 3 * kAvgBlocks + 8; }

cudaError_t launch_densify_accumulate(const uint2* rect, const float* screen, int n,
                                      int n_sets, float* stats, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  ProfScope ps(kProfDensify, st);
  count_launch();
  densify_acc_kernel<<<div_up(n, 256), 256, 0, st>>>(rect, screen, n, n_sets, stats);
  return cudaGetLastError();
}

cudaError_t launch_densify_select(int64_t n, const float* stats, const float* scale, float omega,
                                  float grad_thr, float eta_thr, uint8_t* mask, float* g_out,
                                  float* k_out, double* tmp, cudaStream_t st) {
  ProfScope ps(kProfDensify, st);
  count_launch(n > 0 ? 3 : 2);
  densify_avg_kernel<<<kAvgBlocks, 256, 0, st>>>(stats, n, tmp);
  densify_scale_kernel<<<1, 256, 0, st>>>(tmp, kAvgBlocks, omega, k_out);
  if (n > 0)
    densify_select_kernel<<<div_up(n, 256), 256, 0, st>>>(stats, scale, n, tmp, grad_thr, eta_thr,
                                                          mask, g_out);
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
