// Photometric and depth losses with their adjoints (Sec. 3.1: L1 + D-SSIM;
// Sec. 3.2: L1 on inverse depth).
//
// Kernel 1, per 32 x 32 tile and colour channel: stages a 42 x 42 halo of
// the render and the target in shared memory, forms the five windowed
// moments (mu_x, mu_y, E[x^2], E[y^2], E[xy]) with the separable 11-tap
// Gaussian (zero padded), the SSIM map and its partials with respect to
// mu_x, E[x^2] and E[xy]; the partials go to scratch, the map and |x - y| to
// per-block sums.  Kernel 2 blurs the three partial maps again (the window
// is symmetric, so the adjoint of the windowed sum is the same windowed sum)
// and writes the adjoint planes of the weighted SSIM term, the weighted L1
// term and their sum, plus the inverse-depth adjoint.  A last one-block
// kernel reduces the per-block sums in double.
//
// Both blurs slide the window in registers: a thread of the horizontal pass
// reads 18 inputs of one row and produces 8 outputs, a thread of the
// vertical pass reads 14 rows of one column and produces 4, so each staged
// value is read from shared memory a few times instead of 22.
#include <math.h>

#include <mutex>
#include <string>

#include "gs2d_internal.cuh"

namespace gs2d {
namespace {

constexpr int kT = 32;              // output tile side
constexpr int kR = 5;               // window radius (11 taps)
constexpr int kHalo = kT + 2 * kR;  // 42
constexpr int kTaps = 2 * kR + 1;
constexpr int kThr = 256;
constexpr int kHS = 8;              // outputs per horizontal item
constexpr int kVS = 4;              // outputs per vertical item
constexpr int kSX = kHalo + 1;      // odd row stride of the staged halo
constexpr int kSH = kT + 1;         // row stride of the horizontal sums
constexpr int kHItems = kHalo * (kT / kHS);  // 168
static_assert((kT / kVS) * kT == kThr, "one vertical item per thread");

struct Gauss {
  float w[kTaps];
};

// Stage a kHalo x kHalo window (top-left at (ox, oy)) of NP planes of a
// W x H image, zero outside the image; all loads of a thread are issued
// before the first store.  Thread t takes column t % kHalo of rows
// t / kHalo, + kStageRows, ...: its index arithmetic is done once.
constexpr int kStageRows = kThr / kHalo;                           // 6
constexpr int kStageIt = (kHalo + kStageRows - 1) / kStageRows;    // 7
template <int NP>
struct Planes {
  const float* p[NP];
};
template <int NP>
__device__ __forceinline__ void stage_halo(float (*dst)[kHalo][kSX], Planes<NP> src, int W, int H, int ox,
                                           int oy) {
  const int r0 = threadIdx.x / kHalo, hx = threadIdx.x - r0 * kHalo;
  if (r0 >= kStageRows) return;
  const int gx = ox + hx;
  const bool inx = gx >= 0 && gx < W;
  float v[NP][kStageIt];
#pragma unroll
  for (int k = 0; k < kStageIt; ++k) {
    const int hy = r0 + k * kStageRows, gy = oy + hy;
    const bool in = inx && hy < kHalo && gy >= 0 && gy < H;
#pragma unroll
    for (int q = 0; q < NP; ++q) v[q][k] = in ? src.p[q][(size_t)gy * W + gx] : 0.f;
  }
#pragma unroll
  for (int k = 0; k < kStageIt; ++k) {
    const int hy = r0 + k * kStageRows;
    if (hy < kHalo) {
#pragma unroll
      for (int q = 0; q < NP; ++q) dst[q][hy][hx] = v[q][k];
    }
  }
}

// out[i] = sum_k w[k] in[i + k] for kHS (or kVS) consecutive outputs, with
// the inputs already in registers.
template <int NO>
__device__ __forceinline__ void slide(const float* in, const Gauss& g, float* o) {
#pragma unroll
  for (int j = 0; j < NO + kTaps - 1; ++j)
#pragma unroll
    for (int i = 0; i < NO; ++i) {
      if (j == i) o[i] = g.w[0] * in[j];
      else if (j - i > 0 && j - i < kTaps) o[i] = fmaf(g.w[j - i], in[j], o[i]);
    }
}

__global__ void __launch_bounds__(kThr) ssim_fwd_kernel(int W, int H, const float* __restrict__ out,
                                                        const float* __restrict__ tgt, Gauss g,
                                                        float* __restrict__ part,
                                                        float* __restrict__ bsum) {
  __shared__ float sxy[2][kHalo][kSX];
  float (*sx)[kSX] = sxy[0];
  float (*sy)[kSX] = sxy[1];
  __shared__ float hm[5][kHalo][kSH];
  const int c = blockIdx.z;
  const size_t HW = (size_t)W * H;
  const int ox = blockIdx.x * kT - kR, oy = blockIdx.y * kT - kR;
  const int t = threadIdx.x;
  stage_halo<2>(sxy, Planes<2>{{out + c * HW, tgt + c * HW}}, W, H, ox, oy);
  __syncthreads();
  // horizontal pass over all halo rows: item = (row, 8-column segment)
  if (t < kHItems) {
    const int r = t % kHalo, c0 = (t / kHalo) * kHS;
    float in[kHS + kTaps - 1], o[kHS];
#pragma unroll
    for (int j = 0; j < kHS + kTaps - 1; ++j) in[j] = sx[r][c0 + j];
    slide<kHS>(in, g, o);
#pragma unroll
    for (int i = 0; i < kHS; ++i) hm[0][r][c0 + i] = o[i];
#pragma unroll
    for (int j = 0; j < kHS + kTaps - 1; ++j) in[j] *= in[j];
    slide<kHS>(in, g, o);
#pragma unroll
    for (int i = 0; i < kHS; ++i) hm[2][r][c0 + i] = o[i];
    float iy[kHS + kTaps - 1];
#pragma unroll
    for (int j = 0; j < kHS + kTaps - 1; ++j) iy[j] = sy[r][c0 + j];
    slide<kHS>(iy, g, o);
#pragma unroll
    for (int i = 0; i < kHS; ++i) hm[1][r][c0 + i] = o[i];
#pragma unroll
    for (int j = 0; j < kHS + kTaps - 1; ++j) in[j] = sx[r][c0 + j] * iy[j];
    slide<kHS>(in, g, o);
#pragma unroll
    for (int i = 0; i < kHS; ++i) hm[4][r][c0 + i] = o[i];
#pragma unroll
    for (int j = 0; j < kHS + kTaps - 1; ++j) iy[j] *= iy[j];
    slide<kHS>(iy, g, o);
#pragma unroll
    for (int i = 0; i < kHS; ++i) hm[3][r][c0 + i] = o[i];
  }
  __syncthreads();
  // vertical pass: item = (column, 4-row segment), then the SSIM terms
  const int col = t % kT, r0 = (t / kT) * kVS;
  float m[5][kVS];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    float in[kVS + kTaps - 1];
#pragma unroll
    for (int j = 0; j < kVS + kTaps - 1; ++j) in[j] = hm[q][r0 + j][col];
    slide<kVS>(in, g, m[q]);
  }
  const int px = blockIdx.x * kT + col;
  float ssim = 0.f, l1 = 0.f;
  const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
#pragma unroll
  for (int i = 0; i < kVS; ++i) {
    const int py = blockIdx.y * kT + r0 + i;
    if (px < W && py < H) {
      const float ux = m[0][i], uy = m[1][i];
      const float vx = m[2][i] - ux * ux, vy = m[3][i] - uy * uy, cxy = m[4][i] - ux * uy;
      const float A1 = 2.f * ux * uy + C1, A2 = 2.f * cxy + C2;
      const float B1 = ux * ux + uy * uy + C1, B2 = vx + vy + C2;
      const float iB = 1.f / (B1 * B2);
      const float s = A1 * A2 * iB;
      const float dux = 2.f * uy * A2 * iB - s * 2.f * ux / B1;
      const float dvx = -s / B2;
      const float dcxy = 2.f * A1 * iB;
      const size_t pix = (size_t)py * W + px;
      part[(0 * 3 + c) * HW + pix] = dux - 2.f * ux * dvx - uy * dcxy;
      part[(1 * 3 + c) * HW + pix] = dvx;
      part[(2 * 3 + c) * HW + pix] = dcxy;
      ssim += s;
      l1 += fabsf(sx[r0 + i + kR][col + kR] - sy[r0 + i + kR][col + kR]);
    }
  }
  // block sums
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ssim += __shfl_xor_sync(0xffffffffu, ssim, o);
    l1 += __shfl_xor_sync(0xffffffffu, l1, o);
  }
  __shared__ float ws[2][kThr / 32];
  if ((t & 31) == 0) { ws[0][t >> 5] = l1; ws[1][t >> 5] = ssim; }
  __syncthreads();
  if (t == 0) {
    float a = 0.f, b = 0.f;
    for (int i = 0; i < kThr / 32; ++i) { a += ws[0][i]; b += ws[1][i]; }
    const size_t bi = ((size_t)c * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    bsum[2 * bi] = a;
    bsum[2 * bi + 1] = b;
  }
}

__global__ void __launch_bounds__(kThr) ssim_bwd_kernel(
    int W, int H, const float* __restrict__ out, const float* __restrict__ tgt,
    const float* __restrict__ tinv, Gauss g, gs_loss_weights wt, const float* __restrict__ part,
    float* __restrict__ adj_total, float* __restrict__ adj_ssim, float* __restrict__ adj_l1,
    float* __restrict__ dsum) {
  __shared__ float sp[3][kHalo][kSX];
  __shared__ float hm[3][kHalo][kSH];
  const int c = blockIdx.z;
  const size_t HW = (size_t)W * H;
  const int ox = blockIdx.x * kT - kR, oy = blockIdx.y * kT - kR;
  const int t = threadIdx.x;
  // partial q of channel c is plane 3 q + c
  stage_halo<3>(sp, Planes<3>{{part + c * HW, part + (3 + c) * HW, part + (6 + c) * HW}}, W, H, ox, oy);
  __syncthreads();
  if (t < kHItems) {
    const int r = t % kHalo, c0 = (t / kHalo) * kHS;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float in[kHS + kTaps - 1], o[kHS];
#pragma unroll
      for (int j = 0; j < kHS + kTaps - 1; ++j) in[j] = sp[q][r][c0 + j];
      slide<kHS>(in, g, o);
#pragma unroll
      for (int i = 0; i < kHS; ++i) hm[q][r][c0 + i] = o[i];
    }
  }
  __syncthreads();
  const int col = t % kT, r0 = (t / kT) * kVS;
  float b[3][kVS];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    float in[kVS + kTaps - 1];
#pragma unroll
    for (int j = 0; j < kVS + kTaps - 1; ++j) in[j] = hm[q][r0 + j][col];
    slide<kVS>(in, g, b[q]);
  }
  const int px = blockIdx.x * kT + col;
  const float inv = 1.f / (3.f * (float)HW);
  float dl = 0.f;
#pragma unroll
  for (int i = 0; i < kVS; ++i) {
    const int py = blockIdx.y * kT + r0 + i;
    if (px < W && py < H) {
      const size_t pix = (size_t)py * W + px;
      const float x = out[c * HW + pix], y = tgt[c * HW + pix];
      const float dssim = b[0][i] + 2.f * x * b[1][i] + y * b[2][i];
      const float as = -wt.w_ssim * dssim * inv;
      const float d = x - y;
      const float al = wt.w_l1 * (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f)) * inv;
      adj_total[c * HW + pix] = as + al;
      if (adj_ssim) adj_ssim[c * HW + pix] = as;
      if (adj_l1) adj_l1[c * HW + pix] = al;
      if (c == 0 && tinv) {
        const float e = out[5 * HW + pix] - tinv[pix];
        dl += fabsf(e);
        adj_total[5 * HW + pix] = wt.w_depth * (e > 0.f ? 1.f : (e < 0.f ? -1.f : 0.f)) / (float)HW;
      }
    }
  }
  if (c == 0 && dsum) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dl += __shfl_xor_sync(0xffffffffu, dl, o);
    __shared__ float ws[kThr / 32];
    if ((t & 31) == 0) ws[t >> 5] = dl;
    __syncthreads();
    if (t == 0) {
      float a = 0.f;
      for (int i = 0; i < kThr / 32; ++i) a += ws[i];
      dsum[blockIdx.y * gridDim.x + blockIdx.x] = a;
    }
  }
}

__global__ void loss_reduce_kernel(const float* __restrict__ bsum, int nb, const float* __restrict__ dsum,
                                   int nd, int W, int H, gs_loss_weights wt, int has_depth,
                                   float* __restrict__ losses) {
  __shared__ double red[3][1024];
  // per-thread partial sums in FP32 (a few dozen terms each), the tree in FP64
  float a = 0.f, b = 0.f, d = 0.f;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    a += bsum[2 * i];
    b += bsum[2 * i + 1];
  }
  if (has_depth)
    for (int i = threadIdx.x; i < nd; i += blockDim.x) d += dsum[i];
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  red[2][threadIdx.x] = d;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[0][threadIdx.x] += red[0][threadIdx.x + s];
      red[1][threadIdx.x] += red[1][threadIdx.x + s];
      red[2][threadIdx.x] += red[2][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double n3 = 3.0 * (double)W * (double)H;
    const double l1 = red[0][0] / n3, ss = red[1][0] / n3;
    const double ld = has_depth ? red[2][0] / ((double)W * H) : 0.0;
    losses[0] = (float)l1;
    losses[1] = (float)ss;
    losses[2] = (float)ld;
    losses[3] = (float)(wt.w_l1 * l1 + wt.w_ssim * (1.0 - ss) + wt.w_depth * ld);
  }
}

}  // namespace

size_t loss_tmp_floats(int W, int H) {
  const size_t gx = div_up(W, kT), gy = div_up(H, kT);
  return 9 * (size_t)W * H + 2 * 3 * gx * gy + gx * gy + 64;
}

cudaError_t launch_loss(int W, int H, const float* out, const float* tgt, const float* tinv,
                        const gs_loss_weights& w, float* adj_total, float* adj_ssim,
                        float* adj_l1, float* losses, float* tmp, cudaStream_t st) {
  Gauss g;
  double s = 0.0, e[2 * kR + 1];
  for (int i = 0; i < 2 * kR + 1; ++i) {
    e[i] = exp(-((i - kR) * (i - kR)) / (2.0 * 1.5 * 1.5));
    s += e[i];
  }
  for (int i = 0; i < 2 * kR + 1; ++i) g.w[i] = (float)(e[i] / s);
  const unsigned gx = div_up(W, kT), gy = div_up(H, kT);
  float* part = tmp;
  float* bsum = tmp + 9 * (size_t)W * H;
  float* dsum = bsum + 2 * 3 * (size_t)gx * gy;
  const dim3 grid(gx, gy, 3);
  ProfScope ps(kProfLoss, st);
  count_launch(3);
  ssim_fwd_kernel<<<grid, kThr, 0, st>>>(W, H, out, tgt, g, part, bsum);
  ssim_bwd_kernel<<<grid, kThr, 0, st>>>(W, H, out, tgt, tinv, g, w, part, adj_total, adj_ssim,
                                        adj_l1, dsum);
  loss_reduce_kernel<<<1, 1024, 0, st>>>(bsum, 3 * gx * gy, dsum, gx * gy, W, H, w, tinv != nullptr,
                                        losses);
  return cudaGetLastError();
}

}  // namespace gs2d

// ---------------------------------------------------------------------------
// Loss without any device allocation (gs_loss_noalloc).
//
// Some callers cannot allocate device memory at the moment they need the
// loss: a renderer or trainer that runs under an external memory manager
// which owns every byte of the GPU (allocating behind its back would break
// its budget), a real-time loop where an allocation's latency or possible
// failure is not acceptable, or a host that hands this library a device it
// may only compute on.  For them the loss's scratch (the SSIM partial maps
// and the per-block sums) lives in one fixed array in this file, sized for
// images of up to kNoAllocMaxPixels pixels with sides up to kNoAllocMaxSide.
// Every GPU that loads the library reserves it (about 9.5 MB) until the
// process exits.  Every call uses the same array, so calls whose work can
// overlap on the GPU (different streams, or different host threads) race.
namespace gs2d {
namespace {

constexpr int kNoAllocMaxPixels = 512 * 512;
constexpr int kNoAllocMaxSide = 4096;
// per-block sums: at most HW/256 + (W + H)/16 + 1 blocks (an upper bound
// for the loss kernels' 32 x 32 tiles as well)
constexpr size_t kNoAllocTiles = kNoAllocMaxPixels / 256 + (2 * kNoAllocMaxSide) / 16 + 1;
constexpr size_t kNoAllocFloats = 9 * (size_t)kNoAllocMaxPixels + 7 * kNoAllocTiles + 64;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) float g_noalloc_loss_scratch[kNoAllocFloats];

std::mutex g_noalloc_mu;
float* g_noalloc_addr[kNoAllocMaxDevices] = {};

}  // namespace
}  // namespace gs2d

extern "C" gs_status gs_loss_noalloc(int32_t W, int32_t H, const float* out, const float* tgt,
                                     const float* tinv, const gs_loss_weights* w, float* adj_total,
                                     float* adj_ssim, float* adj_l1, float* losses, void* stream) {
  using namespace gs2d;
  if (W <= 0 || H <= 0 || !out || !tgt || !w || !adj_total || !losses) {
    set_last_error("gs_loss_noalloc: bad argument");
    return GS_ERR_ARG;
  }
  if ((int64_t)W * H > kNoAllocMaxPixels || W > kNoAllocMaxSide || H > kNoAllocMaxSide ||
      loss_tmp_floats(W, H) > kNoAllocFloats) {
    set_last_error(("gs_loss_noalloc: image " + std::to_string(W) + "x" + std::to_string(H) +
                    " exceeds the fixed scratch (at most " + std::to_string(kNoAllocMaxPixels) +
                    " pixels, sides up to " + std::to_string(kNoAllocMaxSide) + "); use gs_loss")
                       .c_str());
    return GS_ERR_CAPACITY;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
    set_last_error("gs_loss_noalloc: no usable current device");
    return GS_ERR_CUDA;
  }
  float* scratch = nullptr;
  {
    // once per device, with that device current: the device address of the
    // scratch array (its name in host code is only a host-side handle)
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_loss_scratch);
      if (e != cudaSuccess || !ptr) {
        set_last_error((std::string("gs_loss_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
        return GS_ERR_CUDA;
      }
      g_noalloc_addr[dev] = static_cast<float*>(ptr);
    }
    scratch = g_noalloc_addr[dev];
  }
  // Nothing in the scratch must start at zero: every partial map entry and
  // per-block sum the kernels read is written earlier in the same call.
  e = launch_loss(W, H, out, tgt, tinv, *w, adj_total, adj_ssim, adj_l1, losses, scratch,
                  (cudaStream_t)stream);
  if (e != cudaSuccess) {
    set_last_error((std::string("gs_loss_noalloc: ") + cudaGetErrorString(e)).c_str());
    return GS_ERR_CUDA;
  }
  return GS_OK;
}
