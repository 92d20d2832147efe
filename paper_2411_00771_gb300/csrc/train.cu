// Training-loop kernels beyond the rasterizer: the geometric terms of the
// loss (depth-normal consistency, depth distortion) and the Adam update.
//
// Normal consistency (2DGS's surface smoothness term, weight 0.0125 in
// Sec. 5.1): per pixel L = A - N~ . N_r, where A is the rendered alpha, N_r the
// rendered (weight-summed) normal and N~ the unit normal of the surface seen
// at the pixel: the cross product of the central differences of the points
// P = median depth * ray of its four neighbours, turned towards the camera.
// Interior pixels whose four neighbours have a depth and a non-degenerate
// cross product count; the loss is weight * mean over all pixels.  The depth
// distortion term (2DGS's, weight 0 in Sec. 5.1) is its weight times the mean
// of the rendered distortion plane.  Pass 1
// (per pixel) adds the adjoints of A and N_r at the pixel and writes the
// adjoint of each neighbour's depth; pass 2 (per pixel) gathers the depth
// adjoint from the four pixels whose stencil holds it.
//
// Adam: the usual bias-corrected update, in FP32, one thread per element.
// Densification and the activations of the trained parametrisation follow.
#include <math.h>

#include "gs2d_internal.cuh"

namespace gs2d {
namespace {

constexpr int kBx = 32, kBy = 8;

struct Ray {
  float fx, fy, cx, cy;
  __device__ __forceinline__ float3 at(int i, int j) const {
    return make_float3(((float)i + 0.5f - cx) / fx, ((float)j + 0.5f - cy) / fy, 1.f);
  }
};

__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 mul3(float3 a, float s) { return make_float3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dot3f(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3f(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__global__ void __launch_bounds__(kBx* kBy) normal_pass1(int W, int H, Ray rc, const float* __restrict__ out,
                                                         float s, float* __restrict__ adj,
                                                         float4* __restrict__ part, float* __restrict__ bsum) {
  const int i = blockIdx.x * kBx + threadIdx.x, j = blockIdx.y * kBy + threadIdx.y;
  const size_t HW = (size_t)W * H;
  float L = 0.f;
  float4 pt = make_float4(0.f, 0.f, 0.f, 0.f);  // depth adjoints of the right, left, lower, upper neighbours
  if (i > 0 && j > 0 && i < W - 1 && j < H - 1) {
    const float* med = out + 6 * HW;
    const float dr = med[(size_t)j * W + i + 1], dl = med[(size_t)j * W + i - 1];
    const float dd = med[(size_t)(j + 1) * W + i], du = med[(size_t)(j - 1) * W + i];
    if (dr > 0.f && dl > 0.f && dd > 0.f && du > 0.f) {
      const float3 rr = rc.at(i + 1, j), rl = rc.at(i - 1, j), rd = rc.at(i, j + 1), ru = rc.at(i, j - 1);
      const float3 a = sub3(mul3(rr, dr), mul3(rl, dl));
      const float3 b = sub3(mul3(rd, dd), mul3(ru, du));
      const float3 c = cross3f(a, b);
      const float cn = sqrtf(dot3f(c, c));
      if (cn > 0.f) {
        const size_t p = (size_t)j * W + i;
        const float sg = dot3f(c, rc.at(i, j)) > 0.f ? -1.f : 1.f;
        const float ic = 1.f / cn;
        const float3 ch = mul3(c, ic);
        const float3 n = mul3(ch, sg);
        const float3 N = make_float3(out[7 * HW + p], out[8 * HW + p], out[9 * HW + p]);
        L = out[3 * HW + p] - dot3f(n, N);
        adj[3 * HW + p] += s;
        adj[7 * HW + p] -= s * n.x;
        adj[8 * HW + p] -= s * n.y;
        adj[9 * HW + p] -= s * n.z;
        // d(-n.N)/dc = -sg (I - ch ch^T) N / |c|
        const float cN = dot3f(ch, N);
        const float3 gc = mul3(sub3(N, mul3(ch, cN)), -sg * ic * s);
        const float3 ga = cross3f(b, gc), gb = cross3f(gc, a);
        pt = make_float4(dot3f(rr, ga), -dot3f(rl, ga), dot3f(rd, gb), -dot3f(ru, gb));
      }
    }
  }
  if (i < W && j < H) part[(size_t)j * W + i] = pt;
  // block sum of the loss terms
  const int t = threadIdx.y * kBx + threadIdx.x;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) L += __shfl_xor_sync(0xffffffffu, L, o);
  __shared__ float ws[kBx * kBy / 32];
  if ((t & 31) == 0) ws[t >> 5] = L;
  __syncthreads();
  if (t == 0) {
    float a = 0.f;
    for (int k = 0; k < kBx * kBy / 32; ++k) a += ws[k];
    bsum[blockIdx.y * gridDim.x + blockIdx.x] = a;
  }
}

// Pass 2: the depth adjoint gathered from the four stencils that hold the
// pixel, and the distortion term's constant adjoint (wd = its weight / (W H)).
__global__ void __launch_bounds__(kBx* kBy) normal_pass2(int W, int H, const float4* __restrict__ part, float wd,
                                                         const float* __restrict__ out, float* __restrict__ adj,
                                                         float* __restrict__ dsum) {
  const int i = blockIdx.x * kBx + threadIdx.x, j = blockIdx.y * kBy + threadIdx.y;
  const size_t HW = (size_t)W * H;
  float dv = 0.f;
  if (i < W && j < H && wd != 0.f) {
    adj[10 * HW + (size_t)j * W + i] += wd;
    dv = out[10 * HW + (size_t)j * W + i];
  }
  if (dsum) {
    const int t = threadIdx.y * kBx + threadIdx.x;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dv += __shfl_xor_sync(0xffffffffu, dv, o);
    __shared__ float ws[kBx * kBy / 32];
    if ((t & 31) == 0) ws[t >> 5] = dv;
    __syncthreads();
    if (t == 0) {
      float a = 0.f;
      for (int k = 0; k < kBx * kBy / 32; ++k) a += ws[k];
      dsum[blockIdx.y * gridDim.x + blockIdx.x] = a;
    }
  }
  if (i >= W || j >= H) return;
  float g = 0.f;
  if (i > 0) g += part[(size_t)j * W + i - 1].x;      // I am the right neighbour of (i-1, j)
  if (i < W - 1) g += part[(size_t)j * W + i + 1].y;  // the left neighbour of (i+1, j)
  if (j > 0) g += part[(size_t)(j - 1) * W + i].z;    // the lower neighbour of (i, j-1)
  if (j < H - 1) g += part[(size_t)(j + 1) * W + i].w;
  if (g != 0.f) adj[6 * (size_t)W * H + (size_t)j * W + i] += g;
}

// loss[0] = normal term, loss[1] = distortion term (block sums reduced in double)
__global__ void normal_reduce(const float* __restrict__ bsum, const float* __restrict__ dsum, int nb, double sn,
                              double sd, float* __restrict__ loss) {
  __shared__ double red[2][256];
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) {
    a += bsum[k];
    b += dsum[k];
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    loss[0] = (float)(red[0][0] * sn);
    loss[1] = (float)(red[1][0] * sd);
  }
}

struct AdamK {
  float lr, b1, b2, eps, bc1, bc2;
};
__device__ __forceinline__ void adam_one(float& p, float g, float& m, float& v, const AdamK& k) {
  m = fmaf(k.b1, m, (1.f - k.b1) * g);
  v = fmaf(k.b2, v, (1.f - k.b2) * g * g);
  p -= k.lr * (m / k.bc1) / (sqrtf(v / k.bc2) + k.eps);
}
__global__ void adam_kernel(int64_t n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, AdamK k) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    adam_one(p[i], g[i], m[i], v[i], k);
}
// The same update four values at a time (all arrays 16-byte aligned; n4 = n / 4).
__global__ void adam4_kernel(int64_t n4, float4* __restrict__ p, const float4* __restrict__ g, float4* __restrict__ m,
                             float4* __restrict__ v, AdamK k) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    float4 pi = p[i], mi = m[i], vi = v[i];
    const float4 gi = g[i];
    adam_one(pi.x, gi.x, mi.x, vi.x, k);
    adam_one(pi.y, gi.y, mi.y, vi.y, k);
    adam_one(pi.z, gi.z, mi.z, vi.z, k);
    adam_one(pi.w, gi.w, mi.w, vi.w, k);
    p[i] = pi;
    m[i] = mi;
    v[i] = vi;
  }
}

}  // namespace

size_t geometry_tmp_bytes(int W, int H) {
  const size_t nb = (size_t)div_up(W, kBx) * div_up(H, kBy);
  return sizeof(float4) * (size_t)W * H + 2 * sizeof(float) * nb;
}

cudaError_t launch_geometry_loss(int W, int H, float fx, float fy, float cx, float cy, const float* out,
                                 float w_normal, float w_dist, float* adj, float* loss, void* tmp, cudaStream_t st) {
  const dim3 blk(kBx, kBy), grid(div_up(W, kBx), div_up(H, kBy));
  const int nb = (int)(grid.x * grid.y);
  float4* part = static_cast<float4*>(tmp);
  float* bsum = reinterpret_cast<float*>(part + (size_t)W * H);
  float* dsum = bsum + nb;
  const Ray rc{fx, fy, cx, cy};
  const double hw = (double)W * H;
  ProfScope ps(kProfLoss, st);
  count_launch(3);
  normal_pass1<<<grid, blk, 0, st>>>(W, H, rc, out, (float)(w_normal / hw), adj, part, bsum);
  normal_pass2<<<grid, blk, 0, st>>>(W, H, part, (float)(w_dist / hw), out, adj, dsum);
  normal_reduce<<<1, 256, 0, st>>>(bsum, dsum, nb, w_normal / hw, w_dist / hw, loss);
  return cudaGetLastError();
}

cudaError_t launch_adam(int64_t n, float* p, const float* g, float* m, float* v, float lr, float b1, float b2,
                        float eps, float bc1, float bc2, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const AdamK k{lr, b1, b2, eps, bc1, bc2};
  const bool vec = (((uintptr_t)p | (uintptr_t)g | (uintptr_t)m | (uintptr_t)v) & 15u) == 0;
  const int64_t n4 = vec ? n / 4 : 0;
  if (n4 > 0) {
    const int64_t b = (n4 + 255) / 256;
    count_launch();
    adam4_kernel<<<(unsigned)(b < 2432 ? b : 2432), 256, 0, st>>>(n4, reinterpret_cast<float4*>(p),
                                                                  reinterpret_cast<const float4*>(g),
                                                                  reinterpret_cast<float4*>(m),
                                                                  reinterpret_cast<float4*>(v), k);
  }
  const int64_t rest = n - 4 * n4;
  if (rest > 0) {
    const int64_t b = (rest + 255) / 256;
    count_launch();
    adam_kernel<<<(unsigned)(b < 2432 ? b : 2432), 256, 0, st>>>(rest, p + 4 * n4, g + 4 * n4, m + 4 * n4,
                                                                 v + 4 * n4, k);
  }
  return cudaGetLastError();
}

}  // namespace gs2d

// ---------------------------------------------------------------------------
// Densification (the clone / split / prune of the training schedule the paper
// keeps from CityGaussian, Sec. 5.1, with the selection of Eq. 2 and the
// elongation filter of Sec. 3.2):
//   action 0  drop   (opacity below min_opacity, or a split parent),
//          1  keep,
//          2  clone  (selected, max scale <= dense_thr): itself, then a copy,
//          3  split  (selected, max scale >  dense_thr): two children at
//                    mu + t_u s_u xi_0 + t_v s_v xi_1 (t_u, t_v the surfel's
//                    tangents, xi standard normals given per child), scales
//                    s / 1.6, the rest copied; the parent is dropped.
// Output rows follow the source order (a surfel's rows are contiguous).

namespace gs2d {
namespace {

__global__ void densify_plan_kernel(int64_t n, const uint8_t* __restrict__ sel, const uint8_t* __restrict__ keep,
                                    const float* __restrict__ scale, const float* __restrict__ opac, float dense_thr,
                                    float min_opacity, uint8_t* __restrict__ action, uint32_t* __restrict__ rows) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint8_t a;
    if (sel[i] && (!keep || keep[i])) a = fmaxf(scale[2 * i], scale[2 * i + 1]) <= dense_thr ? 2 : 3;
    else a = opac[i] < min_opacity ? 0 : 1;
    action[i] = a;
    rows[i] = a == 0 ? 0u : (a == 1 ? 1u : 2u);
  }
}

__global__ void densify_apply_kernel(int64_t n, int K3, bool log_scale, const uint8_t* __restrict__ action,
                                     const uint32_t* __restrict__ off, const float* __restrict__ xi,
                                     const float* __restrict__ mu, const float* __restrict__ quat,
                                     const float* __restrict__ scale, const float* __restrict__ opac,
                                     const float* __restrict__ sh, float* __restrict__ mu_o,
                                     float* __restrict__ quat_o, float* __restrict__ scale_o,
                                     float* __restrict__ opac_o, float* __restrict__ sh_o, int32_t* __restrict__ src,
                                     uint8_t* __restrict__ fresh) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t a = action[i];
    if (a == 0) continue;
    const int nr = a == 1 ? 1 : 2;
    const int64_t r0 = off[i];
    // tangents of the surfel (first two columns of its rotation)
    float qw = quat[4 * i], qx = quat[4 * i + 1], qy = quat[4 * i + 2], qz = quat[4 * i + 3];
    const float iq = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    qw *= iq; qx *= iq; qy *= iq; qz *= iq;
    const float tu[3] = {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy + qw * qz), 2.f * (qx * qz - qw * qy)};
    const float tv[3] = {2.f * (qx * qy - qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz + qw * qx)};
    for (int c = 0; c < nr; ++c) {
      const int64_t r = r0 + c;
      const bool child = a == 3;
      float su = scale[2 * i], sv = scale[2 * i + 1];  // activated or log-scales
      const float au = log_scale ? expf(su) : su, av = log_scale ? expf(sv) : sv;
      for (int k = 0; k < 3; ++k) {
        float m = mu[3 * i + k];
        if (child) m += tu[k] * au * xi[4 * i + 2 * c] + tv[k] * av * xi[4 * i + 2 * c + 1];
        mu_o[3 * r + k] = m;
      }
      if (child) {
        if (log_scale) {
          su -= 0.47000362924573558f;  // ln 1.6
          sv -= 0.47000362924573558f;
        } else {
          su /= 1.6f;
          sv /= 1.6f;
        }
      }
      scale_o[2 * r] = su;
      scale_o[2 * r + 1] = sv;
      for (int k = 0; k < 4; ++k) quat_o[4 * r + k] = quat[4 * i + k];
      opac_o[r] = opac[i];
      for (int k = 0; k < K3; ++k) sh_o[(size_t)K3 * r + k] = sh[(size_t)K3 * i + k];
      src[r] = (int32_t)i;
      fresh[r] = (a == 3 || (a == 2 && c == 1)) ? 1u : 0u;
    }
  }
}

__global__ void gather_rows_kernel(int64_t n_out, int width, const int32_t* __restrict__ src,
                                   const uint8_t* __restrict__ fresh, const float* __restrict__ in,
                                   float* __restrict__ out) {
  const int64_t total = n_out * width;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / width;
    const int k = (int)(e - r * width);
    out[e] = (fresh && fresh[r]) ? 0.f : in[(size_t)src[r] * width + k];
  }
}

// Activations of the trained parametrisation: scale = exp(log-scale),
// opacity = sigmoid(logit); and the chain of their gradients, in place.
__global__ void activate_kernel(int64_t n, const float* __restrict__ ls, const float* __restrict__ lo,
                                float* __restrict__ scale, float* __restrict__ opac) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    scale[2 * i] = expf(ls[2 * i]);
    scale[2 * i + 1] = expf(ls[2 * i + 1]);
    opac[i] = 1.f / (1.f + expf(-lo[i]));
  }
}

__global__ void activate_grad_kernel(int64_t n, const float* __restrict__ scale, const float* __restrict__ opac,
                                     float* __restrict__ gs, float* __restrict__ go) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    gs[2 * i] *= scale[2 * i];
    gs[2 * i + 1] *= scale[2 * i + 1];
    go[i] *= opac[i] * (1.f - opac[i]);
  }
}

unsigned grid_of(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 2432 ? 2432 : b));
}

}  // namespace

cudaError_t launch_densify_plan(int64_t n, const uint8_t* sel, const uint8_t* keep, const float* scale,
                                const float* opac, float dense_thr, float min_opacity, uint8_t* action, uint32_t* rows,
                                cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  ProfScope ps(kProfDensify, st);
  count_launch();
  densify_plan_kernel<<<grid_of(n), 256, 0, st>>>(n, sel, keep, scale, opac, dense_thr, min_opacity, action, rows);
  return cudaGetLastError();
}

cudaError_t launch_densify_apply(int64_t n, int sh_degree, bool log_scale, const uint8_t* action, const uint32_t* off,
                                 const float* xi, const float* mu, const float* quat, const float* scale,
                                 const float* opac, const float* sh, float* mu_o, float* quat_o, float* scale_o,
                                 float* opac_o, float* sh_o, int32_t* src, uint8_t* fresh, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  ProfScope ps(kProfDensify, st);
  count_launch();
  const int K3 = (sh_degree + 1) * (sh_degree + 1) * 3;
  densify_apply_kernel<<<grid_of(n), 256, 0, st>>>(n, K3, log_scale, action, off, xi, mu, quat, scale, opac, sh, mu_o, quat_o,
                                                   scale_o, opac_o, sh_o, src, fresh);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(int64_t n_out, int width, const int32_t* src, const uint8_t* fresh, const float* in,
                               float* out, cudaStream_t st) {
  if (n_out <= 0 || width <= 0) return cudaSuccess;
  count_launch();
  gather_rows_kernel<<<grid_of(n_out * width), 256, 0, st>>>(n_out, width, src, fresh, in, out);
  return cudaGetLastError();
}

cudaError_t launch_activate(int64_t n, const float* ls, const float* lo, float* scale, float* opac, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  count_launch();
  activate_kernel<<<grid_of(n), 256, 0, st>>>(n, ls, lo, scale, opac);
  return cudaGetLastError();
}

cudaError_t launch_activate_grad(int64_t n, const float* scale, const float* opac, float* gs, float* go,
                                 cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  count_launch();
  activate_grad_kernel<<<grid_of(n), 256, 0, st>>>(n, scale, opac, gs, go);
  return cudaGetLastError();
}

}  // namespace gs2d
