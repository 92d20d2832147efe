// Per-pixel compositing (forward) and its adjoint (reverse replay).
//
// Forward (Eq. 1, Sec. 3.1, with the 2DGS surfel model and the low-pass
// filter of Sec. 3.2): one CTA per 16 x 16 tile, one thread per pixel.  The
// tile's depth-sorted surfel list is staged through shared memory in
// batches of 256 records; each pixel intersects its ray with every surfel
// plane (rho_obj), takes the screen-space filter (rho_scr) where smaller,
// and composites front to back until the transmittance would drop below
// T_min.  Colour, alpha, expected and inverse depth, median depth, normal
// and the depth-distortion sum are accumulated in registers.
//
// Backward: the same tiles replay each pixel's list back to front from the
// final transmittance, T_before = T_after / (1 - alpha), with suffix sums
// for d L / d alpha.  Per-pair gradients are reduced across each warp with a
// reduce-scatter of shuffles, summed per tile in shared memory, and added
// to global memory once per (surfel, tile).
#include <math.h>

#include "gs2d_internal.cuh"

namespace gs2d {
namespace {

struct Pair {
  float dx, dy;    // pixel offset from the projected centre
  float nu, nv;    // Ji d
  float rden;      // 1 / (1 + e.d)
  float rho;       // min(rho_obj, rho_scr)
  float G;         // exp(-rho / 2)
  float alpha;     // min(alpha_max, o G)
  bool obj;        // object-space branch
  bool hit;        // rho <= rho_max and alpha >= alpha_min
};

// Shared by both blends; written with explicit round-to-nearest intrinsics
// so that forward and backward take bit-identical decisions.
__device__ __forceinline__ Pair eval_pair(float px, float py, float4 r0, float4 r1, float4 r2,
                                          const SetDev& set) {
  Pair q;
  q.dx = __fsub_rn(__fsub_rn(px, r0.x), r0.z);
  q.dy = __fsub_rn(__fsub_rn(py, r0.y), r0.w);
  const float den = __fmaf_rn(r2.x, q.dx, __fmaf_rn(r2.y, q.dy, 1.0f));
  q.nu = __fmaf_rn(r1.x, q.dx, __fmul_rn(r1.y, q.dy));
  q.nv = __fmaf_rn(r1.z, q.dx, __fmul_rn(r1.w, q.dy));
  q.rden = __frcp_rn(den);
  const float u = __fmul_rn(q.nu, q.rden), v = __fmul_rn(q.nv, q.rden);
  const float rho_obj = den > 0.f ? __fmaf_rn(u, u, __fmul_rn(v, v)) : INFINITY;
  const float rho_scr = __fmul_rn(set.sinv, __fmaf_rn(q.dx, q.dx, __fmul_rn(q.dy, q.dy)));
  q.obj = rho_obj <= rho_scr;  // false for NaN (edge-on disks)
  q.rho = q.obj ? rho_obj : rho_scr;
  q.G = __expf(__fmul_rn(-0.5f, q.rho));
  q.alpha = fminf(set.alpha_max, __fmul_rn(r2.w, q.G));
  q.hit = (q.rho <= set.rho_max) && (q.alpha >= set.alpha_min);
  return q;
}

__global__ void __launch_bounds__(kBlock) blend_fwd_kernel(
    CamDev cam, SetDev set, const float4* __restrict__ rec, const uint32_t* __restrict__ vals,
    const int2* __restrict__ ranges, float* __restrict__ out, int32_t* __restrict__ n_contrib,
    int32_t* __restrict__ last, int32_t* __restrict__ med, unsigned long long* __restrict__ counters) {
  __shared__ float4 s0[kBlock], s1[kBlock], s2[kBlock], s3[kBlock], s4[kBlock];
  const int tile = blockIdx.y * cam.tiles_x + blockIdx.x;
  const int px = blockIdx.x * kTile + (threadIdx.x & (kTile - 1));
  const int py = blockIdx.y * kTile + (threadIdx.x >> 4);
  const bool inside = px < cam.W && py < cam.H;
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
  const int2 rg = ranges[tile];
  const int len = rg.y - rg.x;
  bool done = !inside;
  // Z is accumulated relative to zr, the depth of the first blended pair:
  // sum w (z - zr) keeps the distortion terms z A - Z free of the
  // cancellation between depths of hundreds of metres (both are invariant
  // under a common shift of z), and sum w z = sum w (z - zr) + zr A.
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, A = 0.f, Zs = 0.f, zr = 0.f, I = 0.f;
  float N0 = 0.f, N1 = 0.f, N2 = 0.f, D = 0.f, M = 0.f;
  int cnt = 0, lastpos = 0, medpos = -1;
  unsigned evaluated = 0;
  for (int b0 = 0; b0 < len; b0 += kBlock) {
    if (__syncthreads_count(done) == kBlock) break;
    const int j = b0 + threadIdx.x;
    if (j < len) {
      const float4* R = rec + (size_t)vals[rg.x + j] * kRecF4;
      s0[threadIdx.x] = R[0];
      s1[threadIdx.x] = R[1];
      s2[threadIdx.x] = R[2];
      s3[threadIdx.x] = R[3];
      s4[threadIdx.x] = R[4];
    }
    __syncthreads();
    const int nb = min(kBlock, len - b0);
    for (int k = 0; k < nb && !done; ++k) {
      ++evaluated;
      const float4 r2 = s2[k];
      const Pair q = eval_pair(fx, fy, s0[k], s1[k], r2, set);
      if (!q.hit) continue;
      const float Tn = T * (1.f - q.alpha);
      if (Tn < set.T_min) {
        done = true;
        break;
      }
      const float w = q.alpha * T;
      const float z = q.obj ? r2.z * q.rden : r2.z;
      const float4 r3 = s3[k], r4 = s4[k];
      C0 = fmaf(w, r3.x, C0);
      C1 = fmaf(w, r3.y, C1);
      C2 = fmaf(w, r3.z, C2);
      if (cnt == 0) zr = z;
      const float zs = z - zr;
      D = fmaf(2.f * w, fmaf(zs, A, -Zs), D);
      A += w;
      Zs = fmaf(w, zs, Zs);
      I += w / z;
      N0 = fmaf(w, r3.w, N0);
      N1 = fmaf(w, r4.x, N1);
      N2 = fmaf(w, r4.y, N2);
      if (T > 0.5f) {
        M = z;
        medpos = b0 + k;
      }
      T = Tn;
      ++cnt;
      lastpos = b0 + k + 1;
    }
  }
  if (inside) {
    const size_t HW = (size_t)cam.W * cam.H;
    const size_t p = (size_t)py * cam.W + px;
    out[p] = C0 + T * set.bg[0];
    out[HW + p] = C1 + T * set.bg[1];
    out[2 * HW + p] = C2 + T * set.bg[2];
    out[3 * HW + p] = A;
    out[4 * HW + p] = fmaf(zr, A, Zs);
    out[5 * HW + p] = I;
    out[6 * HW + p] = M;
    out[7 * HW + p] = N0;
    out[8 * HW + p] = N1;
    out[9 * HW + p] = N2;
    out[10 * HW + p] = D;
    out[11 * HW + p] = T;
    if (n_contrib) n_contrib[p] = cnt;
    if (last) last[p] = lastpos;
    if (med) med[p] = medpos;
  }
  if (counters) {
    // per-tile totals of evaluated and blended pairs (performance counters)
    __shared__ unsigned long long tot[2];
    if (threadIdx.x == 0) tot[0] = tot[1] = 0ull;
    __syncthreads();
    unsigned e = evaluated, c = (unsigned)cnt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, o);
      c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&tot[0], (unsigned long long)e);
      atomicAdd(&tot[1], (unsigned long long)c);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      atomicAdd(&counters[0], tot[0]);
      atomicAdd(&counters[1], tot[1]);
    }
  }
}

// ---------------------------------------------------------------------------
// Backward.

constexpr int kSlots = 32;  // padded length of the per-pair gradient vector
constexpr int kMaxSets = 3;
// gradient vector layout: [0..15] per-surfel record, [16 + 2 s, 17 + 2 s]
// screen-space gradient of set s
constexpr int kAcc = kGradRec + 2 * kMaxSets;  // 22

// Sum of v[q] over the warp for every q; afterwards lane q holds the sum of
// slot q.  31 shuffles for 32 slots (reduce-scatter by halving).
__device__ __forceinline__ float warp_reduce_scatter(float (&v)[kSlots]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const float send = up ? v[i] : v[i + o];
      const float keep = up ? v[i + o] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0];
}

__global__ void __launch_bounds__(kBlock) blend_bwd_kernel(
    CamDev cam, SetDev set, const float4* __restrict__ rec, const uint32_t* __restrict__ vals,
    const int2* __restrict__ ranges, const float* __restrict__ out, const int32_t* __restrict__ last,
    const int32_t* __restrict__ med, AdjDev adj, float* __restrict__ grec,
    float* __restrict__ screen, int n, unsigned long long* __restrict__ counters) {
  __shared__ float4 s0[kBlock], s1[kBlock], s2[kBlock], s3[kBlock], s4[kBlock];
  __shared__ uint32_t sid[kBlock];
  __shared__ float acc[kBlock][kAcc + 1];
  __shared__ int smax;
  const int tile = blockIdx.y * cam.tiles_x + blockIdx.x;
  const int px = blockIdx.x * kTile + (threadIdx.x & (kTile - 1));
  const int py = blockIdx.y * kTile + (threadIdx.x >> 4);
  const bool inside = px < cam.W && py < cam.H;
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
  const int2 rg = ranges[tile];
  const size_t HW = (size_t)cam.W * cam.H;
  const size_t p = inside ? (size_t)py * cam.W + px : 0;
  const int lane = threadIdx.x & 31;
  const int nsets = adj.n_sets;

  int lastpos = 0, medpos = -1;
  float T = 1.f, A = 0.f, Z = 0.f, Af = 0.f, Zf = 0.f;
  float gC[kMaxSets][3];
  float gA = 0.f, gZ = 0.f, gI = 0.f, gMed = 0.f, gD = 0.f, gN0 = 0.f, gN1 = 0.f, gN2 = 0.f;
  float S[kMaxSets];
#pragma unroll
  for (int s = 0; s < kMaxSets; ++s) {
    gC[s][0] = gC[s][1] = gC[s][2] = 0.f;
    S[s] = 0.f;
  }
  if (inside) {
    lastpos = last[p];
    medpos = med[p];
    T = out[11 * HW + p];
    Af = A = out[3 * HW + p];
    Zf = Z = out[4 * HW + p];
#pragma unroll
    for (int s = 0; s < kMaxSets; ++s) {
      if (s >= nsets) break;
      const float* a = adj.set[s];
      const uint32_t m = adj.mask[s];
#pragma unroll
      for (int c = 0; c < 3; ++c) gC[s][c] = (m >> c) & 1u ? a[c * HW + p] : 0.f;
      S[s] = T * (gC[s][0] * set.bg[0] + gC[s][1] * set.bg[1] + gC[s][2] * set.bg[2]);
    }
    const float* a = adj.set[0];
    const uint32_t m = adj.mask[0];
    if (m & (1u << 3)) gA = a[3 * HW + p];
    if (m & (1u << 4)) gZ = a[4 * HW + p];
    if (m & (1u << 5)) gI = a[5 * HW + p];
    if (m & (1u << 6)) gMed = a[6 * HW + p];
    if (m & (1u << 7)) gN0 = a[7 * HW + p];
    if (m & (1u << 8)) gN1 = a[8 * HW + p];
    if (m & (1u << 9)) gN2 = a[9 * HW + p];
    if (m & (1u << 10)) gD = a[10 * HW + p];
  }
  if (threadIdx.x == 0) smax = 0;
  __syncthreads();
  atomicMax(&smax, lastpos);
  __syncthreads();
  const int maxlast = smax;
  unsigned replayed = 0;

  for (int bend = maxlast; bend > 0; bend -= kBlock) {
    const int b0 = bend > kBlock ? bend - kBlock : 0;
    const int nb = bend - b0;
    __syncthreads();
    if (threadIdx.x < nb) {
      const uint32_t s = vals[rg.x + b0 + threadIdx.x];
      sid[threadIdx.x] = s;
      const float4* R = rec + (size_t)s * kRecF4;
      s0[threadIdx.x] = R[0];
      s1[threadIdx.x] = R[1];
      s2[threadIdx.x] = R[2];
      s3[threadIdx.x] = R[3];
      s4[threadIdx.x] = R[4];
    }
    for (int i = threadIdx.x; i < nb * (kAcc + 1); i += kBlock) (&acc[0][0])[i] = 0.f;
    __syncthreads();
    for (int kk = nb - 1; kk >= 0; --kk) {
      const int k = b0 + kk;
      Pair q;
      q.hit = false;
      const float4 r1 = s1[kk], r2 = s2[kk];
      if (k < lastpos) {
        ++replayed;
        q = eval_pair(fx, fy, s0[kk], r1, r2, set);
      }
      const bool contrib = q.hit;
      if (__ballot_sync(0xffffffffu, contrib) == 0u) continue;
      float v[kSlots];
#pragma unroll
      for (int i = 0; i < kSlots; ++i) v[i] = 0.f;
      {
        if (contrib) {
          const float4 r3 = s3[kk], r4 = s4[kk];
          const float om = 1.f - q.alpha;
          const float rom = 1.f / om;
          T = T * rom;  // transmittance before this pair
          const float w = q.alpha * T;
          const float z = q.obj ? r2.z * q.rden : r2.z;
          const float Ap = A - w, Zp = Z - w * z;
          const float dDdw = 2.f * (z * Ap - Zp + (Zf - Z) - z * (Af - A));
          const float rz = 1.f / z;
          const float dLdw = gC[0][0] * r3.x + gC[0][1] * r3.y + gC[0][2] * r3.z + gA + gZ * z +
                             gI * rz + gN0 * r3.w + gN1 * r4.x + gN2 * r4.y + gD * dDdw;
          float dLda[kMaxSets];
          dLda[0] = T * dLdw - S[0] * rom;
          S[0] += w * dLdw;
#pragma unroll
          for (int s = 1; s < kMaxSets; ++s) {
            if (s < nsets) {
              const float dw = gC[s][0] * r3.x + gC[s][1] * r3.y + gC[s][2] * r3.z;
              dLda[s] = T * dw - S[s] * rom;
              S[s] += w * dw;
            } else {
              dLda[s] = 0.f;
            }
          }
          const float dzv = w * (gZ - gI * rz * rz) + gD * 2.f * w * (Ap - (Af - A)) +
                            (k == medpos ? gMed : 0.f);
          A = Ap;
          Z = Zp;
          // alpha -> rho (zero where alpha is clamped at alpha_max)
          const bool unclamped = r2.w * q.G < set.alpha_max;
          const float dadrho = unclamped ? -0.5f * r2.w * q.G : 0.f;
          const float drho = dLda[0] * dadrho;
          // d rho / d offset
          float rx, ry;
          float gdx, gdy, gpz;
          if (q.obj) {
            const float u = q.nu * q.rden, vv = q.nv * q.rden;
            const float r2d = q.rden * q.rden;
            rx = 2.f * r2d * (q.nu * r1.x + q.nv * r1.z) - 2.f * q.rho * q.rden * r2.x;
            ry = 2.f * r2d * (q.nu * r1.y + q.nv * r1.w) - 2.f * q.rho * q.rden * r2.y;
            const float dLdu = 2.f * u * drho, dLdv = 2.f * vv * drho;
            const float drden = dLdu * q.nu + dLdv * q.nv + dzv * r2.z;
            const float dnu = dLdu * q.rden, dnv = dLdv * q.rden;
            const float dden = -drden * r2d;
            v[0] = dnu * q.dx;
            v[1] = dnu * q.dy;
            v[2] = dnv * q.dx;
            v[3] = dnv * q.dy;
            v[4] = dden * q.dx;
            v[5] = dden * q.dy;
            gdx = dnu * r1.x + dnv * r1.z + dden * r2.x;
            gdy = dnu * r1.y + dnv * r1.w + dden * r2.y;
            gpz = dzv * q.rden;
          } else {
            rx = 2.f * set.sinv * q.dx;
            ry = 2.f * set.sinv * q.dy;
            gdx = drho * rx;
            gdy = drho * ry;
            gpz = dzv;
          }
          v[6] = -gdx;
          v[7] = -gdy;
          v[8] = gpz;
          v[9] = unclamped ? dLda[0] * q.G : 0.f;
          v[10] = w * gC[0][0];
          v[11] = w * gC[0][1];
          v[12] = w * gC[0][2];
          v[13] = w * gN0;
          v[14] = w * gN1;
          v[15] = w * gN2;
#pragma unroll
          for (int s = 0; s < kMaxSets; ++s) {
            const float dr = dLda[s] * dadrho;
            v[kGradRec + 2 * s] = -dr * rx;
            v[kGradRec + 2 * s + 1] = -dr * ry;
          }
        }
      }
      const unsigned ballot = __ballot_sync(0xffffffffu, contrib);
      if (ballot == 0u) continue;
      if (__popc(ballot) == 1) {
        if (contrib) {
#pragma unroll
          for (int i = 0; i < kAcc; ++i)
            if (v[i] != 0.f) atomicAdd(&acc[kk][i], v[i]);
        }
      } else {
        const float r = warp_reduce_scatter(v);
        if (lane < kAcc && r != 0.f) atomicAdd(&acc[kk][lane], r);
      }
    }
    __syncthreads();
    // flush this batch: one (surfel, tile) gradient record per entry
    if (threadIdx.x < nb) {
      const uint32_t s = sid[threadIdx.x];
      float* g = grec + (size_t)s * kGradRec;
#pragma unroll
      for (int i = 0; i < kGradRec; ++i) {
        const float x = acc[threadIdx.x][i];
        if (x != 0.f) atomicAdd(&g[i], x);
      }
      if (screen) {
        for (int st = 0; st < nsets; ++st) {
          const float x0 = acc[threadIdx.x][kGradRec + 2 * st];
          const float x1 = acc[threadIdx.x][kGradRec + 2 * st + 1];
          float* sg = screen + ((size_t)st * n + s) * 2;
          if (x0 != 0.f) atomicAdd(&sg[0], x0);
          if (x1 != 0.f) atomicAdd(&sg[1], x1);
        }
      }
    }
  }
  if (counters) {
    unsigned e = replayed;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if (lane == 0) atomicAdd(&counters[2], (unsigned long long)e);
  }
}

}  // namespace

cudaError_t launch_blend_fwd(const CamDev& cam, const SetDev& set, const float4* rec,
                             const uint32_t* vals, const int2* ranges, float* out,
                             int32_t* n_contrib, int32_t* last, int32_t* med,
                             unsigned long long* counters, cudaStream_t st) {
  const dim3 grid(cam.tiles_x, cam.tiles_y);
  ProfScope ps(kProfBlendFwd, st);
  blend_fwd_kernel<<<grid, kBlock, 0, st>>>(cam, set, rec, vals, ranges, out, n_contrib, last, med,
                                            counters);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_blend_bwd(const CamDev& cam, const SetDev& set, const float4* rec,
                             const uint32_t* vals, const int2* ranges, const float* out,
                             const int32_t* last, const int32_t* med, const AdjDev& adj,
                             float* grec, float* screen, int n, unsigned long long* counters,
                             cudaStream_t st) {
  const dim3 grid(cam.tiles_x, cam.tiles_y);
  ProfScope ps(kProfBlendBwd, st);
  blend_bwd_kernel<<<grid, kBlock, 0, st>>>(cam, set, rec, vals, ranges, out, last, med, adj, grec,
                                            screen, n, counters);
  count_launch();
  return cudaGetLastError();
}

}  // namespace gs2d
