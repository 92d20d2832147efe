// Per-surfel preprocess (forward) and its adjoint (backward).
//
// Forward (Sec. 3.1 surfel model; Sec. 3.2 antialiasing filter): for each
// surfel compute the view-space frame, cull disks whose 3-sigma extent
// reaches the near plane, the projected centre c, the centred homography
// of the tangent plane in inverse form (Ji, e), the conservative screen
// bounding box of {rho <= rho_max} (ellipse of the disk union the screen
// filter disk) and its tile rectangle, SH colour and the camera-facing
// normal.  The geometry runs in double-float (pairs of FP32 values, about
// 48 bits) so that pixel offsets from c and the inverse Jacobian of nearly
// edge-on disks are accurate to FP32 rounding; the record the blends read is
// FP32 with c split into two floats.
//
// Backward: chains the per-surfel gradient record of the blend backward
// (d Ji, d e, d c, d p_z, d opacity, d rgb, d normal) to the parameters,
// in FP32, recomputing the forward intermediates.
#include <math.h>

#include "gs2d_df.cuh"
#include "gs2d_internal.cuh"

namespace gs2d {
namespace {

// Real SH basis (degree <= 3, Condon-Shortley phase), as Cartesian
// polynomials of the unit direction (x, y, z).  Constants:
// 1/(2 sqrt(pi)), sqrt(3/(4 pi)), sqrt(15/pi)/2, sqrt(5/pi)/4,
// sqrt(15/pi)/4, sqrt(35/(2 pi))/4, sqrt(105/pi)/2, sqrt(21/(2 pi))/4,
// sqrt(7/pi)/4, sqrt(105/pi)/4.
constexpr float kY0 = 0.28209479177387814f;
constexpr float kY1 = 0.48860251190291992f;
constexpr float kY2a = 1.0925484305920792f;
constexpr float kY2b = 0.31539156525252005f;
constexpr float kY2c = 0.54627421529603959f;
constexpr float kY3a = 0.59004358992664352f;
constexpr float kY3b = 2.8906114426405538f;
constexpr float kY3c = 0.45704579946446572f;
constexpr float kY3d = 0.37317633259011546f;
constexpr float kY3e = 1.4453057213202769f;

__device__ __forceinline__ void sh_basis(float x, float y, float z, int deg, float* Y) {
  Y[0] = kY0;
  if (deg < 1) return;
  Y[1] = -kY1 * y;
  Y[2] = kY1 * z;
  Y[3] = -kY1 * x;
  if (deg < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = kY2a * x * y;
  Y[5] = -kY2a * y * z;
  Y[6] = kY2b * (2.f * zz - xx - yy);
  Y[7] = -kY2a * x * z;
  Y[8] = kY2c * (xx - yy);
  if (deg < 3) return;
  Y[9] = -kY3a * y * (3.f * xx - yy);
  Y[10] = kY3b * x * y * z;
  Y[11] = -kY3c * y * (4.f * zz - xx - yy);
  Y[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
  Y[13] = -kY3c * x * (4.f * zz - xx - yy);
  Y[14] = kY3e * z * (xx - yy);
  Y[15] = -kY3a * x * (xx - 3.f * yy);
}

// gradient of the polynomial basis, dY[k] = (dY/dx, dY/dy, dY/dz)
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, int deg, float3* dY) {
  dY[0] = make_float3(0.f, 0.f, 0.f);
  if (deg < 1) return;
  dY[1] = make_float3(0.f, -kY1, 0.f);
  dY[2] = make_float3(0.f, 0.f, kY1);
  dY[3] = make_float3(-kY1, 0.f, 0.f);
  if (deg < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  dY[4] = make_float3(kY2a * y, kY2a * x, 0.f);
  dY[5] = make_float3(0.f, -kY2a * z, -kY2a * y);
  dY[6] = make_float3(-2.f * kY2b * x, -2.f * kY2b * y, 4.f * kY2b * z);
  dY[7] = make_float3(-kY2a * z, 0.f, -kY2a * x);
  dY[8] = make_float3(2.f * kY2c * x, -2.f * kY2c * y, 0.f);
  if (deg < 3) return;
  dY[9] = make_float3(-kY3a * 6.f * x * y, -kY3a * (3.f * xx - 3.f * yy), 0.f);
  dY[10] = make_float3(kY3b * y * z, kY3b * x * z, kY3b * x * y);
  dY[11] = make_float3(kY3c * 2.f * x * y, -kY3c * (4.f * zz - xx - 3.f * yy), -kY3c * 8.f * y * z);
  dY[12] = make_float3(-kY3d * 6.f * x * z, -kY3d * 6.f * y * z, kY3d * (6.f * zz - 3.f * xx - 3.f * yy));
  dY[13] = make_float3(-kY3c * (4.f * zz - 3.f * xx - yy), kY3c * 2.f * x * y, -kY3c * 8.f * x * z);
  dY[14] = make_float3(kY3e * 2.f * x * z, -kY3e * 2.f * y * z, kY3e * (xx - yy));
  dY[15] = make_float3(-kY3a * (3.f * xx - 3.f * yy), kY3a * 6.f * x * y, 0.f);
}

template <typename T>
struct V3 {
  T x, y, z;
};

// Columns of the rotation of the unit quaternion (w, x, y, z).
template <typename T>
__device__ __forceinline__ void quat_cols(T w, T x, T y, T z, V3<T>& r1, V3<T>& r2, V3<T>& r3) {
  r1 = {T(1) - T(2) * (y * y + z * z), T(2) * (x * y + w * z), T(2) * (x * z - w * y)};
  r2 = {T(2) * (x * y - w * z), T(1) - T(2) * (x * x + z * z), T(2) * (y * z + w * x)};
  r3 = {T(2) * (x * z + w * y), T(2) * (y * z - w * x), T(1) - T(2) * (x * x + y * y)};
}

// R v and R^T v; R in the precision of v (FP32 kernels take the camera's
// FP32 copy).
template <typename T>
__device__ __forceinline__ V3<T> rot(const T* R, V3<T> v) {
  return {R[0] * v.x + R[1] * v.y + R[2] * v.z,
          R[3] * v.x + R[4] * v.y + R[5] * v.z,
          R[6] * v.x + R[7] * v.y + R[8] * v.z};
}
template <typename T>
__device__ __forceinline__ V3<T> rotT(const T* R, V3<T> v) {
  return {R[0] * v.x + R[3] * v.y + R[6] * v.z,
          R[1] * v.x + R[4] * v.y + R[7] * v.z,
          R[2] * v.x + R[5] * v.y + R[8] * v.z};
}

// Stage 1 (FP32, every surfel): defaults for the sort inputs and a
// conservative visibility test, appending possibly visible surfels to a
// candidate list.  It rejects only surfels that stage 2 would reject: the
// 3-sigma disk lies inside the sphere of radius 3 max(s_u, s_v) around mu,
// so a sphere entirely behind the near plane, or whose camera-space box
// projects (with the screen-filter radius, one pixel and a relative error
// margin added) entirely outside the image, has an empty tile rectangle.
__global__ void __launch_bounds__(256) preprocess_cull_kernel(ParamsDev P, CamDev cam, SetDev set,
                                                              uint2* __restrict__ rect,
                                                              uint32_t* __restrict__ tcount,
                                                              uint32_t* __restrict__ flags) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  bool keep = false;
  if (n < P.n) {
    tcount[n] = 0u;
    rect[n] = make_uint2(0u, 0u);
    const float4 q4 = load_quat(P, n);
    const float qw = q4.x, qx = q4.y, qy = q4.z, qz = q4.w;
    const df qn2 = two_prod(qw, qw) + two_prod(qx, qx) + two_prod(qy, qy) + two_prod(qz, qz);
    const V3<float> mu = {P.mu[3 * n], P.mu[3 * n + 1], P.mu[3 * n + 2]};
    V3<float> p = rot<float>(cam.Rf, mu);
    p.x += cam.tf[0]; p.y += cam.tf[1]; p.z += cam.tf[2];
    const float2 s2 = load_scale(P, n);
    const float R = 3.0f * fmaxf(s2.x, s2.y) * sqrtf(set.rho_max / 9.0f);
    // FP32 error of p is far below this margin (a few ulp of |mu| + |t|)
    const float eps = 1e-4f * (fabsf(mu.x) + fabsf(mu.y) + fabsf(mu.z) + cam.tabs + 1.0f) + 1e-3f * R;
    keep = df_pos(qn2) && p.z + R + eps > set.near_plane;
    const float zlo = p.z - R - eps, zhi = p.z + R + eps;
    if (keep && zlo > 0.f) {
      const float rpix = sqrtf(set.rho_max / set.sinv) + 1.0f;
      const float fx = cam.fxf, fy = cam.fyf;
      const float xa = p.x - R - eps, xb = p.x + R + eps, ya = p.y - R - eps, yb = p.y + R + eps;
      const float sx0 = fx * (xa < 0.f ? xa / zlo : xa / zhi) + cam.cxf - rpix;
      const float sx1 = fx * (xb > 0.f ? xb / zlo : xb / zhi) + cam.cxf + rpix;
      const float sy0 = fy * (ya < 0.f ? ya / zlo : ya / zhi) + cam.cyf - rpix;
      const float sy1 = fy * (yb > 0.f ? yb / zlo : yb / zhi) + cam.cyf + rpix;
      const float m = 1e-3f * (fabsf(sx0) + fabsf(sx1) + fabsf(sy0) + fabsf(sy1)) + 1.0f;
      keep = !(sx1 < -m || sx0 > (float)cam.W + m || sy1 < -m || sy0 > (float)cam.H + m);
    }
  }
  if (n < P.n) flags[n] = keep ? 1u : 0u;
}

// Candidates in surfel-index order (the compositing order breaks depth ties
// by index, and the stable depth sort keeps this order for equal keys).
__global__ void __launch_bounds__(256) compact_kernel(const uint32_t* __restrict__ flags,
                                                      const uint32_t* __restrict__ pos, int n,
                                                      uint32_t* __restrict__ cand) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && flags[i]) cand[pos[i]] = (uint32_t)i;
}

// Double-float vector helpers for the preprocess geometry.
struct D3 {
  df x, y, z;
};
__device__ __forceinline__ df dot3(const D3& a, const D3& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
// R v with R the camera rotation in double-float (row-major)
__device__ __forceinline__ D3 cam_rot(const CamDev& c, const D3& v) {
  D3 r;
  df* o[3] = {&r.x, &r.y, &r.z};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const df r0 = df_make(c.Rf[3 * i], c.Rlo[3 * i]);
    const df r1 = df_make(c.Rf[3 * i + 1], c.Rlo[3 * i + 1]);
    const df r2 = df_make(c.Rf[3 * i + 2], c.Rlo[3 * i + 2]);
    *o[i] = r0 * v.x + r1 * v.y + r2 * v.z;
  }
  return r;
}
__device__ __forceinline__ D3 cam_rot(const CamDev& c, float x, float y, float z) {
  D3 r;
  df* o[3] = {&r.x, &r.y, &r.z};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const df r0 = df_make(c.Rf[3 * i], c.Rlo[3 * i]);
    const df r1 = df_make(c.Rf[3 * i + 1], c.Rlo[3 * i + 1]);
    const df r2 = df_make(c.Rf[3 * i + 2], c.Rlo[3 * i + 2]);
    *o[i] = r0 * x + r1 * y + r2 * z;
  }
  return r;
}

// Stage 2 (candidates only): the definition's preprocess, the footprint's
// exact tile-row coverage and the blend record.  The geometry that decides
// where a surfel lands (view transform, projection, the centred inverse
// homography, the bound of {rho <= rho_max} and its tile rectangle) is
// computed in double-float (about 48 bits; the FP64 pipe is too slow for a
// million surfels per view), colour and normal in FP32.
template <int DEG>
__global__ void __launch_bounds__(256) preprocess_main_kernel(ParamsDev P, CamDev cam, SetDev set,
                                                              const uint32_t* __restrict__ cand,
                                                              const uint32_t* __restrict__ ncand,
                                                              float4* __restrict__ rec,
                                                              uint2* __restrict__ rect,
                                                              uint32_t* __restrict__ tcount,
                                                              uint32_t* __restrict__ dkey,
                                                              uint32_t* __restrict__ idx,
                                                              RowGeom* __restrict__ geom) {
  const uint32_t total = *ncand;
  const df rf = df_sqrt(df_make(set.rho_max) / df_make(set.sinv));
  const float rff = df_float(rf);
  const df fx = df_make(cam.fxf, cam.fxlo), fy = df_make(cam.fyf, cam.fylo);
  const df cx0 = df_make(cam.cxf, cam.cxlo), cy0 = df_make(cam.cyf, cam.cylo);
  for (uint32_t ci = blockIdx.x * blockDim.x + threadIdx.x; ci < total; ci += gridDim.x * blockDim.x) {
    const int n = (int)cand[ci];
    idx[ci] = (uint32_t)n;
    dkey[ci] = 0xFFFFFFFFu;  // not visible unless set below
    const float4 q4 = load_quat(P, n);
    const float qw0 = q4.x, qx0 = q4.y, qy0 = q4.z, qz0 = q4.w;
    const df qn2 = two_prod(qw0, qw0) + two_prod(qx0, qx0) + two_prod(qy0, qy0) + two_prod(qz0, qz0);
    if (!df_pos(qn2)) continue;
    const df iq = df_rsqrt(qn2);
    const df qw = iq * qw0, qx = iq * qx0, qy = iq * qy0, qz = iq * qz0;
    // columns of the rotation of the unit quaternion
    const df one = df_make(1.f);
    const D3 r1 = {one - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy + qw * qz), 2.f * (qx * qz - qw * qy)};
    const D3 r2 = {2.f * (qx * qy - qw * qz), one - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz + qw * qx)};
    const D3 r3 = {2.f * (qx * qz + qw * qy), 2.f * (qy * qz - qw * qx), one - 2.f * (qx * qx + qy * qy)};
    const float mux = P.mu[3 * n], muy = P.mu[3 * n + 1], muz = P.mu[3 * n + 2];
    D3 p = cam_rot(cam, mux, muy, muz);
    p.x = p.x + df_make(cam.tf[0], cam.tlo[0]);
    p.y = p.y + df_make(cam.tf[1], cam.tlo[1]);
    p.z = p.z + df_make(cam.tf[2], cam.tlo[2]);
    const D3 tu = cam_rot(cam, r1), tv = cam_rot(cam, r2), nv = cam_rot(cam, r3);
    const float2 s2 = load_scale(P, n);
    const float su = s2.x, sv = s2.y;
    const D3 a = {tu.x * su, tu.y * su, tu.z * su}, b = {tv.x * sv, tv.y * sv, tv.z * sv};
    const df zmin = p.z - df_sqrt((a.z * a.z + b.z * b.z) * set.rho_max);
    if (!df_pos(zmin - set.near_plane)) continue;
    const df iz = df_rcp(p.z);
    const df xi = p.x * iz, yi = p.y * iz;
    const df cx = fx * xi + cx0, cy = fy * yi + cy0;
    const df J11 = fx * (a.x - a.z * xi) * iz, J12 = fx * (b.x - b.z * xi) * iz;
    const df J21 = fy * (a.y - a.z * yi) * iz, J22 = fy * (b.y - b.z * yi) * iz;
    const df w1 = a.z * iz, w2 = b.z * iz;
    // bounding box of {rho_obj <= rho_max} in offsets from c: dual conic of
    // the centred homography H = [[J, 0], [w^T, 1]]; scaled to C33 = 1 it is
    // [[e0 e0^T - G, e0], [e0^T, 1]] for the ellipse (d - e0)^T G^-1 (d - e0) <= 1
    const float rm = set.rho_max;
    const df C11 = (J11 * J11 + J12 * J12) * rm, C22 = (J21 * J21 + J22 * J22) * rm;
    const df C12 = (J11 * J21 + J12 * J22) * rm;
    const df C13 = (J11 * w1 + J12 * w2) * rm, C23 = (J21 * w1 + J22 * w2) * rm;
    const df C33 = (w1 * w1 + w2 * w2) * rm - 1.f;
    const df ex = df_sqrt(df_max(C13 * C13 - C11 * C33, df_make(0.f)));
    const df ey = df_sqrt(df_max(C23 * C23 - C22 * C33, df_make(0.f)));
    const df i33 = df_rcp(C33);
    const df x0 = (C13 - ex) * i33, x1 = (C13 + ex) * i33;
    const df y0 = (C23 - ey) * i33, y1 = (C23 + ey) * i33;
    const df xmin = cx + df_min(df_min(x0, x1), -rf), xmax = cx + df_max(df_max(x0, x1), rf);
    const df ymin = cy + df_min(df_min(y0, y1), -rf), ymax = cy + df_max(df_max(y0, y1), rf);
    float ilo = df_ceil(xmin - 0.5f), ihi = df_floor(xmax - 0.5f);
    float jlo = df_ceil(ymin - 0.5f), jhi = df_floor(ymax - 0.5f);
    ilo = fmaxf(ilo, 0.f); jlo = fmaxf(jlo, 0.f);
    ihi = fminf(ihi, (float)(cam.W - 1)); jhi = fminf(jhi, (float)(cam.H - 1));
    if (!(ilo <= ihi && jlo <= jhi)) continue;
    RowGeom gm;
    {
      const df e0x = C13 * i33, e0y = C23 * i33;
      const df g11 = e0x * e0x - C11 * i33, g12 = e0x * e0y - C12 * i33, g22 = e0y * e0y - C22 * i33;
      gm.cx_hi = cx.hi; gm.cx_lo = cx.lo;
      gm.cy_hi = cy.hi; gm.cy_lo = cy.lo;
      gm.e0x = df_float(e0x); gm.e0y = df_float(e0y);
      if (df_pos(g11) && df_pos(g22)) {
        // rounded once to FP32; the row rule's margin covers their error
        const df dg = g11 * g22 - g12 * g12;
        const float det = df_pos(dg) ? df_float(dg) : 0.f;
        const float f11 = df_float(g11), f12 = df_float(g12), f22 = df_float(g22);
        gm.hy = sqrtf(f22);
        gm.t = f12 * rsqrtf(f11);
        gm.slope = f12 / f22;
        gm.wsc = sqrtf(det) / f22;
      } else {
        gm.hy = -1.f; gm.t = 0.f; gm.slope = 0.f; gm.wsc = 0.f;  // disk only
      }
    }
    gm.ilo = (int)ilo; gm.ihi = (int)ihi; gm.jlo = (int)jlo; gm.jhi = (int)jhi;
    const int tx0 = gm.ilo / kTile, tx1 = gm.ihi / kTile + 1;
    const int ty0 = gm.jlo / kTile, ty1 = gm.jhi / kTile + 1;
    rect[n] = make_uint2((uint32_t)tx0 | ((uint32_t)ty0 << 16), (uint32_t)tx1 | ((uint32_t)ty1 << 16));
    uint32_t cnt = 0;
    for (int ty = ty0; ty < ty1; ++ty) {
      int a0, a1;
      if (row_tiles(gm, ty, rff, &a0, &a1)) cnt += (uint32_t)(a1 - a0);
    }
    if (cnt == 0) continue;
    geom[n] = gm;
    tcount[n] = cnt;
    const float pz = df_float(p.z);
    dkey[ci] = __float_as_uint(pz);
    const df det = J11 * J22 - J12 * J21;
    // Ji, split for the blends' exact tile-relative evaluation of (u, v):
    // on a power-of-two grid 2^g chosen so that |Ji d| < 2^(g+22) for every
    // pixel and tile origin of the surfel's tile rectangle, Jh (multiples of
    // 2^(g+1)) and nref_h (Ji (o_ref - c) on multiples of 2^g, o_ref the
    // rectangle's first tile origin) make every partial sum of
    // nref_h + Jh (o - o_ref) + Jh (lx, ly) exact in FP32; the low parts Jl =
    // Ji - Jh and nref_l = Ji (o_ref - c) - nref_h (both about 2^g) carry the
    // rest (see blend.cu).
    float4 jh, jl, nref;  // nref = (nref_h.u, nref_h.v, nref_l.u, nref_l.v)
    float ugrid = 1.f;    // 2^-g
    float2 ef;
    const float orx = (float)(tx0 * kTile), ory = (float)(ty0 * kTile);
    if (df_nonzero(det)) {
      const df id = df_rcp(det);
      const df i11 = J22 * id, i12 = -(J12 * id), i21 = -(J21 * id), i22 = J11 * id;
      const float4 r1f = make_float4(df_float(i11), df_float(i12), df_float(i21), df_float(i22));
      const float4 r5f = make_float4(df_float(i11 - r1f.x), df_float(i12 - r1f.y), df_float(i21 - r1f.z),
                                     df_float(i22 - r1f.w));
      ef = make_float2(df_float(-(i11 * w1 + i21 * w2)), df_float(-(i12 * w1 + i22 * w2)));
      const df d0x = two_sum(orx, -cx.hi) - cx.lo, d0y = two_sum(ory, -cy.hi) - cy.lo;
      const df nu0 = i11 * d0x + i12 * d0y, nv0 = i21 * d0x + i22 * d0y;
      const float Dx = fmaxf(fabsf(orx - cx.hi), fabsf((float)(tx1 * kTile) - cx.hi));
      const float Dy = fmaxf(fabsf(ory - cy.hi), fabsf((float)(ty1 * kTile) - cy.hi));
      const float Rs = fmaxf(fabsf(r1f.x) + fabsf(r1f.y), fabsf(r1f.z) + fabsf(r1f.w));
      const float M = __fmul_rn(__fmul_rn(Rs, fmaxf(Dx, Dy) + 2.f), 1.0009765625f);
      const int E = min(max(((__float_as_int(M) >> 23) & 0xff) - 127, -100), 100);  // M < 2^(E+1)
      const int g = E - 21;
      const float ug = __int_as_float((127 - g) << 23), dg = __int_as_float((127 + g) << 23);
      const float uj = __int_as_float((126 - g) << 23), dj = __int_as_float((128 + g) << 23);
      jh = make_float4(__fmul_rn(rintf(__fmul_rn(r1f.x, uj)), dj), __fmul_rn(rintf(__fmul_rn(r1f.y, uj)), dj),
                       __fmul_rn(rintf(__fmul_rn(r1f.z, uj)), dj), __fmul_rn(rintf(__fmul_rn(r1f.w, uj)), dj));
      jl = make_float4(__fadd_rn(__fsub_rn(r1f.x, jh.x), r5f.x), __fadd_rn(__fsub_rn(r1f.y, jh.y), r5f.y),
                       __fadd_rn(__fsub_rn(r1f.z, jh.z), r5f.z), __fadd_rn(__fsub_rn(r1f.w, jh.w), r5f.w));
      const float uh = __fmul_rn(rintf(__fmul_rn(nu0.hi, ug)), dg);
      const float vh = __fmul_rn(rintf(__fmul_rn(nv0.hi, ug)), dg);
      nref = make_float4(uh, vh, __fadd_rn(__fsub_rn(nu0.hi, uh), nu0.lo), __fadd_rn(__fsub_rn(nv0.hi, vh), nv0.lo));
      ugrid = ug;
    } else {
      // edge-on disk: no object-space footprint (rho_obj is NaN, the
      // screen filter decides)
      const float qnan = __int_as_float(0x7fffffff);
      jh = make_float4(qnan, qnan, qnan, qnan);
      jl = nref = make_float4(0.f, 0.f, 0.f, 0.f);
      ef = make_float2(0.f, 0.f);
    }
    // colour: SH at the world direction from the camera centre
    const float dx = mux - cam.camposf[0], dy = muy - cam.camposf[1], dz = muz - cam.camposf[2];
    const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
    constexpr int K = (DEG + 1) * (DEG + 1);
    float Y[16];
    sh_basis(dx * il, dy * il, dz * il, DEG, Y);
    float col[3] = {0.f, 0.f, 0.f};
    if (P.sh_table) {
      const uint16_t* f = P.sh_table + (size_t)P.sh_row[n] * K * 3;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        col[0] = fmaf(h2f(f[k * 3]), Y[k], col[0]);
        col[1] = fmaf(h2f(f[k * 3 + 1]), Y[k], col[1]);
        col[2] = fmaf(h2f(f[k * 3 + 2]), Y[k], col[2]);
      }
    } else {
      const float* f = P.sh + (size_t)n * K * 3;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        col[0] = fmaf(f[k * 3], Y[k], col[0]);
        col[1] = fmaf(f[k * 3 + 1], Y[k], col[1]);
        col[2] = fmaf(f[k * 3 + 2], Y[k], col[2]);
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) col[c] = fmaxf(col[c] + 0.5f, 0.f);
    const float sg = df_pos(dot3(nv, p)) ? -1.f : 1.f;
    float4* Rr = rec + (size_t)n * kRecF4;
    Rr[0] = make_float4(cx.hi, cy.hi, cx.lo, cy.lo);
    Rr[1] = jh;
    Rr[2] = make_float4(ef.x, ef.y, pz, load_opacity(P, n));
    Rr[3] = make_float4(col[0], col[1], col[2], sg * df_float(nv.x));
    Rr[4] = make_float4(sg * df_float(nv.y), sg * df_float(nv.z), nref.x, nref.y);
    Rr[5] = jl;
    // the first tile of the rectangle (tile indices, packed) and 2^-g, g the grid's exponent
    Rr[6] = make_float4(nref.z, nref.w, __uint_as_float((uint32_t)tx0 | ((uint32_t)ty0 << 16)), ugrid);
  }
}

// ---------------------------------------------------------------------------
// Backward.

// Gradient of one visible surfel n: chain the per-surfel record (d Ji, d e,
// d c, d p_z, d opacity, d rgb, d normal) back to mu, q, s, o and SH,
// accumulated into G.  kVec: SH rows and gradient rows are float4-aligned.
// Every load that does not depend on the computation (the surfel's tile
// count tc, its gradient record, parameters and the current values of the
// small gradient arrays) is issued before the first use, so that a surfel
// costs two memory round trips (these loads, then the SH gradient row) and
// not one per dependent access.  The gradient arrays must not overlap one
// another or the parameters.
template <int DEG, bool kVec>
__device__ __forceinline__ void bwd_one(const ParamsDev& P, const CamDev& cam, int n, uint32_t tc,
                                        const float* __restrict__ grec, const gs_param_grads& G) {
  static_assert(kGradRec == 16, "gradient record of four float4");
  float* __restrict__ Gq = G.quat;
  float* __restrict__ Gm = G.mu;
  float* __restrict__ Gs = G.scale;
  float* __restrict__ Go = G.opacity;
  const float4* g4 = reinterpret_cast<const float4*>(grec + (size_t)n * kGradRec);
  const float4 ga4 = g4[0], gb4 = g4[1], gc4 = g4[2], gd4 = g4[3];
  float oq[4] = {0.f, 0.f, 0.f, 0.f}, om[3] = {0.f, 0.f, 0.f}, os[2] = {0.f, 0.f}, oo = 0.f;
  if (Gq) {
#pragma unroll
    for (int i = 0; i < 4; ++i) oq[i] = Gq[4 * n + i];
  }
  if (Gm) {
#pragma unroll
    for (int i = 0; i < 3; ++i) om[i] = Gm[3 * n + i];
  }
  if (Gs) {
    os[0] = Gs[2 * n];
    os[1] = Gs[2 * n + 1];
  }
  if (Go) oo = Go[n];
  float gJi11 = ga4.x, gJi12 = ga4.y, gJi21 = ga4.z, gJi22 = ga4.w;
  const float ge1 = gb4.x, ge2 = gb4.y, gcx = gb4.z, gcy = gb4.w, gpz0 = gc4.x, gop = gc4.y;
  const float grgb[3] = {gc4.z, gc4.w, gd4.x};
  const V3<float> gnrm = {gd4.y, gd4.z, gd4.w};
  // forward intermediates, FP32
  const float qw0 = P.quat[4 * n], qx0 = P.quat[4 * n + 1], qy0 = P.quat[4 * n + 2], qz0 = P.quat[4 * n + 3];
  const float qn = sqrtf(qw0 * qw0 + qx0 * qx0 + qy0 * qy0 + qz0 * qz0);
  const float iqn = 1.f / qn;
  const float qw = qw0 * iqn, qx = qx0 * iqn, qy = qy0 * iqn, qz = qz0 * iqn;
  V3<float> r1, r2, r3;
  quat_cols<float>(qw, qx, qy, qz, r1, r2, r3);
  const V3<float> mu = {P.mu[3 * n], P.mu[3 * n + 1], P.mu[3 * n + 2]};
  V3<float> p = rot<float>(cam.Rf, mu);
  p.x += cam.tf[0]; p.y += cam.tf[1]; p.z += cam.tf[2];
  const V3<float> tu = rot<float>(cam.Rf, r1), tv = rot<float>(cam.Rf, r2), nv = rot<float>(cam.Rf, r3);
  const float su = P.scale[2 * n], sv = P.scale[2 * n + 1];
  const V3<float> a = {su * tu.x, su * tu.y, su * tu.z}, b = {sv * tv.x, sv * tv.y, sv * tv.z};
  const float fx = cam.fxf, fy = cam.fyf;
  const float iz = 1.f / p.z;
  const float xi = p.x * iz, yi = p.y * iz;
  const float J11 = fx * (a.x - a.z * xi) * iz, J12 = fx * (b.x - b.z * xi) * iz;
  const float J21 = fy * (a.y - a.z * yi) * iz, J22 = fy * (b.y - b.z * yi) * iz;
  const float w1 = a.z * iz, w2 = b.z * iz;
  const float det = J11 * J22 - J12 * J21;
  float gJ11 = 0.f, gJ12 = 0.f, gJ21 = 0.f, gJ22 = 0.f, gw1 = 0.f, gw2 = 0.f;
  if (det != 0.f) {
    const float id = 1.f / det;
    const float i11 = J22 * id, i12 = -J12 * id, i21 = -J21 * id, i22 = J11 * id;
    // e = -Ji^T w
    gJi11 -= w1 * ge1; gJi12 -= w1 * ge2; gJi21 -= w2 * ge1; gJi22 -= w2 * ge2;
    gw1 = -(i11 * ge1 + i12 * ge2);
    gw2 = -(i21 * ge1 + i22 * ge2);
    // Ji = J^-1:  dJ = -Ji^T dJi Ji^T
    const float m11 = gJi11 * i11 + gJi12 * i12, m12 = gJi11 * i21 + gJi12 * i22;
    const float m21 = gJi21 * i11 + gJi22 * i12, m22 = gJi21 * i21 + gJi22 * i22;
    gJ11 = -(i11 * m11 + i21 * m21);
    gJ12 = -(i11 * m12 + i21 * m22);
    gJ21 = -(i12 * m11 + i22 * m21);
    gJ22 = -(i12 * m12 + i22 * m22);
  }
  // J_1k = fx (g_x - g_z xi) / p_z, J_2k = fy (g_y - g_z yi) / p_z, w_k = g_z / p_z
  const V3<float> ga = {fx * gJ11 * iz, fy * gJ21 * iz, (-fx * xi * gJ11 - fy * yi * gJ21 + gw1) * iz};
  const V3<float> gb = {fx * gJ12 * iz, fy * gJ22 * iz, (-fx * xi * gJ12 - fy * yi * gJ22 + gw2) * iz};
  const float gxi = -fx * (a.z * gJ11 + b.z * gJ12) * iz + fx * gcx;
  const float gyi = -fy * (a.z * gJ21 + b.z * gJ22) * iz + fy * gcy;
  float gpz = gpz0 - (J11 * gJ11 + J12 * gJ12 + J21 * gJ21 + J22 * gJ22) * iz - (w1 * gw1 + w2 * gw2) * iz;
  const V3<float> gp = {gxi * iz, gyi * iz, gpz - (xi * gxi + yi * gyi) * iz};
  V3<float> gmu = rotT<float>(cam.Rf, gp);
  const float gsu = ga.x * tu.x + ga.y * tu.y + ga.z * tu.z;
  const float gsv = gb.x * tv.x + gb.y * tv.y + gb.z * tv.z;
  const V3<float> gr1 = rotT<float>(cam.Rf, V3<float>{su * ga.x, su * ga.y, su * ga.z});
  const V3<float> gr2 = rotT<float>(cam.Rf, V3<float>{sv * gb.x, sv * gb.y, sv * gb.z});
  const float sgn = (nv.x * p.x + nv.y * p.y + nv.z * p.z) > 0.f ? -1.f : 1.f;
  const V3<float> gr3 = rotT<float>(cam.Rf, V3<float>{sgn * gnrm.x, sgn * gnrm.y, sgn * gnrm.z});
  // colour
  const V3<float> dd = {mu.x - cam.camposf[0], mu.y - cam.camposf[1], mu.z - cam.camposf[2]};
  const float dl = sqrtf(dd.x * dd.x + dd.y * dd.y + dd.z * dd.z);
  const float il = 1.f / dl;
  const float dx = dd.x * il, dy = dd.y * il, dz = dd.z * il;
  constexpr int K = (DEG + 1) * (DEG + 1);
  float Y[16];
  float3 dY[16];
  sh_basis(dx, dy, dz, DEG, Y);
  sh_basis_grad(dx, dy, dz, DEG, dY);
  const float* f = P.sh + (size_t)n * K * 3;
  float fv[K * 3];
  if constexpr (kVec) {
#pragma unroll
    for (int i = 0; i < K * 3 / 4; ++i) {
      const float4 x = reinterpret_cast<const float4*>(f)[i];
      fv[4 * i] = x.x; fv[4 * i + 1] = x.y; fv[4 * i + 2] = x.z; fv[4 * i + 3] = x.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < K * 3; ++i) fv[i] = f[i];
  }
  if (tc == 0u) return;  // no tile: nothing to add
  float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[c] = fmaf(fv[k * 3 + c], Y[k], acc[c]);
  float gc[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) gc[c] = (acc[c] + 0.5f > 0.f) ? grgb[c] : 0.f;  // clamped: no gradient
  V3<float> gdir = {0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float fk = fv[k * 3] * gc[0] + fv[k * 3 + 1] * gc[1] + fv[k * 3 + 2] * gc[2];
    gdir.x += fk * dY[k].x;
    gdir.y += fk * dY[k].y;
    gdir.z += fk * dY[k].z;
  }
  if (G.sh) {
    float* gs = G.sh + (size_t)n * K * 3;
    if constexpr (kVec) {
      // element j of the row is (basis j / 3, channel j % 3)
#pragma unroll
      for (int i = 0; i < K * 3 / 4; ++i) {
        float4* q4 = reinterpret_cast<float4*>(gs) + i;
        float4 x = *q4;
        x.x += gc[(4 * i) % 3] * Y[(4 * i) / 3];
        x.y += gc[(4 * i + 1) % 3] * Y[(4 * i + 1) / 3];
        x.z += gc[(4 * i + 2) % 3] * Y[(4 * i + 2) / 3];
        x.w += gc[(4 * i + 3) % 3] * Y[(4 * i + 3) / 3];
        *q4 = x;
      }
    } else {
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (gc[c] != 0.f) gs[k * 3 + c] += gc[c] * Y[k];
    }
  }
  const float gdd = dx * gdir.x + dy * gdir.y + dz * gdir.z;
  gmu.x += (gdir.x - dx * gdd) * il;
  gmu.y += (gdir.y - dy * gdd) * il;
  gmu.z += (gdir.z - dz * gdd) * il;
  // rotation: dL/dR with columns gr1, gr2, gr3 -> unit quaternion
  const float R00 = gr1.x, R10 = gr1.y, R20 = gr1.z;
  const float R01 = gr2.x, R11 = gr2.y, R21 = gr2.z;
  const float R02 = gr3.x, R12 = gr3.y, R22 = gr3.z;
  const float dqw = 2.f * (-qz * R01 + qy * R02 + qz * R10 - qx * R12 - qy * R20 + qx * R21);
  const float dqx = 2.f * (qy * R01 + qz * R02 + qy * R10 - 2.f * qx * R11 - qw * R12 + qz * R20 +
                           qw * R21 - 2.f * qx * R22);
  const float dqy = 2.f * (-2.f * qy * R00 + qx * R01 + qw * R02 + qx * R10 + qz * R12 - qw * R20 +
                           qz * R21 - 2.f * qy * R22);
  const float dqz = 2.f * (-2.f * qz * R00 - qw * R01 + qx * R02 + qw * R10 - 2.f * qz * R11 +
                           qy * R12 + qx * R20 + qy * R21);
  const float qd = qw * dqw + qx * dqx + qy * dqy + qz * dqz;
  if (Gq) {
    Gq[4 * n] = oq[0] + (dqw - qw * qd) * iqn;
    Gq[4 * n + 1] = oq[1] + (dqx - qx * qd) * iqn;
    Gq[4 * n + 2] = oq[2] + (dqy - qy * qd) * iqn;
    Gq[4 * n + 3] = oq[3] + (dqz - qz * qd) * iqn;
  }
  if (Gm) {
    Gm[3 * n] = om[0] + gmu.x;
    Gm[3 * n + 1] = om[1] + gmu.y;
    Gm[3 * n + 2] = om[2] + gmu.z;
  }
  if (Gs) {
    Gs[2 * n] = os[0] + gsu;
    Gs[2 * n + 1] = os[1] + gsv;
  }
  if (Go) Go[n] = oo + gop;
}

// Over the render's candidates (a grid-stride loop over the device-side
// count); surfels with no tile contribute nothing.
template <int DEG, bool kVec>
__global__ void __launch_bounds__(256, 2) preprocess_bwd_kernel(ParamsDev P, CamDev cam,
                                                             const uint32_t* __restrict__ cand,
                                                             const uint32_t* __restrict__ ncand,
                                                             const uint32_t* __restrict__ tcount,
                                                             const float* __restrict__ grec,
                                                             gs_param_grads G) {
  const int nc = (int)*ncand;
  for (int ci = blockIdx.x * blockDim.x + threadIdx.x; ci < nc; ci += gridDim.x * blockDim.x) {
    const int n = (int)cand[ci];
    bwd_one<DEG, kVec>(P, cam, n, tcount[n], grec, G);
  }
}

template <int DEG>
void launch_bwd_deg(const ParamsDev& P, const CamDev& cam, const uint32_t* cand, const uint32_t* ncand,
                    const uint32_t* tcount, const float* grec, const gs_param_grads& G, unsigned blocks,
                    cudaStream_t st) {
  constexpr int K3 = (DEG + 1) * (DEG + 1) * 3;
  const bool vec = K3 % 4 == 0 && ((uintptr_t)P.sh % 16u) == 0 && ((uintptr_t)G.sh % 16u) == 0;
  if constexpr (K3 % 4 == 0) {
    if (vec) {
      preprocess_bwd_kernel<DEG, true><<<blocks, 256, 0, st>>>(P, cam, cand, ncand, tcount, grec, G);
      return;
    }
  }
  preprocess_bwd_kernel<DEG, false><<<blocks, 256, 0, st>>>(P, cam, cand, ncand, tcount, grec, G);
}

}  // namespace

cudaError_t launch_preprocess(const ParamsDev& P, const CamDev& cam, const SetDev& set,
                              float4* rec, uint2* rect, uint32_t* tcount, uint32_t* dkey,
                              uint32_t* idx, uint32_t* cand, uint32_t* ncand, RowGeom* geom,
                              uint32_t* flags, uint32_t* scan_tmp, cudaStream_t st) {
  if (P.n == 0) return cudaMemsetAsync(ncand, 0, sizeof(uint32_t), st);
  ProfScope ps(kProfPreprocess, st);
  preprocess_cull_kernel<<<div_up(P.n, 256), 256, 0, st>>>(P, cam, set, rect, tcount, flags);
  count_launch();
  // positions of the candidates: exclusive scan of the flags (into cand's
  // second half is not needed: dkey is free until the main pass writes it)
  cudaError_t e = launch_scan(flags, dkey, P.n, ncand, scan_tmp, st);
  if (e != cudaSuccess) return e;
  compact_kernel<<<div_up(P.n, 256), 256, 0, st>>>(flags, dkey, P.n, cand);
  // candidates are a subset of the surfels; a grid-stride loop over the
  // device-side count, three CTAs per SM (what its registers allow)
  static const unsigned resident = [] {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return 3u * (unsigned)sms;
  }();
  const unsigned blocks = div_up(P.n, 256) < resident ? div_up(P.n, 256) : resident;
  switch (P.sh_degree) {
    case 0: preprocess_main_kernel<0><<<blocks, 256, 0, st>>>(P, cam, set, cand, ncand, rec, rect, tcount, dkey, idx, geom); break;
    case 1: preprocess_main_kernel<1><<<blocks, 256, 0, st>>>(P, cam, set, cand, ncand, rec, rect, tcount, dkey, idx, geom); break;
    case 2: preprocess_main_kernel<2><<<blocks, 256, 0, st>>>(P, cam, set, cand, ncand, rec, rect, tcount, dkey, idx, geom); break;
    default: preprocess_main_kernel<3><<<blocks, 256, 0, st>>>(P, cam, set, cand, ncand, rec, rect, tcount, dkey, idx, geom); break;
  }
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_preprocess_bwd(const ParamsDev& P, const CamDev& cam, const uint32_t* cand,
                                  const uint32_t* ncand, const uint32_t* tcount, const float* grec,
                                  const gs_param_grads& G, cudaStream_t st) {
  if (P.n == 0) return cudaSuccess;
  ProfScope ps(kProfPreprocessBwd, st);
  // candidates are a subset of the surfels: a grid-stride loop over the
  // device-side count, two CTAs per SM
  const unsigned blocks = div_up(P.n, 256) < 304u ? div_up(P.n, 256) : 304u;
  switch (P.sh_degree) {
    case 0: launch_bwd_deg<0>(P, cam, cand, ncand, tcount, grec, G, blocks, st); break;
    case 1: launch_bwd_deg<1>(P, cam, cand, ncand, tcount, grec, G, blocks, st); break;
    case 2: launch_bwd_deg<2>(P, cam, cand, ncand, tcount, grec, G, blocks, st); break;
    default: launch_bwd_deg<3>(P, cam, cand, ncand, tcount, grec, G, blocks, st); break;
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace gs2d
