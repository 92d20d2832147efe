// Internal declarations of the CUDA library (sm_103a).  Not part of the C ABI.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/gs2d.h"

namespace gs2d {

constexpr int kTile = 16;              // 16 x 16 pixel tiles
constexpr int kRecF4 = 7;              // per-surfel blend record, 7 x float4

// Camera as the kernels see it (by value).  Geometry that decides where a
// surfel lands on screen is carried in double precision.
struct CamDev {
  double R[9];
  double t[3];
  double fx, fy, cx, cy;
  double campos[3];  // camera centre in world coordinates, -R^T t
  int W, H, tiles_x, tiles_y;
  // FP32 copies for the FP32 kernels (converting doubles per use is slow);
  // with the *lo parts (value - FP32 copy, rounded) they are the double-float
  // form the preprocess computes in
  float Rf[9], tf[3], camposf[3];
  float fxf, fyf, cxf, cyf;
  float Rlo[9], tlo[3], fxlo, fylo, cxlo, cylo;
  float tabs;  // |t_x| + |t_y| + |t_z|
};

// Fill a CamDev from a camera (everything derived is computed here, once).
inline void cam_from(const gs_camera& c, CamDev& cam) {
  for (int i = 0; i < 9; ++i) cam.R[i] = c.R[i];
  for (int i = 0; i < 3; ++i) cam.t[i] = c.t[i];
  cam.fx = c.fx; cam.fy = c.fy; cam.cx = c.cx; cam.cy = c.cy;
  for (int i = 0; i < 3; ++i) cam.campos[i] = -(c.R[i] * c.t[0] + c.R[3 + i] * c.t[1] + c.R[6 + i] * c.t[2]);
  cam.W = c.width; cam.H = c.height;
  cam.tiles_x = (c.width + 15) / 16;
  cam.tiles_y = (c.height + 15) / 16;
  for (int i = 0; i < 9; ++i) cam.Rf[i] = (float)c.R[i];
  for (int i = 0; i < 3; ++i) cam.tf[i] = (float)c.t[i];
  for (int i = 0; i < 3; ++i) cam.camposf[i] = (float)cam.campos[i];
  cam.fxf = (float)c.fx; cam.fyf = (float)c.fy; cam.cxf = (float)c.cx; cam.cyf = (float)c.cy;
  for (int i = 0; i < 9; ++i) cam.Rlo[i] = (float)(c.R[i] - (double)cam.Rf[i]);
  for (int i = 0; i < 3; ++i) cam.tlo[i] = (float)(c.t[i] - (double)cam.tf[i]);
  cam.fxlo = (float)(c.fx - (double)cam.fxf); cam.fylo = (float)(c.fy - (double)cam.fyf);
  cam.cxlo = (float)(c.cx - (double)cam.cxf); cam.cylo = (float)(c.cy - (double)cam.cyf);
  cam.tabs = (float)(fabs(c.t[0]) + fabs(c.t[1]) + fabs(c.t[2]));
}

struct SetDev {
  float near_plane, alpha_min, T_min, alpha_max, rho_max, sinv;
  float bg[3];
};

// Per-surfel blend record (written by the preprocess, read by both blends):
//  r0 = (c_hi.x, c_hi.y, c_lo.x, c_lo.y)   projected centre, two-float split
//  r1 = Jh                                 inverse of the centred Jacobian,
//  r5 = Jl                                 split Ji = Jh + Jl on the surfel's grid
//  r2 = (e.x, e.y, p_z, opacity)           projective row, centre depth
//  r3 = (r, g, b, n.x)                     colour, view-space normal
//  r4 = (n.y, n.z, nref_h.u, nref_h.v)     Ji (o_ref - c), high parts
//  r6 = (nref_l.u, nref_l.v, tile, 2^-g)   its low parts; o_ref the origin of
//                                          the rectangle's first tile, whose
//                                          indices are packed in `tile`'s bits
//                                          (x | y << 16); g the grid exponent
// For a pixel offset d = x - c:  den = 1 + e.d,  (u, v) = Ji d / den,
// rho_obj = u^2 + v^2, z_obj = p_z / den.  Jh and nref_h lie on a grid 2^g
// coarse enough that nref_h + Jh (o - o_ref) + Jh (lx, ly) sums exactly in
// FP32 for every tile origin o and pixel offset (lx, ly) of the rectangle
// (see the preprocess).

// Footprint shape for tile-row coverage, FP32 (offsets from c): the ellipse
// {rho_obj <= rho_max} is (d - e0)^T G^-1 (d - e0) <= 1; its boundary at
// height dy (relative to e0) is x = e0x + slope dy +- wsc sqrt(hy^2 - dy^2)
// with slope = g12 / g22, wsc = sqrt(det G) / g22, hy = sqrt(g22); its
// rightmost point is at dy = t = g12 / sqrt(g11), the leftmost at -t.  The
// screen-filter disk is |d| <= rf.  [ilo, ihi] x [jlo, jhi] is the
// pixel-centre index box of the whole footprint (FP64, clipped to the image).
// Derived terms are computed in FP64 and rounded once.
struct RowGeom {
  float cx_hi, cx_lo, cy_hi, cy_lo;
  float e0x, e0y, hy, t, slope, wsc;
  int ilo, ihi, jlo, jhi;
};

// Pixel columns [*ilo, *ihi] that the footprint reaches in the band of
// pixel rows ja..jb.  Over the band, the ellipse's right boundary x(y) is
// concave, so its maximum is at the rightmost point's y clamped to the band
// (likewise the left boundary); the disk is widest at its centre's y
// clamped to the band.  Pixel centres inside the hull of the two intervals,
// widened by a margin that covers the FP32 rounding of these few
// operations, are reported: the result is a superset of the exact cover,
// clipped to the footprint's pixel box.  Written with explicit
// round-to-nearest operations because several kernels evaluate it on the
// same stored values and must agree bit for bit.
__device__ __forceinline__ bool band_pixels(const RowGeom& g, int ja, int jb, float rf, int* pilo,
                                            int* pihi) {
  ja = max(ja, g.jlo);
  jb = min(jb, g.jhi);
  if (ja > jb) return false;
  const float ya = __fsub_rn(__fsub_rn((float)ja + 0.5f, g.cy_hi), g.cy_lo);
  const float yb = __fsub_rn(__fsub_rn((float)jb + 0.5f, g.cy_hi), g.cy_lo);
  const float my = __fmaf_rn(1e-5f, __fadd_rn(fabsf(ya), fabsf(yb)), 1e-3f);
  float lo = INFINITY, hi = -INFINITY;
  if (g.hy > 0.f) {
    const float dya = __fsub_rn(ya, g.e0y), dyb = __fsub_rn(yb, g.e0y);
    if (dyb >= -__fadd_rn(g.hy, my) && dya <= __fadd_rn(g.hy, my)) {
      const float yr = fminf(fmaxf(g.t, dya), dyb);
      const float yl = fminf(fmaxf(-g.t, dya), dyb);
      const float qr = fmaxf(__fmul_rn(__fsub_rn(g.hy, yr), __fadd_rn(g.hy, yr)), 0.f);
      const float ql = fmaxf(__fmul_rn(__fsub_rn(g.hy, yl), __fadd_rn(g.hy, yl)), 0.f);
      hi = __fmaf_rn(g.wsc, __fsqrt_rn(qr), __fmaf_rn(g.slope, yr, g.e0x));
      lo = __fmaf_rn(-g.wsc, __fsqrt_rn(ql), __fmaf_rn(g.slope, yl, g.e0x));
      // the y rounding moves the boundary by up to |slope| my
      const float ms = __fmul_rn(fabsf(g.slope), my);
      hi = __fadd_rn(hi, ms);
      lo = __fsub_rn(lo, ms);
    }
  }
  const float yn = fminf(fmaxf(0.f, ya), yb);
  const float r2 = __fsub_rn(__fmul_rn(rf, rf), __fmul_rn(yn, yn));
  if (r2 >= -__fmul_rn(2.f * rf, my)) {
    const float h = __fadd_rn(__fsqrt_rn(fmaxf(r2, 0.f)), my);
    lo = fminf(lo, -h);
    hi = fmaxf(hi, h);
  }
  if (!(lo <= hi)) return false;
  const float m = __fmaf_rn(1e-5f, __fadd_rn(fabsf(lo), fabsf(hi)), 1e-3f);
  const float xlo = __fadd_rn(__fadd_rn(g.cx_hi, __fsub_rn(lo, m)), g.cx_lo);
  const float xhi = __fadd_rn(__fadd_rn(g.cx_hi, __fadd_rn(hi, m)), g.cx_lo);
  const int ilo = max((int)ceilf(__fsub_rn(fmaxf(xlo, -1.f), 0.5f)), g.ilo);
  const int ihi = min((int)floorf(__fsub_rn(fminf(xhi, 1.0e9f), 0.5f)), g.ihi);
  if (ilo > ihi) return false;
  *pilo = ilo;
  *pihi = ihi;
  return true;
}

// Tile columns [tx0, tx1) that the footprint reaches in tile row ty (the
// preprocess counts with it, the emission writes with it).
__device__ __forceinline__ bool row_tiles(const RowGeom& g, int ty, float rf, int* tx0, int* tx1) {
  int ilo, ihi;
  if (!band_pixels(g, ty * kTile, ty * kTile + kTile - 1, rf, &ilo, &ihi)) return false;
  *tx0 = ilo / kTile;
  *tx1 = ihi / kTile + 1;
  return true;
}

struct Workspace;  // allocator wrapper

struct ParamsDev {
  const float* mu;
  const float* quat;
  const float* scale;
  const float* opacity;
  const float* sh;
  int n;
  int sh_degree;
  // Compressed store (render only; null for FP32 scenes): quat, scale and
  // opacity as IEEE binary16, and the SH of surfel n in row sh_row[n] of
  // sh_table (binary16, rows of 3 (deg+1)^2 values: the codebook of the
  // vector quantisation, then the kept surfels' own SH).
  const uint16_t* quat16 = nullptr;
  const uint16_t* scale16 = nullptr;
  const uint16_t* opacity16 = nullptr;
  const uint32_t* sh_row = nullptr;
  const uint16_t* sh_table = nullptr;
};

// Parameter loads for either store (a kernel-uniform branch).
__device__ __forceinline__ float h2f(uint16_t b) { return __half2float(__ushort_as_half(b)); }
__device__ __forceinline__ float4 load_quat(const ParamsDev& P, int n) {
  if (P.quat16) {
    const uint2 v = *reinterpret_cast<const uint2*>(P.quat16 + 4 * (size_t)n);
    return make_float4(h2f((uint16_t)(v.x & 0xFFFFu)), h2f((uint16_t)(v.x >> 16)), h2f((uint16_t)(v.y & 0xFFFFu)),
                       h2f((uint16_t)(v.y >> 16)));
  }
  return make_float4(P.quat[4 * n], P.quat[4 * n + 1], P.quat[4 * n + 2], P.quat[4 * n + 3]);
}
__device__ __forceinline__ float2 load_scale(const ParamsDev& P, int n) {
  if (P.scale16) {
    const uint32_t v = *reinterpret_cast<const uint32_t*>(P.scale16 + 2 * (size_t)n);
    return make_float2(h2f((uint16_t)(v & 0xFFFFu)), h2f((uint16_t)(v >> 16)));
  }
  return make_float2(P.scale[2 * n], P.scale[2 * n + 1]);
}
__device__ __forceinline__ float load_opacity(const ParamsDev& P, int n) {
  return P.opacity16 ? h2f(P.opacity16[n]) : P.opacity[n];
}

// ---- launch wrappers (each returns cudaError_t from the launch) ----------
// Writes, for the ncand candidates (device count) in surfel-index order,
// depth_key[i] (FP32 depth bits, or all ones when not visible) and idx[i]
// (surfel index); per surfel: rec, rect, tcount, geom.  flags and scan_tmp
// are scratch (n and scan_tmp_words(n) words).
cudaError_t launch_preprocess(const ParamsDev& P, const CamDev& cam, const SetDev& set,
                              float4* rec, uint2* rect, uint32_t* tcount, uint32_t* depth_key,
                              uint32_t* idx, uint32_t* cand, uint32_t* ncand, RowGeom* geom,
                              uint32_t* flags, uint32_t* scan_tmp, cudaStream_t st);

// device-wide exclusive scan of n uint32 values; total (uint32) written to
// *total_dev; tmp must hold scan_tmp_words(n) uint32 words.
size_t scan_tmp_words(int64_t n);
// n_dev (optional): device-side item count <= n (n sizes the grid).
cudaError_t launch_scan(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_dev,
                        uint32_t* tmp, cudaStream_t st, const uint32_t* n_dev = nullptr);

// LSD radix sort of (key, value) pairs over key bits [0, bits); stable.
// Result ends in (keys_out, vals_out) (double-buffering through the alt
// buffers); tmp must hold radix_tmp_words(n) uint32 words.  gsrc/gout
// (optional): also gout[i] = gsrc[vals_out[i]] for the sorted pairs.
size_t radix_tmp_words(int64_t n);
cudaError_t radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                             uint32_t* vals_alt, int64_t n, int bits, uint32_t* tmp,
                             uint32_t** keys_out, uint32_t** vals_out, cudaStream_t st,
                             const uint32_t* n_dev = nullptr, const uint32_t* gsrc = nullptr,
                             uint32_t* gout = nullptr);

cudaError_t launch_gather_counts(const uint32_t* order, const uint32_t* tcount, uint32_t* out,
                                 int64_t n, cudaStream_t st, const uint32_t* n_dev = nullptr);
cudaError_t launch_emit(const uint32_t* order, const uint32_t* offs, const uint32_t* counts,
                        const uint2* rect, const RowGeom* geom, float rf, int64_t n, int tiles_x,
                        uint32_t* keys, uint32_t* vals, cudaStream_t st, const uint32_t* n_dev = nullptr);
cudaError_t launch_ranges(const uint32_t* keys, int64_t K, int2* ranges, int ntiles,
                          cudaStream_t st);
// Tile ids ordered by list length, longest first (launch order of the blends);
// for images with more tiles than the ordering kernel holds, nothing is
// written and the blends take the natural order (pass a null order).
bool tile_order_supported(int ntiles);
cudaError_t launch_tile_order(const int2* ranges, int ntiles, uint32_t* order, cudaStream_t st);

cudaError_t launch_blend_fwd(const CamDev& cam, const SetDev& set, const uint32_t* order, const float4* rec,
                             const RowGeom* geom, const uint32_t* vals, const int2* ranges, float* out,
                             int32_t* n_contrib, int32_t* last, int32_t* med,
                             unsigned long long* counters, cudaStream_t st);

// Long lists composited in segments (see blend.cu).  A tile whose list is
// longer than lseg entries is cut into segments of lseg; the buffers hold up
// to nseg_max segments (split_nseg_max bounds their number).
struct SegBufs {
  int lseg = 0;
  unsigned nseg_max = 0;
  uint32_t* segcnt = nullptr;    // [ntiles] segments per tile (0: whole)
  uint32_t* segoff = nullptr;    // [ntiles] exclusive scan of segcnt
  uint32_t* nseg = nullptr;      // [1] number of segments (device)
  uint32_t* scan_tmp = nullptr;  // scan_tmp_words(ntiles)
  uint32_t* seg_tile = nullptr;  // [nseg_max]
  uint32_t* seg_idx = nullptr;   // [nseg_max]
  float* trans = nullptr;        // [nseg_max][256]
  void* part = nullptr;          // [nseg_max][256] records of seg_part_bytes()
};
size_t seg_part_bytes();
// Segment length for a view of ntiles tiles and K instances on a GPU of sms
// SMs, or 0 to composite whole tiles: views with fewer than two waves of
// tiles (five CTAs per SM) and more than 1024 instances are split so that the
// segments make about two waves (at least 1024 entries each).
inline int split_lseg(int ntiles, int64_t K, int sms) {
  const int64_t slots2 = 2 * (int64_t)sms * 5;
  if (ntiles >= slots2 || K <= 1024) return 0;
  const int64_t per = (K + slots2 - 1) / slots2;
  const int64_t l = (per + 255) / 256 * 256;
  return (int)(l < 1024 ? 1024 : l);
}
// Upper bound of the number of segments, the sum over the split tiles of
// ceil(len / lseg): a split tile has len > lseg, so ceil(len / lseg) <
// 2 len / lseg, and the lengths sum to at most K.
inline int64_t split_nseg_max(int64_t K, int lseg) { return (2 * K + lseg - 1) / lseg; }
cudaError_t launch_blend_fwd_split(const CamDev& cam, const SetDev& set, const uint32_t* order, const float4* rec,
                                   const RowGeom* geom, const uint32_t* vals, const int2* ranges, float* out,
                                   int32_t* n_contrib, int32_t* last, int32_t* med, unsigned long long* counters,
                                   const SegBufs& sb, cudaStream_t st);

// One view of a batched (serving) forward blend.
struct BlendJob {
  CamDev cam;
  SetDev set;
  float rf;
  int tile_begin;  // first work item of this view in the batch
  const float4* rec;
  const RowGeom* geom;
  const uint32_t* vals;
  const int2* ranges;
  float* out;
  int32_t* n_contrib;
};
constexpr int kMaxBatch = 16;
struct BlendBatch {
  BlendJob job[kMaxBatch];
  int njobs;
  int total_tiles;
  unsigned* counter;  // zeroed before the launch
  unsigned long long* work;  // [2] evaluated and blended pairs, added to (may be null)
};
cudaError_t launch_blend_fwd_batched(const BlendBatch& batch, int grid, cudaStream_t st);

struct AdjDev {
  const float* set[3];
  uint32_t mask[3];
  int n_sets;
};

// Per-surfel intermediate gradient record of the blend backward.
constexpr int kGradRec = 16;  // Ji(4) e(2) c(2) p_z(1) opacity(1) rgb(3) n(3)

cudaError_t launch_blend_bwd(const CamDev& cam, const SetDev& set, const uint32_t* order, const float4* rec,
                             const RowGeom* geom, const uint32_t* vals, const int2* ranges, const float* out,
                             const int32_t* last, const int32_t* med, const AdjDev& adj,
                             float* grec, float* screen, int n, int64_t K, unsigned long long* counters,
                             cudaStream_t st);

// Trim contribution (Sec. 3.3, Eq. 3) of one view over the frame's tile
// lists: per surfel the support count and the sum of alpha^gamma T^(1-gamma)
// (csum, ccnt: [N], accumulated).
cudaError_t launch_blend_contrib(const CamDev& cam, const SetDev& set, float gamma, const uint32_t* order,
                                 const float4* rec, const RowGeom* geom, const uint32_t* vals,
                                 const int2* ranges, float* csum, uint32_t* ccnt, cudaStream_t st);
// Zero the candidates' csum/ccnt (when zero_cand), run the contribution blend
// and add weight * csum / ccnt to contrib[n] for the candidates (contrib may
// be null).
cudaError_t launch_contribution(const CamDev& cam, const SetDev& set, float gamma, float weight,
                                const uint32_t* order, const float4* rec, const RowGeom* geom,
                                const uint32_t* vals, const int2* ranges, const uint32_t* cand,
                                const uint32_t* ncand, int64_t n, bool zero_cand, float* csum, uint32_t* ccnt,
                                float* contrib, cudaStream_t st);
// Visible frequency of points (Sec. 4 crop volume): a view as the count
// kernel reads it (world-to-camera rotation row-major, translation,
// intrinsics, image size).
struct VisCam {
  float R[9], t[3];
  float fx, fy, cx, cy, W, H;
};
cudaError_t launch_visibility_count(const float* pts, int64_t n, float sigma, float lowpass, float near_plane,
                                    const VisCam* cams, int nviews, uint32_t* counts, cudaStream_t st);
// keep[j] = counts[j] >= min_count; zrange = (min z, max z) of the kept
// points (NaN when none); tmp: 2 ints of device scratch.
cudaError_t launch_visibility_keep(const float* pts, int64_t n, const uint32_t* counts, uint32_t min_count,
                                   uint8_t* keep, float* zrange, int* tmp, cudaStream_t st);
// Geometric loss terms (see train.cu): depth-normal consistency and depth
// distortion; adds their adjoints to adj ([11][H][W]) and writes loss[0..1];
// tmp: geometry_tmp_bytes(W, H).
size_t geometry_tmp_bytes(int W, int H);
cudaError_t launch_geometry_loss(int W, int H, float fx, float fy, float cx, float cy, const float* out,
                                 float w_normal, float w_dist, float* adj, float* loss, void* tmp, cudaStream_t st);
// Bias-corrected Adam step (bc1 = 1 - beta1^t, bc2 = 1 - beta2^t).
cudaError_t launch_adam(int64_t n, float* p, const float* g, float* m, float* v, float lr, float b1, float b2,
                        float eps, float bc1, float bc2, cudaStream_t st);
// Densification actions (0 drop, 1 keep, 2 clone, 3 split) and output row
// counts; the rows themselves; row gather (fresh rows zero); activations.
cudaError_t launch_densify_plan(int64_t n, const uint8_t* sel, const uint8_t* keep, const float* scale,
                                const float* opac, float dense_thr, float min_opacity, uint8_t* action, uint32_t* rows,
                                cudaStream_t st);
cudaError_t launch_densify_apply(int64_t n, int sh_degree, bool log_scale, const uint8_t* action, const uint32_t* off,
                                 const float* xi, const float* mu, const float* quat, const float* scale,
                                 const float* opac, const float* sh, float* mu_o, float* quat_o, float* scale_o,
                                 float* opac_o, float* sh_o, int32_t* src, uint8_t* fresh, cudaStream_t st);
cudaError_t launch_gather_rows(int64_t n_out, int width, const int32_t* src, const uint8_t* fresh, const float* in,
                               float* out, cudaStream_t st);
cudaError_t launch_activate(int64_t n, const float* ls, const float* lo, float* scale, float* opac, cudaStream_t st);
cudaError_t launch_activate_grad(int64_t n, const float* scale, const float* opac, float* gs, float* go,
                                 cudaStream_t st);
// Percentile pruning (Sec. 3.3): the k-th smallest value of contrib (k >= 1;
// radix select on order-preserving keys), keep[i] = contrib[i] > it, the
// bound to *bound (device, may be null); k = 0 keeps everything and writes
// -inf.  tmp: select_tmp_words() words.
size_t select_tmp_words();
cudaError_t launch_prune(int64_t n, const float* contrib, int64_t k, uint8_t* keep, float* bound,
                         uint32_t* tmp, cudaStream_t st);

cudaError_t launch_preprocess_bwd(const ParamsDev& P, const CamDev& cam, const uint32_t* cand,
                                  const uint32_t* ncand, const uint32_t* tcount, const float* grec,
                                  const gs_param_grads& G, cudaStream_t st);

cudaError_t launch_loss(int W, int H, const float* out, const float* tgt, const float* tinv,
                        const gs_loss_weights& w, float* adj_total, float* adj_ssim,
                        float* adj_l1, float* losses, float* tmp, cudaStream_t st);
size_t loss_tmp_floats(int W, int H);

cudaError_t launch_densify_accumulate(const uint2* rect, const float* screen, int n,
                                      int n_sets, float* stats, cudaStream_t st);
cudaError_t launch_densify_select(int64_t n, const float* stats, const float* scale, float omega,
                                  float grad_thr, float eta_thr, uint8_t* mask, float* g_out,
                                  float* k_out, double* tmp, cudaStream_t st);
size_t densify_tmp_doubles(int64_t n);
cudaError_t launch_elongation(int64_t n, const float* scale, float eta_thr, uint8_t* keep,
                              cudaStream_t st);

inline unsigned div_up(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// Launch accounting and optional per-kernel CUDA-event timing (diagnostics:
// gs_kernel_launches, gs_profile_enable, gs_profile_read).
enum ProfId {
  kProfPreprocess = 0,
  kProfSort = 1,
  kProfBlendFwd = 2,
  kProfLoss = 3,
  kProfBlendBwd = 4,
  kProfPreprocessBwd = 5,
  kProfDensify = 6,
  kProfContrib = 7,
  kProfVqAssign = 8,
  kProfCount = 9
};
void count_launch(int n = 1);
void set_last_error(const char* msg);
void prof_begin(int id, cudaStream_t st);
void prof_end(int id, cudaStream_t st);

struct ProfScope {
  int id;
  cudaStream_t st;
  ProfScope(int i, cudaStream_t s) : id(i), st(s) { prof_begin(id, st); }
  ~ProfScope() { prof_end(id, st); }
};


// ---- Vector quantisation of SH (vq.cu) --------------------------------------
// Scratch of one K-means / assignment call (m quantised vectors of C
// coefficients, width D = C + 2 rounded up to 16, K entries).
struct VqBufs {
  uint32_t* rows = nullptr;              // [m] quantised surfels in index order
  uint16_t* xr = nullptr;                // [m][C] binary16 vectors, row-major
  uint16_t* xt = nullptr;                // [m_pad][D] augmented vectors, core-matrix layout
  uint16_t* ct = nullptr;                // [K][D] augmented codebook, core-matrix layout
  float2* hl = nullptr;                  // [K] ||c||^2 as two binary16 values
  unsigned long long* best64 = nullptr;  // [m_pad] (score key, entry)
  int32_t* best_idx = nullptr;           // [m]
  unsigned long long* sums = nullptr;    // [K][C] exact sums (units of 2^-24)
  unsigned int* cnt = nullptr;           // [K]
  int* err = nullptr;                    // [1] 0 ok, 1 pipeline timeout, 2 value outside binary16
};
// D for an SH degree; *C = 3 (deg + 1)^2.
int vq_width(int sh_degree, int* C);
// Lists the surfels with (keep[i] != 0) == want (rows may be null: offsets and total only).
cudaError_t launch_vq_list(const uint8_t* keep, int n, int want, uint32_t* flags, uint32_t* offs, uint32_t* total,
                           uint32_t* scan_tmp, uint32_t* rows, cudaStream_t st);
cudaError_t launch_vq_pack_x(const float* sh, const VqBufs& b, int m, int C, int D, cudaStream_t st);
cudaError_t launch_vq_init(const VqBufs& b, int m, int C, const float* u, int K, uint16_t* cb, cudaStream_t st);
// tensor: tcgen05 kernel (K a multiple of 256), else the CUDA-core kernel.
cudaError_t launch_vq_assign(const VqBufs& b, int m, int C, int D, const uint16_t* cb, int K, bool tensor, int num_sms,
                             cudaStream_t st);
cudaError_t launch_vq_accum(const VqBufs& b, int m, int C, const uint16_t* cb, int K, bool with_sums,
                            double* objective, cudaStream_t st);
cudaError_t launch_vq_update(const VqBufs& b, int C, uint16_t* cb, int K, cudaStream_t st);
cudaError_t launch_vq_scatter(const VqBufs& b, int m, int32_t* assign, cudaStream_t st);
cudaError_t launch_vq_pack_scene(int n, int C, int K, const float* quat, const float* scale, const float* opacity,
                                 const float* sh, const uint8_t* keep, const int32_t* assign,
                                 const uint32_t* kept_offs, const uint16_t* codebook, uint16_t* q16, uint16_t* s16,
                                 uint16_t* o16, uint32_t* sh_row, uint16_t* table, int* err, cudaStream_t st);
cudaError_t launch_vq_check_rows(const uint32_t* sh_row, int n, uint32_t rows, int* err, cudaStream_t st);

}  // namespace gs2d
