// Per-pixel compositing (forward) and its adjoint (reverse replay).
//
// Forward (Eq. 1, Sec. 3.1, with the 2DGS surfel model and the low-pass
// filter of Sec. 3.2): one CTA of 128 threads per 16 x 16 tile; each warp
// covers an 8 x 8 block of pixels and each thread two pixels of one column,
// four rows apart, so that an entry read from shared memory serves two
// pixels and the two per-pixel dependency chains interleave.  The tile's
// depth-sorted surfel list is staged through shared memory in batches of
// 256 entries; while staging, each entry's footprint is tested against the
// tile's four warp blocks (a conservative cover from the stored footprint
// shape) and warps skip entries that cannot touch them.  Each pixel
// intersects its ray with the surfel plane (rho_obj), takes the
// screen-space filter (rho_scr) where smaller, and composites front to back
// until the transmittance would drop below T_min.
//
// Backward: the same tiles replay each pixel's list back to front from the
// final transmittance, T_before = T_after / (1 - alpha), with suffix sums
// for d L / d alpha.  A thread adds the gradients of its two pixels, the
// warp reduces them with a reduce-scatter of shuffles (one reduction per 64
// pixels), the tile sums them in shared memory, and they reach global
// memory once per (surfel, tile).
#include <math.h>

#include "gs2d_internal.cuh"

namespace gs2d {
namespace {

constexpr int kThreads = 128;  // threads per tile CTA, two pixels each
constexpr int kBatch = 256;    // list entries staged per batch
constexpr int kTilePix = 2 * kThreads;  // pixels of a tile, two per thread

// Hardware approximations (relative error about 2^-22), the same
// instructions in both blends so that the replay reproduces the forward's
// decisions exactly.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
constexpr float kNegHalfLog2e = -0.72134752044448170f;  // -log2(e) / 2

// Pixels of thread t within its tile: warp w covers columns 8 (w & 1) .. +7
// and rows 8 (w >> 1) .. +7; lane l takes column l & 7 and rows l >> 3 and
// (l >> 3) + 4 of that block.
__device__ __forceinline__ int local_x(int t) { return (((t >> 5) & 1) << 3) | (t & 7); }
__device__ __forceinline__ int local_y(int t) { return ((t >> 6) << 3) | ((t >> 3) & 3); }

// Staged entry: s0 = (c.x, c.y relative to the tile origin, e.x, e.y),
// s1 = Jh, s2 = (p_z, opacity, r, g), s3 = (b, n.x, n.y, n.z), s4 = Jl,
// s5 = (nu0h, nv0h, nu0l, nv0l); wmask bit w set when the footprint may
// reach warp w's pixel block.
//
// Tile-relative ray-splat coordinates.  For a pixel at offset (lx, ly) from
// the tile origin o, Ji d = Ji (o - c) + Ji (lx, ly) = n0 + Ji (lx, ly).  Held
// in FP32 as Ji d, the coordinates of an ill-conditioned footprint (a nearly
// edge-on or elongated disk: large Ji, pixel far from c along the long axis)
// would carry an absolute error of about 2^-24 |Ji| |d|, far above the
// error of the exact value near the support boundary.  The preprocess splits
// Ji = Jh + Jl and the offset of the surfel's first tile origin o_ref,
// Ji (o_ref - c) = nref_h + nref_l, on a power-of-two grid 2^g chosen from the
// magnitudes over the surfel's tile rectangle: the high parts (nref_h on
// multiples of 2^g, Jh on multiples of 2^(g+1)) are so coarse that
// nref_h + Jh (o - o_ref) + Jh (lx, ly) is exact in FP32 (o - o_ref are
// multiples of 16, lx, ly half-integers below 16, every partial sum stays
// below 2^(g+24)); the low parts (about 2^g) carry the rest with negligible
// FP32 rounding.  Per (entry, tile) the staging forms
// n0h = nref_h + Jh (o - o_ref) (exact) and n0l = nref_l + Jl (o - o_ref) with
// four FMAs each; per pixel
// Ji d = [n0h + Jh (lx, ly)] + [n0l + Jl (lx, ly)] is then accurate to the
// FP32 rounding of the result itself, whatever the conditioning of Ji.
struct Staged {
  float4 s0, s1, s2, s3, s4, s5;
  uint32_t wmask;
};


__device__ __forceinline__ Staged stage_entry(const float4* __restrict__ rec,
                                              const RowGeom* __restrict__ geom, uint32_t s,
                                              int tx0, int ty0, int H, float rf) {
  const float4* R = rec + (size_t)s * kRecF4;
  const float4 r0 = R[0], r1 = R[1], r2 = R[2], r3 = R[3], r4 = R[4], r5 = R[5], r6 = R[6];
  Staged e;
  // centre relative to the tile origin: (c_hi - x0) + c_lo keeps the
  // offset accurate to its own rounding
  e.s0 = make_float4(__fadd_rn(__fsub_rn(r0.x, (float)tx0), r0.z),
                     __fadd_rn(__fsub_rn(r0.y, (float)ty0), r0.w), r2.x, r2.y);
  e.s2 = make_float4(r2.z, r2.w, r3.x, r3.y);
  e.s3 = make_float4(r3.z, r3.w, r4.x, r4.y);
  e.s1 = r1;
  e.s4 = r5;
  // n0 at this tile's origin (o - o_ref: multiples of 16, exact); the low
  // part's grid rounding q moves to the high part (both sums exact), so the
  // low part stays below 2^(g-1) whatever the tile's distance from o_ref
  const uint32_t rt = __float_as_uint(r6.z);
  const float dox = (float)(tx0 - (int)(rt & 0xFFFFu) * kTile), doy = (float)(ty0 - (int)(rt >> 16) * kTile);
  const float ug = r6.w, dg = __frcp_rn(ug);
  const float hu = __fmaf_rn(r1.x, dox, __fmaf_rn(r1.y, doy, r4.z));
  const float hv = __fmaf_rn(r1.z, dox, __fmaf_rn(r1.w, doy, r4.w));
  const float lu = __fmaf_rn(r5.x, dox, __fmaf_rn(r5.y, doy, r6.x));
  const float lv = __fmaf_rn(r5.z, dox, __fmaf_rn(r5.w, doy, r6.y));
  const float qu = __fmul_rn(rintf(__fmul_rn(lu, ug)), dg), qv = __fmul_rn(rintf(__fmul_rn(lv, ug)), dg);
  e.s5 = make_float4(__fadd_rn(hu, qu), __fadd_rn(hv, qv), __fsub_rn(lu, qu), __fsub_rn(lv, qv));
  const RowGeom g = geom[s];
  uint32_t m = 0u;
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    const int ja = ty0 + 8 * b;
    if (ja >= H) break;
    int ilo, ihi;
    if (!band_pixels(g, ja, min(ja + 7, H - 1), rf, &ilo, &ihi)) continue;
    if (ilo <= tx0 + 7 && ihi >= tx0) m |= 1u << (2 * b);
    if (ilo <= tx0 + 15 && ihi >= tx0 + 8) m |= 1u << (2 * b + 1);
  }
  e.wmask = m;
  return e;
}

// Per warp, the batch's entries whose footprint may reach the warp's pixel
// block, as kBatch / 32 bit words (ballots of the staged masks); the loops
// below visit only their set bits, so entries that miss the block cost
// nothing (long lists, where most entries miss a given block).
constexpr int kWords = kBatch / 32;
template <int NW = kWords>
__device__ __forceinline__ void warp_entry_bits(const uint32_t* sm, int nb, int warp, int lane,
                                                uint32_t* wb) {
#pragma unroll
  for (int j = 0; j < NW; ++j) {
    const int e = 32 * j + lane;
    const uint32_t w = __ballot_sync(0xffffffffu, e < nb && ((sm[e] >> warp) & 1u));
    if (lane == 0) wb[j] = w;
  }
  __syncwarp();
}

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

// The rest of one pair's evaluation from its plane coordinates (nu, nv) =
// Ji d.  Shared by every blend; explicit round-to-nearest operations so that
// the forward and the backward take bit-identical decisions.
__device__ __forceinline__ void finish_pair(float lx, float ly, float4 s0, float nu, float nv, float opac,
                                            const SetDev& set, Pair& q) {
  q.dx = __fsub_rn(lx, s0.x);
  q.dy = __fsub_rn(ly, s0.y);
  const float den = __fmaf_rn(s0.z, q.dx, __fmaf_rn(s0.w, q.dy, 1.0f));
  q.nu = nu;
  q.nv = nv;
  q.rden = rcp_approx(den);
  const float u = __fmul_rn(q.nu, q.rden), v = __fmul_rn(q.nv, q.rden);
  const float rho_obj = den > 0.f ? __fmaf_rn(u, u, __fmul_rn(v, v)) : INFINITY;
  const float rho_scr = __fmul_rn(set.sinv, __fmaf_rn(q.dx, q.dx, __fmul_rn(q.dy, q.dy)));
  q.obj = rho_obj <= rho_scr;  // false for NaN (edge-on disks)
  q.rho = q.obj ? rho_obj : rho_scr;
  q.G = ex2_approx(__fmul_rn(kNegHalfLog2e, q.rho));
  q.alpha = fminf(set.alpha_max, __fmul_rn(opac, q.G));
  q.hit = (q.rho <= set.rho_max) && (q.alpha >= set.alpha_min);
}

// One entry against a thread's two pixels, (lx, ly) and (lx, ly + 4) from
// the tile origin: the exact grid sums nu0h + Jh (lx, ly) (row B adds 4 Jh
// exactly), plus the small low-part corrections (see Staged).
__device__ __forceinline__ void eval_two(float lx, float ly, float4 s0, float4 jh, float4 jl, float4 n0,
                                         float opac, const SetDev& set, Pair& qa, Pair& qb) {
  const float suA = __fmaf_rn(jh.x, lx, __fmaf_rn(jh.y, ly, n0.x));
  const float svA = __fmaf_rn(jh.z, lx, __fmaf_rn(jh.w, ly, n0.y));
  const float cuA = __fmaf_rn(jl.x, lx, __fmaf_rn(jl.y, ly, n0.z));
  const float cvA = __fmaf_rn(jl.z, lx, __fmaf_rn(jl.w, ly, n0.w));
  const float suB = __fmaf_rn(jh.y, 4.f, suA), svB = __fmaf_rn(jh.w, 4.f, svA);
  const float cuB = __fmaf_rn(jl.y, 4.f, cuA), cvB = __fmaf_rn(jl.w, 4.f, cvA);
  finish_pair(lx, ly, s0, __fadd_rn(suA, cuA), __fadd_rn(svA, cvA), opac, set, qa);
  finish_pair(lx, __fadd_rn(ly, 4.f), s0, __fadd_rn(suB, cuB), __fadd_rn(svB, cvB), opac, set, qb);
}

// ---------------------------------------------------------------------------
// Forward.

// Running sums of one pixel.  Z is accumulated relative to zr, the depth of
// the first blended pair: sum w (z - zr) keeps the distortion terms z A - Z
// free of the cancellation between depths of hundreds of metres (both are
// invariant under a common shift of z), and sum w z = sum w (z - zr) + zr A.
struct FwdPix {
  float T, C0, C1, C2, A, Zs, zr, I, N0, N1, N2, D, M;
  int cnt, lastpos, medpos;
  unsigned evaluated;
  bool done;
};

__device__ __forceinline__ void fwd_init(FwdPix& p, bool inside) {
  p.T = 1.f;
  p.C0 = p.C1 = p.C2 = p.A = p.Zs = p.zr = p.I = p.N0 = p.N1 = p.N2 = p.D = p.M = 0.f;
  p.cnt = 0;
  p.lastpos = 0;
  p.medpos = -1;
  p.evaluated = 0;
  p.done = !inside;
}

// One list entry (position pos, already evaluated as q) against one pixel.
// Branch-free, so that the two pixels of a thread interleave: a pair that is
// not blended updates the sums with weight 0 (and a finite depth of 1), which
// leaves them unchanged.
template <bool kFixedRef = false>
__device__ __forceinline__ void fwd_step(FwdPix& p, const Pair& q, float4 e2, float4 e3, int pos,
                                         const SetDev& set) {
  p.evaluated += p.done ? 0u : 1u;
  const bool h = !p.done && q.hit;
  const float Tn = p.T * (1.f - q.alpha);
  const bool stop = h && Tn < set.T_min;
  const bool bl = h && !stop;
  p.done = p.done || stop;
  const float w = bl ? q.alpha * p.T : 0.f;
  const float z = bl ? (q.obj ? e2.x * q.rden : e2.x) : 1.f;
  p.C0 = fmaf(w, e2.z, p.C0);
  p.C1 = fmaf(w, e2.w, p.C1);
  p.C2 = fmaf(w, e3.x, p.C2);
  if constexpr (!kFixedRef) p.zr = (bl && p.cnt == 0) ? z : p.zr;
  const float zs = z - p.zr;
  p.D = fmaf(2.f * w, fmaf(zs, p.A, -p.Zs), p.D);
  p.A += w;
  p.Zs = fmaf(w, zs, p.Zs);
  p.I = fmaf(w, rcp_approx(z), p.I);
  p.N0 = fmaf(w, e3.y, p.N0);
  p.N1 = fmaf(w, e3.z, p.N1);
  p.N2 = fmaf(w, e3.w, p.N2);
  const bool m = bl && p.T > 0.5f;
  p.M = m ? z : p.M;
  p.medpos = m ? pos : p.medpos;
  p.T = bl ? Tn : p.T;
  p.cnt += bl ? 1 : 0;
  p.lastpos = bl ? pos + 1 : p.lastpos;
}

__device__ __forceinline__ void fwd_store(const FwdPix& p, const CamDev& cam, const SetDev& set, int px,
                                          int py, float* __restrict__ out, int32_t* __restrict__ n_contrib,
                                          int32_t* __restrict__ last, int32_t* __restrict__ med) {
  if (px >= cam.W || py >= cam.H) return;
  const size_t HW = (size_t)cam.W * cam.H;
  const size_t i = (size_t)py * cam.W + px;
  out[i] = p.C0 + p.T * set.bg[0];
  out[HW + i] = p.C1 + p.T * set.bg[1];
  out[2 * HW + i] = p.C2 + p.T * set.bg[2];
  out[3 * HW + i] = p.A;
  out[4 * HW + i] = fmaf(p.zr, p.A, p.Zs);
  out[5 * HW + i] = p.I;
  out[6 * HW + i] = p.M;
  out[7 * HW + i] = p.N0;
  out[8 * HW + i] = p.N1;
  out[9 * HW + i] = p.N2;
  out[10 * HW + i] = p.D;
  out[11 * HW + i] = p.T;
  if (n_contrib) n_contrib[i] = p.cnt;
  if (last) last[i] = p.lastpos;
  if (med) med[i] = p.medpos;
}

// Shared-memory staging area of one CTA.
struct FwdSmem {
  float4 s0[kBatch], s1[kBatch], s2[kBatch], s3[kBatch], s4[kBatch], s5[kBatch];
  uint32_t sm[kBatch];
  uint32_t wbits[kThreads / 32][kWords];
  unsigned long long tot[2];
};

// Forward blend of tile (bx, by) of one view by the whole CTA.
__device__ __forceinline__ void blend_fwd_tile(
    FwdSmem& sh, const CamDev& cam, const SetDev& set, float rf, const float4* __restrict__ rec,
    const RowGeom* __restrict__ geom, const uint32_t* __restrict__ vals, const int2* __restrict__ ranges,
    float* __restrict__ out, int32_t* __restrict__ n_contrib, int32_t* __restrict__ last,
    int32_t* __restrict__ med, unsigned long long* __restrict__ counters, int bx, int by, int lseg = 0) {
  const int tile = by * cam.tiles_x + bx;
  const int tx0 = bx * kTile, ty0 = by * kTile;
  const int lxi = local_x(threadIdx.x), lyi = local_y(threadIdx.x);
  const int px = tx0 + lxi, pyA = ty0 + lyi, pyB = pyA + 4;
  const int warp = threadIdx.x >> 5;
  const float lx = (float)lxi + 0.5f, lyA = (float)lyi + 0.5f;
  const int2 rg = ranges[tile];
  const int len = rg.y - rg.x;
  if (lseg > 0 && len > lseg) return;  // a long list: composited in segments
  FwdPix a, b;
  fwd_init(a, px < cam.W && pyA < cam.H);
  fwd_init(b, px < cam.W && pyB < cam.H);
  for (int b0 = 0; b0 < len; b0 += kBatch) {
    if (__syncthreads_count(a.done && b.done) == kThreads) break;
    for (int t = threadIdx.x; t < kBatch; t += kThreads) {
      if (b0 + t < len) {
        const Staged e = stage_entry(rec, geom, vals[rg.x + b0 + t], tx0, ty0, cam.H, rf);
        sh.s0[t] = e.s0;
        sh.s1[t] = e.s1;
        sh.s2[t] = e.s2;
        sh.s3[t] = e.s3;
        sh.s4[t] = e.s4;
        sh.s5[t] = e.s5;
        sh.sm[t] = e.wmask;
      }
    }
    __syncthreads();
    const int nb = min(kBatch, len - b0);
    warp_entry_bits(sh.sm, nb, warp, threadIdx.x & 31, sh.wbits[warp]);
    for (int j = 0; j < kWords && !(a.done && b.done); ++j) {
      uint32_t bits = sh.wbits[warp][j];
      while (bits != 0u && !(a.done && b.done)) {
        const int k = 32 * j + __ffs(bits) - 1;
        bits &= bits - 1u;
        const float4 e0 = sh.s0[k], e1 = sh.s1[k], e2 = sh.s2[k], e3 = sh.s3[k];
        Pair qa, qb;
        eval_two(lx, lyA, e0, e1, sh.s4[k], sh.s5[k], e2.y, set, qa, qb);
        fwd_step(a, qa, e2, e3, b0 + k, set);
        fwd_step(b, qb, e2, e3, b0 + k, set);
      }
    }
  }
  fwd_store(a, cam, set, px, pyA, out, n_contrib, last, med);
  fwd_store(b, cam, set, px, pyB, out, n_contrib, last, med);
  if (counters) {
    // per-tile totals of evaluated and blended pairs (performance counters)
    unsigned long long* tot = sh.tot;
    if (threadIdx.x == 0) tot[0] = tot[1] = 0ull;
    __syncthreads();
    unsigned e = a.evaluated + b.evaluated, c = (unsigned)(a.cnt + b.cnt);
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

// One CTA per tile; block b takes tile order[b] (longest lists first).
__global__ void __launch_bounds__(kThreads, 5) blend_fwd_kernel(
    CamDev cam, SetDev set, float rf, const uint32_t* __restrict__ order, const float4* __restrict__ rec,
    const RowGeom* __restrict__ geom, const uint32_t* __restrict__ vals, const int2* __restrict__ ranges,
    float* __restrict__ out, int32_t* __restrict__ n_contrib, int32_t* __restrict__ last,
    int32_t* __restrict__ med, unsigned long long* __restrict__ counters, int lseg) {
  __shared__ FwdSmem sh;
  const int t = order ? (int)order[blockIdx.x] : (int)blockIdx.x;
  blend_fwd_tile(sh, cam, set, rf, rec, geom, vals, ranges, out, n_contrib, last, med, counters,
                 t % cam.tiles_x, t / cam.tiles_x, lseg);
}

// ---------------------------------------------------------------------------
// Long lists, composited in segments.
//
// When an image has too few tiles to fill the GPU and some tiles carry long
// lists (a small view of a large scene), a tile's list is cut into segments
// of lseg entries that separate CTAs process:
//   1. seg_trans_kernel: per segment and pixel, the product of (1 - alpha)
//      over the segment's pairs that pass the support and cutoff tests (no
//      stop);
//   2. seg_blend_kernel: per segment, the pixel enters with the product of
//      the segments in front (the transmittance it would have there had
//      nothing stopped) and composites the segment with the forward's rules,
//      the stop included.  A pixel that stopped in an earlier segment enters
//      below T_min and blends nothing;
//   3. seg_merge_kernel: per tile and pixel, the segments are combined in
//      order.  Sums add; the distortion adds the cross terms
//      2 (A_front Zs_seg - Zs_front A_seg) (depths relative to one reference,
//      the tile's first centre depth); the median comes from the last
//      segment that has one; T and the stop from the segment where blending
//      ended.
// The result equals the one-CTA compositing up to the rounding of T's
// products (decisions within a hair of a threshold may differ).

struct SegPart {
  float4 f0;  // C0, C1, C2, A
  float4 f1;  // Zs (relative to the reference), I, N0, N1
  float4 f2;  // N2, D, M, T after the segment
  int4 f3;    // median position, count, last position, stopped
};

// Segment b of the split tiles: its tile and its index within the tile.
__device__ __forceinline__ bool seg_of(const uint32_t* seg_tile, const uint32_t* seg_idx, const uint32_t* nseg,
                                       int b, int* tile, int* s) {
  if ((uint32_t)b >= *nseg) return false;
  *tile = (int)seg_tile[b];
  *s = (int)seg_idx[b];
  return true;
}

// Stage entries [b0, b0 + nb) of the tile's list (shared by the segment kernels).
__device__ __forceinline__ void stage_batch(FwdSmem& sh, const float4* __restrict__ rec,
                                            const RowGeom* __restrict__ geom, const uint32_t* __restrict__ vals,
                                            int base, int nb, int tx0, int ty0, int H, float rf) {
  for (int t = threadIdx.x; t < kBatch; t += kThreads) {
    if (t < nb) {
      const Staged e = stage_entry(rec, geom, vals[base + t], tx0, ty0, H, rf);
      sh.s0[t] = e.s0;
      sh.s1[t] = e.s1;
      sh.s2[t] = e.s2;
      sh.s3[t] = e.s3;
      sh.s4[t] = e.s4;
      sh.s5[t] = e.s5;
      sh.sm[t] = e.wmask;
    }
  }
}

__global__ void __launch_bounds__(kThreads) seg_trans_kernel(
    CamDev cam, SetDev set, float rf, const float4* __restrict__ rec, const RowGeom* __restrict__ geom,
    const uint32_t* __restrict__ vals, const int2* __restrict__ ranges, int lseg,
    const uint32_t* __restrict__ seg_tile, const uint32_t* __restrict__ seg_idx, const uint32_t* __restrict__ nseg,
    float* __restrict__ trans) {
  __shared__ FwdSmem sh;
  int tile, s;
  if (!seg_of(seg_tile, seg_idx, nseg, blockIdx.x, &tile, &s)) return;
  const int tx0 = (tile % cam.tiles_x) * kTile, ty0 = (tile / cam.tiles_x) * kTile;
  const int lxi = local_x(threadIdx.x), lyi = local_y(threadIdx.x);
  const int warp = threadIdx.x >> 5;
  const float lx = (float)lxi + 0.5f, lyA = (float)lyi + 0.5f;
  const int2 rg = ranges[tile];
  const int e0 = s * lseg, e1 = min(rg.y - rg.x, e0 + lseg);
  float TA = 1.f, TB = 1.f;
  for (int b0 = e0; b0 < e1; b0 += kBatch) {
    const int nb = min(kBatch, e1 - b0);
    __syncthreads();
    stage_batch(sh, rec, geom, vals, rg.x + b0, nb, tx0, ty0, cam.H, rf);
    __syncthreads();
    warp_entry_bits(sh.sm, nb, warp, threadIdx.x & 31, sh.wbits[warp]);
    for (int j = 0; j < kWords; ++j) {
      uint32_t bits = sh.wbits[warp][j];
      while (bits != 0u) {
        const int k = 32 * j + __ffs(bits) - 1;
        bits &= bits - 1u;
        const float4 f0 = sh.s0[k], f1 = sh.s1[k], f2 = sh.s2[k];
        Pair qa, qb;
        eval_two(lx, lyA, f0, f1, sh.s4[k], sh.s5[k], f2.y, set, qa, qb);
        TA = qa.hit ? TA * (1.f - qa.alpha) : TA;
        TB = qb.hit ? TB * (1.f - qb.alpha) : TB;
      }
    }
  }
  trans[(size_t)blockIdx.x * kTilePix + threadIdx.x] = TA;
  trans[(size_t)blockIdx.x * kTilePix + kThreads + threadIdx.x] = TB;
}

__device__ __forceinline__ void seg_store(const FwdPix& p, bool inside, SegPart* __restrict__ part, int slot) {
  SegPart q;
  q.f0 = make_float4(p.C0, p.C1, p.C2, p.A);
  q.f1 = make_float4(p.Zs, p.I, p.N0, p.N1);
  q.f2 = make_float4(p.N2, p.D, p.M, p.T);
  q.f3 = make_int4(p.medpos, p.cnt, p.lastpos, (inside && p.done) ? 1 : 0);
  part[slot] = q;
}

__global__ void __launch_bounds__(kThreads) seg_blend_kernel(
    CamDev cam, SetDev set, float rf, const float4* __restrict__ rec, const RowGeom* __restrict__ geom,
    const uint32_t* __restrict__ vals, const int2* __restrict__ ranges, int lseg,
    const uint32_t* __restrict__ seg_tile, const uint32_t* __restrict__ seg_idx, const uint32_t* __restrict__ nseg,
    const float* __restrict__ trans, SegPart* __restrict__ part, unsigned long long* __restrict__ counters) {
  __shared__ FwdSmem sh;
  int tile, s;
  if (!seg_of(seg_tile, seg_idx, nseg, blockIdx.x, &tile, &s)) return;
  const int tx0 = (tile % cam.tiles_x) * kTile, ty0 = (tile / cam.tiles_x) * kTile;
  const int lxi = local_x(threadIdx.x), lyi = local_y(threadIdx.x);
  const int px = tx0 + lxi, pyA = ty0 + lyi, pyB = pyA + 4;
  const int warp = threadIdx.x >> 5;
  const float lx = (float)lxi + 0.5f, lyA = (float)lyi + 0.5f;
  const int2 rg = ranges[tile];
  const int e0 = s * lseg, e1 = min(rg.y - rg.x, e0 + lseg);
  const bool inA = px < cam.W && pyA < cam.H, inB = px < cam.W && pyB < cam.H;
  FwdPix a, b;
  fwd_init(a, inA);
  fwd_init(b, inB);
  // transmittance in front: the segments before this one (contiguous)
  const int first = (int)blockIdx.x - s;
  for (int q = 0; q < s; ++q) {
    a.T *= trans[(size_t)(first + q) * kTilePix + threadIdx.x];
    b.T *= trans[(size_t)(first + q) * kTilePix + kThreads + threadIdx.x];
  }
  const float zref = rec[(size_t)vals[rg.x] * kRecF4 + 2].z;  // the tile's first centre depth
  a.zr = zref;
  b.zr = zref;
  for (int b0 = e0; b0 < e1; b0 += kBatch) {
    if (__syncthreads_count(a.done && b.done) == kThreads) break;
    const int nb = min(kBatch, e1 - b0);
    stage_batch(sh, rec, geom, vals, rg.x + b0, nb, tx0, ty0, cam.H, rf);
    __syncthreads();
    warp_entry_bits(sh.sm, nb, warp, threadIdx.x & 31, sh.wbits[warp]);
    for (int j = 0; j < kWords && !(a.done && b.done); ++j) {
      uint32_t bits = sh.wbits[warp][j];
      while (bits != 0u && !(a.done && b.done)) {
        const int k = 32 * j + __ffs(bits) - 1;
        bits &= bits - 1u;
        const float4 f0 = sh.s0[k], f1 = sh.s1[k], f2 = sh.s2[k], f3 = sh.s3[k];
        Pair qa, qb;
        eval_two(lx, lyA, f0, f1, sh.s4[k], sh.s5[k], f2.y, set, qa, qb);
        fwd_step<true>(a, qa, f2, f3, b0 + k, set);
        fwd_step<true>(b, qb, f2, f3, b0 + k, set);
      }
    }
  }
  SegPart* pp = part + (size_t)blockIdx.x * kTilePix;
  seg_store(a, inA, pp, threadIdx.x);
  seg_store(b, inB, pp, kThreads + threadIdx.x);
  if (counters) {
    unsigned e = a.evaluated + b.evaluated, c = (unsigned)(a.cnt + b.cnt);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, o);
      c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&counters[0], (unsigned long long)e);
      atomicAdd(&counters[1], (unsigned long long)c);
    }
  }
}

// Combine the segments of one pixel in order (slot = its index within the
// segment records).
__device__ __forceinline__ FwdPix seg_merge_pixel(const SegPart* __restrict__ part, int first, int nseg_tile,
                                                  int slot, float zref) {
  FwdPix p;
  fwd_init(p, true);
  p.zr = zref;
  bool stopped = false;
  for (int q = 0; q < nseg_tile && !stopped; ++q) {
    const SegPart g = part[(size_t)(first + q) * kTilePix + slot];
    p.C0 += g.f0.x;
    p.C1 += g.f0.y;
    p.C2 += g.f0.z;
    p.D += g.f2.y + 2.f * (p.A * g.f1.x - p.Zs * g.f0.w);
    p.A += g.f0.w;
    p.Zs += g.f1.x;
    p.I += g.f1.y;
    p.N0 += g.f1.z;
    p.N1 += g.f1.w;
    p.N2 += g.f2.x;
    if (g.f3.x >= 0) {
      p.M = g.f2.z;
      p.medpos = g.f3.x;
    }
    if (g.f3.y > 0) p.lastpos = g.f3.z;
    p.cnt += g.f3.y;
    p.T = g.f2.w;
    stopped = g.f3.w != 0;
  }
  return p;
}

__global__ void __launch_bounds__(kThreads) seg_merge_kernel(
    CamDev cam, SetDev set, const float4* __restrict__ rec, const uint32_t* __restrict__ vals,
    const int2* __restrict__ ranges, const uint32_t* __restrict__ segcnt, const uint32_t* __restrict__ seg_tile,
    const uint32_t* __restrict__ seg_idx, const uint32_t* __restrict__ nseg, const SegPart* __restrict__ part,
    float* __restrict__ out, int32_t* __restrict__ n_contrib, int32_t* __restrict__ last,
    int32_t* __restrict__ med) {
  int tile, s;
  if (!seg_of(seg_tile, seg_idx, nseg, blockIdx.x, &tile, &s) || s != 0) return;
  const int tx0 = (tile % cam.tiles_x) * kTile, ty0 = (tile / cam.tiles_x) * kTile;
  const int lxi = local_x(threadIdx.x), lyi = local_y(threadIdx.x);
  const int px = tx0 + lxi, pyA = ty0 + lyi, pyB = pyA + 4;
  const int2 rg = ranges[tile];
  const float zref = rec[(size_t)vals[rg.x] * kRecF4 + 2].z;
  const int ns = (int)segcnt[tile];
  const FwdPix a = seg_merge_pixel(part, blockIdx.x, ns, threadIdx.x, zref);
  const FwdPix b = seg_merge_pixel(part, blockIdx.x, ns, kThreads + threadIdx.x, zref);
  fwd_store(a, cam, set, px, pyA, out, n_contrib, last, med);
  fwd_store(b, cam, set, px, pyB, out, n_contrib, last, med);
}

// Segments per tile (0 for tiles composited whole).
__global__ void seg_count_kernel(const int2* __restrict__ ranges, int ntiles, int lseg, uint32_t* __restrict__ segcnt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  const int len = ranges[t].y - ranges[t].x;
  segcnt[t] = len > lseg ? (uint32_t)((len + lseg - 1) / lseg) : 0u;
}

__global__ void seg_list_kernel(const uint32_t* __restrict__ segcnt, const uint32_t* __restrict__ segoff, int ntiles,
                                uint32_t* __restrict__ seg_tile, uint32_t* __restrict__ seg_idx) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  const uint32_t c = segcnt[t], o = segoff[t];
  for (uint32_t q = 0; q < c; ++q) {
    seg_tile[o + q] = (uint32_t)t;
    seg_idx[o + q] = q;
  }
}

// Persistent forward blend over the tiles of several views (serving): each
// CTA takes (view, tile) work items from a device counter until all tiles
// of all views in the batch are done; views of different sizes and scenes
// share one launch.
__global__ void __launch_bounds__(kThreads) blend_fwd_batched_kernel(BlendBatch batch) {
  __shared__ FwdSmem sh;
  __shared__ int item;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) item = (int)atomicAdd(batch.counter, 1u);
    __syncthreads();
    const int t = item;
    if (t >= batch.total_tiles) break;
    int j = 0;
    while (j + 1 < batch.njobs && batch.job[j + 1].tile_begin <= t) ++j;
    const BlendJob& jb = batch.job[j];
    const int local = t - jb.tile_begin;
    blend_fwd_tile(sh, jb.cam, jb.set, jb.rf, jb.rec, jb.geom, jb.vals, jb.ranges, jb.out, jb.n_contrib,
                   nullptr, nullptr, batch.work, local % jb.cam.tiles_x, local / jb.cam.tiles_x);
  }
}

// ---------------------------------------------------------------------------
// Backward.

constexpr int kMaxSets = 3;
// Entries staged per batch in the backward, by the CTAs per SM its variant
// is sized for: 128 for five (a small batch leaves more of the SM's shared
// memory to L1: 0.939 -> 0.921 ms on the 1M-surfel view, against 224), 224
// for four (the dense variant's long lists: 128 made the 4M-surfel training
// step 2.5 % slower).  The gradient accumulators and the six staged vectors
// per entry fit either way.
constexpr int batch_b(int min_ctas) { return min_ctas >= 5 ? 128 : 224; }
// Average tile-list length from which the backward takes the 4-CTA variant:
// 200 (the 1M-surfel aerial view) ran best with 5 CTAs per SM, 590 (the
// 4M-surfel orbit view) with 4.
constexpr int kDenseListLen = 400;

// Per-pair gradient vector.  General layout (any adjoint planes):
//   [0..5] d Ji, d e; [6] Zc, the depth term of the centre gradient (below);
//   [7] d p_z, [8] d opacity, [9..11] d rgb, [12..14] d normal;
//   [15 + 2 s, 16 + 2 s] screen-space gradient of set s.
// Loss layout (set 0 on colour and inverse depth only, later sets on
// colour): the normal slots are dropped, [0..11] as above without d normal,
// [12 + 2 s, 13 + 2 s] screen gradients.
// The centre gradient is not accumulated on its own: per pair it is set 0's
// screen gradient plus, on the object-space branch, the term of the depth
// z = p_z / (1 + e.d) through d, (d rden / d d) p_z dz = -e p_z rden^2 dz;
// so d c = (screen gradient of set 0) + e * Zc with Zc the sum of
// p_z rden^2 dz, formed once per entry at the flush.
template <bool kLoss>
struct Layout {
  static constexpr int kRec = kLoss ? 12 : kGradRec - 1;
  static constexpr int kN = kRec + 2 * kMaxSets;  // 18 or 21
};

// Balanced reduce-scatter of N values over the warp: at each halving level
// the lanes whose bit is clear keep the first ceil(N/2) values and the others
// the rest, exchanging the halves they do not keep; N values need about
// N + 5 shuffles.  Afterwards v[0] holds the warp sum of one slot, given by
// rs_slot() for the lane (or nothing when rs_slot() returns -1).
template <int O, int N>
__device__ __forceinline__ void rs_level(float* v, int lane) {
  constexpr int L = (N + 1) / 2, H = N - L;
  const bool up = (lane & O) != 0;
#pragma unroll
  for (int i = 0; i < L; ++i) {
    const float hi = (i < H) ? v[L + i] : 0.f;
    const float send = up ? v[i] : hi;
    const float keep = up ? hi : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
  }
  if constexpr (O > 1) rs_level<O / 2, L>(v, lane);
}

template <int N>
__device__ __forceinline__ int rs_slot(int lane) {
  int n = N, real = N, slot = 0;
  for (int o = 16; o >= 1; o >>= 1) {
    const int L = (n + 1) / 2;
    if (lane & o) {
      slot += L;
      real = real - L > 0 ? real - L : 0;
    } else {
      real = real < L ? real : L;
    }
    n = L;
  }
  return real > 0 ? slot : -1;
}

// Per-pixel state of the reverse replay: transmittance, suffix sums S of
// each adjoint set, the pixel's adjoints, and (general layout) the running
// opacity A and depth sum Z with their final values for the distortion.
struct BwdPix {
  float T, A, Z, Af, Zf;
  float S[kMaxSets];
  float gC[kMaxSets][3];
  float gA, gZ, gI, gMed, gD, gN0, gN1, gN2;
  int last, med;
};

template <bool kLoss>
__device__ __forceinline__ void bwd_init(BwdPix& p, bool inside, size_t pix, size_t HW,
                                         const float* __restrict__ out, const int32_t* __restrict__ last,
                                         const int32_t* __restrict__ med, const AdjDev& adj,
                                         const SetDev& set) {
  p.T = 1.f;
  p.A = p.Z = p.Af = p.Zf = 0.f;
  p.gA = p.gZ = p.gI = p.gMed = p.gD = p.gN0 = p.gN1 = p.gN2 = 0.f;
  p.last = 0;
  p.med = -1;
#pragma unroll
  for (int s = 0; s < kMaxSets; ++s) {
    p.gC[s][0] = p.gC[s][1] = p.gC[s][2] = 0.f;
    p.S[s] = 0.f;
  }
  if (!inside) return;
  p.last = last[pix];
  p.T = out[11 * HW + pix];
#pragma unroll
  for (int s = 0; s < kMaxSets; ++s) {
    if (s >= adj.n_sets) break;
    const float* a = adj.set[s];
    const uint32_t m = adj.mask[s];
#pragma unroll
    for (int c = 0; c < 3; ++c) p.gC[s][c] = (m >> c) & 1u ? a[c * HW + pix] : 0.f;
    p.S[s] = p.T * (p.gC[s][0] * set.bg[0] + p.gC[s][1] * set.bg[1] + p.gC[s][2] * set.bg[2]);
  }
  const float* a = adj.set[0];
  const uint32_t m = adj.mask[0];
  if (m & (1u << 5)) p.gI = a[5 * HW + pix];
  if constexpr (!kLoss) {
    p.med = med[pix];
    p.Af = p.A = out[3 * HW + pix];
    p.Zf = p.Z = out[4 * HW + pix];
    if (m & (1u << 3)) p.gA = a[3 * HW + pix];
    if (m & (1u << 4)) p.gZ = a[4 * HW + pix];
    if (m & (1u << 6)) p.gMed = a[6 * HW + pix];
    if (m & (1u << 7)) p.gN0 = a[7 * HW + pix];
    if (m & (1u << 8)) p.gN1 = a[8 * HW + pix];
    if (m & (1u << 9)) p.gN2 = a[9 * HW + pix];
    if (m & (1u << 10)) p.gD = a[10 * HW + pix];
  }
}

// A pair that was not blended (or lies past the pixel's last blended
// entry) is masked so that every term of bwd_pair is a finite zero and the
// pixel's state passes through unchanged: alpha = G = 0 and the
// screen-space branch, whose terms are finite for any offset.
__device__ __forceinline__ void mask_pair(Pair& q, bool live) {
  const bool h = live && q.hit;
  q.hit = h;
  q.alpha = h ? q.alpha : 0.f;
  q.G = h ? q.G : 0.f;
  q.obj = h && q.obj;
}

// Gradient of one pair at list position k, added into v (gradient-vector
// layout), and the pixel's replay state moved past it.  Branch-free, so that
// the two pixels of a thread interleave: both branches of the ray-splat are
// formed and the one the forward took is selected.
template <bool kLoss>
__device__ __forceinline__ void bwd_pair(BwdPix& p, const Pair& q, float4 e0, float4 e1, float4 e2,
                                         float4 e3, int k, int nsets, const SetDev& set, float* v) {
  using LY = Layout<kLoss>;
  const float rom = rcp_approx(1.f - q.alpha);
  p.T = q.hit ? p.T * rom : p.T;  // transmittance before this pair
  const float w = q.alpha * p.T;
  const float pz = e2.x;
  const float z = q.obj ? pz * q.rden : pz;
  const float rz = rcp_approx(z);
  float dLdw = p.gC[0][0] * e2.z + p.gC[0][1] * e2.w + p.gC[0][2] * e3.x + p.gI * rz;
  float dzv = -w * p.gI * rz * rz;
  if constexpr (!kLoss) {
    const float Ap = p.A - w, Zp = p.Z - w * z;
    const float dDdw = 2.f * (z * Ap - Zp + (p.Zf - p.Z) - z * (p.Af - p.A));
    dLdw += p.gA + p.gZ * z + p.gN0 * e3.y + p.gN1 * e3.z + p.gN2 * e3.w + p.gD * dDdw;
    dzv += w * p.gZ + p.gD * 2.f * w * (Ap - (p.Af - p.A)) + (k == p.med ? p.gMed : 0.f);
    p.A = Ap;
    p.Z = Zp;
  }
  float dLda[kMaxSets];
  dLda[0] = p.T * dLdw - p.S[0] * rom;
  p.S[0] += w * dLdw;
#pragma unroll
  for (int s = 1; s < kMaxSets; ++s) {
    if (s < nsets) {
      const float dw = p.gC[s][0] * e2.z + p.gC[s][1] * e2.w + p.gC[s][2] * e3.x;
      dLda[s] = p.T * dw - p.S[s] * rom;
      p.S[s] += w * dw;
    } else {
      dLda[s] = 0.f;
    }
  }
  // alpha -> rho (zero where alpha is clamped at alpha_max).  Every
  // derivative of rho below carries a factor 2; it is kept in
  // dadrho2 = 2 d alpha / d rho and drho2 = 2 dL / d rho (exact scalings),
  // and rx, ry are half of d rho / d d.
  const bool unclamped = e2.y * q.G < set.alpha_max;
  const float dadrho2 = unclamped ? -q.alpha : 0.f;
  const float drho2 = dLda[0] * dadrho2;
  // object-space branch: rho = u^2 + v^2 with (u, v) = (nu, nv) rden,
  // z = p_z rden (its terms may be non-finite where it was not taken)
  const float r2d = q.rden * q.rden;
  const float tx = q.nu * e1.x + q.nv * e1.z, ty = q.nu * e1.y + q.nv * e1.w;
  const float c1 = q.rho * q.rden;
  const float u = q.nu * q.rden, vv = q.nv * q.rden;
  const float dnu = u * q.rden * drho2, dnv = vv * q.rden * drho2;
  const float zr2 = dzv * pz * r2d;
  const float drden = drho2 * (u * q.nu + vv * q.nv) + dzv * pz;
  const float dden = -drden * r2d;
  const bool ob = q.obj;
  const float rx = ob ? r2d * tx - c1 * e0.z : set.sinv * q.dx;
  const float ry = ob ? r2d * ty - c1 * e0.w : set.sinv * q.dy;
  const float gpz = ob ? dzv * q.rden : dzv;
  // the object-space terms of Ji, e and the centre's depth term, zero (and
  // finite) where the screen branch was taken
  const float dnu_o = ob ? dnu : 0.f, dnv_o = ob ? dnv : 0.f, dden_o = ob ? dden : 0.f;
  v[0] = fmaf(dnu_o, q.dx, v[0]);
  v[1] = fmaf(dnu_o, q.dy, v[1]);
  v[2] = fmaf(dnv_o, q.dx, v[2]);
  v[3] = fmaf(dnv_o, q.dy, v[3]);
  v[4] = fmaf(dden_o, q.dx, v[4]);
  v[5] = fmaf(dden_o, q.dy, v[5]);
  v[6] += ob ? zr2 : 0.f;
  v[7] += gpz;
  v[8] = fmaf(dLda[0], unclamped ? q.G : 0.f, v[8]);
  v[9] += w * p.gC[0][0];
  v[10] += w * p.gC[0][1];
  v[11] += w * p.gC[0][2];
  if constexpr (!kLoss) {
    v[12] += w * p.gN0;
    v[13] += w * p.gN1;
    v[14] += w * p.gN2;
  }
#pragma unroll
  for (int s = 0; s < kMaxSets; ++s) {
    const float dr = dLda[s] * dadrho2;
    v[LY::kRec + 2 * s] -= dr * rx;
    v[LY::kRec + 2 * s + 1] -= dr * ry;
  }
}

// Shared-memory staging of the backward (one batch of kBB entries).
template <int kAcc, int kBB>
struct BwdSmem {
  float4 s0[kBB], s1[kBB], s2[kBB], s3[kBB], s4[kBB], s5[kBB];
  uint32_t sm[kBB];
  uint32_t sid[kBB];
  float acc[kBB][kAcc];
  uint32_t wbits[kThreads / 32][kBB / 32];
  int smax;
};

// Reverse replay of entry kk (list position k) for a thread's two pixels:
// the pair's gradients, reduced over the warp into the entry's accumulator.
template <bool kLoss, int kN, int kAcc, int kBB>
__device__ __forceinline__ void bwd_entry(BwdSmem<kAcc, kBB>& sh, int kk, int k, float lx, float ly, BwdPix& a,
                                          BwdPix& b, int nsets, const SetDev& set, int lane, int myslot,
                                          unsigned& wentries, unsigned& wlanes) {
  const float4 e0 = sh.s0[kk], jh = sh.s1[kk], e2 = sh.s2[kk];
  const bool liveA = k < a.last, liveB = k < b.last;
  Pair qa, qb;
  const float4 jl = sh.s4[kk];
  eval_two(lx, ly, e0, jh, jl, sh.s5[kk], e2.y, set, qa, qb);
  mask_pair(qa, liveA);
  mask_pair(qb, liveB);
  const bool contrib = qa.hit || qb.hit;
  const unsigned ballot = __ballot_sync(0xffffffffu, contrib);
  if (ballot == 0u) return;
  ++wentries;
  wlanes += __popc(ballot);
  float v[kN];
#pragma unroll
  for (int i = 0; i < kN; ++i) v[i] = 0.f;
  const float4 e3 = sh.s3[kk];
  // Ji = Jh + Jl (FP32) for the chain rule
  const float4 e1 = make_float4(jh.x + jl.x, jh.y + jl.y, jh.z + jl.z, jh.w + jl.w);
  // a pixel row with no hit in the whole warp needs no gradient pass (a
  // masked pair leaves the pixel's state and the sums unchanged)
  const bool anyA = __any_sync(0xffffffffu, qa.hit), anyB = __any_sync(0xffffffffu, qb.hit);
  if (anyA && anyB) {
    bwd_pair<kLoss>(a, qa, e0, e1, e2, e3, k, nsets, set, v);
    bwd_pair<kLoss>(b, qb, e0, e1, e2, e3, k, nsets, set, v);
  } else if (anyA) {
    bwd_pair<kLoss>(a, qa, e0, e1, e2, e3, k, nsets, set, v);
  } else {
    bwd_pair<kLoss>(b, qb, e0, e1, e2, e3, k, nsets, set, v);
  }
  if (__popc(ballot) == 1) {
    if (contrib) {
#pragma unroll
      for (int i = 0; i < kN; ++i)
        if (v[i] != 0.f) atomicAdd(&sh.acc[kk][i], v[i]);
    }
  } else {
    rs_level<16, kN>(v, lane);
    if (myslot >= 0 && v[0] != 0.f) atomicAdd(&sh.acc[kk][myslot], v[0]);
  }
}

// kMinCtas: the CTAs per SM the register budget is sized for (5: 96
// registers; 4: up to 128, for dense lists of small footprints).
template <bool kLoss, int kMinCtas>
__global__ void __launch_bounds__(kThreads, kMinCtas) blend_bwd_kernel(
    CamDev cam, SetDev set, float rf, const uint32_t* __restrict__ order, const float4* __restrict__ rec,
    const RowGeom* __restrict__ geom, const uint32_t* __restrict__ vals, const int2* __restrict__ ranges,
    const float* __restrict__ out, const int32_t* __restrict__ last, const int32_t* __restrict__ med,
    AdjDev adj, float* __restrict__ grec, float* __restrict__ screen, int n,
    unsigned long long* __restrict__ counters) {
  using LY = Layout<kLoss>;
  constexpr int kN = LY::kN;
  constexpr int kAcc = kN | 1;  // odd row stride: the flush's column reads are conflict-free
  constexpr int kBatchB = batch_b(kMinCtas), kWordsB = kBatchB / 32;
  __shared__ BwdSmem<kAcc, kBatchB> sh;
  const int tile = order ? (int)order[blockIdx.x] : (int)blockIdx.x;
  const int tx0 = (tile % cam.tiles_x) * kTile, ty0 = (tile / cam.tiles_x) * kTile;
  const int lxi = local_x(threadIdx.x), lyi = local_y(threadIdx.x);
  const int px = tx0 + lxi, pyA = ty0 + lyi, pyB = pyA + 4;
  const int warp = threadIdx.x >> 5;
  const float lx = (float)lxi + 0.5f, lyA = (float)lyi + 0.5f;
  const int2 rg = ranges[tile];
  const size_t HW = (size_t)cam.W * cam.H;
  const int lane = threadIdx.x & 31;
  const int nsets = adj.n_sets;
  const int myslot = rs_slot<kN>(lane);
  const bool inA = px < cam.W && pyA < cam.H, inB = px < cam.W && pyB < cam.H;
  BwdPix a, b;
  bwd_init<kLoss>(a, inA, inA ? (size_t)pyA * cam.W + px : 0, HW, out, last, med, adj, set);
  bwd_init<kLoss>(b, inB, inB ? (size_t)pyB * cam.W + px : 0, HW, out, last, med, adj, set);
  if (threadIdx.x == 0) sh.smax = 0;
  __syncthreads();
  atomicMax(&sh.smax, max(a.last, b.last));
  __syncthreads();
  const int maxlast = sh.smax;
  // the warp's own last blended position: entries behind it are dead for all
  // of its pixels and are not visited
  int wlast = max(a.last, b.last);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wlast = max(wlast, __shfl_xor_sync(0xffffffffu, wlast, o));
  unsigned replayed = 0, wentries = 0, wlanes = 0;

  for (int bend = maxlast; bend > 0; bend -= kBatchB) {
    const int b0 = bend > kBatchB ? bend - kBatchB : 0;
    const int nb = bend - b0;
    __syncthreads();
    for (int t = threadIdx.x; t < nb; t += kThreads) {
      const uint32_t s = vals[rg.x + b0 + t];
      sh.sid[t] = s;
      const Staged e = stage_entry(rec, geom, s, tx0, ty0, cam.H, rf);
      sh.s0[t] = e.s0;
      sh.s1[t] = e.s1;
      sh.s2[t] = e.s2;
      sh.s3[t] = e.s3;
      sh.s4[t] = e.s4;
      sh.s5[t] = e.s5;
      sh.sm[t] = e.wmask;
    }
    for (int i = threadIdx.x; i < nb * kAcc; i += kThreads) (&sh.acc[0][0])[i] = 0.f;
    __syncthreads();
    warp_entry_bits<kWordsB>(sh.sm, nb, warp, lane, sh.wbits[warp]);
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < kWordsB; ++j) {
        const int lw = wlast - b0 - 32 * j;
        sh.wbits[warp][j] &= lw >= 32 ? 0xffffffffu : (lw > 0 ? (1u << lw) - 1u : 0u);
      }
    }
    __syncwarp();
    if (counters) {
      // the batch's entries before each pixel's last blended one that the
      // warp visits (performance counter)
#pragma unroll
      for (int j = 0; j < kWordsB; ++j) {
        const uint32_t bits = sh.wbits[warp][j];
        const int la = a.last - b0 - 32 * j, lb = b.last - b0 - 32 * j;
        replayed += (unsigned)__popc(la >= 32 ? bits : (la > 0 ? bits & ((1u << la) - 1u) : 0u));
        replayed += (unsigned)__popc(lb >= 32 ? bits : (lb > 0 ? bits & ((1u << lb) - 1u) : 0u));
      }
    }
    for (int j = kWordsB - 1; j >= 0; --j) {
      uint32_t bits = sh.wbits[warp][j];
      while (bits != 0u) {  // back to front: highest set bit first
        const int hb = 31 - __clz(bits);
        bits &= ~(1u << hb);
        bwd_entry<kLoss, kN, kAcc, kBatchB>(sh, 32 * j + hb, b0 + 32 * j + hb, lx, lyA, a, b, nsets, set, lane, myslot,
                                   wentries, wlanes);
      }
    }
    __syncthreads();
    // flush this batch: one (surfel, tile) gradient record per entry, the
    // centre gradient formed from set 0's screen gradient and Zc
    for (int t = threadIdx.x; t < nb; t += kThreads) {
      const uint32_t s = sh.sid[t];
      float* g = grec + (size_t)s * kGradRec;
      const float* x = sh.acc[t];
      const float4 e0 = sh.s0[t];
      float r[kGradRec];
#pragma unroll
      for (int i = 0; i < 6; ++i) r[i] = x[i];
      r[6] = fmaf(e0.z, x[6], x[LY::kRec]);
      r[7] = fmaf(e0.w, x[6], x[LY::kRec + 1]);
#pragma unroll
      for (int i = 7; i < LY::kRec; ++i) r[i + 1] = x[i];
#pragma unroll
      for (int i = 0; i < LY::kRec + 1; ++i)
        if (r[i] != 0.f) atomicAdd(&g[i], r[i]);
      if (screen) {
        for (int st = 0; st < nsets; ++st) {
          const float x0 = sh.acc[t][LY::kRec + 2 * st];
          const float x1 = sh.acc[t][LY::kRec + 2 * st + 1];
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
    if (lane == 0) {
      atomicAdd(&counters[2], (unsigned long long)e);
      atomicAdd(&counters[3], (unsigned long long)wentries);
      atomicAdd(&counters[4], (unsigned long long)wlanes);
    }
  }
}

// ---------------------------------------------------------------------------
// Trim contribution (Sec. 3.3, Eq. 3).
//
// The tiles of the render walk their lists front to back as the forward
// does, with the forward's decisions (same evaluation, same transmittance
// sequence), but every pixel goes through the whole list: a pair that lies
// in the surfel's support (rho <= rho_max) counts towards |P_k| even behind
// the pixel's stop.  A blended pair adds alpha^gamma T^(1 - gamma), T the
// transmittance in front of it.  Per entry the warp counts its support
// pixels with ballots and sums its contributions with shuffles; the tile sums
// them in shared memory and adds them to the surfel's totals once.

__device__ __forceinline__ float contrib_step(float& T, bool& stopped, const Pair& q, const SetDev& set,
                                              float gamma) {
  float c = 0.f;
  if (!stopped && q.hit) {
    const float Tn = T * (1.f - q.alpha);
    if (Tn < set.T_min) {
      stopped = true;
    } else {
      c = gamma == 0.5f ? sqrtf(q.alpha * T) : exp2f(gamma * log2f(q.alpha) + (1.f - gamma) * log2f(T));
      T = Tn;
    }
  }
  return c;
}

__global__ void __launch_bounds__(kThreads) blend_contrib_kernel(
    CamDev cam, SetDev set, float rf, float gamma, const uint32_t* __restrict__ order,
    const float4* __restrict__ rec, const RowGeom* __restrict__ geom, const uint32_t* __restrict__ vals,
    const int2* __restrict__ ranges, float* __restrict__ csum, uint32_t* __restrict__ ccnt) {
  __shared__ float4 s0[kBatch], s1[kBatch], s2[kBatch], s4[kBatch], s5[kBatch];
  __shared__ uint32_t sm[kBatch], sid[kBatch];
  __shared__ float asum[kBatch];
  __shared__ uint32_t acnt[kBatch];
  __shared__ uint32_t wbits[kThreads / 32][kWords];
  const int tile = order ? (int)order[blockIdx.x] : (int)blockIdx.x;
  const int tx0 = (tile % cam.tiles_x) * kTile, ty0 = (tile / cam.tiles_x) * kTile;
  const int lxi = local_x(threadIdx.x), lyi = local_y(threadIdx.x);
  const int px = tx0 + lxi, pyA = ty0 + lyi, pyB = pyA + 4;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float lx = (float)lxi + 0.5f, lyA = (float)lyi + 0.5f;
  const bool inA = px < cam.W && pyA < cam.H, inB = px < cam.W && pyB < cam.H;
  const int2 rg = ranges[tile];
  const int len = rg.y - rg.x;
  float TA = 1.f, TB = 1.f;
  bool stA = !inA, stB = !inB;
  for (int b0 = 0; b0 < len; b0 += kBatch) {
    const int nb = min(kBatch, len - b0);
    __syncthreads();
    for (int t = threadIdx.x; t < kBatch; t += kThreads) {
      if (t < nb) {
        const uint32_t sidx = vals[rg.x + b0 + t];
        const Staged e = stage_entry(rec, geom, sidx, tx0, ty0, cam.H, rf);
        s0[t] = e.s0;
        s1[t] = e.s1;
        s2[t] = e.s2;
        s4[t] = e.s4;
        s5[t] = e.s5;
        sm[t] = e.wmask;
        sid[t] = sidx;
        asum[t] = 0.f;
        acnt[t] = 0u;
      }
    }
    __syncthreads();
    warp_entry_bits(sm, nb, warp, lane, wbits[warp]);
    for (int j = 0; j < kWords; ++j) {
      uint32_t bits = wbits[warp][j];
      while (bits != 0u) {
        const int k = 32 * j + __ffs(bits) - 1;
        bits &= bits - 1u;
        const float4 e0 = s0[k], e1 = s1[k], e2 = s2[k];
        Pair qa, qb;
        eval_two(lx, lyA, e0, e1, s4[k], s5[k], e2.y, set, qa, qb);
        const unsigned ba = __ballot_sync(0xffffffffu, inA && qa.rho <= set.rho_max);
        const unsigned bb = __ballot_sync(0xffffffffu, inB && qb.rho <= set.rho_max);
        const uint32_t cnt = (uint32_t)(__popc(ba) + __popc(bb));
        float c = contrib_step(TA, stA, qa, set, gamma) + contrib_step(TB, stB, qb, set, gamma);
        if (cnt == 0u) continue;
  #pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) {
          atomicAdd(&acnt[k], cnt);
          if (c != 0.f) atomicAdd(&asum[k], c);
        }
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nb; t += kThreads) {
      if (acnt[t] != 0u) {
        atomicAdd(&ccnt[sid[t]], acnt[t]);
        if (asum[t] != 0.f) atomicAdd(&csum[sid[t]], asum[t]);
      }
    }
  }
}

}  // namespace

cudaError_t launch_blend_fwd(const CamDev& cam, const SetDev& set, const uint32_t* order, const float4* rec,
                             const RowGeom* geom, const uint32_t* vals, const int2* ranges, float* out,
                             int32_t* n_contrib, int32_t* last, int32_t* med,
                             unsigned long long* counters, cudaStream_t st) {
  const unsigned grid = (unsigned)cam.tiles_x * (unsigned)cam.tiles_y;
  const float rf = (float)sqrt((double)set.rho_max / (double)set.sinv);
  ProfScope ps(kProfBlendFwd, st);
  blend_fwd_kernel<<<grid, kThreads, 0, st>>>(cam, set, rf, order, rec, geom, vals, ranges, out, n_contrib,
                                              last, med, counters, 0);
  count_launch();
  return cudaGetLastError();
}

size_t seg_part_bytes() { return sizeof(SegPart); }

cudaError_t launch_blend_fwd_split(const CamDev& cam, const SetDev& set, const uint32_t* order, const float4* rec,
                                   const RowGeom* geom, const uint32_t* vals, const int2* ranges, float* out,
                                   int32_t* n_contrib, int32_t* last, int32_t* med, unsigned long long* counters,
                                   const SegBufs& sb, cudaStream_t st) {
  const int ntiles = cam.tiles_x * cam.tiles_y;
  const float rf = (float)sqrt((double)set.rho_max / (double)set.sinv);
  ProfScope ps(kProfBlendFwd, st);
  count_launch(2);
  seg_count_kernel<<<div_up(ntiles, 256), 256, 0, st>>>(ranges, ntiles, sb.lseg, sb.segcnt);
  cudaError_t e = launch_scan(sb.segcnt, sb.segoff, ntiles, sb.nseg, sb.scan_tmp, st);
  if (e != cudaSuccess) return e;
  seg_list_kernel<<<div_up(ntiles, 256), 256, 0, st>>>(sb.segcnt, sb.segoff, ntiles, sb.seg_tile, sb.seg_idx);
  // the whole tiles, then the segments (grids sized for the bound, the device
  // count decides)
  count_launch(4);
  blend_fwd_kernel<<<(unsigned)ntiles, kThreads, 0, st>>>(cam, set, rf, order, rec, geom, vals, ranges, out,
                                                          n_contrib, last, med, counters, sb.lseg);
  seg_trans_kernel<<<sb.nseg_max, kThreads, 0, st>>>(cam, set, rf, rec, geom, vals, ranges, sb.lseg, sb.seg_tile,
                                                     sb.seg_idx, sb.nseg, sb.trans);
  seg_blend_kernel<<<sb.nseg_max, kThreads, 0, st>>>(cam, set, rf, rec, geom, vals, ranges, sb.lseg, sb.seg_tile,
                                                     sb.seg_idx, sb.nseg, sb.trans,
                                                     static_cast<SegPart*>(sb.part), counters);
  seg_merge_kernel<<<sb.nseg_max, kThreads, 0, st>>>(cam, set, rec, vals, ranges, sb.segcnt, sb.seg_tile,
                                                     sb.seg_idx, sb.nseg, static_cast<const SegPart*>(sb.part),
                                                     out, n_contrib, last, med);
  return cudaGetLastError();
}

cudaError_t launch_blend_fwd_batched(const BlendBatch& batch, int grid, cudaStream_t st) {
  ProfScope ps(kProfBlendFwd, st);
  blend_fwd_batched_kernel<<<grid, kThreads, 0, st>>>(batch);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_blend_bwd(const CamDev& cam, const SetDev& set, const uint32_t* order, const float4* rec,
                             const RowGeom* geom, const uint32_t* vals, const int2* ranges, const float* out,
                             const int32_t* last, const int32_t* med, const AdjDev& adj,
                             float* grec, float* screen, int n, int64_t K, unsigned long long* counters,
                             cudaStream_t st) {
  const unsigned grid = (unsigned)cam.tiles_x * (unsigned)cam.tiles_y;
  const float rf = (float)sqrt((double)set.rho_max / (double)set.sinv);
  // the training loss drives set 0 through colour and inverse depth only and
  // the other sets through colour: a leaner kernel for that layout
  bool loss_layout = (adj.mask[0] & ~(GS_MASK_RGB | (1u << GS_PLANE_INVDEPTH))) == 0u;
  for (int s = 1; s < adj.n_sets; ++s) loss_layout = loss_layout && (adj.mask[s] & ~GS_MASK_RGB) == 0u;
  // long lists (many small footprints per tile) run faster with more
  // registers per thread than with a fifth CTA per SM; both compute the same
  const bool dense = K >= (int64_t)kDenseListLen * (int64_t)grid;
  ProfScope ps(kProfBlendBwd, st);
#define GS_BWD(L, M)                                                                                           \
  blend_bwd_kernel<L, M><<<grid, kThreads, 0, st>>>(cam, set, rf, order, rec, geom, vals, ranges, out, last, med, \
                                                    adj, grec, screen, n, counters)
  if (loss_layout) {
    if (dense) GS_BWD(true, 4);
    else GS_BWD(true, 5);
  } else {
    if (dense) GS_BWD(false, 4);
    else GS_BWD(false, 5);
  }
#undef GS_BWD
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_blend_contrib(const CamDev& cam, const SetDev& set, float gamma, const uint32_t* order,
                                 const float4* rec, const RowGeom* geom, const uint32_t* vals,
                                 const int2* ranges, float* csum, uint32_t* ccnt, cudaStream_t st) {
  const unsigned grid = (unsigned)cam.tiles_x * (unsigned)cam.tiles_y;
  const float rf = (float)sqrt((double)set.rho_max / (double)set.sinv);
  ProfScope ps(kProfContrib, st);
  blend_contrib_kernel<<<grid, kThreads, 0, st>>>(cam, set, rf, gamma, order, rec, geom, vals, ranges, csum,
                                                  ccnt);
  count_launch();
  return cudaGetLastError();
}

}  // namespace gs2d
