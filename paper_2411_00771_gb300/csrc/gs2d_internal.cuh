// Internal declarations of the CUDA library (sm_103a).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gs2d.h"

namespace gs2d {

constexpr int kTile = 16;              // 16 x 16 pixel tiles
constexpr int kBlock = kTile * kTile;  // one thread per pixel
constexpr int kRecF4 = 5;              // per-surfel blend record, 5 x float4

// Camera as the kernels see it (by value).  Geometry that decides where a
// surfel lands on screen is carried in double precision.
struct CamDev {
  double R[9];
  double t[3];
  double fx, fy, cx, cy;
  double campos[3];  // camera centre in world coordinates, -R^T t
  int W, H, tiles_x, tiles_y;
};

struct SetDev {
  float near_plane, alpha_min, T_min, alpha_max, rho_max, sinv;
  float bg[3];
};

// Per-surfel blend record (written by the preprocess, read by both blends):
//  r0 = (c_hi.x, c_hi.y, c_lo.x, c_lo.y)   projected centre, two-float split
//  r1 = (Ji11, Ji12, Ji21, Ji22)           inverse of the centred Jacobian
//  r2 = (e.x, e.y, p_z, opacity)           projective row, centre depth
//  r3 = (r, g, b, n.x)                     colour, view-space normal
//  r4 = (n.y, n.z, 0, 0)
// For a pixel offset d = x - c:  den = 1 + e.d,  (u, v) = Ji d / den,
// rho_obj = u^2 + v^2, z_obj = p_z / den.

struct Workspace;  // allocator wrapper

struct ParamsDev {
  const float* mu;
  const float* quat;
  const float* scale;
  const float* opacity;
  const float* sh;
  int n;
  int sh_degree;
};

// ---- launch wrappers (each returns cudaError_t from the launch) ----------
cudaError_t launch_preprocess(const ParamsDev& P, const CamDev& cam, const SetDev& set,
                              float4* rec, uint2* rect, uint32_t* tcount, uint32_t* depth_key,
                              uint32_t* idx, cudaStream_t st);

// device-wide exclusive scan of n uint32 values; total (uint32) written to
// *total_dev; tmp must hold scan_tmp_words(n) uint32 words.
size_t scan_tmp_words(int64_t n);
cudaError_t launch_scan(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_dev,
                        uint32_t* tmp, cudaStream_t st);

// LSD radix sort of (key, value) pairs over key bits [0, bits); stable.
// Result ends in (keys_out, vals_out) (double-buffering through the alt
// buffers); tmp must hold radix_tmp_words(n) uint32 words.
size_t radix_tmp_words(int64_t n);
cudaError_t radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                             uint32_t* vals_alt, int64_t n, int bits, uint32_t* tmp,
                             uint32_t** keys_out, uint32_t** vals_out, cudaStream_t st);

cudaError_t launch_gather_counts(const uint32_t* order, const uint32_t* tcount, uint32_t* out,
                                 int64_t n, cudaStream_t st);
cudaError_t launch_emit(const uint32_t* order, const uint32_t* offs, const uint2* rect,
                        int64_t n, int tiles_x, uint32_t* keys, uint32_t* vals, cudaStream_t st);
cudaError_t launch_ranges(const uint32_t* keys, int64_t K, int2* ranges, int ntiles,
                          cudaStream_t st);

cudaError_t launch_blend_fwd(const CamDev& cam, const SetDev& set, const float4* rec,
                             const uint32_t* vals, const int2* ranges, float* out,
                             int32_t* n_contrib, int32_t* last, int32_t* med,
                             unsigned long long* counters, cudaStream_t st);

struct AdjDev {
  const float* set[3];
  uint32_t mask[3];
  int n_sets;
};

// Per-surfel intermediate gradient record of the blend backward.
constexpr int kGradRec = 16;  // Ji(4) e(2) c(2) p_z(1) opacity(1) rgb(3) n(3)

cudaError_t launch_blend_bwd(const CamDev& cam, const SetDev& set, const float4* rec,
                             const uint32_t* vals, const int2* ranges, const float* out,
                             const int32_t* last, const int32_t* med, const AdjDev& adj,
                             float* grec, float* screen, int n, unsigned long long* counters,
                             cudaStream_t st);

cudaError_t launch_preprocess_bwd(const ParamsDev& P, const CamDev& cam, const uint32_t* tcount,
                                  const float* grec, const gs_param_grads& G, cudaStream_t st);

cudaError_t launch_loss(int W, int H, const float* out, const float* tgt, const float* tinv,
                        const gs_loss_weights& w, float* adj_total, float* adj_ssim,
                        float* adj_l1, float* losses, float* tmp, cudaStream_t st);
size_t loss_tmp_floats(int W, int H);

cudaError_t launch_densify_accumulate(const uint32_t* tcount, const float* screen, int n,
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
  kProfCount = 7
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

}  // namespace gs2d
