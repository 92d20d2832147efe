// C ABI of the library: scene and frame objects, buffer management and the
// order of kernel launches for render, loss, backward and densification.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "gs2d_internal.cuh"

using namespace gs2d;

namespace {

thread_local std::string g_last_error;

gs_status fail(gs_status code, const std::string& msg) {
  g_last_error = msg;
  return code;
}
gs_status cuda_fail(cudaError_t e, const char* where) {
  return fail(GS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define GS_CK(expr)                                   \
  do {                                                \
    cudaError_t e_ = (expr);                          \
    if (e_ != cudaSuccess) return cuda_fail(e_, #expr); \
  } while (0)

// Allocations through the caller's allocator (or the stream-ordered pool).
struct Alloc {
  gs_allocator a{};
  void* get(size_t bytes, cudaStream_t st) const {
    if (bytes == 0) bytes = 16;
    if (a.alloc) return a.alloc(bytes, a.ctx, st);
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void put(void* p, size_t bytes, cudaStream_t st) const {
    if (!p) return;
    if (a.free) a.free(p, bytes, a.ctx, st);
    else cudaFreeAsync(p, st);
  }
};

// A list of buffers freed together.
struct Buffers {
  struct B {
    void* p;
    size_t bytes;
  };
  std::vector<B> list;
  const Alloc* al = nullptr;
  template <typename T>
  T* get(size_t count, cudaStream_t st) {
    void* p = al->get(count * sizeof(T), st);
    if (p) list.push_back({p, count * sizeof(T)});
    return static_cast<T*>(p);
  }
  void release(void* p, cudaStream_t st) {
    for (size_t i = 0; i < list.size(); ++i)
      if (list[i].p == p) {
        al->put(p, list[i].bytes, st);
        list.erase(list.begin() + (long)i);
        return;
      }
  }
  void release_all(cudaStream_t st) {
    for (auto& b : list) al->put(b.p, b.bytes, st);
    list.clear();
  }
};

void set_pool_threshold() {
  static bool done = false;
  if (done) return;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  done = true;
}

SetDev to_dev(const gs_settings& s) {
  SetDev d;
  d.near_plane = s.near_plane;
  d.alpha_min = s.alpha_min;
  d.T_min = s.T_min;
  d.alpha_max = s.alpha_max;
  d.rho_max = s.rho_max;
  d.sinv = s.screen_inv_sigma2;
  d.bg[0] = s.bg[0];
  d.bg[1] = s.bg[1];
  d.bg[2] = s.bg[2];
  return d;
}

int bits_for(int64_t v) {
  int b = 0;
  while ((int64_t(1) << b) < v) ++b;
  return b;
}

}  // namespace

// ---- launch accounting and optional per-kernel event timing ---------------
namespace gs2d {
namespace {
std::atomic<unsigned long long> g_launches{0};
std::atomic<int> g_prof_on{0};
std::mutex g_prof_mu;
struct EvPair {
  cudaEvent_t a, b;
};
std::vector<EvPair> g_prof_pending[kProfCount];
std::vector<cudaEvent_t> g_prof_free;
thread_local cudaEvent_t g_prof_open[kProfCount] = {};
cudaEvent_t prof_event() {
  if (!g_prof_free.empty()) {
    cudaEvent_t e = g_prof_free.back();
    g_prof_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}
}  // namespace

__global__ void api_unpack_rect_kernel(const uint2* __restrict__ rect, const uint32_t* __restrict__ tcount,
                                   int n, int32_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint2 r = rect[i];
  const bool v = (r.y & 0xFFFF) > (r.x & 0xFFFF);
  (void)tcount;
  out[4 * i] = v ? (int)(r.x & 0xFFFF) : 0;
  out[4 * i + 1] = v ? (int)(r.x >> 16) : 0;
  out[4 * i + 2] = v ? (int)(r.y & 0xFFFF) : 0;
  out[4 * i + 3] = v ? (int)(r.y >> 16) : 0;
}

void set_last_error(const char* msg) { g_last_error = msg; }

void count_launch(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

// Scopes of one group may nest (a sort calls a scan); only the outermost
// scope of each group records.
thread_local int g_prof_depth[kProfCount] = {};

void prof_begin(int id, cudaStream_t st) {
  if (!g_prof_on.load(std::memory_order_relaxed)) return;
  if (g_prof_depth[id]++ > 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEvent_t e = prof_event();
  if (e && cudaEventRecord(e, st) == cudaSuccess) g_prof_open[id] = e;
  else g_prof_open[id] = nullptr;
}

void prof_end(int id, cudaStream_t st) {
  if (g_prof_depth[id] > 0 && --g_prof_depth[id] > 0) return;
  if (!g_prof_on.load(std::memory_order_relaxed) || !g_prof_open[id]) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEvent_t e = prof_event();
  if (e && cudaEventRecord(e, st) == cudaSuccess) g_prof_pending[id].push_back({g_prof_open[id], e});
  g_prof_open[id] = nullptr;
}
}  // namespace gs2d

struct gs_scene {
  ParamsDev P;
  gs_settings settings;
  Alloc al;
};

struct gs_frame {
  gs_scene* scene = nullptr;
  CamDev cam{};
  int n = 0;
  int sh_degree = 0;
  int64_t K = 0;
  int64_t n_visible = 0;
  Buffers buf;
  float4* rec = nullptr;
  uint2* rect = nullptr;
  RowGeom* geom = nullptr;
  uint32_t* tcount = nullptr;
  uint32_t* vals = nullptr;
  int2* ranges = nullptr;
  uint32_t* order = nullptr;  // tiles by list length, longest first
  int32_t* last = nullptr;
  int32_t* med = nullptr;
  uint32_t* cand = nullptr;   // candidate surfels of the render (index order)
  uint32_t* ncand = nullptr;  // their count (device; in counters[6])
  unsigned long long* counters = nullptr;  // evaluated, blended, bwd replayed, visible
  const float* out = nullptr;
};

namespace gs2d {
const ParamsDev& scene_params(const gs_scene* sc) { return sc->P; }
const gs_settings& scene_settings(const gs_scene* sc) { return sc->settings; }
}  // namespace gs2d

extern "C" gs_status gs_frame_release(gs_frame* f, void* stream);

namespace {

// A frame of scene sc seen by camera c (host side; no device memory yet).
gs_frame* new_frame(gs_scene* sc, const gs_camera* c, const float* out, const char* who, gs_status* err) {
  if (!sc || !c) {
    *err = fail(GS_ERR_ARG, std::string(who) + ": null argument");
    return nullptr;
  }
  if (c->width <= 0 || c->height <= 0 || c->width > 16 * 65535 || c->height > 16 * 65535) {
    *err = fail(GS_ERR_ARG, std::string(who) + ": bad image size");
    return nullptr;
  }
  if (!(c->fx > 0) || !(c->fy > 0)) {
    *err = fail(GS_ERR_ARG, std::string(who) + ": focal lengths must be > 0");
    return nullptr;
  }
  gs_frame* f = new (std::nothrow) gs_frame();
  if (!f) {
    *err = fail(GS_ERR_OOM, std::string(who) + ": host allocation");
    return nullptr;
  }
  f->scene = sc;
  f->n = sc->P.n;
  f->sh_degree = sc->P.sh_degree;
  f->out = out;
  f->buf.al = &sc->al;
  cam_from(*c, f->cam);
  return f;
}

// Every step of a render before the blend: preprocess, candidate depth order,
// tile lists, ranges and the tiles' launch order, into frame f.  Reads the
// 4-byte instance count back once.  On failure f keeps what it allocated
// (the caller releases it).
gs_status build_lists(gs_scene* sc, gs_frame* f, const char* who, cudaStream_t st) {
  const CamDev& cam = f->cam;
  const int ntiles = cam.tiles_x * cam.tiles_y;
  const int64_t n = f->n;
  const SetDev set = to_dev(sc->settings);
  Buffers tmp;
  tmp.al = &sc->al;
  auto failed = [&](gs_status s) {
    tmp.release_all(st);
    return s;
  };
  // per-surfel buffers
  f->rec = f->buf.get<float4>((size_t)(n > 0 ? n : 1) * kRecF4, st);
  f->rect = f->buf.get<uint2>(n > 0 ? n : 1, st);
  f->tcount = f->buf.get<uint32_t>(n > 0 ? n : 1, st);
  f->ranges = f->buf.get<int2>(ntiles, st);
  f->order = f->buf.get<uint32_t>(ntiles, st);
  f->counters = f->buf.get<unsigned long long>(8, st);
  f->cand = f->buf.get<uint32_t>(n > 0 ? n : 1, st);
  f->geom = f->buf.get<RowGeom>(n > 0 ? n : 1, st);
  uint32_t* dkey = tmp.get<uint32_t>(n > 0 ? n : 1, st);
  uint32_t* idx = tmp.get<uint32_t>(n > 0 ? n : 1, st);
  uint32_t* dkey2 = tmp.get<uint32_t>(n > 0 ? n : 1, st);
  uint32_t* idx2 = tmp.get<uint32_t>(n > 0 ? n : 1, st);
  uint32_t* cnts = tmp.get<uint32_t>(n > 0 ? n : 1, st);
  uint32_t* offs = tmp.get<uint32_t>(n > 0 ? n : 1, st);
  uint32_t* rtmp = tmp.get<uint32_t>(radix_tmp_words(n) + scan_tmp_words(n) + 4, st);
  if (!f->rec || !f->rect || !f->tcount || !f->ranges || !f->order || !f->counters || !f->cand || !f->geom ||
      !dkey || !idx || !dkey2 || !idx2 || !cnts || !offs || !rtmp)
    return failed(fail(GS_ERR_OOM, std::string(who) + ": device allocation failed"));
  uint32_t* total = rtmp + radix_tmp_words(n) + scan_tmp_words(n);
  cudaError_t e;
#define GS_CKC(expr)                                         \
  do {                                                       \
    e = (expr);                                              \
    if (e != cudaSuccess) return failed(cuda_fail(e, #expr)); \
  } while (0)
  GS_CKC(cudaMemsetAsync(f->counters, 0, 8 * sizeof(unsigned long long), st));
  // candidates (possibly visible surfels) in index order; only they are sorted
  uint32_t* ncand = reinterpret_cast<uint32_t*>(f->counters + 6);
  f->ncand = ncand;
  GS_CKC(launch_preprocess(sc->P, cam, set, f->rec, f->rect, f->tcount, dkey, idx, f->cand, ncand, f->geom,
                           cnts, rtmp + radix_tmp_words(n), st));
  uint32_t *skey = dkey, *sidx = idx;
  // the last pass also gathers each sorted candidate's instance count
  GS_CKC(radix_sort_pairs(dkey, idx, dkey2, idx2, n, 32, rtmp, &skey, &sidx, st, ncand, f->tcount, cnts));
  GS_CKC(launch_scan(cnts, offs, n, total, rtmp + radix_tmp_words(n), st, ncand));
  uint32_t Kh = 0;
  GS_CKC(cudaMemcpyAsync(&Kh, total, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  GS_CKC(cudaStreamSynchronize(st));
  const int64_t K = Kh;
  if (K >= (int64_t(1) << 31)) return failed(fail(GS_ERR_CAPACITY, std::string(who) + ": more than 2^31 tile instances"));
  f->K = K;
  uint32_t* keys = tmp.get<uint32_t>(K > 0 ? K : 1, st);
  uint32_t* vals = f->buf.get<uint32_t>(K > 0 ? K : 1, st);
  uint32_t* keys2 = tmp.get<uint32_t>(K > 0 ? K : 1, st);
  uint32_t* vals2 = f->buf.get<uint32_t>(K > 0 ? K : 1, st);
  uint32_t* ktmp = tmp.get<uint32_t>(radix_tmp_words(K), st);
  if (!keys || !vals || !keys2 || !vals2 || !ktmp)
    return failed(fail(GS_ERR_OOM, std::string(who) + ": device allocation failed (tile lists)"));
  const float rf = (float)sqrt((double)sc->settings.rho_max / (double)sc->settings.screen_inv_sigma2);
  GS_CKC(launch_emit(sidx, offs, cnts, f->rect, f->geom, rf, n, cam.tiles_x, keys, vals, st, ncand));
  uint32_t *tk = keys, *tv = vals;
  GS_CKC(radix_sort_pairs(keys, vals, keys2, vals2, K, bits_for(ntiles), ktmp, &tk, &tv, st));
  f->vals = tv;
  f->buf.release(tv == vals ? vals2 : vals, st);
  GS_CKC(launch_ranges(tk, K, f->ranges, ntiles, st));
  if (tile_order_supported(ntiles)) GS_CKC(launch_tile_order(f->ranges, ntiles, f->order, st));
  else f->order = nullptr;  // natural tile order (the buffer stays owned by f->buf)
#undef GS_CKC
  tmp.release_all(st);
  return GS_OK;
}

// The forward blend of a built frame.  An image with too few tiles to fill
// the GPU (under two waves of five CTAs per SM) has its long tile lists
// composited in segments of lseg entries, lseg chosen so that the segments
// make about two waves.
gs_status blend_forward(gs_scene* sc, gs_frame* f, float* out, int32_t* n_contrib, cudaStream_t st) {
  const CamDev& cam = f->cam;
  const SetDev set = to_dev(sc->settings);
  const int ntiles = cam.tiles_x * cam.tiles_y;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  SegBufs sb;
  sb.lseg = split_lseg(ntiles, f->K, sms);
  if (sb.lseg == 0) {
    e = launch_blend_fwd(cam, set, f->order, f->rec, f->geom, f->vals, f->ranges, out, n_contrib, f->last, f->med,
                         f->counters, st);
    return e == cudaSuccess ? GS_OK : cuda_fail(e, "gs_render: blend");
  }
  const int64_t nmax = split_nseg_max(f->K, sb.lseg);
  sb.nseg_max = (unsigned)nmax;
  Buffers tmp;
  tmp.al = &sc->al;
  sb.segcnt = tmp.get<uint32_t>(ntiles, st);
  sb.segoff = tmp.get<uint32_t>(ntiles, st);
  sb.nseg = tmp.get<uint32_t>(1, st);
  sb.scan_tmp = tmp.get<uint32_t>(scan_tmp_words(ntiles), st);
  sb.seg_tile = tmp.get<uint32_t>(nmax, st);
  sb.seg_idx = tmp.get<uint32_t>(nmax, st);
  sb.trans = tmp.get<float>((size_t)nmax * 256, st);
  sb.part = tmp.get<unsigned char>((size_t)nmax * 256 * seg_part_bytes(), st);
  if (!sb.segcnt || !sb.segoff || !sb.nseg || !sb.scan_tmp || !sb.seg_tile || !sb.seg_idx || !sb.trans || !sb.part) {
    tmp.release_all(st);
    return fail(GS_ERR_OOM, "gs_render: device allocation failed (segments)");
  }
  e = launch_blend_fwd_split(cam, set, f->order, f->rec, f->geom, f->vals, f->ranges, out, n_contrib, f->last,
                             f->med, f->counters, sb, st);
  tmp.release_all(st);
  return e == cudaSuccess ? GS_OK : cuda_fail(e, "gs_render: blend");
}

}  // namespace

extern "C" {

uint64_t gs_kernel_launches(void) { return gs2d::g_launches.load(); }

gs_status gs_profile_enable(int32_t on) {
  gs2d::g_prof_on.store(on ? 1 : 0);
  return GS_OK;
}

gs_status gs_profile_read(int32_t kernel, double* total_ms, int64_t* launches) {
  if (kernel < 0 || kernel >= kProfCount || !total_ms || !launches)
    return fail(GS_ERR_ARG, "gs_profile_read: bad argument");
  std::lock_guard<std::mutex> lk(gs2d::g_prof_mu);
  double t = 0.0;
  int64_t k = 0;
  for (auto& pr : gs2d::g_prof_pending[kernel]) {
    float ms = 0.f;
    if (cudaEventSynchronize(pr.b) == cudaSuccess && cudaEventElapsedTime(&ms, pr.a, pr.b) == cudaSuccess) {
      t += ms;
      ++k;
    }
    cudaGetLastError();
    gs2d::g_prof_free.push_back(pr.a);
    gs2d::g_prof_free.push_back(pr.b);
  }
  gs2d::g_prof_pending[kernel].clear();
  *total_ms = t;
  *launches = k;
  return GS_OK;
}

const char* gs_version(void) { return "gs2d-gb300 0.1 (sm_103a)"; }

const char* gs_last_error(void) { return g_last_error.c_str(); }

gs_status gs_default_settings(gs_settings* s) {
  if (!s) return fail(GS_ERR_ARG, "gs_default_settings: null");
  s->near_plane = 0.2f;
  s->alpha_min = 1.0f / 255.0f;
  s->T_min = 1e-4f;
  s->alpha_max = 0.99f;
  s->rho_max = 9.0f;
  s->screen_inv_sigma2 = 2.0f;
  s->bg[0] = s->bg[1] = s->bg[2] = 0.0f;
  return GS_OK;
}

gs_status gs_set_params(gs_scene* sc, int64_t n, const float* mu, const float* quat,
                        const float* scale, const float* opacity, const float* sh) {
  if (!sc) return fail(GS_ERR_ARG, "gs_set_params: null scene");
  if (sc->P.sh_table) return fail(GS_ERR_ARG, "gs_set_params: the scene is compressed");
  if (n < 0 || n >= (int64_t(1) << 31)) return fail(GS_ERR_ARG, "gs_set_params: n out of range");
  if (n > 0 && (!mu || !quat || !scale || !opacity || !sh))
    return fail(GS_ERR_ARG, "gs_set_params: null parameter array");
  sc->P.n = (int)n;
  sc->P.mu = mu;
  sc->P.quat = quat;
  sc->P.scale = scale;
  sc->P.opacity = opacity;
  sc->P.sh = sh;
  return GS_OK;
}

gs_status gs_create_scene(gs_scene** out, const gs_scene_desc* d) {
  if (!out || !d) return fail(GS_ERR_ARG, "gs_create_scene: null argument");
  *out = nullptr;
  if (d->sh_degree < 0 || d->sh_degree > 3) return fail(GS_ERR_ARG, "gs_create_scene: sh_degree must be 0..3");
  const gs_settings& s = d->settings;
  if (!(s.rho_max > 0.f) || !(s.screen_inv_sigma2 > 0.f) || !(s.alpha_max > 0.f) ||
      !(s.alpha_max < 1.f) || !(s.T_min > 0.f) || !(s.near_plane > 0.f))
    return fail(GS_ERR_ARG, "gs_create_scene: invalid settings");
  gs_scene* sc = new (std::nothrow) gs_scene();
  if (!sc) return fail(GS_ERR_OOM, "gs_create_scene: host allocation");
  sc->settings = s;
  sc->al.a = d->allocator;
  sc->P.sh_degree = d->sh_degree;
  gs_status st = gs_set_params(sc, d->n, d->mu, d->quat, d->scale, d->opacity, d->sh);
  if (st != GS_OK) {
    delete sc;
    return st;
  }
  set_pool_threshold();
  *out = sc;
  return GS_OK;
}

gs_status gs_destroy_scene(gs_scene* sc) {
  delete sc;
  return GS_OK;
}

gs_status gs_frame_release(gs_frame* f, void* stream) {
  if (!f) return GS_OK;
  f->buf.release_all((cudaStream_t)stream);
  delete f;
  return GS_OK;
}

gs_status gs_render(gs_scene* sc, const gs_camera* c, float* out, int32_t* n_contrib,
                    gs_frame** saved, void* stream) {
  if (saved) *saved = nullptr;
  if (!out) return fail(GS_ERR_ARG, "gs_render: null argument");
  gs_status s = GS_OK;
  gs_frame* f = new_frame(sc, c, out, "gs_render", &s);
  if (!f) return s;
  cudaStream_t st = (cudaStream_t)stream;
  f->last = f->buf.get<int32_t>((size_t)f->cam.W * f->cam.H, st);
  f->med = f->buf.get<int32_t>((size_t)f->cam.W * f->cam.H, st);
  if (!f->last || !f->med) {
    gs_frame_release(f, stream);
    return fail(GS_ERR_OOM, "gs_render: device allocation failed");
  }
  s = build_lists(sc, f, "gs_render", st);
  if (s == GS_OK) s = blend_forward(sc, f, out, n_contrib, st);
  if (s != GS_OK || !saved) {
    gs_frame_release(f, stream);
    return s;
  }
  *saved = f;
  return GS_OK;
}

gs_status gs_contribution(gs_scene* sc, const gs_camera* c, float gamma, float weight, float* contrib,
                          float* view_sum, uint32_t* view_count, void* stream) {
  if (!contrib && !view_sum && !view_count) return fail(GS_ERR_ARG, "gs_contribution: no output");
  if (!(gamma >= 0.f && gamma <= 1.f)) return fail(GS_ERR_ARG, "gs_contribution: gamma must be in [0, 1]");
  gs_status s = GS_OK;
  gs_frame* f = new_frame(sc, c, nullptr, "gs_contribution", &s);
  if (!f) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = f->n;
  // per-view sums and support counts: the caller's arrays (overwritten, zero
  // outside the candidates) or scratch (zeroed for the candidates only)
  float* csum = view_sum ? view_sum : f->buf.get<float>(n > 0 ? n : 1, st);
  uint32_t* ccnt = view_count ? view_count : f->buf.get<uint32_t>(n > 0 ? n : 1, st);
  if (!csum || !ccnt) {
    gs_frame_release(f, stream);
    return fail(GS_ERR_OOM, "gs_contribution: device allocation failed");
  }
  cudaError_t e = cudaSuccess;
  if (view_sum && n > 0) e = cudaMemsetAsync(view_sum, 0, sizeof(float) * (size_t)n, st);
  if (e == cudaSuccess && view_count && n > 0) e = cudaMemsetAsync(view_count, 0, sizeof(uint32_t) * (size_t)n, st);
  if (e != cudaSuccess) {
    gs_frame_release(f, stream);
    return cuda_fail(e, "gs_contribution");
  }
  s = build_lists(sc, f, "gs_contribution", st);
  if (s == GS_OK) {
    const bool zero_cand = !view_sum || !view_count;
    e = launch_contribution(f->cam, to_dev(sc->settings), gamma, weight, f->order, f->rec, f->geom, f->vals,
                            f->ranges, f->cand, f->ncand, n, zero_cand, csum, ccnt, contrib, st);
    if (e != cudaSuccess) s = cuda_fail(e, "gs_contribution");
  }
  gs_frame_release(f, stream);
  return s;
}

gs_status gs_prune_by_contribution(int64_t n, const float* contrib, double ratio, uint8_t* keep, float* bound,
                                   void* stream) {
  if (n < 0 || (n > 0 && (!contrib || !keep))) return fail(GS_ERR_ARG, "gs_prune_by_contribution: bad argument");
  if (!(ratio >= 0.0 && ratio <= 1.0)) return fail(GS_ERR_ARG, "gs_prune_by_contribution: ratio must be in [0, 1]");
  const double kd = ceil(ratio * (double)n);
  const int64_t k = kd < 0.0 ? 0 : (kd > (double)n ? n : (int64_t)kd);
  cudaStream_t st = (cudaStream_t)stream;
  set_pool_threshold();
  Alloc al;
  uint32_t* tmp = static_cast<uint32_t*>(al.get(select_tmp_words() * sizeof(uint32_t), st));
  if (!tmp) return fail(GS_ERR_OOM, "gs_prune_by_contribution: scratch allocation failed");
  const cudaError_t e = launch_prune(n, contrib, k, keep, bound, tmp, st);
  al.put(tmp, 0, st);
  if (e != cudaSuccess) return cuda_fail(e, "gs_prune_by_contribution");
  return GS_OK;
}

gs_status gs_frame_get_info(gs_frame* f, gs_frame_info* info, void* stream) {
  if (!f || !info) return fail(GS_ERR_ARG, "gs_frame_get_info: null argument");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long h[8];
  GS_CK(cudaMemcpyAsync(h, f->counters, sizeof h, cudaMemcpyDeviceToHost, st));
  GS_CK(cudaStreamSynchronize(st));
  info->n_instances = f->K;
  info->pairs_evaluated = (int64_t)h[0];
  info->pairs_blended = (int64_t)h[1];
  info->bwd_pairs_evaluated = (int64_t)h[2];
  info->bwd_warp_entries = (int64_t)h[3];
  info->bwd_warp_lanes = (int64_t)h[4];
  info->tiles_x = f->cam.tiles_x;
  info->tiles_y = f->cam.tiles_y;
  info->n_candidates = (int64_t)(h[6] & 0xFFFFFFFFull);
  // visible surfels (non-empty tile rectangle), counted on the host (debug path)
  std::vector<uint2> rc((size_t)f->n);
  if (f->n > 0) {
    GS_CK(cudaMemcpyAsync(rc.data(), f->rect, sizeof(uint2) * (size_t)f->n, cudaMemcpyDeviceToHost, st));
    GS_CK(cudaStreamSynchronize(st));
  }
  int64_t v = 0;
  for (const uint2& r : rc) v += (r.y & 0xFFFF) > (r.x & 0xFFFF);
  info->n_visible = v;
  return GS_OK;
}

gs_status gs_frame_copy_lists(gs_frame* f, int32_t* values, int64_t cap, int32_t* ranges,
                              int32_t* rects, void* stream) {
  if (!f) return fail(GS_ERR_ARG, "gs_frame_copy_lists: null frame");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t k = f->K < cap ? f->K : cap;
  if (values && k > 0)
    GS_CK(cudaMemcpyAsync(values, f->vals, sizeof(uint32_t) * (size_t)k, cudaMemcpyDeviceToDevice, st));
  if (ranges)
    GS_CK(cudaMemcpyAsync(ranges, f->ranges, sizeof(int2) * (size_t)f->cam.tiles_x * f->cam.tiles_y,
                          cudaMemcpyDeviceToDevice, st));
  if (rects && f->n > 0) {
    api_unpack_rect_kernel<<<div_up(f->n, 256), 256, 0, st>>>(f->rect, f->tcount, f->n, rects);
    count_launch();
    GS_CK(cudaGetLastError());
  }
  return GS_OK;
}

static_assert(sizeof(RowGeom) == 14 * sizeof(int32_t), "RowGeom is 14 words");

__global__ void api_depth_kernel(const float4* __restrict__ rec, const uint32_t* __restrict__ tcount, int n,
                                 float* __restrict__ depth) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) depth[i] = tcount[i] > 0u ? rec[(size_t)i * kRecF4 + 2].z : 0.f;
}

gs_status gs_frame_copy_cover(gs_frame* f, int32_t* geom, float* depth, int32_t* tile_count, void* stream) {
  if (!f) return fail(GS_ERR_ARG, "gs_frame_copy_cover: null frame");
  cudaStream_t st = (cudaStream_t)stream;
  if (f->n <= 0) return GS_OK;
  if (geom) GS_CK(cudaMemcpyAsync(geom, f->geom, sizeof(RowGeom) * (size_t)f->n, cudaMemcpyDeviceToDevice, st));
  if (tile_count)
    GS_CK(cudaMemcpyAsync(tile_count, f->tcount, sizeof(uint32_t) * (size_t)f->n, cudaMemcpyDeviceToDevice, st));
  if (depth) {
    api_depth_kernel<<<div_up(f->n, 256), 256, 0, st>>>(f->rec, f->tcount, f->n, depth);
    count_launch();
    GS_CK(cudaGetLastError());
  }
  return GS_OK;
}

gs_status gs_loss(int32_t W, int32_t H, const float* out, const float* tgt, const float* tinv,
                  const gs_loss_weights* w, float* adj_total, float* adj_ssim, float* adj_l1,
                  float* losses, void* stream) {
  if (W <= 0 || H <= 0 || !out || !tgt || !w || !adj_total || !losses)
    return fail(GS_ERR_ARG, "gs_loss: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  set_pool_threshold();
  Alloc al;
  float* tmp = static_cast<float*>(al.get(loss_tmp_floats(W, H) * sizeof(float), st));
  if (!tmp) return fail(GS_ERR_OOM, "gs_loss: scratch allocation failed");
  cudaError_t e = launch_loss(W, H, out, tgt, tinv, *w, adj_total, adj_ssim, adj_l1, losses, tmp, st);
  al.put(tmp, 0, st);
  if (e != cudaSuccess) return cuda_fail(e, "gs_loss");
  return GS_OK;
}

gs_status gs_backward(gs_scene* sc, gs_frame* f, const float* const* adj_sets,
                      const uint32_t* plane_masks, int32_t n_sets, const gs_param_grads* grads,
                      float* screen_grads, void* stream) {
  if (!sc || !f || !adj_sets || !plane_masks || !grads) return fail(GS_ERR_ARG, "gs_backward: null argument");
  if (sc->P.sh_table) return fail(GS_ERR_ARG, "gs_backward: compressed scenes are render-only");
  if (f->scene != sc) return fail(GS_ERR_STATE, "gs_backward: frame belongs to another scene");
  if (sc->P.n != f->n) return fail(GS_ERR_STATE, "gs_backward: surfel count changed since the render");
  if (n_sets < 1 || n_sets > 3) return fail(GS_ERR_ARG, "gs_backward: n_sets must be 1..3");
  AdjDev adj{};
  adj.n_sets = n_sets;
  for (int s = 0; s < n_sets; ++s) {
    if (!adj_sets[s]) return fail(GS_ERR_ARG, "gs_backward: null adjoint set");
    if (s > 0 && (plane_masks[s] & ~GS_MASK_RGB)) return fail(GS_ERR_ARG, "gs_backward: sets after the first may use only colour planes");
    adj.set[s] = adj_sets[s];
    adj.mask[s] = plane_masks[s] & GS_MASK_ALL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int n = f->n;
  float* grec = static_cast<float*>(sc->al.get(sizeof(float) * kGradRec * (size_t)(n > 0 ? n : 1), st));
  if (!grec) return fail(GS_ERR_OOM, "gs_backward: scratch allocation failed");
  cudaError_t e = cudaMemsetAsync(grec, 0, sizeof(float) * kGradRec * (size_t)n, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->counters + 2, 0, 3 * sizeof(unsigned long long), st);
  const SetDev set = to_dev(sc->settings);
  if (e == cudaSuccess)
    e = launch_blend_bwd(f->cam, set, f->order, f->rec, f->geom, f->vals, f->ranges, f->out, f->last, f->med, adj,
                         grec, screen_grads, n, f->K, f->counters, st);
  if (e == cudaSuccess) e = launch_preprocess_bwd(sc->P, f->cam, f->cand, f->ncand, f->tcount, grec, *grads, st);
  sc->al.put(grec, sizeof(float) * kGradRec * (size_t)(n > 0 ? n : 1), st);
  if (e != cudaSuccess) return cuda_fail(e, "gs_backward");
  return GS_OK;
}

gs_status gs_densify_accumulate(gs_scene* sc, gs_frame* f, const float* screen, int32_t n_sets,
                                float* stats, void* stream) {
  if (!sc || !f || !screen || !stats) return fail(GS_ERR_ARG, "gs_densify_accumulate: null argument");
  if (sc->P.sh_table) return fail(GS_ERR_ARG, "gs_densify_accumulate: compressed scenes are render-only");
  if (f->n != sc->P.n) return fail(GS_ERR_STATE, "gs_densify_accumulate: surfel count changed");
  if (n_sets < 1) return fail(GS_ERR_ARG, "gs_densify_accumulate: n_sets must be >= 1");
  cudaError_t e = launch_densify_accumulate(f->rect, screen, f->n, n_sets, stats, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_densify_accumulate");
  return GS_OK;
}

gs_status gs_densify_select(int64_t n, const float* stats, const float* scale, float omega,
                            float grad_thr, float eta_thr, uint8_t* mask, float* g_out, float* k_out,
                            void* stream) {
  if (n < 0 || (n > 0 && (!stats || !scale || !mask))) return fail(GS_ERR_ARG, "gs_densify_select: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  set_pool_threshold();
  Alloc al;
  double* tmp = static_cast<double*>(al.get(densify_tmp_doubles(n) * sizeof(double), st));
  if (!tmp) return fail(GS_ERR_OOM, "gs_densify_select: scratch allocation failed");
  cudaError_t e = launch_densify_select(n, stats, scale, omega, grad_thr, eta_thr, mask, g_out, k_out, tmp, st);
  al.put(tmp, 0, st);
  if (e != cudaSuccess) return cuda_fail(e, "gs_densify_select");
  return GS_OK;
}

gs_status gs_elongation_filter(int64_t n, const float* scale, float eta_thr, uint8_t* keep, void* stream) {
  if (n < 0 || (n > 0 && (!scale || !keep))) return fail(GS_ERR_ARG, "gs_elongation_filter: bad argument");
  cudaError_t e = launch_elongation(n, scale, eta_thr, keep, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_elongation_filter");
  return GS_OK;
}

gs_status gs_visibility_count(int64_t n, const float* points, float sigma, const gs_camera* cams, int32_t n_views,
                              float near_plane, float lowpass, uint32_t* counts, void* stream) {
  if (n < 0 || n_views < 0 || (n > 0 && (!points || !counts)) || (n_views > 0 && !cams))
    return fail(GS_ERR_ARG, "gs_visibility_count: bad argument");
  if (!(sigma >= 0.f) || !(lowpass >= 0.f)) return fail(GS_ERR_ARG, "gs_visibility_count: sigma and lowpass must be >= 0");
  if (n == 0 || n_views == 0) return GS_OK;
  std::vector<VisCam> hc((size_t)n_views);
  for (int32_t v = 0; v < n_views; ++v) {
    const gs_camera& c = cams[v];
    if (c.width <= 0 || c.height <= 0 || !(c.fx > 0) || !(c.fy > 0))
      return fail(GS_ERR_ARG, "gs_visibility_count: bad camera " + std::to_string(v));
    VisCam& k = hc[(size_t)v];
    for (int i = 0; i < 9; ++i) k.R[i] = (float)c.R[i];
    for (int i = 0; i < 3; ++i) k.t[i] = (float)c.t[i];
    k.fx = (float)c.fx; k.fy = (float)c.fy; k.cx = (float)c.cx; k.cy = (float)c.cy;
    k.W = (float)c.width; k.H = (float)c.height;
  }
  cudaStream_t st = (cudaStream_t)stream;
  set_pool_threshold();
  Alloc al;
  const size_t bytes = sizeof(VisCam) * (size_t)n_views;
  VisCam* dc = static_cast<VisCam*>(al.get(bytes, st));
  if (!dc) return fail(GS_ERR_OOM, "gs_visibility_count: device allocation failed");
  // pageable source: the copy is staged before the call returns
  cudaError_t e = cudaMemcpyAsync(dc, hc.data(), bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_visibility_count(points, n, sigma, lowpass, near_plane, dc, n_views, counts, st);
  al.put(dc, bytes, st);
  if (e != cudaSuccess) return cuda_fail(e, "gs_visibility_count");
  return GS_OK;
}

gs_status gs_visibility_bounds(int64_t n, const float* points, const uint32_t* counts, uint32_t min_count,
                               uint8_t* keep, float* zrange, void* stream) {
  if (n < 0 || (n > 0 && (!points || !counts || !keep)) || !zrange)
    return fail(GS_ERR_ARG, "gs_visibility_bounds: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  set_pool_threshold();
  Alloc al;
  int* tmp = static_cast<int*>(al.get(2 * sizeof(int), st));
  if (!tmp) return fail(GS_ERR_OOM, "gs_visibility_bounds: scratch allocation failed");
  const cudaError_t e = launch_visibility_keep(points, n, counts, min_count, keep, zrange, tmp, st);
  al.put(tmp, 2 * sizeof(int), st);
  if (e != cudaSuccess) return cuda_fail(e, "gs_visibility_bounds");
  return GS_OK;
}

gs_status gs_geometry_loss(int32_t W, int32_t H, const gs_camera* cam, const float* out, float w_normal,
                           float w_dist, float* adj, float* losses, void* stream) {
  if (W <= 0 || H <= 0 || !cam || !out || !adj || !losses) return fail(GS_ERR_ARG, "gs_geometry_loss: bad argument");
  if (cam->width != W || cam->height != H || !(cam->fx > 0) || !(cam->fy > 0))
    return fail(GS_ERR_ARG, "gs_geometry_loss: camera does not match the image");
  cudaStream_t st = (cudaStream_t)stream;
  set_pool_threshold();
  Alloc al;
  const size_t bytes = geometry_tmp_bytes(W, H);
  void* tmp = al.get(bytes, st);
  if (!tmp) return fail(GS_ERR_OOM, "gs_geometry_loss: scratch allocation failed");
  const cudaError_t e = launch_geometry_loss(W, H, (float)cam->fx, (float)cam->fy, (float)cam->cx, (float)cam->cy,
                                             out, w_normal, w_dist, adj, losses, tmp, st);
  al.put(tmp, bytes, st);
  if (e != cudaSuccess) return cuda_fail(e, "gs_geometry_loss");
  return GS_OK;
}

gs_status gs_adam_step(int64_t n, float* param, const float* grad, float* m, float* v, float lr, float beta1,
                       float beta2, float eps, int32_t step, void* stream) {
  if (n < 0 || (n > 0 && (!param || !grad || !m || !v)) || step < 1 || !(beta1 >= 0.f && beta1 < 1.f) ||
      !(beta2 >= 0.f && beta2 < 1.f))
    return fail(GS_ERR_ARG, "gs_adam_step: bad argument");
  const double bc1 = 1.0 - pow((double)beta1, step), bc2 = 1.0 - pow((double)beta2, step);
  const cudaError_t e = launch_adam(n, param, grad, m, v, lr, beta1, beta2, eps, (float)bc1, (float)bc2,
                                    (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_adam_step");
  return GS_OK;
}

gs_status gs_densify_plan(int64_t n, const uint8_t* select, const uint8_t* keep, const float* scale,
                          const float* opacity, int32_t raw, float dense_thr, float min_opacity, uint8_t* action,
                          uint32_t* offset, int64_t* n_out, void* stream) {
  if (n < 0 || !n_out || (n > 0 && (!select || !scale || !opacity || !action || !offset)))
    return fail(GS_ERR_ARG, "gs_densify_plan: bad argument");
  *n_out = 0;
  if (n == 0) return GS_OK;
  if (n >= (int64_t(1) << 31)) return fail(GS_ERR_CAPACITY, "gs_densify_plan: more than 2^31 surfels");
  cudaStream_t st = (cudaStream_t)stream;
  set_pool_threshold();
  Alloc al;
  const size_t words = (size_t)n + scan_tmp_words(n) + 2;
  uint32_t* tmp = static_cast<uint32_t*>(al.get(words * 4, st));
  if (!tmp) return fail(GS_ERR_OOM, "gs_densify_plan: scratch allocation failed");
  uint32_t* rows = tmp;
  uint32_t* total = tmp + n;
  uint32_t* stmp = total + 1;
  // raw parametrisation (log-scale, logit-opacity): the thresholds move with it
  const float thr_s = raw ? (float)log((double)dense_thr) : dense_thr;
  const float thr_o = raw ? (float)log((double)min_opacity / (1.0 - (double)min_opacity)) : min_opacity;
  cudaError_t e = launch_densify_plan(n, select, keep, scale, opacity, thr_s, thr_o, action, rows, st);
  if (e == cudaSuccess) e = launch_scan(rows, offset, n, total, stmp, st);
  uint32_t h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, total, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  al.put(tmp, words * 4, st);
  if (e != cudaSuccess) return cuda_fail(e, "gs_densify_plan");
  *n_out = h;
  return GS_OK;
}

gs_status gs_densify_apply(int64_t n, int32_t sh_degree, int32_t raw, const uint8_t* action,
                           const uint32_t* offset, const float* xi, const float* mu, const float* quat, const float* scale,
                           const float* opacity, const float* sh, float* mu_out, float* quat_out, float* scale_out,
                           float* opacity_out, float* sh_out, int32_t* src, uint8_t* fresh, void* stream) {
  if (n < 0 || sh_degree < 0 || sh_degree > 3 ||
      (n > 0 && (!action || !offset || !xi || !mu || !quat || !scale || !opacity || !sh || !mu_out || !quat_out ||
                 !scale_out || !opacity_out || !sh_out || !src || !fresh)))
    return fail(GS_ERR_ARG, "gs_densify_apply: bad argument");
  const cudaError_t e = launch_densify_apply(n, sh_degree, raw != 0, action, offset, xi, mu, quat, scale, opacity, sh,
                                             mu_out, quat_out, scale_out, opacity_out, sh_out, src, fresh,
                                             (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_densify_apply");
  return GS_OK;
}

gs_status gs_gather_rows(int64_t n_out, int32_t width, const int32_t* src, const uint8_t* fresh, const float* in,
                         float* out, void* stream) {
  if (n_out < 0 || width < 0 || (n_out > 0 && width > 0 && (!src || !in || !out)))
    return fail(GS_ERR_ARG, "gs_gather_rows: bad argument");
  const cudaError_t e = launch_gather_rows(n_out, width, src, fresh, in, out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_gather_rows");
  return GS_OK;
}

gs_status gs_activate(int64_t n, const float* log_scale, const float* logit_opacity, float* scale, float* opacity,
                      void* stream) {
  if (n < 0 || (n > 0 && (!log_scale || !logit_opacity || !scale || !opacity)))
    return fail(GS_ERR_ARG, "gs_activate: bad argument");
  const cudaError_t e = launch_activate(n, log_scale, logit_opacity, scale, opacity, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_activate");
  return GS_OK;
}

gs_status gs_activate_grad(int64_t n, const float* scale, const float* opacity, float* grad_scale, float* grad_opacity,
                           void* stream) {
  if (n < 0 || (n > 0 && (!scale || !opacity || !grad_scale || !grad_opacity)))
    return fail(GS_ERR_ARG, "gs_activate_grad: bad argument");
  const cudaError_t e = launch_activate_grad(n, scale, opacity, grad_scale, grad_opacity, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_activate_grad");
  return GS_OK;
}

gs_status gs_sync(void* stream, int32_t timeout_ms) {
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaStreamQuery((cudaStream_t)stream);
    if (e == cudaSuccess) return GS_OK;
    if (e != cudaErrorNotReady) return cuda_fail(e, "gs_sync");
    const auto dt = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0);
    if (dt.count() >= timeout_ms) return fail(GS_ERR_TIMEOUT, "gs_sync: stream still busy");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

}  // extern "C"

// ---- Vector quantisation of SH and compressed scenes ------------------------------

namespace {

int device_sms() {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

// Lists the quantised vectors and packs their operands: fills b (owned by
// buf), m, C, D.  Synchronises once (m).
gs_status vq_prepare(const char* who, int64_t n, int32_t deg, const float* sh, const uint8_t* keep, int32_t K,
                     int32_t method, bool kmeans, cudaStream_t st, Buffers& buf, VqBufs& b, int& m, int& C, int& D,
                     bool& tensor) {
  const std::string w(who);
  if (n < 0 || n >= (int64_t(1) << 31) || (n > 0 && (!sh || !keep)))
    return fail(GS_ERR_ARG, w + ": bad n or null array");
  if (deg < 0 || deg > 3) return fail(GS_ERR_ARG, w + ": sh_degree must be 0..3");
  if (K < 1 || K > (1 << 24)) return fail(GS_ERR_ARG, w + ": K must be in [1, 2^24]");
  if (method < 0 || method > 2) return fail(GS_ERR_ARG, w + ": method must be 0, 1 or 2");
  if (method == 1 && K % 256 != 0) return fail(GS_ERR_ARG, w + ": the tensor-core path needs K % 256 == 0");
  tensor = method == 1 || (method == 0 && K % 256 == 0);
  D = vq_width(deg, &C);
  b.err = buf.get<int>(1, st);
  uint32_t* total = buf.get<uint32_t>(1, st);
  if (!b.err || !total) return fail(GS_ERR_OOM, w + ": scratch allocation failed");
  GS_CK(cudaMemsetAsync(b.err, 0, sizeof(int), st));
  uint32_t hm = 0;
  if (n > 0) {
    uint32_t* flags = buf.get<uint32_t>((size_t)n, st);
    uint32_t* offs = buf.get<uint32_t>((size_t)n, st);
    uint32_t* stmp = buf.get<uint32_t>(scan_tmp_words(n), st);
    b.rows = buf.get<uint32_t>((size_t)n, st);
    if (!flags || !offs || !stmp || !b.rows) return fail(GS_ERR_OOM, w + ": scratch allocation failed");
    GS_CK(launch_vq_list(keep, (int)n, 0, flags, offs, total, stmp, b.rows, st));
    GS_CK(cudaMemcpyAsync(&hm, total, sizeof hm, cudaMemcpyDeviceToHost, st));
    GS_CK(cudaStreamSynchronize(st));
    buf.release(flags, st);
    buf.release(offs, st);
    buf.release(stmp, st);
  }
  m = (int)hm;
  const size_t m_pad = ((size_t)m + 127) / 128 * 128;
  b.xr = buf.get<uint16_t>((size_t)m * C + 1, st);
  b.xt = buf.get<uint16_t>(m_pad * D + 1, st);
  b.ct = tensor ? buf.get<uint16_t>((size_t)K * D, st) : nullptr;
  b.hl = buf.get<float2>((size_t)K, st);
  b.best64 = buf.get<unsigned long long>(m_pad + 1, st);
  b.best_idx = buf.get<int32_t>((size_t)m + 1, st);
  if (kmeans) {
    b.sums = buf.get<unsigned long long>((size_t)K * C, st);
    b.cnt = buf.get<unsigned int>((size_t)K, st);
  }
  if (!b.xr || !b.xt || (tensor && !b.ct) || !b.hl || !b.best64 || !b.best_idx || (kmeans && (!b.sums || !b.cnt)))
    return fail(GS_ERR_OOM, w + ": scratch allocation failed");
  GS_CK(launch_vq_pack_x(sh, b, m, C, D, st));
  return GS_OK;
}

gs_status vq_check(const char* who, const int* err_dev, cudaStream_t st) {
  int err = 0;
  GS_CK(cudaMemcpyAsync(&err, err_dev, sizeof err, cudaMemcpyDeviceToHost, st));
  GS_CK(cudaStreamSynchronize(st));
  if (err == 1) return fail(GS_ERR_CUDA, std::string(who) + ": the assignment pipeline timed out");
  if (err == 2) return fail(GS_ERR_ARG, std::string(who) + ": a value is outside the binary16 range");
  if (err == 3) return fail(GS_ERR_ARG, std::string(who) + ": an entry index is outside [0, K)");
  return GS_OK;
}

}  // namespace

gs_status gs_vq_kmeans(int64_t n, int32_t sh_degree, const float* sh, const uint8_t* keep, int32_t K, int32_t iters,
                       const float* init_u, uint16_t* codebook, int32_t* assign, double* objective, int32_t method,
                       int64_t* m_out, void* stream) {
  if (iters < 0 || !init_u || !codebook || (n > 0 && !assign)) return fail(GS_ERR_ARG, "gs_vq_kmeans: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  set_pool_threshold();
  Alloc al;
  Buffers buf;
  buf.al = &al;
  VqBufs b;
  int m = 0, C = 0, D = 0;
  bool tensor = false;
  gs_status s = vq_prepare("gs_vq_kmeans", n, sh_degree, sh, keep, K, method, true, st, buf, b, m, C, D, tensor);
  if (s != GS_OK) {
    buf.release_all(st);
    return s;
  }
  const int sms = device_sms();
  cudaError_t e = launch_vq_init(b, m, C, init_u, K, codebook, st);
  if (e == cudaSuccess && objective) e = cudaMemsetAsync(objective, 0, sizeof(double) * (size_t)(iters + 1), st);
  for (int t = 0; t < iters && e == cudaSuccess; ++t) {
    e = launch_vq_assign(b, m, C, D, codebook, K, tensor, sms, st);
    if (e == cudaSuccess) e = launch_vq_accum(b, m, C, codebook, K, true, objective ? objective + t : nullptr, st);
    if (e == cudaSuccess) e = launch_vq_update(b, C, codebook, K, st);
  }
  if (e == cudaSuccess) e = launch_vq_assign(b, m, C, D, codebook, K, tensor, sms, st);
  if (e == cudaSuccess) e = launch_vq_accum(b, m, C, codebook, K, false, objective ? objective + iters : nullptr, st);
  if (e == cudaSuccess && n > 0) e = cudaMemsetAsync(assign, 0xFF, sizeof(int32_t) * (size_t)n, st);
  if (e == cudaSuccess) e = launch_vq_scatter(b, m, assign, st);
  s = e == cudaSuccess ? vq_check("gs_vq_kmeans", b.err, st) : cuda_fail(e, "gs_vq_kmeans");
  buf.release_all(st);
  if (s == GS_OK && m_out) *m_out = m;
  return s;
}

gs_status gs_vq_assign(int64_t n, int32_t sh_degree, const float* sh, const uint8_t* keep, int32_t K,
                       const uint16_t* codebook, int32_t* assign, int32_t method, void* stream) {
  if (!codebook || (n > 0 && !assign)) return fail(GS_ERR_ARG, "gs_vq_assign: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  set_pool_threshold();
  Alloc al;
  Buffers buf;
  buf.al = &al;
  VqBufs b;
  int m = 0, C = 0, D = 0;
  bool tensor = false;
  gs_status s = vq_prepare("gs_vq_assign", n, sh_degree, sh, keep, K, method, false, st, buf, b, m, C, D, tensor);
  if (s != GS_OK) {
    buf.release_all(st);
    return s;
  }
  cudaError_t e = launch_vq_assign(b, m, C, D, codebook, K, tensor, device_sms(), st);
  if (e == cudaSuccess) e = launch_vq_accum(b, m, C, codebook, K, false, nullptr, st);
  if (e == cudaSuccess && n > 0) e = cudaMemsetAsync(assign, 0xFF, sizeof(int32_t) * (size_t)n, st);
  if (e == cudaSuccess) e = launch_vq_scatter(b, m, assign, st);
  s = e == cudaSuccess ? vq_check("gs_vq_assign", b.err, st) : cuda_fail(e, "gs_vq_assign");
  buf.release_all(st);
  return s;
}

gs_status gs_vq_pack(int64_t n, int32_t sh_degree, const float* quat, const float* scale, const float* opacity,
                     const float* sh, const uint8_t* keep, const int32_t* assign, int32_t K, const uint16_t* codebook,
                     uint16_t* quat16, uint16_t* scale16, uint16_t* opacity16, uint32_t* sh_row, uint16_t* sh_table,
                     int64_t* rows_out, void* stream) {
  if (n < 0 || n >= (int64_t(1) << 31) || sh_degree < 0 || sh_degree > 3 || K < 0 || !rows_out ||
      (K > 0 && (!codebook || !sh_table)) ||
      (n > 0 && (!quat || !scale || !opacity || !sh || !keep || !assign || !quat16 || !scale16 || !opacity16 ||
                 !sh_row || !sh_table)))
    return fail(GS_ERR_ARG, "gs_vq_pack: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  set_pool_threshold();
  Alloc al;
  Buffers buf;
  buf.al = &al;
  int C = 0;
  vq_width(sh_degree, &C);
  int* err = buf.get<int>(1, st);
  uint32_t* total = buf.get<uint32_t>(1, st);
  uint32_t* flags = buf.get<uint32_t>((size_t)n + 1, st);
  uint32_t* offs = buf.get<uint32_t>((size_t)n + 1, st);
  uint32_t* stmp = buf.get<uint32_t>(scan_tmp_words(n), st);
  gs_status s = GS_OK;
  if (!err || !total || !flags || !offs || !stmp) {
    s = fail(GS_ERR_OOM, "gs_vq_pack: scratch allocation failed");
  } else {
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = launch_vq_list(keep, (int)n, 1, flags, offs, total, stmp, nullptr, st);
    if (e == cudaSuccess)
      e = launch_vq_pack_scene((int)n, C, K, quat, scale, opacity, sh, keep, assign, offs, codebook, quat16, scale16,
                               opacity16, sh_row, sh_table, err, st);
    uint32_t kept = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&kept, total, sizeof kept, cudaMemcpyDeviceToHost, st);
    s = e == cudaSuccess ? vq_check("gs_vq_pack", err, st) : cuda_fail(e, "gs_vq_pack");
    if (s == GS_OK) *rows_out = (int64_t)K + kept;
  }
  buf.release_all(st);
  return s;
}

gs_status gs_create_compressed_scene(gs_scene** out, const gs_compressed_scene_desc* d, void* stream) {
  if (!out || !d) return fail(GS_ERR_ARG, "gs_create_compressed_scene: null argument");
  *out = nullptr;
  if (d->sh_degree < 0 || d->sh_degree > 3)
    return fail(GS_ERR_ARG, "gs_create_compressed_scene: sh_degree must be 0..3");
  const gs_settings& se = d->settings;
  if (!(se.rho_max > 0.f) || !(se.screen_inv_sigma2 > 0.f) || !(se.alpha_max > 0.f) || !(se.alpha_max < 1.f) ||
      !(se.T_min > 0.f) || !(se.near_plane > 0.f))
    return fail(GS_ERR_ARG, "gs_create_compressed_scene: invalid settings");
  if (d->n < 0 || d->n >= (int64_t(1) << 31)) return fail(GS_ERR_ARG, "gs_create_compressed_scene: n out of range");
  if (d->n > 0 && (!d->mu || !d->quat || !d->scale || !d->opacity || !d->sh_row || !d->sh_table))
    return fail(GS_ERR_ARG, "gs_create_compressed_scene: null parameter array");
  if (d->n > 0 && (d->sh_rows < 1 || d->sh_rows > (int64_t)0xFFFFFFFFu))
    return fail(GS_ERR_ARG, "gs_create_compressed_scene: sh_rows out of range");
  if (((uintptr_t)d->quat % 8) || ((uintptr_t)d->scale % 4) || ((uintptr_t)d->opacity % 2) ||
      ((uintptr_t)d->sh_table % 2) || ((uintptr_t)d->sh_row % 4) || ((uintptr_t)d->mu % 4))
    return fail(GS_ERR_ARG, "gs_create_compressed_scene: misaligned array");
  cudaStream_t st = (cudaStream_t)stream;
  set_pool_threshold();
  Alloc al;
  al.a = d->allocator;
  if (d->n > 0) {
    int* err = static_cast<int*>(al.get(sizeof(int), st));
    if (!err) return fail(GS_ERR_OOM, "gs_create_compressed_scene: scratch allocation failed");
    int h = 0;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = launch_vq_check_rows(d->sh_row, (int)d->n, (uint32_t)d->sh_rows, err, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    al.put(err, sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(e, "gs_create_compressed_scene");
    if (h) return fail(GS_ERR_ARG, "gs_create_compressed_scene: an sh_row is outside [0, sh_rows)");
  }
  gs_scene* sc = new (std::nothrow) gs_scene();
  if (!sc) return fail(GS_ERR_OOM, "gs_create_compressed_scene: host allocation");
  sc->settings = se;
  sc->al = al;
  sc->P.n = (int)d->n;
  sc->P.sh_degree = d->sh_degree;
  sc->P.mu = d->mu;
  sc->P.quat = sc->P.scale = sc->P.opacity = sc->P.sh = nullptr;
  sc->P.quat16 = d->quat;
  sc->P.scale16 = d->scale;
  sc->P.opacity16 = d->opacity;
  sc->P.sh_row = d->sh_row;
  sc->P.sh_table = d->sh_table;
  *out = sc;
  return GS_OK;
}
