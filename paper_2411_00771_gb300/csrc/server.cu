// Serving loop: continuous batching of forward renders over resident scenes.
//
// Clients submit (scene, camera, output buffer) requests from any thread; a
// worker thread owned by the server runs each request through the render
// stages on one of `max_slots` streams and polls events instead of blocking:
//   stage A  preprocess, depth sort, instance count (count copied to pinned
//            host memory),
//   stage B  instance buffers, emission, tile sort, tile ranges,
//   blend    the views whose stage B has finished are blended together by
//            one persistent launch over all their tiles (blend_fwd_batched);
//            a view with too few tiles to fill the GPU and long lists gets
//            its own launches with the lists composited in segments, as
//            gs_render does for it.
// Requests that arrive while others are on the GPU enter as soon as a slot
// and memory are free, so stages of different requests overlap on the
// device.  Each slot keeps its buffers (per-surfel records, sort buffers,
// tile lists) resident between requests and grows them on demand; the sum
// of all slots' buffers never exceeds the server's memory budget.  A request
// whose buffers cannot fit is held until other slots finish (their idle
// buffers are then released) or fails with GS_ERR_CAPACITY if it cannot fit
// even alone.  Results are identical to gs_render's: the same kernels run
// in the same per-pixel order.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gs2d_internal.cuh"

// The scene object is defined in api.cu; the server needs its parameters.
namespace gs2d {
const ParamsDev& scene_params(const gs_scene* sc);
const gs_settings& scene_settings(const gs_scene* sc);
}  // namespace gs2d

using namespace gs2d;

namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Ticket {
  int64_t id = 0;
  gs_request req{};
  gs_scene* scene = nullptr;
  int state = 0;  // 0 queued, 1 running, 2 done, 3 failed
  gs_status err = GS_OK;
  std::string msg;
  double t_submit = 0.0, t_done = 0.0;
};

// Grow-only device buffer.
struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

enum SlotState { kIdle, kStageA, kWaitMem, kStageB, kReady, kBlending };

struct Slot {
  SlotState state = kIdle;
  cudaStream_t st = nullptr;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;
  uint32_t* k_host = nullptr;  // pinned
  Ticket* t = nullptr;
  // resident buffers
  Buf rec, geom, rect, tcount, dkey, idx, dkey2, idx2, cnts, offs, cand, rtmp;  // per surfel
  Buf keys, vals, keys2, vals2, ktmp;                                             // per instance
  Buf ranges;                                                                     // per tile
  Buf seg_tiles, seg_list, seg_trans, seg_part;  // long lists composited in segments
  int lseg = 0;                                  // 0: whole tiles
  unsigned nseg_max = 0;
  // request-specific
  CamDev cam{};
  SetDev set{};
  ParamsDev P{};
  float rf = 0.f;
  int64_t K = 0;
  uint32_t* sidx = nullptr;  // sorted surfel order (one of idx / idx2)
  uint32_t* ncand = nullptr; // device count of sorted candidates
  uint32_t* vals_final = nullptr;
  size_t bytes() const {
    return rec.bytes + geom.bytes + rect.bytes + tcount.bytes + dkey.bytes + idx.bytes + dkey2.bytes +
           idx2.bytes + cnts.bytes + offs.bytes + cand.bytes + rtmp.bytes + keys.bytes + vals.bytes +
           keys2.bytes + vals2.bytes + ktmp.bytes + ranges.bytes + seg_tiles.bytes + seg_list.bytes +
           seg_trans.bytes + seg_part.bytes;
  }
};

struct Batch {
  cudaEvent_t ev = nullptr;
  std::vector<int> slots;
};

}  // namespace

struct gs_server {
  int device = 0;
  size_t budget = 0;
  gs_allocator al{};
  std::vector<Slot> slots;
  cudaStream_t blend_st = nullptr;
  unsigned* counters = nullptr;  // one work counter per in-flight batch
  unsigned long long* work = nullptr;  // [2] evaluated and blended pairs of the served views
  int max_batches = 2;  // one running and one queued: views that get ready meanwhile join the next
  std::vector<Batch> batches;  // in flight
  std::vector<cudaEvent_t> free_events;
  std::vector<gs_scene*> scenes;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Ticket*> queue;
  std::unordered_map<int64_t, Ticket*> tickets;
  int64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  // statistics
  std::vector<double> lat;
  int64_t completed = 0, failed = 0, batches_launched = 0, batched_views = 0;
  size_t bytes_in_use = 0;
  std::string fatal;
};

namespace {

void* dev_alloc(gs_server* s, size_t bytes, cudaStream_t st) {
  if (bytes == 0) bytes = 16;
  if (s->al.alloc) return s->al.alloc(bytes, s->al.ctx, st);
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}
void dev_free(gs_server* s, Buf& b, cudaStream_t st) {
  if (!b.p) return;
  if (s->al.free) s->al.free(b.p, b.bytes, s->al.ctx, st);
  else cudaFreeAsync(b.p, st);
  s->bytes_in_use -= b.bytes;
  b.p = nullptr;
  b.bytes = 0;
}
// Ensure b holds `bytes`: 0 done, 1 over the budget, 2 the allocator failed.
// headroom: allocate an eighth more when it fits (buffers whose size varies
// from view to view: the instance lists); the stage-A buffers, whose sizes
// the admission reserves exactly, take none.
int ensure(gs_server* s, Buf& b, size_t bytes, cudaStream_t st, bool headroom = true) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return 0;
  size_t grow = headroom ? bytes + bytes / 8 : bytes;
  if (s->bytes_in_use - b.bytes + grow > s->budget) grow = bytes;
  if (s->bytes_in_use - b.bytes + grow > s->budget) return 1;
  dev_free(s, b, st);
  void* p = dev_alloc(s, grow, st);
  if (!p) return 2;
  b.p = p;
  b.bytes = grow;
  s->bytes_in_use += grow;
  return 0;
}

size_t stage_a_bytes_needed(int64_t n, int ntiles) {
  const size_t N = (size_t)(n > 0 ? n : 1);
  return N * (kRecF4 * sizeof(float4) + sizeof(RowGeom) + sizeof(uint2) + 9 * sizeof(uint32_t)) +
         (radix_tmp_words(n) + scan_tmp_words(n) + 4) * sizeof(uint32_t) + ntiles * sizeof(int2);
}

// Bytes a slot's stage-A buffers must grow by for a request of n surfels
// and ntiles tiles (the same sizes stage_a ensures).
size_t stage_a_growth(const Slot& sl, int64_t n, int ntiles) {
  const size_t N = (size_t)(n > 0 ? n : 1);
  const struct {
    const Buf* b;
    size_t bytes;
  } need[] = {{&sl.rec, N * kRecF4 * sizeof(float4)}, {&sl.geom, N * sizeof(RowGeom)},
              {&sl.rect, N * sizeof(uint2)}, {&sl.tcount, N * 4}, {&sl.dkey, N * 4}, {&sl.idx, N * 4},
              {&sl.dkey2, N * 4}, {&sl.idx2, N * 4}, {&sl.cnts, N * 4}, {&sl.offs, N * 4},
              {&sl.cand, N * 4}, {&sl.rtmp, (radix_tmp_words(n) + scan_tmp_words(n) + 4) * 4},
              {&sl.ranges, (size_t)ntiles * sizeof(int2)}};
  size_t g = 0;
  for (const auto& x : need) g += x.b->bytes < x.bytes ? x.bytes - x.b->bytes : 0;
  return g;
}

void release_all(gs_server* s, Slot& sl) {
  Buf* all[] = {&sl.rec, &sl.geom, &sl.rect, &sl.tcount, &sl.dkey, &sl.idx, &sl.dkey2, &sl.idx2, &sl.cnts,
                &sl.offs, &sl.cand, &sl.rtmp, &sl.keys, &sl.vals, &sl.keys2, &sl.vals2, &sl.ktmp, &sl.ranges,
                &sl.seg_tiles, &sl.seg_list, &sl.seg_trans, &sl.seg_part};
  for (Buf* b : all) dev_free(s, *b, sl.st);
}

void finish(gs_server* s, Slot& sl, gs_status err, const std::string& msg) {
  Ticket* t = sl.t;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    t->t_done = now_ms();
    if (err == GS_OK) {
      t->state = 2;
      s->completed++;
      s->lat.push_back(t->t_done - t->t_submit);
    } else {
      t->state = 3;
      t->err = err;
      t->msg = msg;
      s->failed++;
    }
  }
  s->cv_done.notify_all();
  sl.t = nullptr;
  sl.state = kIdle;
}

// Stage A: preprocess, depth sort, instance count -> pinned host.
// Returns GS_OK when launched.
gs_status stage_a(gs_server* s, Slot& sl, std::string* msg) {
  const int64_t n = sl.P.n;
  const size_t N = (size_t)(n > 0 ? n : 1);
  const int ntiles = sl.cam.tiles_x * sl.cam.tiles_y;
  cudaStream_t st = sl.st;
  struct Need {
    Buf* b;
    size_t bytes;
  } need[] = {{&sl.rec, N * kRecF4 * sizeof(float4)}, {&sl.geom, N * sizeof(RowGeom)},
              {&sl.rect, N * sizeof(uint2)}, {&sl.tcount, N * 4}, {&sl.dkey, N * 4}, {&sl.idx, N * 4},
              {&sl.dkey2, N * 4}, {&sl.idx2, N * 4}, {&sl.cnts, N * 4}, {&sl.offs, N * 4},
              {&sl.cand, N * 4}, {&sl.rtmp, (radix_tmp_words(n) + scan_tmp_words(n) + 4) * 4},
              {&sl.ranges, (size_t)ntiles * sizeof(int2)}};
  for (const Need& x : need) {
    const int r = ensure(s, *x.b, x.bytes, st, false);
    if (r == 1) {
      *msg = "device buffers for the surfels do not fit the memory budget";
      return GS_ERR_CAPACITY;
    }
    if (r == 2) {
      *msg = "the allocator failed";
      return GS_ERR_OOM;
    }
  }
  uint32_t* rtmp = (uint32_t*)sl.rtmp.p;
  uint32_t* total = rtmp + radix_tmp_words(n) + scan_tmp_words(n);
  uint32_t* ncand = total + 1;
  sl.ncand = ncand;
  cudaError_t e = launch_preprocess(sl.P, sl.cam, sl.set, (float4*)sl.rec.p, (uint2*)sl.rect.p,
                                    (uint32_t*)sl.tcount.p, (uint32_t*)sl.dkey.p, (uint32_t*)sl.idx.p,
                                    (uint32_t*)sl.cand.p, ncand, (RowGeom*)sl.geom.p, (uint32_t*)sl.cnts.p,
                                    rtmp + radix_tmp_words(n), st);
  uint32_t *skey = nullptr, *sidx = nullptr;
  if (e == cudaSuccess)
    e = radix_sort_pairs((uint32_t*)sl.dkey.p, (uint32_t*)sl.idx.p, (uint32_t*)sl.dkey2.p,
                         (uint32_t*)sl.idx2.p, n, 32, rtmp, &skey, &sidx, st, ncand, (uint32_t*)sl.tcount.p,
                         (uint32_t*)sl.cnts.p);
  if (e == cudaSuccess)
    e = launch_scan((uint32_t*)sl.cnts.p, (uint32_t*)sl.offs.p, n, total, rtmp + radix_tmp_words(n), st,
                    ncand);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sl.k_host, total, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaEventRecord(sl.ev_a, st);
  if (e != cudaSuccess) {
    *msg = std::string("stage A: ") + cudaGetErrorString(e);
    return GS_ERR_CUDA;
  }
  sl.sidx = sidx;
  return GS_OK;
}

// Stage B: instance buffers, emission, tile sort, ranges.  Returns 1 when
// launched, 0 when the buffers do not fit the budget yet, -1 on a CUDA
// error, -2 when the allocator failed.
int stage_b(gs_server* s, Slot& sl, std::string* msg) {
  const int64_t K = sl.K;
  const size_t KK = (size_t)(K > 0 ? K : 1);
  cudaStream_t st = sl.st;
  const int ntiles_v = sl.cam.tiles_x * sl.cam.tiles_y;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
  // the same choice as a lone render, so that served images equal it
  sl.lseg = split_lseg(ntiles_v, K, sms);
  const int64_t nmax = sl.lseg ? split_nseg_max(K, sl.lseg) : 0;
  sl.nseg_max = (unsigned)nmax;
  const size_t tiles_words = 2 * (size_t)ntiles_v + 1 + scan_tmp_words(ntiles_v);
  Buf* bufs[] = {&sl.keys, &sl.vals, &sl.keys2, &sl.vals2, &sl.ktmp, &sl.seg_tiles, &sl.seg_list, &sl.seg_trans,
                 &sl.seg_part};
  const size_t sizes[] = {KK * 4, KK * 4, KK * 4, KK * 4, radix_tmp_words(K) * 4,
                          sl.lseg ? tiles_words * 4 : 0, (size_t)nmax * 2 * 4, (size_t)nmax * 256 * 4,
                          (size_t)nmax * 256 * seg_part_bytes()};
  for (int i = 0; i < 9; ++i) {
    if (sizes[i] == 0) continue;
    const int r = ensure(s, *bufs[i], sizes[i], st);
    if (r == 1) return 0;
    if (r == 2) {
      *msg = "the allocator failed";
      return -2;
    }
  }
  const int ntiles = sl.cam.tiles_x * sl.cam.tiles_y;
  int bits = 0;
  while ((int64_t(1) << bits) < ntiles) ++bits;
  cudaError_t e = launch_emit(sl.sidx, (uint32_t*)sl.offs.p, (uint32_t*)sl.cnts.p, (uint2*)sl.rect.p,
                              (RowGeom*)sl.geom.p, sl.rf, sl.P.n, sl.cam.tiles_x, (uint32_t*)sl.keys.p,
                              (uint32_t*)sl.vals.p, st, sl.ncand);
  uint32_t *tk = nullptr, *tv = nullptr;
  if (e == cudaSuccess)
    e = radix_sort_pairs((uint32_t*)sl.keys.p, (uint32_t*)sl.vals.p, (uint32_t*)sl.keys2.p,
                         (uint32_t*)sl.vals2.p, K, bits, (uint32_t*)sl.ktmp.p, &tk, &tv, st);
  if (e == cudaSuccess) e = launch_ranges(tk, K, (int2*)sl.ranges.p, ntiles, st);
  if (e == cudaSuccess) e = cudaEventRecord(sl.ev_b, st);
  if (e != cudaSuccess) {
    *msg = std::string("stage B: ") + cudaGetErrorString(e);
    return -1;
  }
  sl.vals_final = tv;
  return 1;
}

cudaEvent_t get_event(gs_server* s) {
  if (!s->free_events.empty()) {
    cudaEvent_t e = s->free_events.back();
    s->free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  return e;
}

bool launch_batch(gs_server* s, const std::vector<int>& ready, std::string* msg) {
  BlendBatch b;
  memset(&b, 0, sizeof b);
  int tiles = 0, nj = 0;
  for (size_t i = 0; i < ready.size(); ++i) {
    Slot& sl = s->slots[ready[i]];
    if (cudaStreamWaitEvent(s->blend_st, sl.ev_b, 0) != cudaSuccess) {
      *msg = "cudaStreamWaitEvent failed";
      return false;
    }
    if (sl.lseg > 0) {
      // a view with few tiles and long lists: its own launches, in segments
      const int nt = sl.cam.tiles_x * sl.cam.tiles_y;
      uint32_t* tw = (uint32_t*)sl.seg_tiles.p;
      uint32_t* lw = (uint32_t*)sl.seg_list.p;
      SegBufs sb;
      sb.lseg = sl.lseg;
      sb.nseg_max = sl.nseg_max;
      sb.segcnt = tw;
      sb.segoff = tw + nt;
      sb.nseg = tw + 2 * nt;
      sb.scan_tmp = tw + 2 * nt + 1;
      sb.seg_tile = lw;
      sb.seg_idx = lw + sl.nseg_max;
      sb.trans = (float*)sl.seg_trans.p;
      sb.part = sl.seg_part.p;
      const cudaError_t es = launch_blend_fwd_split(sl.cam, sl.set, nullptr, (const float4*)sl.rec.p,
                                                    (const RowGeom*)sl.geom.p, sl.vals_final,
                                                    (const int2*)sl.ranges.p, sl.t->req.out, sl.t->req.n_contrib,
                                                    nullptr, nullptr, s->work, sb, s->blend_st);
      if (es != cudaSuccess) {
        *msg = std::string("blend: ") + cudaGetErrorString(es);
        return false;
      }
      continue;
    }
    BlendJob& j = b.job[nj++];
    j.cam = sl.cam;
    j.set = sl.set;
    j.rf = sl.rf;
    j.tile_begin = tiles;
    j.rec = (const float4*)sl.rec.p;
    j.geom = (const RowGeom*)sl.geom.p;
    j.vals = sl.vals_final;
    j.ranges = (const int2*)sl.ranges.p;
    j.out = sl.t->req.out;
    j.n_contrib = sl.t->req.n_contrib;
    tiles += sl.cam.tiles_x * sl.cam.tiles_y;
  }
  b.njobs = nj;
  b.total_tiles = tiles;
  const int bi = (int)s->batches.size();
  b.counter = s->counters + bi;
  b.work = s->work;
  cudaError_t e = nj ? cudaMemsetAsync(b.counter, 0, sizeof(unsigned), s->blend_st) : cudaSuccess;
  if (e == cudaSuccess && nj) {
    // persistent grid: four CTAs per SM (the blend's occupancy), no more
    // CTAs than tiles
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    e = launch_blend_fwd_batched(b, std::max(1, std::min(4 * sms, tiles)), s->blend_st);
  }
  Batch bt;
  bt.ev = get_event(s);
  if (e == cudaSuccess) e = cudaEventRecord(bt.ev, s->blend_st);
  if (e != cudaSuccess) {
    *msg = std::string("blend: ") + cudaGetErrorString(e);
    s->free_events.push_back(bt.ev);
    return false;
  }
  bt.slots = ready;
  s->batches.push_back(bt);
  s->batches_launched++;
  s->batched_views += (int64_t)ready.size();
  for (int i : ready) s->slots[i].state = kBlending;
  return true;
}

void worker_loop(gs_server* s) {
  cudaSetDevice(s->device);
  std::vector<Ticket*> incoming;
  while (true) {
    bool progress = false;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop) break;
    }
    // 1. finished blend batches
    for (size_t bi = 0; bi < s->batches.size();) {
      Batch& b = s->batches[bi];
      const cudaError_t q = cudaEventQuery(b.ev);
      if (q == cudaErrorNotReady) {
        ++bi;
        continue;
      }
      for (int i : b.slots) finish(s, s->slots[i], q == cudaSuccess ? GS_OK : GS_ERR_CUDA,
                                   q == cudaSuccess ? "" : cudaGetErrorString(q));
      s->free_events.push_back(b.ev);
      // keep the per-batch work counters aligned with their batch index
      s->batches.erase(s->batches.begin() + (long)bi);
      progress = true;
    }
    // 2. stage A finished -> stage B; stage B finished -> ready
    for (size_t i = 0; i < s->slots.size(); ++i) {
      Slot& sl = s->slots[i];
      if (sl.state == kStageA) {
        const cudaError_t q = cudaEventQuery(sl.ev_a);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) {
          finish(s, sl, GS_ERR_CUDA, cudaGetErrorString(q));
          progress = true;
          continue;
        }
        sl.K = *sl.k_host;
        sl.state = kWaitMem;
        progress = true;
      }
      if (sl.state == kWaitMem) {
        std::string msg;
        const int r = stage_b(s, sl, &msg);
        if (r == 1) {
          sl.state = kStageB;
          progress = true;
        } else if (r < 0) {
          finish(s, sl, r == -2 ? GS_ERR_OOM : GS_ERR_CUDA, msg);
          progress = true;
        } else {
          // release idle slots' buffers; a running slot will free memory
          // when it finishes.  When only waiting slots remain, the oldest
          // request keeps its buffers and the others go back to the head of
          // the queue (no two waiting slots can block each other); if the
          // oldest then still does not fit, it never will.
          bool running = false;
          for (size_t j = 0; j < s->slots.size(); ++j) {
            if (j == i) continue;
            const SlotState o = s->slots[j].state;
            if (o == kIdle && s->slots[j].bytes() > 0) release_all(s, s->slots[j]);
            else if (o != kIdle && o != kWaitMem) running = true;
          }
          bool oldest = true;
          for (size_t j = 0; j < s->slots.size(); ++j)
            if (j != i && s->slots[j].state == kWaitMem && s->slots[j].t->id < sl.t->id) oldest = false;
          if (!running && oldest) {
            std::vector<Ticket*> back;
            for (size_t j = 0; j < s->slots.size(); ++j) {
              Slot& o = s->slots[j];
              if (j == i || o.state != kWaitMem) continue;
              release_all(s, o);
              back.push_back(o.t);
              o.t = nullptr;
              o.state = kIdle;
            }
            if (!back.empty()) {
              std::sort(back.begin(), back.end(), [](const Ticket* a, const Ticket* b) { return a->id > b->id; });
              std::lock_guard<std::mutex> lk(s->mu);
              for (Ticket* t : back) {
                t->state = 0;
                s->queue.push_front(t);
              }
            }
            const int r2 = stage_b(s, sl, &msg);
            if (r2 == 1) sl.state = kStageB;
            else if (r2 < 0) finish(s, sl, r2 == -2 ? GS_ERR_OOM : GS_ERR_CUDA, msg);
            else finish(s, sl, GS_ERR_CAPACITY, "tile lists do not fit the memory budget");
            progress = true;
          }
        }
      }
      if (sl.state == kStageB) {
        const cudaError_t q = cudaEventQuery(sl.ev_b);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) {
          finish(s, sl, GS_ERR_CUDA, cudaGetErrorString(q));
        } else {
          sl.state = kReady;
        }
        progress = true;
      }
    }
    // 3. one persistent blend launch for every view that is ready
    if ((int)s->batches.size() < s->max_batches) {
      std::vector<int> ready;
      for (size_t i = 0; i < s->slots.size() && (int)ready.size() < kMaxBatch; ++i)
        if (s->slots[i].state == kReady) ready.push_back((int)i);
      if (!ready.empty()) {
        std::string msg;
        if (!launch_batch(s, ready, &msg))
          for (int i : ready) finish(s, s->slots[i], GS_ERR_CUDA, msg);
        progress = true;
      }
    }
    // 4. admission: queued requests into idle slots, by memory footprint
    {
      std::unique_lock<std::mutex> lk(s->mu);
      // stage-A growth of the requests admitted in this pass (their buffers
      // are allocated after the pass, so bytes_in_use does not hold them yet)
      size_t reserved = 0;
      for (size_t i = 0; i < s->slots.size() && !s->queue.empty(); ++i) {
        Slot& sl = s->slots[i];
        if (sl.state != kIdle) continue;
        Ticket* t = s->queue.front();
        gs_scene* sc = t->scene;
        const ParamsDev& P = scene_params(sc);
        const int tx = (t->req.camera.width + kTile - 1) / kTile, ty = (t->req.camera.height + kTile - 1) / kTile;
        const size_t need = stage_a_bytes_needed(P.n, tx * ty);
        size_t grow = stage_a_growth(sl, P.n, tx * ty);
        if (grow > 0 && s->bytes_in_use + reserved + grow > s->budget) {
          bool others = false;
          for (const Slot& o : s->slots) others = others || o.state != kIdle;
          if (others) break;  // wait for memory to free up (head of line keeps its place)
          // nothing in flight: drop idle buffers, then it fits or never will
          for (Slot& o : s->slots) release_all(s, o);
          if (need > s->budget) {
            s->queue.pop_front();
            t->state = 3;
            t->err = GS_ERR_CAPACITY;
            t->msg = "request does not fit the memory budget";
            t->t_done = now_ms();
            s->failed++;
            s->cv_done.notify_all();
            progress = true;
            continue;
          }
          grow = need;
        }
        reserved += grow;
        s->queue.pop_front();
        t->state = 1;
        incoming.push_back(t);
        sl.t = t;
        sl.state = kStageA;  // reserved; launched below without the lock
      }
    }
    for (Ticket* t : incoming) {
      for (Slot& sl : s->slots) {
        if (sl.t != t) continue;
        gs_scene* sc = t->scene;
        sl.P = scene_params(sc);
        const gs_settings& g = scene_settings(sc);
        sl.set.near_plane = g.near_plane;
        sl.set.alpha_min = g.alpha_min;
        sl.set.T_min = g.T_min;
        sl.set.alpha_max = g.alpha_max;
        sl.set.rho_max = g.rho_max;
        sl.set.sinv = g.screen_inv_sigma2;
        for (int c = 0; c < 3; ++c) sl.set.bg[c] = g.bg[c];
        sl.rf = (float)sqrt((double)g.rho_max / (double)g.screen_inv_sigma2);
        const gs_camera& c = t->req.camera;
        cam_from(c, sl.cam);
        std::string msg;
        const gs_status r = stage_a(s, sl, &msg);
        if (r != GS_OK) finish(s, sl, r, msg);
        progress = true;
        break;
      }
    }
    incoming.clear();
    if (!progress) {
      std::unique_lock<std::mutex> lk(s->mu);
      bool busy = !s->batches.empty();
      for (const Slot& sl : s->slots) busy = busy || sl.state != kIdle;
      if (busy)
        s->cv_work.wait_for(lk, std::chrono::microseconds(20));
      else
        s->cv_work.wait_for(lk, std::chrono::milliseconds(5), [&] { return s->stop || !s->queue.empty(); });
    }
  }
}

}  // namespace

extern "C" {

gs_status gs_server_create(gs_server** out, size_t budget_bytes, int32_t max_slots, const gs_allocator* al) {
  if (!out || max_slots < 1 || max_slots > 64 || budget_bytes == 0) {
    set_last_error("gs_server_create: bad argument");
    return GS_ERR_ARG;
  }
  *out = nullptr;
  gs_server* s = new (std::nothrow) gs_server();
  if (!s) {
    set_last_error("gs_server_create: host allocation");
    return GS_ERR_OOM;
  }
  if (al) s->al = *al;
  s->budget = budget_bytes;
  cudaError_t e = cudaGetDevice(&s->device);
  s->slots.resize((size_t)max_slots);
  for (Slot& sl : s->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev_a, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev_b, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&sl.k_host, sizeof(uint32_t));
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->blend_st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->counters, sizeof(unsigned) * 8);
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->work, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(s->work, 0, 2 * sizeof(unsigned long long));
  if (e != cudaSuccess) {
    set_last_error((std::string("gs_server_create: ") + cudaGetErrorString(e)).c_str());
    gs_server_destroy(s);
    return GS_ERR_CUDA;
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return GS_OK;
}

gs_status gs_server_add_scene(gs_server* s, gs_scene* scene, int32_t* scene_id) {
  if (!s || !scene || !scene_id) {
    set_last_error("gs_server_add_scene: null argument");
    return GS_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->scenes.push_back(scene);
  *scene_id = (int32_t)s->scenes.size() - 1;
  return GS_OK;
}

gs_status gs_server_submit(gs_server* s, const gs_request* req, int64_t* ticket) {
  if (!s || !req || !ticket || !req->out) {
    set_last_error("gs_server_submit: null argument");
    return GS_ERR_ARG;
  }
  const gs_camera& c = req->camera;
  if (c.width <= 0 || c.height <= 0 || c.width > 16 * 65535 || c.height > 16 * 65535 || !(c.fx > 0) ||
      !(c.fy > 0)) {
    set_last_error("gs_server_submit: bad camera");
    return GS_ERR_ARG;
  }
  Ticket* t = new (std::nothrow) Ticket();
  if (!t) {
    set_last_error("gs_server_submit: host allocation");
    return GS_ERR_OOM;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (req->scene < 0 || req->scene >= (int32_t)s->scenes.size()) {
      delete t;
      set_last_error("gs_server_submit: unknown scene");
      return GS_ERR_ARG;
    }
    t->id = s->next_id++;
    t->req = *req;
    t->scene = s->scenes[req->scene];
    t->t_submit = now_ms();
    s->tickets[t->id] = t;
    s->queue.push_back(t);
    *ticket = t->id;
  }
  s->cv_work.notify_one();
  return GS_OK;
}

gs_status gs_server_wait(gs_server* s, int64_t ticket, int32_t timeout_ms) {
  if (!s) {
    set_last_error("gs_server_wait: null server");
    return GS_ERR_ARG;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) {
    set_last_error("gs_server_wait: unknown ticket");
    return GS_ERR_ARG;
  }
  Ticket* t = it->second;
  const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                      [&] { return t->state >= 2; });
  if (!ok) {
    set_last_error("gs_server_wait: request still in flight");
    return GS_ERR_TIMEOUT;
  }
  const gs_status r = t->state == 2 ? GS_OK : t->err;
  if (r != GS_OK) set_last_error(("gs_server_wait: " + t->msg).c_str());
  s->tickets.erase(it);
  delete t;
  return r;
}

gs_status gs_server_stats(gs_server* s, gs_server_stats_t* out, int32_t reset) {
  if (!s || !out) {
    set_last_error("gs_server_stats: null argument");
    return GS_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  memset(out, 0, sizeof *out);
  out->completed = s->completed;
  out->failed = s->failed;
  out->queued = (int64_t)s->queue.size();
  out->in_flight = 0;
  for (const auto& kv : s->tickets) out->in_flight += kv.second->state == 1;
  out->batches = s->batches_launched;
  out->batched_views = s->batched_views;
  out->bytes_in_use = (int64_t)s->bytes_in_use;
  std::vector<double> l = s->lat;
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    auto pct = [&](double q) {
      const double pos = q * (double)(l.size() - 1);
      const size_t i = (size_t)pos;
      const double f = pos - (double)i;
      return i + 1 < l.size() ? l[i] * (1.0 - f) + l[i + 1] * f : l[i];
    };
    out->latency_p50_ms = pct(0.50);
    out->latency_p99_ms = pct(0.99);
    double m = 0;
    for (double x : l) m += x;
    out->latency_mean_ms = m / (double)l.size();
  }
  // blend work of the served views (a snapshot: the counters are device words)
  unsigned long long w[2] = {0ull, 0ull};
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  if (cudaMemcpy(w, s->work, sizeof w, cudaMemcpyDeviceToHost) == cudaSuccess) {
    out->pairs_evaluated = (int64_t)w[0];
    out->pairs_blended = (int64_t)w[1];
  }
  if (reset) {
    s->lat.clear();
    s->completed = s->failed = s->batches_launched = s->batched_views = 0;
    cudaMemset(s->work, 0, sizeof w);
  }
  cudaSetDevice(prev);
  return GS_OK;
}

gs_status gs_server_destroy(gs_server* s) {
  if (!s) return GS_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (Slot& sl : s->slots) {
    if (sl.st) cudaStreamSynchronize(sl.st);
    release_all(s, sl);
    if (sl.st) cudaStreamSynchronize(sl.st);
    if (sl.ev_a) cudaEventDestroy(sl.ev_a);
    if (sl.ev_b) cudaEventDestroy(sl.ev_b);
    if (sl.st) cudaStreamDestroy(sl.st);
    if (sl.k_host) cudaFreeHost(sl.k_host);
  }
  if (s->blend_st) {
    cudaStreamSynchronize(s->blend_st);
    cudaStreamDestroy(s->blend_st);
  }
  for (Batch& b : s->batches) cudaEventDestroy(b.ev);
  for (cudaEvent_t e : s->free_events) cudaEventDestroy(e);
  if (s->counters) cudaFree(s->counters);
  if (s->work) cudaFree(s->work);
  for (auto& kv : s->tickets) delete kv.second;
  delete s;
  return GS_OK;
}

}  // extern "C"
