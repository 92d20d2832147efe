// Tile binning and ordering: device-wide scan, key emission, stable LSD
// radix sort of (key, value) pairs and per-tile ranges.
//
// The compositing order (Eq. 1 composites front to back) is (tile, centre
// depth, surfel index).  It is produced in two levels with the same result
// as one sort of 64-bit (tile << 32 | depth bits) keys: the surfels are
// sorted once by depth (32-bit keys, stable, so ties keep index order), the
// (tile, surfel) instances are emitted in that order, and a stable sort by
// tile id alone (13-16 bits) groups them per tile.
#include "gs2d_internal.cuh"

namespace gs2d {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;  // per thread in one-block scans
constexpr int kWarps = kThreads / 32;
constexpr int kRadixBits = 8;
constexpr int kBins = 1 << kRadixBits;

// Items per thread of the scans and radix passes, by the grid's item bound:
// a small block (1024 items, up to 4M items) spreads a few hundred thousand
// items over all SMs and keeps each block's serial ranking short; larger
// inputs take 2048 (up to 16M) and 4096 items per block, to keep the
// per-block digit counts (and the offsets scan over them) small.
inline int items_per_thread(int64_t n) { return n <= (int64_t(1) << 22) ? 4 : (n <= (int64_t(1) << 24) ? 8 : 16); }
inline int64_t blocks_for(int64_t n) {
  const int64_t ti = (int64_t)kThreads * items_per_thread(n);
  return (n > 0 ? n + ti - 1 : ti) / ti;
}

// Item count: a host bound, lowered to a device-side count when one is given
// (the grid is sized for the bound; blocks past the count do nothing).
__device__ __forceinline__ int64_t item_count(int64_t n_max, const uint32_t* n_dev) {
  if (!n_dev) return n_max;
  const int64_t d = (int64_t)*n_dev;
  return d < n_max ? d : n_max;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive block scan of one value per thread (256 threads).  Returns the
// exclusive prefix; *total receives the block sum.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t ws[kWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t inc = warp_incl_scan(v);
  if (lane == 31) ws[w] = inc;
  __syncthreads();
  if (w == 0) {
    const uint32_t x = lane < kWarps ? ws[lane] : 0u;
    const uint32_t xi = warp_incl_scan(x);
    if (lane < kWarps) ws[lane] = xi - x;
    if (lane == kWarps - 1) *total = xi;
  }
  __syncthreads();
  const uint32_t r = ws[w] + inc - v;
  __syncthreads();
  return r;
}

// Last-block election: every block calls this once, after its thread 0 has
// written the block's result to global memory.  Returns true in the block
// that arrives last, to which all blocks' results are then visible (it reads
// them through L2).  atomicInc wraps the counter back to zero, so it is ready
// for the next launch.
__device__ __forceinline__ bool last_block(uint32_t* done) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();  // this block's result before its arrival
    last = atomicInc(done, gridDim.x - 1u) == gridDim.x - 1u;
    if (last) __threadfence();
  }
  __syncthreads();
  return last;
}

// Sum of one value per thread over the block (256 threads), in thread 0.
__device__ __forceinline__ uint32_t block_sum(uint32_t v) {
  __shared__ uint32_t ws[kWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) ws[w] = v;
  __syncthreads();
  uint32_t t = 0;
  if (threadIdx.x == 0)
#pragma unroll
    for (int i = 0; i < kWarps; ++i) t += ws[i];
  return t;
}

// One block: exclusive scan of nb values in place; their sum to *total.
__device__ void block_scan_inplace(uint32_t* __restrict__ v, int nb, uint32_t* __restrict__ total) {
  __shared__ uint32_t tot;
  uint32_t carry = 0;
  for (int base = 0; base < nb; base += kThreads * kItems) {
    // each thread owns kItems consecutive entries of this chunk
    uint32_t x[kItems];
    uint32_t s = 0;
    const int t0 = base + threadIdx.x * kItems;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      x[i] = (t0 + i < nb) ? __ldcg(v + t0 + i) : 0u;
      s += x[i];
    }
    uint32_t pre = block_excl_scan(s, &tot) + carry;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      if (t0 + i < nb) v[t0 + i] = pre;
      pre += x[i];
    }
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

// Block sums of the input; the last block scans them (exclusive, in place)
// and writes the grand total.
template <int kIt>
__global__ void __launch_bounds__(kThreads) scan_reduce(const uint32_t* __restrict__ in, int64_t n_max,
                                                        const uint32_t* __restrict__ n_dev,
                                                        uint32_t* __restrict__ sums,
                                                        uint32_t* __restrict__ total,
                                                        uint32_t* __restrict__ done) {
  const int64_t n = item_count(n_max, n_dev);
  const int64_t base = (int64_t)blockIdx.x * (kThreads * kIt);
  uint32_t x[kIt];
#pragma unroll
  for (int i = 0; i < kIt; ++i) {
    const int64_t k = base + i * kThreads + threadIdx.x;
    x[i] = k < n ? in[k] : 0u;
  }
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kIt; ++i) s += x[i];
  s = block_sum(s);
  if (threadIdx.x == 0) sums[blockIdx.x] = s;
  if (!last_block(done)) return;
  block_scan_inplace(sums, (int)gridDim.x, total);
}

template <int kIt>
__global__ void __launch_bounds__(kThreads) scan_down(const uint32_t* __restrict__ in,
                                                      uint32_t* __restrict__ out, int64_t n_max,
                                                      const uint32_t* __restrict__ n_dev,
                                                      const uint32_t* __restrict__ sums) {
  constexpr int kTI = kThreads * kIt;
  __shared__ uint32_t tile[kTI];
  const int64_t n = item_count(n_max, n_dev);
  const int64_t base = (int64_t)blockIdx.x * kTI;
  if (base >= n) return;
  // coalesced load into shared memory, then each thread scans kIt
  // consecutive entries
  uint32_t x[kIt];
#pragma unroll
  for (int i = 0; i < kIt; ++i) {
    const int64_t k = base + i * kThreads + threadIdx.x;
    x[i] = k < n ? in[k] : 0u;
  }
#pragma unroll
  for (int i = 0; i < kIt; ++i) tile[i * kThreads + threadIdx.x] = x[i];
  __syncthreads();
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kIt; ++i) {
    x[i] = tile[threadIdx.x * kIt + i];
    s += x[i];
  }
  __shared__ uint32_t tot;
  uint32_t pre = block_excl_scan(s, &tot) + sums[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kIt; ++i) {
    tile[threadIdx.x * kIt + i] = pre;
    pre += x[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kIt; ++i) {
    const int64_t k = base + i * kThreads + threadIdx.x;
    if (k < n) out[k] = tile[i * kThreads + threadIdx.x];
  }
}

// ---- radix sort -----------------------------------------------------------
//
// Per pass: every block counts the digits of its kThreads * kIt keys
// (upsweep); one block per digit scans that digit's counts over the blocks
// (offsets; the counts are stored digit-major, so the scan reads them in
// order); every block then ranks its keys stably (per warp, from ballots of the
// lanes' digit bits; the warps of the block in order) and scatters them
// (downsweep).  Only the blocks that hold items (from the device-side count)
// take part.

// Lanes of the warp whose 9-bit digit equals this lane's: the AND over the
// digit's bits of each bit's ballot (or its complement).
__device__ __forceinline__ uint32_t digit_peers(uint32_t d) {
  uint32_t peers = 0xffffffffu;
#pragma unroll
  for (int b = 0; b < 9; ++b) {
    const uint32_t bl = __ballot_sync(0xffffffffu, (d >> b) & 1u);
    peers &= ((d >> b) & 1u) ? bl : ~bl;
  }
  return peers;
}

template <int kIt>
__global__ void __launch_bounds__(kThreads) radix_upsweep(const uint32_t* __restrict__ keys,
                                                          int64_t n_max, const uint32_t* __restrict__ n_dev,
                                                          int shift, int nbins,
                                                          uint32_t* __restrict__ hist) {
  const int64_t n = item_count(n_max, n_dev);
  if ((int64_t)blockIdx.x * (kThreads * kIt) >= n) return;
  __shared__ uint32_t h[kBins];
  for (int i = threadIdx.x; i < kBins; i += kThreads) h[i] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * (kThreads * kIt) + w * (32 * kIt);
  const uint32_t mask = (uint32_t)nbins - 1u;
  uint32_t kk[kIt];
#pragma unroll
  for (int it = 0; it < kIt; ++it) {
    const int64_t k = base + it * 32 + lane;
    kk[it] = k < n ? keys[k] : 0u;
  }
#pragma unroll
  for (int it = 0; it < kIt; ++it) {
    const int64_t k = base + it * 32 + lane;
    const bool valid = k < n;
    if (valid) atomicAdd(&h[(kk[it] >> shift) & mask], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < nbins; d += kThreads) hist[(int64_t)d * gridDim.x + blockIdx.x] = h[d];
}

// Per digit d (one block each): exclusive prefix of the digit's counts over
// the nb_active blocks that hold items, in place, and the digit's total.
__global__ void __launch_bounds__(kThreads) radix_offsets(uint32_t* __restrict__ hist, int nb, int ti,
                                                          int64_t n_max, const uint32_t* __restrict__ n_dev,
                                                          uint32_t* __restrict__ dtot) {
  const int64_t n = item_count(n_max, n_dev);
  const int act = (int)((n + ti - 1) / ti);
  block_scan_inplace(hist + (int64_t)blockIdx.x * nb, act < nb ? act : nb, dtot + blockIdx.x);
}

// gsrc/gout (optional, last pass): gout[dst] = gsrc[value] for every moved
// pair, a gather through the sorted values fused into the scatter.
template <int kIt>
__global__ void __launch_bounds__(kThreads) radix_downsweep(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, int64_t n_max, const uint32_t* __restrict__ n_dev, int shift, int nbins,
    const uint32_t* __restrict__ offs, const uint32_t* __restrict__ dtot,
    const uint32_t* __restrict__ gsrc, uint32_t* __restrict__ gout) {
  const int64_t n = item_count(n_max, n_dev);
  if ((int64_t)blockIdx.x * (kThreads * kIt) >= n) return;
  __shared__ uint32_t wh[kWarps][kBins];
  __shared__ uint32_t dbase[kBins];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * (kThreads * kIt) + w * (32 * kIt);
  uint32_t kk[kIt], vv[kIt], pos[kIt];
#pragma unroll
  for (int it = 0; it < kIt; ++it) {
    const int64_t k = base + it * 32 + lane;
    kk[it] = k < n ? kin[k] : 0u;
    vv[it] = k < n ? vin[k] : 0u;
  }
  {
    __shared__ uint32_t tot;
    const uint32_t x = threadIdx.x < nbins ? dtot[threadIdx.x] : 0u;
    dbase[threadIdx.x] = block_excl_scan(x, &tot);
  }
  for (int i = threadIdx.x; i < kWarps * kBins; i += kThreads) (&wh[0][0])[i] = 0u;
  __syncthreads();
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t mask = (uint32_t)nbins - 1u;
#pragma unroll
  for (int it = 0; it < kIt; ++it) {
    const int64_t k = base + it * 32 + lane;
    const bool valid = k < n;
    const uint32_t d = valid ? ((kk[it] >> shift) & mask) : 0x100u;
    const uint32_t peers = digit_peers(d);
    uint32_t cur = 0u;
    if (valid) cur = wh[w][d];
    __syncwarp();
    if (valid && lane == (31 - __clz(peers))) wh[w][d] = cur + (uint32_t)__popc(peers);
    __syncwarp();
    pos[it] = valid ? cur + (uint32_t)__popc(peers & lt) : 0xFFFFFFFFu;
  }
  __syncthreads();
  for (int d = threadIdx.x; d < nbins; d += kThreads) {
    uint32_t run = dbase[d] + offs[(int64_t)d * gridDim.x + blockIdx.x];
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) {
      const uint32_t t = wh[ww][d];
      wh[ww][d] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kIt; ++it) {
    if (pos[it] == 0xFFFFFFFFu) continue;
    const uint32_t d = (kk[it] >> shift) & mask;
    const uint32_t dst = wh[w][d] + pos[it];
    kout[dst] = kk[it];
    vout[dst] = vv[it];
    if (gout) gout[dst] = gsrc[vv[it]];
  }
}

__global__ void gather_counts_kernel(const uint32_t* __restrict__ order,
                                     const uint32_t* __restrict__ tcount, uint32_t* __restrict__ out,
                                     int64_t n_max, const uint32_t* __restrict__ n_dev) {
  const int64_t n = item_count(n_max, n_dev);
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) out[r] = tcount[order[r]];
}

// Instances of surfel order[r] at offsets offs[r]..: for every tile row of
// its rectangle, the tile columns its footprint reaches (the same row rule,
// on the same stored doubles, that counted them in the preprocess), row by
// row, left to right.  A warp takes 32 consecutive candidates and spreads
// their tile rows over its lanes (a long footprint's rows go to several
// lanes instead of keeping one lane busy while the others wait); each row's
// place within its surfel's run comes from a segmented prefix sum of the
// rows' tile counts.
__device__ __forceinline__ void emit_warp(int64_t r, int64_t n, int lane, const uint32_t* __restrict__ order,
                                          const uint32_t* __restrict__ offs, const uint32_t* __restrict__ counts,
                                          const uint2* __restrict__ rect, const RowGeom* __restrict__ geom,
                                          float rf, int tiles_x, uint32_t* __restrict__ keys,
                                          uint32_t* __restrict__ vals) {
  constexpr unsigned kFull = 0xffffffffu;
  const bool valid = r < n && counts[r] > 0u;
  uint32_t s = 0u, base = 0u;
  int ty0 = 0, nrows = 0;
  if (valid) {
    s = order[r];
    const uint2 rc = rect[s];
    ty0 = (int)(rc.x >> 16);
    nrows = (int)(rc.y >> 16) - ty0;
    base = offs[r];
  }
  // exclusive prefix of the row counts over the warp: lane i's rows are
  // flattened rows [first, first + nrows)
  int incl = nrows;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += t;
  }
  const int first = incl - nrows;
  const int total = __shfl_sync(kFull, incl, 31);
  uint32_t done = 0u;  // tiles written so far for lane's own surfel
  for (int c0 = 0; c0 < total; c0 += 32) {
    const int j = c0 + lane;
    // the row's owner: the last lane whose first row is <= j (lanes with no
    // rows share the next lane's first row and are passed over)
    int own = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const int cand = own + step;
      const int fc = __shfl_sync(kFull, first, cand & 31);
      if (cand < 32 && fc <= j) own = cand;
    }
    const bool live = j < total;
    const uint32_t so = __shfl_sync(kFull, s, own);
    const int tyo = __shfl_sync(kFull, ty0, own) + (j - __shfl_sync(kFull, first, own));
    const uint32_t bo = __shfl_sync(kFull, base, own);
    const uint32_t prev = __shfl_sync(kFull, done, own);
    int a = 0, b = 0;
    if (live) {
      const RowGeom g = geom[so];
      if (!row_tiles(g, tyo, rf, &a, &b)) a = b = 0;
    }
    const int t = b - a;
    // tiles of the owner's earlier rows in this chunk: segmented exclusive scan
    int sc = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int x = __shfl_up_sync(kFull, sc, o);
      if (lane >= o) sc += x;
    }
    const int sx = sc - t;  // exclusive
    const int seg0 = max(__shfl_sync(kFull, first, own) - c0, 0);  // owner's first lane in this chunk
    const int within = sx - __shfl_sync(kFull, sx, seg0);
    uint32_t o = bo + prev + (uint32_t)within;
    for (int tx = a; tx < b; ++tx, ++o) {
      keys[o] = (uint32_t)(tyo * tiles_x + tx);
      vals[o] = so;
    }
    // each surfel's tiles in this chunk, added to its running count
    const int l0 = max(first - c0, 0), l1 = min(first + nrows - c0, 32) - 1;
    const int sum = __shfl_sync(kFull, sc, max(l1, 0)) - __shfl_sync(kFull, sx, min(l0, 31));
    if (nrows > 0 && l0 <= l1) done += (uint32_t)sum;
  }
}

__global__ void __launch_bounds__(256) emit_kernel(const uint32_t* __restrict__ order,
                                                   const uint32_t* __restrict__ offs,
                                                   const uint32_t* __restrict__ counts,
                                                   const uint2* __restrict__ rect,
                                                   const RowGeom* __restrict__ geom, float rf, int64_t n_max,
                                                   const uint32_t* __restrict__ n_dev, int tiles_x,
                                                   uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t n = item_count(n_max, n_dev);
  const int lane = threadIdx.x & 31;
  // grid-stride over warps of 32 candidates (the grid is sized for the
  // resident CTAs, the count is known on the device only)
  for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); r0 < n;
       r0 += (int64_t)gridDim.x * blockDim.x)
    emit_warp(r0 + lane, n, lane, order, offs, counts, rect, geom, rf, tiles_x, keys, vals);
}

__global__ void ranges_kernel(const uint32_t* __restrict__ keys, int64_t K, int2* __restrict__ ranges) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= K) return;
  const uint32_t t = keys[i];
  if (i == 0 || keys[i - 1] != t) ranges[t].x = (int)i;
  if (i == K - 1 || keys[i + 1] != t) ranges[t].y = (int)(i + 1);
}

// Tiles ordered by list length, longest first (by octave of the length;
// order within an octave is arbitrary): launching the blends in this order
// starts the longest tiles first, so the last wave is short ones.  Results
// do not depend on the order.  One block; the octaves are staged in shared
// memory (up to kMaxOrderTiles tiles).
constexpr int kMaxOrderTiles = 40960;
__global__ void __launch_bounds__(1024) tile_order_kernel(const int2* __restrict__ ranges, int ntiles,
                                                          uint32_t* __restrict__ order) {
  __shared__ uint8_t oct[kMaxOrderTiles];
  __shared__ uint32_t cnt[32], cur[32];
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 32) cnt[threadIdx.x] = 0u;
  __syncthreads();
  // per warp and octave one shared-memory atomic (lanes of the same octave
  // are counted together): a few octaves hold most tiles
  for (int t0 = threadIdx.x - lane; t0 < ntiles; t0 += blockDim.x) {
    const int t = t0 + lane;
    const bool valid = t < ntiles;
    uint32_t o = 32u;
    if (valid) {
      const int2 r = ranges[t];
      o = (uint32_t)__clz((uint32_t)(r.y - r.x) | 1u);  // 31 - octave: longest first
      oct[t] = (uint8_t)o;
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, o);
    if (valid && lane == 31 - __clz(peers)) atomicAdd(&cnt[o], (uint32_t)__popc(peers));
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // exclusive scan of the 32 bucket counts in one warp
    const uint32_t c = cnt[threadIdx.x];
    uint32_t v = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, v, d);
      if ((int)threadIdx.x >= d) v += u;
    }
    cur[threadIdx.x] = v - c;
  }
  __syncthreads();
  for (int t0 = threadIdx.x - lane; t0 < ntiles; t0 += blockDim.x) {
    const int t = t0 + lane;
    const bool valid = t < ntiles;
    const uint32_t o = valid ? (uint32_t)oct[t] : 32u;
    const uint32_t peers = __match_any_sync(0xffffffffu, o);
    const int leader = 31 - __clz(peers);
    uint32_t base = 0u;
    if (valid && lane == leader) base = atomicAdd(&cur[o], (uint32_t)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (valid) order[base + (uint32_t)__popc(peers & ((1u << lane) - 1u))] = (uint32_t)t;
  }
}

}  // namespace

// block sums, then the last-block counter
size_t scan_tmp_words(int64_t n) { return (size_t)blocks_for(n) + 2; }

cudaError_t launch_scan(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_dev,
                        uint32_t* tmp, cudaStream_t st, const uint32_t* n_dev) {
  if (n <= 0) {
    return total_dev ? cudaMemsetAsync(total_dev, 0, sizeof(uint32_t), st) : cudaSuccess;
  }
  const unsigned nb = (unsigned)blocks_for(n);
  uint32_t* done = tmp + nb + 1;
  ProfScope ps(kProfSort, st);
  cudaError_t e = cudaMemsetAsync(done, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  count_launch(2);
  switch (items_per_thread(n)) {
    case 4:
      scan_reduce<4><<<nb, kThreads, 0, st>>>(in, n, n_dev, tmp, total_dev, done);
      scan_down<4><<<nb, kThreads, 0, st>>>(in, out, n, n_dev, tmp);
      break;
    case 8:
      scan_reduce<8><<<nb, kThreads, 0, st>>>(in, n, n_dev, tmp, total_dev, done);
      scan_down<8><<<nb, kThreads, 0, st>>>(in, out, n, n_dev, tmp);
      break;
    default:
      scan_reduce<16><<<nb, kThreads, 0, st>>>(in, n, n_dev, tmp, total_dev, done);
      scan_down<16><<<nb, kThreads, 0, st>>>(in, out, n, n_dev, tmp);
      break;
  }
  return cudaGetLastError();
}

// digit-major counts (kBins rows of one word per block), then the digit totals
size_t radix_tmp_words(int64_t n) { return (size_t)blocks_for(n) * kBins + kBins; }

namespace {
template <int kIt>
void radix_pass(const uint32_t* ki, const uint32_t* vi, uint32_t* ko, uint32_t* vo, int64_t n,
                const uint32_t* n_dev, int shift, int nbins, unsigned nb, uint32_t* hist, uint32_t* dtot,
                const uint32_t* gsrc, uint32_t* gout, cudaStream_t st) {
  radix_upsweep<kIt><<<nb, kThreads, 0, st>>>(ki, n, n_dev, shift, nbins, hist);
  radix_offsets<<<nbins, kThreads, 0, st>>>(hist, (int)nb, kThreads * kIt, n, n_dev, dtot);
  radix_downsweep<kIt><<<nb, kThreads, 0, st>>>(ki, vi, ko, vo, n, n_dev, shift, nbins, hist, dtot, gsrc, gout);
}
}  // namespace

cudaError_t radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                             uint32_t* vals_alt, int64_t n, int bits, uint32_t* tmp,
                             uint32_t** keys_out, uint32_t** vals_out, cudaStream_t st,
                             const uint32_t* n_dev, const uint32_t* gsrc, uint32_t* gout) {
  *keys_out = keys;
  *vals_out = vals;
  if (n <= 1 || bits <= 0) {
    // no pass to fuse the gather into
    return gout ? launch_gather_counts(vals, gsrc, gout, n, st, n_dev) : cudaSuccess;
  }
  ProfScope ps(kProfSort, st);
  const unsigned nb = (unsigned)blocks_for(n);
  const int it = items_per_thread(n);
  uint32_t* hist = tmp;
  uint32_t* dtot = tmp + (size_t)nb * kBins;
  uint32_t *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
  for (int shift = 0; shift < bits; shift += kRadixBits) {
    const int pb = bits - shift < kRadixBits ? bits - shift : kRadixBits;
    const int nbins = 1 << pb;
    const bool last = shift + kRadixBits >= bits;
    const uint32_t* gs = last ? gsrc : nullptr;
    uint32_t* go = last ? gout : nullptr;
    count_launch(3);
    if (it == 4) radix_pass<4>(ki, vi, ko, vo, n, n_dev, shift, nbins, nb, hist, dtot, gs, go, st);
    else if (it == 8) radix_pass<8>(ki, vi, ko, vo, n, n_dev, shift, nbins, nb, hist, dtot, gs, go, st);
    else radix_pass<16>(ki, vi, ko, vo, n, n_dev, shift, nbins, nb, hist, dtot, gs, go, st);
    uint32_t* t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
  }
  *keys_out = ki;
  *vals_out = vi;
  return cudaGetLastError();
}

cudaError_t launch_gather_counts(const uint32_t* order, const uint32_t* tcount, uint32_t* out,
                                 int64_t n, cudaStream_t st, const uint32_t* n_dev) {
  if (n <= 0) return cudaSuccess;
  ProfScope ps(kProfSort, st);
  count_launch();
  gather_counts_kernel<<<div_up(n, 256), 256, 0, st>>>(order, tcount, out, n, n_dev);
  return cudaGetLastError();
}

cudaError_t launch_emit(const uint32_t* order, const uint32_t* offs, const uint32_t* counts,
                        const uint2* rect, const RowGeom* geom, float rf, int64_t n, int tiles_x,
                        uint32_t* keys, uint32_t* vals, cudaStream_t st, const uint32_t* n_dev) {
  if (n <= 0) return cudaSuccess;
  ProfScope ps(kProfSort, st);
  count_launch();
  // at most eight CTAs per SM (the count of candidates is on the device; the
  // bound n is usually several times larger)
  static const unsigned resident = [] {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return 8u * (unsigned)sms;
  }();
  const unsigned blocks = div_up(n, 256) < resident ? div_up(n, 256) : resident;
  emit_kernel<<<blocks, 256, 0, st>>>(order, offs, counts, rect, geom, rf, n, n_dev, tiles_x, keys, vals);
  return cudaGetLastError();
}

cudaError_t launch_ranges(const uint32_t* keys, int64_t K, int2* ranges, int ntiles,
                          cudaStream_t st) {
  ProfScope ps(kProfSort, st);
  cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(int2) * (size_t)ntiles, st);
  if (e != cudaSuccess || K <= 0) return e;
  count_launch();
  ranges_kernel<<<div_up(K, 256), 256, 0, st>>>(keys, K, ranges);
  return cudaGetLastError();
}

bool tile_order_supported(int ntiles) { return ntiles > 0 && ntiles <= kMaxOrderTiles; }

cudaError_t launch_tile_order(const int2* ranges, int ntiles, uint32_t* order, cudaStream_t st) {
  if (!tile_order_supported(ntiles)) return cudaSuccess;
  ProfScope ps(kProfSort, st);
  count_launch();
  tile_order_kernel<<<1, 1024, 0, st>>>(ranges, ntiles, order);
  return cudaGetLastError();
}

}  // namespace gs2d
