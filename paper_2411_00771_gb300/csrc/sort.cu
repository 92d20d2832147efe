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
constexpr int kItems = 16;
constexpr int kTileItems = kThreads * kItems;  // 4096 items per block
constexpr int kWarps = kThreads / 32;
constexpr int kRadixBits = 8;
constexpr int kBins = 1 << kRadixBits;

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

// Last-block election: every block calls this once, after its writes to
// global memory.  Returns true in the block that arrives last, to which all
// blocks' writes are then visible (it reads them through L2).  atomicInc
// wraps the counter back to zero, so it is ready for the next launch.
__device__ __forceinline__ bool last_block(uint32_t* done) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicInc(done, gridDim.x - 1u) == gridDim.x - 1u;
  __syncthreads();
  if (last) __threadfence();
  return last;
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
__global__ void __launch_bounds__(kThreads) scan_reduce(const uint32_t* __restrict__ in, int64_t n_max,
                                                        const uint32_t* __restrict__ n_dev,
                                                        uint32_t* __restrict__ sums,
                                                        uint32_t* __restrict__ total,
                                                        uint32_t* __restrict__ done) {
  const int64_t n = item_count(n_max, n_dev);
  const int64_t base = (int64_t)blockIdx.x * kTileItems;
  uint32_t s = 0;
  for (int i = threadIdx.x; i < kTileItems; i += kThreads) {
    const int64_t k = base + i;
    if (k < n) s += in[k];
  }
  __shared__ uint32_t tot;
  block_excl_scan(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
  if (!last_block(done)) return;
  block_scan_inplace(sums, (int)gridDim.x, total);
}

__global__ void __launch_bounds__(kThreads) scan_down(const uint32_t* __restrict__ in,
                                                      uint32_t* __restrict__ out, int64_t n_max,
                                                      const uint32_t* __restrict__ n_dev,
                                                      const uint32_t* __restrict__ sums) {
  __shared__ uint32_t tile[kTileItems];
  const int64_t n = item_count(n_max, n_dev);
  const int64_t base = (int64_t)blockIdx.x * kTileItems;
  // coalesced load into shared memory, then each thread scans kItems
  // consecutive entries
  for (int i = threadIdx.x; i < kTileItems; i += kThreads) {
    const int64_t k = base + i;
    tile[i] = k < n ? in[k] : 0u;
  }
  __syncthreads();
  uint32_t v[kItems];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    v[i] = tile[threadIdx.x * kItems + i];
    s += v[i];
  }
  __shared__ uint32_t tot;
  uint32_t pre = block_excl_scan(s, &tot) + sums[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    tile[threadIdx.x * kItems + i] = pre;
    pre += v[i];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kTileItems; i += kThreads) {
    const int64_t k = base + i;
    if (k < n) out[k] = tile[i];
  }
}

// ---- radix sort -----------------------------------------------------------

__global__ void __launch_bounds__(kThreads) radix_upsweep(const uint32_t* __restrict__ keys,
                                                          int64_t n_max, const uint32_t* __restrict__ n_dev,
                                                          int shift, int nbins,
                                                          uint32_t* __restrict__ hist) {
  const int64_t n = item_count(n_max, n_dev);
  __shared__ uint32_t h[kBins];
  for (int i = threadIdx.x; i < kBins; i += kThreads) h[i] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * kTileItems + w * (32 * kItems);
  const uint32_t mask = (uint32_t)nbins - 1u;
  uint32_t kk[kItems];
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const int64_t k = base + it * 32 + lane;
    kk[it] = k < n ? keys[k] : 0u;
  }
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const int64_t k = base + it * 32 + lane;
    const bool valid = k < n;
    const uint32_t d = valid ? ((kk[it] >> shift) & mask) : 0x100u;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    if (valid && lane == (31 - __clz(peers))) atomicAdd(&h[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  for (int d = threadIdx.x; d < nbins; d += kThreads) hist[(int64_t)blockIdx.x * kBins + d] = h[d];
}

// Per digit d (one block each): exclusive prefix of the digit's per-block
// counts over the blocks, in place, and the digit's total.
__global__ void __launch_bounds__(kThreads) radix_offsets(uint32_t* __restrict__ hist, int nb,
                                                          uint32_t* __restrict__ dtot) {
  const int d = blockIdx.x;
  const int per = (nb + kThreads - 1) / kThreads;
  const int b0 = threadIdx.x * per;
  uint32_t s = 0;
  for (int i = 0; i < per; ++i)
    if (b0 + i < nb) s += hist[(int64_t)(b0 + i) * kBins + d];
  __shared__ uint32_t tot;
  uint32_t run = block_excl_scan(s, &tot);
  for (int i = 0; i < per; ++i) {
    if (b0 + i < nb) {
      uint32_t* h = hist + (int64_t)(b0 + i) * kBins + d;
      const uint32_t x = *h;
      *h = run;
      run += x;
    }
  }
  if (threadIdx.x == 0) dtot[d] = tot;
}

__global__ void __launch_bounds__(kThreads) radix_downsweep(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, int64_t n_max, const uint32_t* __restrict__ n_dev, int shift, int nbins,
    const uint32_t* __restrict__ offs, const uint32_t* __restrict__ dtot) {
  const int64_t n = item_count(n_max, n_dev);
  __shared__ uint32_t wh[kWarps][kBins];
  __shared__ uint32_t dbase[kBins];
  {
    __shared__ uint32_t tot;
    const uint32_t x = threadIdx.x < nbins ? dtot[threadIdx.x] : 0u;
    dbase[threadIdx.x] = block_excl_scan(x, &tot);
  }
  for (int i = threadIdx.x; i < kWarps * kBins; i += kThreads) (&wh[0][0])[i] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const int64_t base = (int64_t)blockIdx.x * kTileItems + w * (32 * kItems);
  const uint32_t mask = (uint32_t)nbins - 1u;
  uint32_t kk[kItems], vv[kItems], pos[kItems];
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const int64_t k = base + it * 32 + lane;
    const bool valid = k < n;
    kk[it] = valid ? kin[k] : 0u;
    vv[it] = valid ? vin[k] : 0u;
    const uint32_t d = valid ? ((kk[it] >> shift) & mask) : 0x100u;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t cur = 0u;
    if (valid) cur = wh[w][d];
    __syncwarp();
    if (valid && lane == (31 - __clz(peers))) wh[w][d] = cur + (uint32_t)__popc(peers);
    __syncwarp();
    pos[it] = valid ? cur + (uint32_t)__popc(peers & lt) : 0xFFFFFFFFu;
  }
  __syncthreads();
  for (int d = threadIdx.x; d < nbins; d += kThreads) {
    uint32_t run = dbase[d] + offs[(int64_t)blockIdx.x * kBins + d];
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) {
      const uint32_t t = wh[ww][d];
      wh[ww][d] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    if (pos[it] == 0xFFFFFFFFu) continue;
    const uint32_t d = (kk[it] >> shift) & mask;
    const uint32_t dst = wh[w][d] + pos[it];
    kout[dst] = kk[it];
    vout[dst] = vv[it];
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
__global__ void __launch_bounds__(256) emit_kernel(const uint32_t* __restrict__ order,
                                                   const uint32_t* __restrict__ offs,
                                                   const uint32_t* __restrict__ counts,
                                                   const uint2* __restrict__ rect,
                                                   const RowGeom* __restrict__ geom, float rf, int64_t n_max,
                                                   const uint32_t* __restrict__ n_dev, int tiles_x,
                                                   uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  constexpr unsigned kFull = 0xffffffffu;
  const int64_t n = item_count(n_max, n_dev);
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
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
  if (threadIdx.x < 32) cnt[threadIdx.x] = 0u;
  __syncthreads();
#pragma unroll 8
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
    const int2 r = ranges[t];
    const int o = __clz((uint32_t)(r.y - r.x) | 1u);  // 31 - octave: longest first
    oct[t] = (uint8_t)o;
    atomicAdd(&cnt[o], 1u);
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
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) order[atomicAdd(&cur[oct[t]], 1u)] = (uint32_t)t;
}

}  // namespace

// block sums, then the last-block counter
size_t scan_tmp_words(int64_t n) { return (size_t)div_up(n > 0 ? n : 1, kTileItems) + 2; }

cudaError_t launch_scan(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_dev,
                        uint32_t* tmp, cudaStream_t st, const uint32_t* n_dev) {
  if (n <= 0) {
    return total_dev ? cudaMemsetAsync(total_dev, 0, sizeof(uint32_t), st) : cudaSuccess;
  }
  const unsigned nb = div_up(n, kTileItems);
  uint32_t* done = tmp + nb + 1;
  ProfScope ps(kProfSort, st);
  cudaError_t e = cudaMemsetAsync(done, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  count_launch(2);
  scan_reduce<<<nb, kThreads, 0, st>>>(in, n, n_dev, tmp, total_dev, done);
  scan_down<<<nb, kThreads, 0, st>>>(in, out, n, n_dev, tmp);
  return cudaGetLastError();
}

// block-major histogram (kBins words per block), then the digit totals
size_t radix_tmp_words(int64_t n) {
  const size_t nb = div_up(n > 0 ? n : 1, kTileItems);
  return nb * kBins + kBins;
}

cudaError_t radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                             uint32_t* vals_alt, int64_t n, int bits, uint32_t* tmp,
                             uint32_t** keys_out, uint32_t** vals_out, cudaStream_t st,
                             const uint32_t* n_dev) {
  *keys_out = keys;
  *vals_out = vals;
  if (n <= 1 || bits <= 0) return cudaSuccess;
  ProfScope ps(kProfSort, st);
  const unsigned nb = div_up(n, kTileItems);
  uint32_t* hist = tmp;
  uint32_t* dtot = tmp + (size_t)nb * kBins;
  uint32_t *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
  for (int shift = 0; shift < bits; shift += kRadixBits) {
    const int pb = bits - shift < kRadixBits ? bits - shift : kRadixBits;
    const int nbins = 1 << pb;
    count_launch(3);
    radix_upsweep<<<nb, kThreads, 0, st>>>(ki, n, n_dev, shift, nbins, hist);
    radix_offsets<<<nbins, kThreads, 0, st>>>(hist, (int)nb, dtot);
    radix_downsweep<<<nb, kThreads, 0, st>>>(ki, vi, ko, vo, n, n_dev, shift, nbins, hist, dtot);
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
  emit_kernel<<<div_up(n, 256), 256, 0, st>>>(order, offs, counts, rect, geom, rf, n, n_dev, tiles_x, keys,
                                               vals);
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
