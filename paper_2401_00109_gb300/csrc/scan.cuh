// scan.cuh -- device-wide exclusive prefix sums (int64) used to turn
// per-series / per-domain counts into offsets.  Three phases: block sums,
// one-block scan of the block sums, block-local scans plus offsets.
#pragma once
#include "jabba_dev.cuh"

namespace jabba {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;  // items per thread
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ long long block_exclusive_scan(long long v, long long* smem_warp, long long& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long x = v;
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    long long w = lane < (kScanThreads / 32) ? smem_warp[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < (kScanThreads / 32)) smem_warp[lane] = w;
  }
  __syncthreads();
  total = smem_warp[kScanThreads / 32 - 1];
  const long long before = warp ? smem_warp[warp - 1] : 0;
  __syncthreads();
  return before + x - v;
}

template <typename T>
static __global__ void k_scan_tile_sums(const T* in, long long n, long long* tile_sums) {
  __shared__ long long sw[kScanThreads / 32];
  const long long base = (long long)blockIdx.x * kScanTile;
  long long v = 0;
  for (int i = 0; i < kScanItems; ++i) {
    const long long k = base + (long long)threadIdx.x * kScanItems + i;
    if (k < n) v += (long long)in[k];
  }
  long long total;
  block_exclusive_scan<T>(v, sw, total);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// One block scans the tile sums in place (exclusive), any number of tiles:
// thread t owns the contiguous range [t c, (t+1) c) of c = ceil(n / threads)
// tiles, sums it, the block scans the per-thread sums once, and every thread
// writes its range's prefixes (one block-wide scan instead of one per 256
// tiles).
static __global__ void k_scan_tile_offsets(long long* tile_sums, long long n_tiles, long long* grand_total) {
  __shared__ long long sw[kScanThreads / 32];
  const long long per = (n_tiles + kScanThreads - 1) / kScanThreads;
  const long long lo = (long long)threadIdx.x * per;
  const long long hi = lo + per < n_tiles ? lo + per : n_tiles;
  long long v = 0;
  for (long long k = lo; k < hi; ++k) v += tile_sums[k];
  long long total;
  long long run = block_exclusive_scan<long long>(v, sw, total);
  for (long long k = lo; k < hi; ++k) {
    const long long c = tile_sums[k];
    tile_sums[k] = run;
    run += c;
  }
  if (threadIdx.x == 0 && grand_total) *grand_total = total;
}

template <typename T>
static __global__ void k_scan_apply(const T* in, long long n, const long long* tile_off, long long* out) {
  __shared__ long long sw[kScanThreads / 32];
  const long long base = (long long)blockIdx.x * kScanTile;
  long long vals[kScanItems];
  long long v = 0;
  for (int i = 0; i < kScanItems; ++i) {
    const long long k = base + (long long)threadIdx.x * kScanItems + i;
    vals[i] = k < n ? (long long)in[k] : 0;
    v += vals[i];
  }
  long long total;
  long long ex = block_exclusive_scan<T>(v, sw, total) + tile_off[blockIdx.x];
  for (int i = 0; i < kScanItems; ++i) {
    const long long k = base + (long long)threadIdx.x * kScanItems + i;
    if (k < n) out[k] = ex;
    ex += vals[i];
  }
}

static __global__ void k_store_total(const long long* total, long long* dst) { *dst = *total; }

// out[0..n] = exclusive scan of in[0..n), out[n] = total.  `tiles` is scratch
// of at least ceil(n / kScanTile) + 1 elements.
template <typename T>
inline void exclusive_scan(const T* in, long long n, long long* out, long long* tiles, cudaStream_t st) {
  const long long n_tiles = (n + kScanTile - 1) / kScanTile;
  if (n_tiles > 0) k_scan_tile_sums<T><<<(unsigned)n_tiles, kScanThreads, 0, st>>>(in, n, tiles);
  k_scan_tile_offsets<<<1, kScanThreads, 0, st>>>(tiles, n_tiles, tiles + n_tiles);
  if (n_tiles > 0) k_scan_apply<T><<<(unsigned)n_tiles, kScanThreads, 0, st>>>(in, n, tiles, out);
  k_store_total<<<1, 1, 0, st>>>(tiles + n_tiles, out + n);
}

inline long long scan_scratch_elems(long long n) { return (n + kScanTile - 1) / kScanTile + 1; }

}  // namespace jabba
