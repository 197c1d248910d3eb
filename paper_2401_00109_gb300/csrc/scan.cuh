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

// A thread's kScanItems consecutive inputs from k: one or two 16-byte loads
// when `vec` (both arrays 16-byte aligned) and all four are in range.
template <typename T>
__device__ __forceinline__ void scan_load4(const T* in, long long k, long long n, bool vec, long long (&v)[4]) {
  static_assert(kScanItems == 4, "four items per thread");
  if (vec && k + 3 < n) {
    if constexpr (sizeof(T) == 4) {
      const int4 w = *(const int4*)(in + k);
      v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
    } else {
      const longlong2 a = *(const longlong2*)(in + k), b = *(const longlong2*)(in + k + 2);
      v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    return;
  }
  for (int i = 0; i < 4; ++i) v[i] = k + i < n ? (long long)in[k + i] : 0;
}

template <typename T>
static __global__ void k_scan_tile_sums(const T* in, long long n, long long* tile_sums, bool vec) {
  __shared__ long long sw[kScanThreads / 32];
  const long long base = (long long)blockIdx.x * kScanTile;
  long long vals[kScanItems];
  scan_load4(in, base + (long long)threadIdx.x * kScanItems, n, vec, vals);
  const long long v = vals[0] + vals[1] + vals[2] + vals[3];
  long long total;
  block_exclusive_scan<T>(v, sw, total);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// One block of kOffThreads scans the tile sums in place (exclusive), any
// number of tiles: thread t owns the contiguous range [t c, (t+1) c) of
// c = ceil(n / threads) tiles, sums it, the block scans the per-thread sums
// once, and every thread writes its range's prefixes (one block-wide scan
// instead of one per 256 tiles).
constexpr int kOffThreads = 1024;

__device__ __forceinline__ long long block_exclusive_scan_1024(long long v, long long* smem_warp, long long& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long x = v;
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    long long w = smem_warp[lane];  // 32 warps
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if (lane >= o) w += y;
    }
    smem_warp[lane] = w;
  }
  __syncthreads();
  total = smem_warp[31];
  const long long before = warp ? smem_warp[warp - 1] : 0;
  __syncthreads();
  return before + x - v;
}

static __global__ void __launch_bounds__(kOffThreads) k_scan_tile_offsets(long long* tile_sums, long long n_tiles,
                                                                         long long* grand_total) {
  __shared__ long long sw[kOffThreads / 32];
  const long long per = (n_tiles + kOffThreads - 1) / kOffThreads;
  const long long lo = (long long)threadIdx.x * per;
  const long long hi = lo + per < n_tiles ? lo + per : n_tiles;
  long long v = 0;
  for (long long k = lo; k < hi; ++k) v += tile_sums[k];
  long long total;
  long long run = block_exclusive_scan_1024(v, sw, total);
  for (long long k = lo; k < hi; ++k) {
    const long long c = tile_sums[k];
    tile_sums[k] = run;
    run += c;
  }
  if (threadIdx.x == 0 && grand_total) *grand_total = total;
}

template <typename T>
static __global__ void k_scan_apply(const T* in, long long n, const long long* tile_off, long long* out, bool vec) {
  __shared__ long long sw[kScanThreads / 32];
  const long long base = (long long)blockIdx.x * kScanTile;
  const long long k0 = base + (long long)threadIdx.x * kScanItems;
  long long vals[kScanItems];
  scan_load4(in, k0, n, vec, vals);
  const long long v = vals[0] + vals[1] + vals[2] + vals[3];
  long long total;
  const long long ex = block_exclusive_scan<T>(v, sw, total) + tile_off[blockIdx.x];
  const long long o0 = ex, o1 = o0 + vals[0], o2 = o1 + vals[1], o3 = o2 + vals[2];
  if (vec && k0 + 3 < n) {
    *(longlong2*)(out + k0) = make_longlong2(o0, o1);
    *(longlong2*)(out + k0 + 2) = make_longlong2(o2, o3);
  } else {
    if (k0 < n) out[k0] = o0;
    if (k0 + 1 < n) out[k0 + 1] = o1;
    if (k0 + 2 < n) out[k0 + 2] = o2;
    if (k0 + 3 < n) out[k0 + 3] = o3;
  }
}

static __global__ void k_store_total(const long long* total, long long* dst) { *dst = *total; }

// out[0..n] = exclusive scan of in[0..n), out[n] = total.  `tiles` is scratch
// of at least ceil(n / kScanTile) + 1 elements.
template <typename T>
inline void exclusive_scan(const T* in, long long n, long long* out, long long* tiles, cudaStream_t st) {
  const long long n_tiles = (n + kScanTile - 1) / kScanTile;
  const bool vec = ((size_t)in % 16) == 0 && ((size_t)out % 16) == 0;
  if (n_tiles > 0) k_scan_tile_sums<T><<<(unsigned)n_tiles, kScanThreads, 0, st>>>(in, n, tiles, vec);
  k_scan_tile_offsets<<<1, kOffThreads, 0, st>>>(tiles, n_tiles, tiles + n_tiles);
  if (n_tiles > 0) k_scan_apply<T><<<(unsigned)n_tiles, kScanThreads, 0, st>>>(in, n, tiles, out, vec);
  k_store_total<<<1, 1, 0, st>>>(tiles + n_tiles, out + n);
}

inline long long scan_scratch_elems(long long n) { return (n + kScanTile - 1) / kScanTile + 1; }

}  // namespace jabba
