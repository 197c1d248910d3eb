// digitize.cu -- Stage I of the two-stage digitization (Sec. 5): per-domain
// greedy aggregation (Sec. 3.2, fABBA) of the normalised pieces (Eq. 4),
// with exact group sums.
//
// One warp aggregates one domain (domains are stolen from a global counter).
// The method's decisions are defined in binary64: X = (scl * len) / sigma_len,
// Y = inc / sigma_inc, key = X*X + Y*Y (order: key, then position), and a
// later piece joins a start when (X_q - X_p)^2 + (Y_q - Y_p)^2 <= alpha^2.
// This GPU runs FP64 at ~1/64 of FP32 and a warp FP64 instruction costs the
// same with one lane active, so every decision is first taken in FP32 with a
// rigorous error interval and recomputed in binary64 (the definition's exact
// operation order) only when the interval straddles the threshold:
//  - keys: key32 = X32^2 + Y32^2 lies within key (1 +- 2^-19) (X32 from a
//    per-length table of the binary64 X rounded to FP32, Y32 = inc32 * (1 /
//    sigma_inc)_32 with inc32 a truncated copy: relative errors 2^-24, 2^-22);
//    after sorting by (key32, position), every run of neighbours whose
//    intervals overlap is re-sorted by the binary64 keys;
//  - distances: |dX32 - dX| <= 2^-23 (|X_q| + |X_p|), |dY32 - dY| <= 2^-20
//    (|Y_q| + |Y_p|); certain when the squared distance with those margins is
//    below / above alpha^2 (1 -+ 2^-20);
//  - the scan from a start stops once key32 (1 - 2^-19) exceeds
//    (sqrt(key32_start (1 + 2^-19)) + alpha (1 + 2^-20))^2: every later piece
//    then lies farther than alpha in binary64 (the Sec. 5 pruning, lossless).
#include "kernels.cuh"

namespace jabba {

constexpr int kLocWarps = 8;
constexpr float kKeyRel = 0x1p-19f;

struct LocalParams {
  const int* piece_len;
  const double* piece_inc;
  const long long* dom_slot_off;
  const int* dom_piece_cnt;
  long long n_domains;
  const double* sigma;    // [2] binary64
  const double* xtab64;   // [cap_len + 1] X(len) in binary64
  const float* xtab32;    // same, rounded to FP32
  const float* rinv32;    // (1 / sigma_inc) rounded to FP32
  long long cap_len;
  double alpha, scl;
  float a2lo, a2hi;       // alpha^2 (1 -+ 2^-20) in FP32 (rounded outward)
  float alpha_up;         // alpha (1 + 2^-20) rounded up
  int* local_label;
  int* dom_group_cnt;
  jabba_group* groups;
  long long group_capacity;
  long long* n_groups;
  unsigned* status;
  unsigned* task_counter;
  unsigned* arena;        // per-warp scratch, kArenaWords * cap_items words each
  long long cap_items;
};

constexpr int kArenaWords = 8;           // key, X32, Y32, sidx, label, tmp key, tmp val, members
constexpr int kSmemItemsArena = 2048;   // domains up to this many pieces use k_local_smem

__device__ __forceinline__ double x64_of(const LocalParams& P, int len) {
  if (len <= P.cap_len) return P.xtab64[len];
  return __ddiv_rn(__dmul_rn(P.scl, (double)len), P.sigma[0]);
}
__device__ __forceinline__ float x32_of(const LocalParams& P, int len) {
  if (len <= P.cap_len) return P.xtab32[len];
  return (float)x64_of(P, len);
}
__device__ __forceinline__ double y64_of(const LocalParams& P, double inc) { return __ddiv_rn(inc, P.sigma[1]); }

__device__ __forceinline__ double key64_of(const LocalParams& P, int len, double inc) {
  const double X = x64_of(P, len), Y = y64_of(P, inc);
  return __dadd_rn(__dmul_rn(X, X), __dmul_rn(Y, Y));
}

// binary64 membership test of the definition
__device__ __noinline__ bool exact_within(const LocalParams& P, int len_a, double inc_a, int len_b, double inc_b,
                                          double a2) {
  const double dx = __dsub_rn(x64_of(P, len_b), x64_of(P, len_a));
  const double dy = __dsub_rn(y64_of(P, inc_b), y64_of(P, inc_a));
  return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) <= a2;
}

// 0 = certainly outside, 1 = certainly within, 2 = undecided
__device__ __forceinline__ int filter_within(float xa, float ya, float xb, float yb, float a2lo, float a2hi) {
  const float dx = fabsf(xb - xa), dy = fabsf(yb - ya);
  const float ex = 0x1p-23f * (fabsf(xa) + fabsf(xb)) + 0x1p-126f;
  const float ey = 0x1p-20f * (fabsf(ya) + fabsf(yb)) + 0x1p-126f;
  const float hx = dx + ex, hy = dy + ey;
  const float lx = fmaxf(dx - ex, 0.f), ly = fmaxf(dy - ey, 0.f);
  const float hi = fmaf(hx, hx, hy * hy) * (1.0f + 0x1p-21f);
  const float lo = fmaf(lx, lx, ly * ly) * (1.0f - 0x1p-21f);
  if (hi < a2lo) return 1;
  if (lo > a2hi) return 0;
  return 2;
}

__device__ __forceinline__ float key_stop(float key_start, float alpha_up) {
  const float r = __fsqrt_ru(key_start * (1.0f + kKeyRel) * (1.0f + 0x1p-22f)) + alpha_up;
  return r * r * (1.0f + 0x1p-18f);
}


// Runs of neighbours whose key intervals overlap, found 32 pairs at a time;
// lane 0 re-sorts each run (insertion sort) by the binary64 keys, ties by
// position.  KeyT/IdxT: the key (FP32 bits) and position arrays of the view.
__device__ __forceinline__ bool keys_overlap32(unsigned k0, unsigned k1) {
  return __uint_as_float(k1) * (1.0f - kKeyRel) <= __uint_as_float(k0) * (1.0f + kKeyRel) * (1.0f + 0x1p-22f);
}

template <typename IdxT>
__device__ void sort_run(const LocalParams& P, const int* plen, const double* pinc, unsigned* key, IdxT* idx, int a,
                         int b) {
  for (int u = a + 1; u <= b; ++u) {
    const int pu = idx[u];
    const unsigned ku32 = key[u];
    const double ku = key64_of(P, plen[pu], pinc[pu]);
    int v = u - 1;
    while (v >= a) {
      const int pv = idx[v];
      const double kv = key64_of(P, plen[pv], pinc[pv]);
      if (kv > ku || (kv == ku && pv > pu)) {
        idx[v + 1] = (IdxT)pv;
        key[v + 1] = key[v];
        --v;
      } else {
        break;
      }
    }
    idx[v + 1] = (IdxT)pu;
    key[v + 1] = ku32;
  }
}

// Runs of neighbours whose key intervals overlap, found 32 pairs at a time
// (links from the keys as sorted: a run's last key bounds all its members, so
// the order across runs is settled by the FP32 keys); lane 0 re-sorts each
// run by the binary64 keys, ties by position.
template <typename IdxT>
__device__ void fix_runs(const LocalParams& P, const int* plen, const double* pinc, unsigned* key, IdxT* idx, int n) {
  const int lane = threadIdx.x & 31;
  int run_start = -1;                          // run open across chunks (uniform)
  for (int a0 = 0; a0 + 1 < n; a0 += 32) {
    const int a = a0 + lane;
    const bool link = a + 1 < n && keys_overlap32(key[a], key[a + 1]);
    const unsigned m = __ballot_sync(0xFFFFFFFFu, link);
    if (m == 0 && run_start < 0) continue;
    for (int l = 0; l < 32 && a0 + l + 1 < n; ++l) {
      const bool lk = (m >> l) & 1u;
      if (lk && run_start < 0) {
        run_start = a0 + l;
      } else if (!lk && run_start >= 0) {
        if (lane == 0) sort_run<IdxT>(P, plen, pinc, key, idx, run_start, a0 + l);
        __syncwarp();
        run_start = -1;
      }
    }
  }
  if (run_start >= 0 && lane == 0) sort_run<IdxT>(P, plen, pinc, key, idx, run_start, n - 1);
  __syncwarp();
}

// Counting-sort scratch view of one warp's arena.
struct Arena {
  unsigned* key;   // key32 bits (sorted in place with sidx)
  float* X;        // by position
  float* Y;        // by position
  int* sidx;       // sorted index -> position
  int* label;      // by position
  unsigned* tk;    // radix ping-pong
  int* tv;
  int* mem;        // group members / counts
};

__device__ __forceinline__ Arena arena_of(const LocalParams& P, long long warp_global) {
  Arena A;
  unsigned* base = P.arena + (size_t)warp_global * kArenaWords * (size_t)P.cap_items;
  const size_t c = (size_t)P.cap_items;
  A.key = base;
  A.X = (float*)(base + c);
  A.Y = (float*)(base + 2 * c);
  A.sidx = (int*)(base + 3 * c);
  A.label = (int*)(base + 4 * c);
  A.tk = base + 5 * c;
  A.tv = (int*)(base + 6 * c);
  A.mem = (int*)(base + 7 * c);
  return A;
}

// Stable LSD radix sort of (key, sidx) by key with 8-bit digits, one warp.
__device__ void warp_radix_sort(unsigned* key, int* val, unsigned* tk, int* tv, int n, unsigned* hist) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  unsigned* kin = key;
  int* vin = val;
  unsigned* kout = tk;
  int* vout = tv;
  for (int shift = 0; shift < 32; shift += 8) {
    for (int i = lane; i < 256; i += 32) hist[i] = 0;
    __syncwarp();
    for (int i = lane; i < n; i += 32) atomicAdd(&hist[(kin[i] >> shift) & 255u], 1u);
    __syncwarp();
    // exclusive scan of 256 counters: 8 per lane
    unsigned loc[8], s = 0;
    for (int j = 0; j < 8; ++j) { loc[j] = hist[lane * 8 + j]; s += loc[j]; }
    unsigned incl = s;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += y;
    }
    unsigned run = incl - s;
    __syncwarp();
    for (int j = 0; j < 8; ++j) { hist[lane * 8 + j] = run; run += loc[j]; }
    __syncwarp();
    for (int i0 = 0; i0 < n; i0 += 32) {
      const int i = i0 + lane;
      const bool v = i < n;
      const unsigned k = v ? kin[i] : 0u;
      const int vv = v ? vin[i] : 0;
      const unsigned d = v ? ((k >> shift) & 255u) : 256u + lane;
      const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
      const unsigned r = __popc(peers & lt);
      if (v) {
        const unsigned pos = hist[d] + r;
        kout[pos] = k;
        vout[pos] = vv;
      }
      __syncwarp();
      if (v && r == 0) hist[d] += __popc(peers);
      __syncwarp();
    }
    unsigned* t = kin; kin = kout; kout = t;
    int* tt = vin; vin = vout; vout = tt;
  }
  // four passes: the result is back in (key, val)
}

__global__ void __launch_bounds__(kLocWarps * 32) k_local_warp(LocalParams P) {
  __shared__ unsigned hist_all[kLocWarps][256];
  __shared__ int cl_flag[kLocWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long warp_global = (long long)blockIdx.x * kLocWarps + warp;
  unsigned* hist = hist_all[warp];
  const Arena A = arena_of(P, warp_global);
  const double a2 = __dmul_rn(P.alpha, P.alpha);
  const float rinv = *P.rinv32;
  for (;;) {
    long long d = 0;
    if (lane == 0) d = (long long)atomicAdd(P.task_counter, 1u);
    d = __shfl_sync(0xFFFFFFFFu, d, 0);
    if (d >= P.n_domains) break;
    const int n = P.dom_piece_cnt[d];
    if (n <= kSmemItemsArena) continue;           // the shared-memory kernel takes it
    const long long slot = P.dom_slot_off[d];
    const int* plen = P.piece_len + slot;
    const double* pinc = P.piece_inc + slot;
    if (n > P.cap_items) {
      if (lane == 0) {
        set_status(P.status, JABBA_ERR_CAPACITY);
        P.dom_group_cnt[d] = 0;
      }
      continue;
    }
    // 1. FP32 coordinates and keys
    for (int i = lane; i < n; i += 32) {
      unsigned mh;
      const float x = x32_of(P, plen[i]);
      const float y = f64_to_f32_trunc(pinc[i], mh) * rinv;
      A.X[i] = x;
      A.Y[i] = y;
      A.key[i] = __float_as_uint(fmaf(x, x, y * y));
      A.sidx[i] = i;
      A.label[i] = -1;
    }
    __syncwarp();
    // 2. sort by (key32, position)
    if (n > 1) warp_radix_sort(A.key, A.sidx, A.tk, A.tv, n, hist);
    __syncwarp();
    // 3. runs of overlapping key intervals: re-sort by the binary64 keys
    fix_runs<int>(P, plen, pinc, A.key, A.sidx, n);
    // 4. greedy in key order
    int G = 0;
    {
      int a = 0;
      for (;;) {
        for (;;) {
          const int aa = a + lane;
          const bool fr = aa < n && A.label[A.sidx[aa]] < 0;
          const unsigned m = __ballot_sync(0xFFFFFFFFu, fr);
          if (m) { a += __ffs(m) - 1; break; }
          a += 32;
          if (a >= n) break;
        }
        if (a >= n) break;
        const int ps = A.sidx[a];
        const float xs = A.X[ps], ys = A.Y[ps];
        const float T = key_stop(__uint_as_float(A.key[a]), P.alpha_up);
        if (lane == 0) A.label[ps] = G;
        for (int b0 = a + 1; b0 < n; b0 += 32) {
          const int b = b0 + lane;
          bool stop = true;
          if (b < n) {
            stop = __uint_as_float(A.key[b]) * (1.0f - kKeyRel) > T;
            if (!stop) {
              const int pb = A.sidx[b];
              if (A.label[pb] < 0) {
                int w = filter_within(xs, ys, A.X[pb], A.Y[pb], P.a2lo, P.a2hi);
                if (w == 2) w = exact_within(P, plen[ps], pinc[ps], plen[pb], pinc[pb], a2) ? 1 : 0;
                if (w) A.label[pb] = G;
              }
            }
          }
          if (__any_sync(0xFFFFFFFFu, stop)) break;
        }
        __syncwarp();
        ++G;
        ++a;
      }
    }
    __syncwarp();
    // 5. members per group (counting sort by label) and exact sums
    int* cnt = A.mem;           // [G] counts, then offsets
    int* mem = A.tv;            // [n] positions grouped by label
    for (int g = lane; g < G; g += 32) cnt[g] = 0;
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
      atomicAdd(&cnt[A.label[i]], 1);
      P.local_label[slot + i] = A.label[i];
    }
    __syncwarp();
    {
      int carry = 0;
      for (int g0 = 0; g0 < G; g0 += 32) {
        const int g = g0 + lane;
        const int c = g < G ? cnt[g] : 0;
        int incl = c;
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
          if (lane >= o) incl += y;
        }
        if (g < G) cnt[g] = carry + incl - c;   // exclusive offset
        carry += __shfl_sync(0xFFFFFFFFu, incl, 31);
      }
    }
    __syncwarp();
    // scatter positions in label order (stable order is not needed: sums are exact)
    for (int i = lane; i < n; i += 32) {
      const int r = atomicAdd(&cnt[A.label[i]], 1);
      mem[r] = i;
    }
    __syncwarp();
    long long base = 0;
    if (lane == 0) {
      base = (long long)atomicAdd((unsigned long long*)P.n_groups, (unsigned long long)G);
      if (base + G > P.group_capacity) {
        set_status(P.status, JABBA_ERR_CAPACITY);
        base = -1;
      }
      P.dom_group_cnt[d] = G;
    }
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (base >= 0) {
      for (int g = lane; g < G; g += 32) {
        const int e = cnt[g];                    // end of group g after the scatter
        const int s = g ? cnt[g - 1] : 0;
        I192 acc = {0, 0, 0};
        long long lensum = 0;
        for (int q = s; q < e; ++q) {
          const int i = mem[q];
          lensum += plen[i];
          bool neg;
          const U128 m = fx_mag(pinc[i], neg);
          acc_signed(acc, m, neg);
        }
        jabba_group rec;
        rec.inc[0] = acc.w0;
        rec.inc[1] = acc.w1;
        rec.inc[2] = acc.w2;
        rec.lensum = lensum;
        rec.count = e - s;
        rec.local_id = g;
        rec.domain = (int)d;
        rec.pad = 0;
        P.groups[base + g] = rec;
      }
    }
    __syncwarp();
  }
  (void)cl_flag;
}

// ------------------------------------------------------------------ shared-memory path
// Domains of at most kSmemItems pieces: the same steps with every per-piece
// array in the warp's slice of shared memory, the coordinates permuted into
// key order after the sort so that the greedy reads contiguous entries.
constexpr int kSmemItems = 2048;
constexpr int kSmemWarps = 4;
// bytes per item: key 4, X/sX 4, Y/sY 4, tmp key 4, idx 2, tmp idx 2, label 2, pad 2
constexpr size_t kSmemPerWarp = (size_t)kSmemItems * 24 + 1024;

__device__ void warp_radix_sort16(unsigned* key, unsigned short* val, unsigned* tk, unsigned short* tv, int n,
                                  unsigned* hist) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  unsigned* kin = key;
  unsigned short* vin = val;
  unsigned* kout = tk;
  unsigned short* vout = tv;
  for (int shift = 0; shift < 32; shift += 8) {
    for (int i = lane; i < 256; i += 32) hist[i] = 0;
    __syncwarp();
    for (int i = lane; i < n; i += 32) atomicAdd(&hist[(kin[i] >> shift) & 255u], 1u);
    __syncwarp();
    unsigned loc[8], sum = 0;
    for (int j = 0; j < 8; ++j) { loc[j] = hist[lane * 8 + j]; sum += loc[j]; }
    unsigned incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += y;
    }
    unsigned run = incl - sum;
    __syncwarp();
    for (int j = 0; j < 8; ++j) { hist[lane * 8 + j] = run; run += loc[j]; }
    __syncwarp();
    for (int i0 = 0; i0 < n; i0 += 32) {
      const int i = i0 + lane;
      const bool v = i < n;
      const unsigned k = v ? kin[i] : 0u;
      const unsigned short vv = v ? vin[i] : 0;
      const unsigned d = v ? ((k >> shift) & 255u) : 256u + lane;
      const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
      const unsigned r = __popc(peers & lt);
      if (v) {
        const unsigned pos = hist[d] + r;
        kout[pos] = k;
        vout[pos] = vv;
      }
      __syncwarp();
      if (v && r == 0) hist[d] += __popc(peers);
      __syncwarp();
    }
    unsigned* t = kin; kin = kout; kout = t;
    unsigned short* tt = vin; vin = vout; vout = tt;
  }
}

__global__ void __launch_bounds__(kSmemWarps * 32) k_local_smem(LocalParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* base = smem_raw + (size_t)warp * kSmemPerWarp;
  unsigned* hist = (unsigned*)base;                                    // 256 words
  unsigned* key = (unsigned*)(base + 1024);                            // [n] sorted keys
  float* X = (float*)(key + kSmemItems);                               // [n] by position, then sY
  float* Y = X + kSmemItems;                                           // [n] by position, then labels/scratch
  unsigned* tk = (unsigned*)(Y + kSmemItems);                          // [n] sort temp, then sX
  unsigned short* idx = (unsigned short*)(tk + kSmemItems);            // [n] sorted index -> position
  unsigned short* tv = idx + kSmemItems;                               // [n] sort temp
  short* lab = (short*)(tv + kSmemItems);                              // [n] label by sorted index
  float* sX = (float*)tk;
  float* sY = X;
  const double a2 = __dmul_rn(P.alpha, P.alpha);
  const float rinv = *P.rinv32;
  for (;;) {
    long long d = 0;
    if (lane == 0) d = (long long)atomicAdd(P.task_counter, 1u);
    d = __shfl_sync(0xFFFFFFFFu, d, 0);
    if (d >= P.n_domains) break;
    const int n = P.dom_piece_cnt[d];
    if (n > kSmemItems) continue;                 // the arena kernel takes it
    const long long slot = P.dom_slot_off[d];
    const int* plen = P.piece_len + slot;
    const double* pinc = P.piece_inc + slot;
    if (n == 0) {
      if (lane == 0) P.dom_group_cnt[d] = 0;
      continue;
    }
    // 1. FP32 coordinates and keys by position
    for (int i = lane; i < n; i += 32) {
      unsigned mh;
      const float x = x32_of(P, plen[i]);
      const float y = f64_to_f32_trunc(pinc[i], mh) * rinv;
      X[i] = x;
      Y[i] = y;
      key[i] = __float_as_uint(fmaf(x, x, y * y));
      idx[i] = (unsigned short)i;
    }
    __syncwarp();
    // 2. sort by (key32, position)
    if (n > 1) warp_radix_sort16(key, idx, tk, tv, n, hist);
    __syncwarp();
    // 3. runs of overlapping key intervals: re-sort by the binary64 keys (rare)
    fix_runs<unsigned short>(P, plen, pinc, key, idx, n);
    // 4. coordinates in key order: sX into the sort temp, then sY into X's slot
    for (int a = lane; a < n; a += 32) sX[a] = X[idx[a]];
    __syncwarp();
    for (int a = lane; a < n; a += 32) sY[a] = Y[idx[a]];
    __syncwarp();
    for (int a = lane; a < n; a += 32) lab[a] = -1;
    __syncwarp();
    // 5. greedy in key order
    int G = 0;
    {
      int a = 0;
      for (;;) {
        for (;;) {
          const int aa = a + lane;
          const bool fr = aa < n && lab[aa] < 0;
          const unsigned m = __ballot_sync(0xFFFFFFFFu, fr);
          if (m) { a += __ffs(m) - 1; break; }
          a += 32;
          if (a >= n) break;
        }
        if (a >= n) break;
        const float xs = sX[a], ys = sY[a];
        const float T = key_stop(__uint_as_float(key[a]), P.alpha_up);
        if (lane == 0) lab[a] = (short)G;
        for (int b0 = a + 1; b0 < n; b0 += 32) {
          const int b = b0 + lane;
          bool stop = true;
          if (b < n) {
            stop = __uint_as_float(key[b]) * (1.0f - kKeyRel) > T;
            if (!stop && lab[b] < 0) {
              int w = filter_within(xs, ys, sX[b], sY[b], P.a2lo, P.a2hi);
              if (w == 2) {
                const int ps = idx[a], pb = idx[b];
                w = exact_within(P, plen[ps], pinc[ps], plen[pb], pinc[pb], a2) ? 1 : 0;
              }
              if (w) lab[b] = (short)G;
            }
          }
          if (__any_sync(0xFFFFFFFFu, stop)) break;
        }
        __syncwarp();
        ++G;
        ++a;
      }
    }
    __syncwarp();
    // 6. labels to positions, member lists (counting sort by label), exact sums
    int* cnt = (int*)key;        // [G + 1] offsets (keys no longer needed)
    unsigned short* mem = tv;    // [n] positions grouped by label
    for (int a = lane; a < n; a += 32) P.local_label[slot + idx[a]] = lab[a];
    for (int g = lane; g <= G; g += 32) cnt[g] = 0;
    __syncwarp();
    for (int a = lane; a < n; a += 32) atomicAdd(&cnt[lab[a]], 1);
    __syncwarp();
    {
      int carry = 0;
      for (int g0 = 0; g0 < G; g0 += 32) {
        const int g = g0 + lane;
        const int c = g < G ? cnt[g] : 0;
        int incl = c;
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
          if (lane >= o) incl += y;
        }
        if (g < G) cnt[g] = carry + incl - c;
        carry += __shfl_sync(0xFFFFFFFFu, incl, 31);
      }
    }
    __syncwarp();
    for (int a = lane; a < n; a += 32) {
      const int r = atomicAdd(&cnt[lab[a]], 1);
      mem[r] = idx[a];
    }
    __syncwarp();
    long long gbase = 0;
    if (lane == 0) {
      gbase = (long long)atomicAdd((unsigned long long*)P.n_groups, (unsigned long long)G);
      if (gbase + G > P.group_capacity) {
        set_status(P.status, JABBA_ERR_CAPACITY);
        gbase = -1;
      }
      P.dom_group_cnt[d] = G;
    }
    gbase = __shfl_sync(0xFFFFFFFFu, gbase, 0);
    if (gbase >= 0) {
      for (int g = lane; g < G; g += 32) {
        const int e = cnt[g];
        const int s0 = g ? cnt[g - 1] : 0;
        I192 acc = {0, 0, 0};
        long long lensum = 0;
#pragma unroll 4
        for (int q = s0; q < e; ++q) {
          const int i = mem[q];
          lensum += plen[i];
          bool neg;
          const U128 m = fx_mag(pinc[i], neg);
          acc_signed(acc, m, neg);
        }
        jabba_group rec;
        rec.inc[0] = acc.w0;
        rec.inc[1] = acc.w1;
        rec.inc[2] = acc.w2;
        rec.lensum = lensum;
        rec.count = e - s0;
        rec.local_id = g;
        rec.domain = (int)d;
        rec.pad = 0;
        P.groups[gbase + g] = rec;
      }
    }
    __syncwarp();
  }
}

// X table and 1/sigma_inc for the FP32 filters (binary64 definitions).
__global__ void k_norm_tables(const double* sigma, double scl, long long cap_len, double* xtab64, float* xtab32,
                              float* rinv32) {
  const double sl = sigma[0];
  for (long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x; l <= cap_len; l += (long long)gridDim.x * blockDim.x) {
    const double X = __ddiv_rn(__dmul_rn(scl, (double)l), sl);
    xtab64[l] = X;
    xtab32[l] = __double2float_rn(X);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *rinv32 = __double2float_rn(__ddiv_rn(1.0, sigma[1]));
}

static float round_down_f(double v) {
  float f = (float)v;
  if ((double)f > v) f = nextafterf(f, 0.0f);
  return f;
}
static float round_up_f(double v) {
  float f = (float)v;
  if ((double)f < v) f = nextafterf(f, INFINITY);
  return f;
}

void launch_local(const int* piece_len, const double* piece_inc, const long long* dom_slot_off,
                  const int* dom_piece_cnt, long long n_domains, const double* sigma, double alpha, double scl,
                  int* local_label, int* dom_group_cnt, long long* dom_group_off, jabba_group* groups,
                  long long group_capacity, long long* n_groups, Scratch& ws, unsigned* status, cudaStream_t st) {
  cudaMemsetAsync(n_groups, 0, sizeof(long long), st);
  cudaMemsetAsync(ws.counters + 4, 0, sizeof(unsigned), st);
  k_norm_tables<<<(unsigned)((ws.cap_len + 256) / 256), 256, 0, st>>>(sigma, scl, ws.cap_len, ws.xtab64, ws.xtab32,
                                                                        ws.rinv32);
  LocalParams P;
  P.piece_len = piece_len;
  P.piece_inc = piece_inc;
  P.dom_slot_off = dom_slot_off;
  P.dom_piece_cnt = dom_piece_cnt;
  P.n_domains = n_domains;
  P.sigma = sigma;
  P.xtab64 = ws.xtab64;
  P.xtab32 = ws.xtab32;
  P.rinv32 = ws.rinv32;
  P.cap_len = ws.cap_len;
  P.alpha = alpha;
  P.scl = scl;
  const double a2 = alpha * alpha;
  P.a2lo = round_down_f(a2 * (1.0 - 0x1p-20));
  P.a2hi = round_up_f(a2 * (1.0 + 0x1p-20));
  P.alpha_up = round_up_f(alpha * (1.0 + 0x1p-20));
  P.local_label = local_label;
  P.dom_group_cnt = dom_group_cnt;
  P.groups = groups;
  P.group_capacity = group_capacity;
  P.n_groups = n_groups;
  P.status = status;
  P.task_counter = ws.counters + 4;
  P.arena = ws.arena;
  P.cap_items = ws.cap_items;
  if (n_domains > 0) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_local_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(kSmemPerWarp * kSmemWarps));
      attr = true;
    }
    k_local_smem<<<(unsigned)(ws.num_sms * 1), kSmemWarps * 32, kSmemPerWarp * kSmemWarps, st>>>(P);
    cudaMemsetAsync(ws.counters + 4, 0, sizeof(unsigned), st);
    k_local_warp<<<(unsigned)ws.loc_ctas, kLocWarps * 32, 0, st>>>(P);
  }
  exclusive_scan<int>(dom_group_cnt, n_domains, dom_group_off, ws.scan_tiles, st);
}

long long local_arena_words(long long cap_items, long long n_warps) { return kArenaWords * cap_items * n_warps; }
int local_warps_per_cta() { return kLocWarps; }

}  // namespace jabba
