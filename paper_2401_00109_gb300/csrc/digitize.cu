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
  int pca;                // sort key: 0 = X*X + Y*Y, 1 = the projection vx X + vy Y on the PCA axis
  int* local_label;
  int* dom_group_cnt;
  jabba_group* groups;
  long long group_capacity;
  long long* n_groups;
  unsigned* status;
  unsigned* task_counter; // arena kernel: next entry of its domain list
  const int* list;        // arena kernel: domains with more pieces than the largest tile
  const unsigned* list_count;
  unsigned* arena;        // per-warp scratch, kArenaWords * cap_items words each
  long long cap_items;
};

constexpr int kArenaWords = 8;           // key, X32, Y32, sidx, label, tmp key, tmp val, members

__device__ __forceinline__ double x64_of(const LocalParams& P, int len) {
  if (len <= P.cap_len) return P.xtab64[len];
  return __ddiv_rn(__dmul_rn(P.scl, (double)len), P.sigma[0]);
}
__device__ __forceinline__ float x32_of(const LocalParams& P, int len) {
  if (len <= P.cap_len) return P.xtab32[len];
  return (float)x64_of(P, len);
}
__device__ __forceinline__ double y64_of(const LocalParams& P, double inc) { return __ddiv_rn(inc, P.sigma[1]); }

// The sort key in binary64 (the definition): X*X + Y*Y, or with the PCA key
// vx * X + vy * Y (the axis in sigma[2..3]); ties by position.
__device__ __forceinline__ double key64_of(const LocalParams& P, int len, double inc) {
  const double X = x64_of(P, len), Y = y64_of(P, inc);
  if (P.pca) return __dadd_rn(__dmul_rn(P.sigma[2], X), __dmul_rn(P.sigma[3], Y));
  return __dadd_rn(__dmul_rn(X, X), __dmul_rn(Y, Y));
}

// FP32 key of a piece from its FP32 coordinates.  Norm key: x*x + y*y lies
// within key (1 +- 2^-19).  PCA key: vx32 x + vy32 y (vx32, vy32 the axis
// rounded to FP32) lies within pca_err of the binary64 projection (|x32 - X|
// <= 2^-24 |X|, |y32 - Y| <= 2^-22 |Y|, |v32 - v| <= 2^-24 |v|, two FP32
// roundings: the error is below 2^-21 (|x| + |y|) + 2^-24 |k|).
__device__ __forceinline__ float key32f(const LocalParams& P, float x, float y, float vx32, float vy32) {
  return P.pca ? fmaf(vx32, x, vy32 * y) : fmaf(x, x, y * y);
}
__device__ __forceinline__ float pca_err(float x, float y, float k) {
  return 0x1p-20f * (fabsf(x) + fabsf(y) + fabsf(k)) + 0x1p-120f;
}
// Order-preserving unsigned image of an FP32 key (signed keys of the PCA
// axis included): the sign bit set for non-negative values, every bit
// flipped for negative ones.
__device__ __forceinline__ unsigned key_bits(float k) {
  const unsigned u = __float_as_uint(k);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_val(unsigned b) {
  return __uint_as_float((b & 0x80000000u) ? (b & 0x7FFFFFFFu) : ~b);
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

// Scan bound of the start at (xs, ys): a later piece past it lies farther
// than alpha from the start in binary64 (Sec. 5 pruning).  Norm key: key32
// (1 - 2^-19) > (sqrt(key32_s (1 + 2^-19)) + alpha)^2; PCA key: the key gap
// exceeds alpha with both error bounds (a projection on a unit axis changes
// by at most the distance).
__device__ __forceinline__ float scan_bound(const LocalParams& P, float xs, float ys, float vx32, float vy32) {
  const float k = key32f(P, xs, ys, vx32, vy32);
  if (P.pca) return (k + pca_err(xs, ys, k)) + P.alpha_up * (1.0f + 0x1p-20f);
  return key_stop(k, P.alpha_up);
}
__device__ __forceinline__ bool past_bound(const LocalParams& P, float xb, float yb, float T, float vx32, float vy32) {
  const float k = key32f(P, xb, yb, vx32, vy32);
  if (P.pca) return k - pca_err(xb, yb, k) > T;
  return k * (1.0f - kKeyRel) > T;
}


// Runs of neighbours whose key intervals overlap, found 32 pairs at a time;
// lane 0 re-sorts each run (insertion sort) by the binary64 keys, ties by
// position.  KeyT/IdxT: the key (FP32 bits) and position arrays of the view.
// Whether the error intervals of two neighbouring sorted keys overlap (then
// their order is settled by the binary64 keys): relative bounds for the norm
// key, the domain's largest absolute bound `edom` for the PCA key.
__device__ __forceinline__ bool keys_overlap32(const LocalParams& P, unsigned k0, unsigned k1, float edom) {
  const float v0 = key_val(k0), v1 = key_val(k1);
  if (P.pca) return v1 - edom <= v0 + edom;
  return v1 * (1.0f - kKeyRel) <= v0 * (1.0f + kKeyRel) * (1.0f + 0x1p-22f);
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

// The same re-sort for a run of at most 32 members: the warp computes each
// member's binary64 key once (lane i, member a + i) into kbuf, then lane 0
// insertion-sorts on those keys.
template <typename IdxT>
__device__ void sort_run32(const LocalParams& P, const int* plen, const double* pinc, unsigned* key, IdxT* idx, int a,
                           int b, double* kbuf) {
  const int lane = threadIdx.x & 31;
  const int r = b - a + 1;
  if (lane < r) {
    const int p = idx[a + lane];
    kbuf[lane] = key64_of(P, plen[p], pinc[p]);
  }
  __syncwarp();
  if (lane == 0) {
    for (int u = 1; u < r; ++u) {
      const double ku = kbuf[u];
      const int pu = idx[a + u];
      const unsigned ku32 = key[a + u];
      int v = u - 1;
      while (v >= 0 && (kbuf[v] > ku || (kbuf[v] == ku && (int)idx[a + v] > pu))) {
        kbuf[v + 1] = kbuf[v];
        idx[a + v + 1] = idx[a + v];
        key[a + v + 1] = key[a + v];
        --v;
      }
      kbuf[v + 1] = ku;
      idx[a + v + 1] = (IdxT)pu;
      key[a + v + 1] = ku32;
    }
  }
  __syncwarp();
}

// Runs of neighbours whose key intervals overlap, found 32 pairs at a time
// (links from the keys as sorted: a run's last key bounds all its members, so
// the order across runs is settled by the FP32 keys); each run is re-sorted by
// the binary64 keys, ties by position.  Whole warp; the run boundaries are
// found by bit scans of the link masks; kbuf: 32 doubles of scratch.
template <typename IdxT>
__device__ void fix_runs(const LocalParams& P, const int* plen, const double* pinc, unsigned* key, IdxT* idx, int n,
                         double* kbuf, float edom) {
  const int lane = threadIdx.x & 31;
  int run_start = -1;                          // run open across chunks (uniform)
  auto sort_members = [&](int a, int b) {
    if (b - a + 1 <= 32) {
      sort_run32<IdxT>(P, plen, pinc, key, idx, a, b, kbuf);
    } else {
      if (lane == 0) sort_run<IdxT>(P, plen, pinc, key, idx, a, b);
      __syncwarp();
    }
  };
  for (int a0 = 0; a0 + 1 < n; a0 += 32) {
    const int a = a0 + lane;
    const bool link = a + 1 < n && keys_overlap32(P, key[a], key[a + 1], edom);
    const int lim = min(32, n - 1 - a0);       // pairs a0 .. a0 + lim - 1 exist
    const unsigned valid = lim >= 32 ? 0xFFFFFFFFu : ((1u << lim) - 1u);
    const unsigned m = __ballot_sync(0xFFFFFFFFu, link) & valid;
    if (m == 0 && run_start < 0) continue;
    int l = 0;
    while (l < lim) {
      if (run_start < 0) {
        const unsigned mm = m & (0xFFFFFFFFu << l);
        if (!mm) break;
        l = __ffs(mm) - 1;
        run_start = a0 + l;
      }
      const unsigned nm = ~m & valid & (0xFFFFFFFFu << l);
      if (!nm) break;                          // the run goes on into the next chunk
      l = __ffs(nm) - 1;                       // first pair past the run: its last member is a0 + l
      sort_members(run_start, a0 + l);
      run_start = -1;
      ++l;
    }
  }
  if (run_start >= 0) sort_members(run_start, n - 1);
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
  __shared__ __align__(16) unsigned hist_all[kLocWarps][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long warp_global = (long long)blockIdx.x * kLocWarps + warp;
  unsigned* hist = hist_all[warp];
  const Arena A = arena_of(P, warp_global);
  const double a2 = __dmul_rn(P.alpha, P.alpha);
  const float rinv = *P.rinv32;
  const float vx32 = P.pca ? __double2float_rn(P.sigma[2]) : 0.f, vy32 = P.pca ? __double2float_rn(P.sigma[3]) : 0.f;
  const unsigned n_list = *P.list_count;
  for (;;) {
    unsigned task = 0;
    if (lane == 0) task = atomicAdd(P.task_counter, 1u);
    task = __shfl_sync(0xFFFFFFFFu, task, 0);
    if (task >= n_list) break;
    const long long d = P.list[task];
    const int n = P.dom_piece_cnt[d];
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
    float edom = 0.f;  // largest error bound of a PCA key of the domain
    for (int i = lane; i < n; i += 32) {
      unsigned mh;
      const float x = x32_of(P, plen[i]);
      const float y = f64_to_f32_trunc(pinc[i], mh) * rinv;
      const float k = key32f(P, x, y, vx32, vy32);
      A.X[i] = x;
      A.Y[i] = y;
      A.key[i] = key_bits(k);
      A.sidx[i] = i;
      A.label[i] = -1;
      if (P.pca) edom = fmaxf(edom, pca_err(x, y, k));
    }
    for (int o = 16; o > 0; o >>= 1) edom = fmaxf(edom, __shfl_xor_sync(0xFFFFFFFFu, edom, o));
    __syncwarp();
    // 2. sort by (key32, position)
    if (n > 1) warp_radix_sort(A.key, A.sidx, A.tk, A.tv, n, hist);
    __syncwarp();
    // 3. runs of overlapping key intervals: re-sort by the binary64 keys
    fix_runs<int>(P, plen, pinc, A.key, A.sidx, n, (double*)hist, edom);
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
        const float T = scan_bound(P, xs, ys, vx32, vy32);
        if (lane == 0) A.label[ps] = G;
        for (int b0 = a + 1; b0 < n; b0 += 32) {
          const int b = b0 + lane;
          bool stop = true;
          if (b < n) {
            const int pb = A.sidx[b];
            const float xb = A.X[pb], yb = A.Y[pb];
            stop = past_bound(P, xb, yb, T, vx32, vy32);
            if (!stop) {
              if (A.label[pb] < 0) {
                int w = filter_within(xs, ys, xb, yb, P.a2lo, P.a2hi);
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
}

// ------------------------------------------------------------------ shared-memory tiles
// Domains of at most CAP pieces: W warps own one domain at a time with every
// per-piece array in shared memory (W = 1: several independent warps per CTA).
// The W warps share the sort, the sums and the greedy's window passes (the
// starts follow one another; each start's window is scanned 32 W pieces per
// step, one ballot per warp and one barrier per step).  Domains are routed to
// the smallest tile that holds them (k_local_classify), so small domains run
// many warps per SM.  After the sort, the W * 512 histogram bytes serve as
// scratch: the binary64 keys of an overlapping-key run, then the greedy's
// per-warp next-start candidates.
//
// Per-tile shared memory: W * 512 histogram bytes, then per piece 4 B key
// (later sY), 4 B sort temp (later sX), 2 B position, 2 B sort temp (later
// the label by sorted index), and 128 misc bytes: 12 B per piece, so the
// 2,048-piece tile of 4 warps fits 8 CTAs per SM.  The FP32 key of a piece is
// recomputed from (sX, sY) by the same expression that produced the sorted
// key, so it is not kept; after the greedy the 8 CAP bytes of sX/sY hold the
// group accumulators (24 B per group, CAP / 4 per pass: 6 CAP bytes) and the
// labels by position (the last 2 CAP bytes).
template <int W, int CAP>
struct TileCfg {
  static constexpr int kThreads = 32 * W;
  static constexpr size_t kBytes = (size_t)W * 512 + (size_t)CAP * 12 + 128;
  // W = 1: independent warps per CTA, as many as fit in ~56 KB (at most 8)
  static constexpr int kTilesPerCta = W > 1 ? 1 : (57344 / (int)kBytes < 1 ? 1 : (57344 / (int)kBytes > 8 ? 8 : 57344 / (int)kBytes));
  static constexpr int kBlock = kThreads * kTilesPerCta;
  static constexpr int kGroupsPerPass = CAP / 4;
};

// Accumulator of one group during the sums: the increments' 2^-64
// fixed-point images (magnitudes below 2^96 under the range contract) in two
// 48-bit limbs, each summed as a signed 64-bit integer (deferred carries: at
// most 4,096 members, so below 2^60), and the member count and length sum
// packed in one word (count << 40 | lensum: a domain of a series has fewer
// than 2^31 intervals): three shared-memory atomics per piece.
struct GroupAcc {
  long long lo48, hi48;
  unsigned long long cnt_len;
};

// 192-bit two's complement value of lo + hi 2^48 (both signed).
__device__ __forceinline__ I192 from_limbs48(long long lo, long long hi) {
  I192 r;
  r.w0 = (u64)lo;
  r.w1 = lo < 0 ? ~0ull : 0ull;
  r.w2 = r.w1;
  const u64 h0 = (u64)hi << 48, h1 = (u64)(hi >> 16), h2 = hi < 0 ? ~0ull : 0ull;  // hi 2^48, sign-extended
  add192(r, h0, h1, h2);
  return r;
}

// Synchronization of the W warps that own one domain.
template <int W>
__device__ __forceinline__ void tile_sync() {
  if (W == 1) __syncwarp(); else __syncthreads();
}
template <int W>
__device__ __forceinline__ bool tile_sync_or(bool p) {
  if (W == 1) {
    __syncwarp();
    return __any_sync(0xFFFFFFFFu, p);
  }
  return __syncthreads_or(p) != 0;
}


// Stable LSD radix sort of (key, val) by key with 8-bit digits over the W
// warps of a tile: warp w ranks the contiguous segment [w seg, (w+1) seg) of
// the input into digit-major, warp-minor positions, so equal digits keep
// their input order.  Thread t owns the 256 / (32 W) consecutive digits
// starting at t * 256 / (32 W) for the offset scan.  hist: W x 256 16-bit
// counters (a tile holds at most 4,096 pieces; counts are added through the
// 32-bit word that holds two counters); wsum: W words.  The result is back in
// (key, val) after four passes.
template <int W>
__device__ void tile_radix_sort16(unsigned* key, unsigned short* val, unsigned* tk, unsigned short* tv, int n,
                                  unsigned short* hist, unsigned* wsum) {
  constexpr int T = 32 * W;
  constexpr int PER = 256 / T;
  static_assert(PER * T == 256, "W must divide 8");
  const int lane = threadIdx.x & 31, w = (threadIdx.x >> 5) % W;
  const int t = threadIdx.x % T;
  const unsigned lt = (1u << lane) - 1u;
  const int seg = (((n + W - 1) / W) + 31) & ~31;
  const int lo = w * seg;
  const int hi = min(n, lo + seg);
  unsigned short* h = hist + w * 256;
  unsigned* hw = (unsigned*)h;  // the same counters, two per word
  unsigned* kin = key;
  unsigned short* vin = val;
  unsigned* kout = tk;
  unsigned short* vout = tv;
  for (int shift = 0; shift < 32; shift += 8) {
    for (int i = lane; i < 128; i += 32) hw[i] = 0;
    __syncwarp();
    for (int i = lo + lane; i < hi; i += 32) {
      const unsigned d = (kin[i] >> shift) & 255u;
      atomicAdd(&hw[d >> 1], 1u << (16 * (d & 1u)));
    }
    tile_sync<W>();
    {
      const int d0 = t * PER;
      unsigned tot[PER];
      unsigned sum = 0;
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        unsigned run = 0;
        for (int v = 0; v < W; ++v) {
          const unsigned c = hist[v * 256 + d0 + k];
          hist[v * 256 + d0 + k] = (unsigned short)run;
          run += c;
        }
        tot[k] = run;
        sum += run;
      }
      unsigned incl = sum;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
      }
      unsigned before = 0;
      if (W > 1) {
        if (lane == 31) wsum[w] = incl;
        tile_sync<W>();
        for (int v = 0; v < w; ++v) before += wsum[v];
      }
      unsigned ex = before + incl - sum;
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        for (int v = 0; v < W; ++v) hist[v * 256 + d0 + k] = (unsigned short)(hist[v * 256 + d0 + k] + ex);
        ex += tot[k];
      }
    }
    tile_sync<W>();
    for (int i0 = lo; i0 < hi; i0 += 32) {
      const int i = i0 + lane;
      const bool v = i < hi;
      const unsigned k = v ? kin[i] : 0u;
      const unsigned short vv = v ? vin[i] : 0;
      const unsigned d = v ? ((k >> shift) & 255u) : 256u + lane;
      const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
      const unsigned r = __popc(peers & lt);
      if (v) {
        const unsigned pos = h[d] + r;
        kout[pos] = k;
        vout[pos] = vv;
      }
      __syncwarp();
      if (v && r == 0) h[d] = (unsigned short)(h[d] + __popc(peers));
      __syncwarp();
    }
    tile_sync<W>();
    unsigned* tt = kin; kin = kout; kout = tt;
    unsigned short* tq = vin; vin = vout; vout = tq;
  }
}

template <int W, int CAP>
__global__ void __launch_bounds__(TileCfg<W, CAP>::kBlock) k_local_tile(LocalParams P, const int* list,
                                                                        const unsigned* list_count,
                                                                        unsigned* task_counter) {
  using Cfg = TileCfg<W, CAP>;
  constexpr int T = Cfg::kThreads;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int tile = threadIdx.x / T;          // W == 1: one tile per warp
  const int t = threadIdx.x % T;
  unsigned char* base = smem_raw + (size_t)tile * Cfg::kBytes;
  unsigned short* hist = (unsigned short*)base;                      // W * 256 16-bit counters
  unsigned* key = (unsigned*)(base + W * 512);                       // [CAP] sorted keys, then sY
  unsigned* tk = key + CAP;                                          // [CAP] sort temp, then sX
  unsigned short* idx = (unsigned short*)(tk + CAP);                 // [CAP] sorted index -> position
  unsigned short* tv = idx + CAP;                                    // [CAP] sort temp, then labels by sorted index
  int* misc = (int*)(tv + CAP);                                      // 32 words
  short* lab = (short*)tv;
  float* sX = (float*)tk;
  float* sY = (float*)key;
  GroupAcc* acc = (GroupAcc*)key;                                    // after the greedy: CAP / 4 groups (6 CAP bytes)
  short* plab = (short*)((unsigned char*)key + 6 * CAP);             // after the greedy: labels by position
  unsigned* wsum = (unsigned*)(misc + 4);                            // [W] sort scan
  long long* gbase_s = (long long*)(misc + 16);                      // group record base
  const double a2 = __dmul_rn(P.alpha, P.alpha);
  const float rinv = *P.rinv32;
  const float vx32 = P.pca ? __double2float_rn(P.sigma[2]) : 0.f, vy32 = P.pca ? __double2float_rn(P.sigma[3]) : 0.f;
  const unsigned n_list = *list_count;
  for (;;) {
    unsigned task = 0;
    if (t == 0) task = atomicAdd(task_counter, 1u);
    if (W == 1) {
      task = __shfl_sync(0xFFFFFFFFu, task, 0);
    } else {
      if (t == 0) {
        misc[12] = (int)task;
        misc[14] = 0;  // the domain's largest PCA key error bound (FP32 bits)
      }
      __syncthreads();
      task = (unsigned)misc[12];
      __syncthreads();
    }
    if (task >= n_list) break;
    const int d = list[task];
    const int n = P.dom_piece_cnt[d];
    const long long slot = P.dom_slot_off[d];
    const int* plen = P.piece_len + slot;
    const double* pinc = P.piece_inc + slot;
    // 1. FP32 keys by position (the loads of four pieces in flight together)
    float edom = 0.f;
    for (int i0 = t; i0 < n; i0 += 4 * T) {
      int L4[4];
      double I4[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * T;
        L4[u] = i < n ? plen[i] : 0;
        I4[u] = i < n ? pinc[i] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * T;
        if (i < n) {
          unsigned mh;
          const float x = x32_of(P, L4[u]);
          const float y = f64_to_f32_trunc(I4[u], mh) * rinv;
          const float k = key32f(P, x, y, vx32, vy32);
          key[i] = key_bits(k);
          idx[i] = (unsigned short)i;
          if (P.pca) edom = fmaxf(edom, pca_err(x, y, k));
        }
      }
    }
    if (P.pca) {
      for (int o = 16; o > 0; o >>= 1) edom = fmaxf(edom, __shfl_xor_sync(0xFFFFFFFFu, edom, o));
      if (W > 1 && lane == 0) atomicMax(&misc[14], __float_as_int(edom));
    }
    tile_sync<W>();
    if (W > 1 && P.pca) edom = __int_as_float(misc[14]);
    // 2. sort by (key32, position)
    if (n > 1) tile_radix_sort16<W>(key, idx, tk, tv, n, hist, wsum);
    tile_sync<W>();
    // 3. runs of overlapping key intervals: re-sort by the binary64 keys (rare;
    // the whole tile first checks whether any neighbouring pair overlaps)
    {
      bool ov = false;
      for (int a = t; a + 1 < n; a += T) ov = ov || keys_overlap32(P, key[a], key[a + 1], edom);
      if (tile_sync_or<W>(ov)) {
        if (t < 32) fix_runs<unsigned short>(P, plen, pinc, key, idx, n, (double*)hist, edom);
        tile_sync<W>();
      }
    }
    // 4. coordinates in key order (gathered again from the pieces, which are
    // in L1/L2), over the keys and the sort temp
    for (int a0 = t; a0 < n; a0 += 4 * T) {
      int L4[4];
      double I4[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int a = a0 + u * T;
        const int p = a < n ? idx[a] : 0;
        L4[u] = a < n ? plen[p] : 0;
        I4[u] = a < n ? pinc[p] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int a = a0 + u * T;
        if (a < n) {
          unsigned mh;
          sX[a] = x32_of(P, L4[u]);
          sY[a] = f64_to_f32_trunc(I4[u], mh) * rinv;
          lab[a] = -1;
        }
      }
    }
    tile_sync<W>();
    // 5. greedy in key order.  One warp (W = 1): each start's window pass
    // also finds the first piece left free behind the start (the next
    // start).  W warps: every window step covers 32 W pieces and the warps
    // agree on the stop and on the next start with one barrier per step.
    if constexpr (W == 1) {
      if (t < 32) {
        int G = 0, a = 0;
        while (a < n) {
          const float xs = sX[a], ys = sY[a];
          const float Tk = scan_bound(P, xs, ys, vx32, vy32);
          if (lane == 0) lab[a] = (short)G;
          int next = n;
          int b0 = a + 1;
          for (; b0 < n; b0 += 32) {
            const int b = b0 + lane;
            bool stop = true, fr = false;
            if (b < n) {
              const float xb = sX[b], yb = sY[b];
              stop = past_bound(P, xb, yb, Tk, vx32, vy32);
              if (lab[b] < 0) {
                bool join = false;
                if (!stop) {
                  int w = filter_within(xs, ys, xb, yb, P.a2lo, P.a2hi);
                  if (w == 2) {
                    const int ps = idx[a], pb = idx[b];
                    w = exact_within(P, plen[ps], pinc[ps], plen[pb], pinc[pb], a2) ? 1 : 0;
                  }
                  join = w != 0;
                }
                if (join) lab[b] = (short)G;
                else fr = true;
              }
            }
            const unsigned mf = __ballot_sync(0xFFFFFFFFu, fr);
            if (mf && next == n) next = b0 + __ffs(mf) - 1;
            if (__any_sync(0xFFFFFFFFu, stop)) break;
          }
          // nothing left free up to the window's last chunk: search on
          if (next == n) {
            for (b0 += 32; b0 < n; b0 += 32) {
              const int b = b0 + lane;
              const unsigned mf = __ballot_sync(0xFFFFFFFFu, b < n && lab[b] < 0);
              if (mf) {
                next = b0 + __ffs(mf) - 1;
                break;
              }
            }
          }
          __syncwarp();
          ++G;
          a = next;
        }
        if (lane == 0) misc[13] = G;
      }
    } else {
      // each warp publishes its first free piece behind the start before every
      // step's barrier; after the last one every thread takes the minimum.
      // Two slots by start parity: a slot is written again only after the
      // next start's barrier, which every reader of it has passed.
      int* cand = (int*)hist;  // [2][W] (the sort's histograms are free now)
      int* srch = misc + 20;   // [2] first free piece found beyond the window
      const int warp = t >> 5;
      int G = 0, a = 0;
      while (a < n) {
        const int sl = G & 1;
        const float xs = sX[a], ys = sY[a];
        const float Tk = scan_bound(P, xs, ys, vx32, vy32);
        if (t == 0) {
          lab[a] = (short)G;
          srch[sl] = n;
        }
        int next = n;  // this warp's first free piece
        int b0 = a + 1;
        const bool stepped = b0 < n;
        for (; b0 < n; b0 += T) {
          const int b = b0 + t;
          bool stop = true, fr = false;
          if (b < n) {
            const float xb = sX[b], yb = sY[b];
            stop = past_bound(P, xb, yb, Tk, vx32, vy32);
            if (lab[b] < 0) {
              bool join = false;
              if (!stop) {
                int w = filter_within(xs, ys, xb, yb, P.a2lo, P.a2hi);
                if (w == 2) {
                  const int ps = idx[a], pb = idx[b];
                  w = exact_within(P, plen[ps], pinc[ps], plen[pb], pinc[pb], a2) ? 1 : 0;
                }
                join = w != 0;
              }
              if (join) lab[b] = (short)G;
              else fr = true;
            }
          }
          const unsigned mf = __ballot_sync(0xFFFFFFFFu, fr);
          if (mf && next == n) next = b0 + warp * 32 + __ffs(mf) - 1;
          if (lane == 0) cand[sl * W + warp] = next;
          if (__syncthreads_or(stop)) break;
        }
        int nx = n;
        if (stepped) {
#pragma unroll
          for (int w = 0; w < W; ++w) nx = min(nx, cand[sl * W + w]);
          if (nx == n) {
            // nothing left free up to the window's last step: search on
            for (b0 += T; b0 < n; b0 += T) {
              const int b = b0 + t;
              const unsigned mf = __ballot_sync(0xFFFFFFFFu, b < n && lab[b] < 0);
              if (mf && lane == 0) atomicMin(&srch[sl], b0 + warp * 32 + __ffs(mf) - 1);
              if (__syncthreads_or(mf != 0)) break;
            }
            nx = srch[sl];
          }
        }
        ++G;
        a = nx;
      }
      if (t == 0) misc[13] = G;
    }
    tile_sync<W>();
    const int G = misc[13];
    // 6. labels by position, written out coalesced
    for (int a = t; a < n; a += T) plab[idx[a]] = lab[a];
    tile_sync<W>();
    for (int i = t; i < n; i += T) P.local_label[slot + i] = plab[i];
    // 7. exact group sums (shared-memory atomics) and the group records
    if (t == 0) {
      long long gb = (long long)atomicAdd((unsigned long long*)P.n_groups, (unsigned long long)G);
      if (gb + G > P.group_capacity) {
        set_status(P.status, JABBA_ERR_CAPACITY);
        gb = -1;
      }
      *gbase_s = gb;
      P.dom_group_cnt[d] = G;
    }
    tile_sync<W>();
    const long long gbase = *gbase_s;
    if (gbase >= 0) {
      for (int g0 = 0; g0 < G; g0 += Cfg::kGroupsPerPass) {
        const int gn = min(G - g0, Cfg::kGroupsPerPass);
        for (int g = t; g < gn; g += T) {
          acc[g].lo48 = 0;
          acc[g].hi48 = 0;
          acc[g].cnt_len = 0;
        }
        tile_sync<W>();
        // four pieces' loads in flight together, then their atomics
        for (int i0 = t; i0 < n; i0 += 4 * T) {
          int L4[4], g4[4];
          double I4[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * T;
            g4[u] = i < n ? plab[i] - g0 : -1;
            L4[u] = i < n ? plen[i] : 0;
            I4[u] = i < n ? pinc[i] : 0.0;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int g = g4[u];
            if (g < 0 || g >= gn) continue;
            bool neg;
            const U128 m = fx_mag(I4[u], neg);          // < 2^96 under the range contract
            long long l0 = (long long)(m.lo & 0xFFFFFFFFFFFFull);
            long long l1 = (long long)((m.lo >> 48) | (m.hi << 16));
            if (neg) { l0 = -l0; l1 = -l1; }
            atomicAdd((unsigned long long*)&acc[g].lo48, (unsigned long long)l0);
            atomicAdd((unsigned long long*)&acc[g].hi48, (unsigned long long)l1);
            atomicAdd(&acc[g].cnt_len, (1ull << 40) | (unsigned long long)(unsigned)L4[u]);
          }
        }
        tile_sync<W>();
        for (int g = t; g < gn; g += T) {
          const I192 s = from_limbs48(acc[g].lo48, acc[g].hi48);
          const unsigned long long cl = acc[g].cnt_len;
          jabba_group rec;
          rec.inc[0] = s.w0;
          rec.inc[1] = s.w1;
          rec.inc[2] = s.w2;
          rec.lensum = (long long)(cl & ((1ull << 40) - 1));
          rec.count = (int)(cl >> 40);
          rec.local_id = g0 + g;
          rec.domain = d;
          rec.pad = 0;
          P.groups[gbase + g0 + g] = rec;
        }
        tile_sync<W>();
      }
    }
    tile_sync<W>();
  }
}

// Routes every domain to the kernel whose tile holds it: list k < kTiers
// holds the domains with kTierCap[k-1] < pieces <= kTierCap[k]; list kTiers
// the larger ones (the global-memory arena kernel).  Empty domains get no
// groups here.
constexpr int kTiers = 5;
constexpr int kTierCap0 = 256, kTierCap1 = 512, kTierCap2 = 1024, kTierCap3 = 2048, kTierCap4 = 4096;

__global__ void k_local_classify(const int* dom_piece_cnt, long long n_domains, int* dom_group_cnt, int* lists,
                                 long long list_stride, unsigned* list_count) {
  const int lane = threadIdx.x & 31;
  for (long long d0 = (long long)blockIdx.x * blockDim.x; d0 < n_domains; d0 += (long long)gridDim.x * blockDim.x) {
    const long long d = d0 + threadIdx.x;
    int tier = -1;
    if (d < n_domains) {
      const int n = dom_piece_cnt[d];
      if (n == 0) dom_group_cnt[d] = 0;
      else tier = n <= kTierCap0 ? 0 : n <= kTierCap1 ? 1 : n <= kTierCap2 ? 2 : n <= kTierCap3 ? 3 : n <= kTierCap4 ? 4 : 5;
    }
    for (int k = 0; k <= kTiers; ++k) {
      const unsigned m = __ballot_sync(0xFFFFFFFFu, tier == k);
      if (!m) continue;
      const int leader = __ffs(m) - 1;
      unsigned b = 0;
      if (lane == leader) b = atomicAdd(&list_count[k], (unsigned)__popc(m));
      b = __shfl_sync(0xFFFFFFFFu, b, leader);
      if (tier == k) lists[k * list_stride + b + __popc(m & ((1u << lane) - 1u))] = (int)d;
    }
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

__global__ void k_set_one(unsigned* p) { *p = 1u; }

// Plain form: list[d] = d, and no groups for empty domains.
__global__ void k_local_plain_prep(const int* dom_piece_cnt, long long n_domains, int* dom_group_cnt, int* list) {
  for (long long d = (long long)blockIdx.x * blockDim.x + threadIdx.x; d < n_domains; d += (long long)gridDim.x * blockDim.x) {
    list[d] = (int)d;
    if (dom_piece_cnt[d] == 0) dom_group_cnt[d] = 0;
  }
}
__global__ void k_set_status(unsigned* status, unsigned code) { set_status(status, code); }

// One launch of a tile kernel for a single domain (the plain form): one CTA
// holding one tile.
template <int W, int CAP>
static void launch_tile_one(const LocalParams& P, const int* list, const unsigned* one, unsigned* ctr,
                            cudaStream_t st) {
  using Cfg = TileCfg<W, CAP>;
  static PerDevice attr;
  attr.get([] {
    cudaFuncSetAttribute(k_local_tile<W, CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)((Cfg::kBlock / Cfg::kThreads) * Cfg::kBytes));
    return 1;
  });
  k_local_tile<W, CAP><<<1, Cfg::kThreads, Cfg::kBytes, st>>>(P, list, one, ctr);
}

template <int W, int CAP>
static void launch_tile(const LocalParams& P, const int* list, const unsigned* cnt, unsigned* ctr, int num_sms,
                        int cap_per_sm, cudaStream_t st) {
  using Cfg = TileCfg<W, CAP>;
  constexpr int kBlock = Cfg::kBlock;
  constexpr size_t kSmem = (size_t)(kBlock / Cfg::kThreads) * Cfg::kBytes;
  static PerDevice occ;
  const int blocks_per_sm = occ.get([] {
    cudaFuncSetAttribute(k_local_tile<W, CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_local_tile<W, CAP>, kBlock, kSmem);
    return b < 1 ? 1 : b;
  });
  const int per_sm = cap_per_sm > 0 && cap_per_sm < blocks_per_sm ? cap_per_sm : blocks_per_sm;
  k_local_tile<W, CAP><<<(unsigned)(num_sms * per_sm), kBlock, kSmem, st>>>(P, list, cnt, ctr);
}

void launch_local(const int* piece_len, const double* piece_inc, const long long* dom_slot_off,
                  const int* dom_piece_cnt, long long n_domains, const double* sigma, double alpha, double scl,
                  int key_mode, int* local_label, int* dom_group_cnt, long long* dom_group_off, jabba_group* groups,
                  long long group_capacity, long long* n_groups, Scratch& ws, unsigned* status, cudaStream_t st) {
  // loc_ctr[0..5]: list sizes of the tiers and the arena; [8..13]: their task counters
  unsigned* list_cnt = ws.loc_ctr;
  unsigned* task_ctr = ws.loc_ctr + 8;
  cudaMemsetAsync(n_groups, 0, sizeof(long long), st);
  cudaMemsetAsync(ws.loc_ctr, 0, 16 * sizeof(unsigned), st);
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
  P.pca = key_mode == 1 ? 1 : 0;
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
  P.task_counter = task_ctr + kTiers;
  P.list = ws.loc_list + kTiers * ws.loc_stride;
  P.list_count = list_cnt + kTiers;
  P.arena = ws.arena;
  P.cap_items = ws.cap_items;
  if (n_domains > 0) {
    const unsigned g = (unsigned)(ws.num_sms * 4);
    if (ws.tune.per_domain_launch) {
      // the plain form: one launch per domain, its tile chosen on the host from
      // the piece count (read back); the list entries are 0..D-1
      unsigned* one = ws.counters + 15;
      k_local_plain_prep<<<g, 256, 0, st>>>(dom_piece_cnt, n_domains, dom_group_cnt, ws.loc_list);
      k_set_one<<<1, 1, 0, st>>>(one);
      cudaMemsetAsync(ws.plain_ctr, 0, sizeof(unsigned) * (size_t)n_domains, st);
      int* cnt_h = (int*)malloc(sizeof(int) * (size_t)n_domains);
      if (!cnt_h) {
        k_set_status<<<1, 1, 0, st>>>(status, JABBA_ERR_CUDA);
      } else {
        cudaMemcpyAsync(cnt_h, dom_piece_cnt, sizeof(int) * (size_t)n_domains, cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        for (long long dd = 0; dd < n_domains; ++dd) {
          const int n = cnt_h[dd];
          if (n == 0) continue;
          const int* l = ws.loc_list + dd;
          unsigned* c = ws.plain_ctr + dd;
          if (n <= kTierCap0) launch_tile_one<1, kTierCap0>(P, l, one, c, st);
          else if (n <= kTierCap1) launch_tile_one<1, kTierCap1>(P, l, one, c, st);
          else if (n <= kTierCap2) launch_tile_one<4, kTierCap2>(P, l, one, c, st);
          else if (n <= kTierCap3) launch_tile_one<4, kTierCap3>(P, l, one, c, st);
          else if (n <= kTierCap4) launch_tile_one<8, kTierCap4>(P, l, one, c, st);
          else {
            LocalParams Q = P;
            Q.list = l;
            Q.list_count = one;
            Q.task_counter = c;
            k_local_warp<<<1, 32 * kLocWarps, 0, st>>>(Q);
          }
        }
        free(cnt_h);
      }
      exclusive_scan<int>(dom_group_cnt, n_domains, dom_group_off, ws.scan_tiles, st);
      return;
    }
    k_local_classify<<<g, 256, 0, st>>>(dom_piece_cnt, n_domains, dom_group_cnt, ws.loc_list, ws.loc_stride,
                                        list_cnt);
    TierEvents* te = ws.tier_ev;
    const long long L = ws.loc_stride;
    const int ns = ws.num_sms;
    launch_tile<1, kTierCap0>(P, ws.loc_list, list_cnt + 0, task_ctr + 0, ns, ws.tune.local_ctas_cap, st);
    launch_tile<1, kTierCap1>(P, ws.loc_list + L, list_cnt + 1, task_ctr + 1, ns, ws.tune.local_ctas_cap, st);
    if (te) cudaEventRecord(te->ev[0][0], st);
    {
      const int* l2 = ws.loc_list + 2 * L;
      if (ws.tune.local_k_warps == 4) launch_tile<4, kTierCap2>(P, l2, list_cnt + 2, task_ctr + 2, ns, ws.tune.local_ctas_cap, st);
      else launch_tile<1, kTierCap2>(P, l2, list_cnt + 2, task_ctr + 2, ns, ws.tune.local_ctas_cap, st);
    }
    if (te) cudaEventRecord(te->ev[0][1], st);
    if (te) cudaEventRecord(te->ev[1][0], st);
    {
      const int* l3 = ws.loc_list + 3 * L;
      switch (ws.tune.local_mid_warps) {
        case 1: launch_tile<1, kTierCap3>(P, l3, list_cnt + 3, task_ctr + 3, ns, ws.tune.local_ctas_cap, st); break;
        case 2: launch_tile<2, kTierCap3>(P, l3, list_cnt + 3, task_ctr + 3, ns, ws.tune.local_ctas_cap, st); break;
        case 8: launch_tile<8, kTierCap3>(P, l3, list_cnt + 3, task_ctr + 3, ns, ws.tune.local_ctas_cap, st); break;
        default: launch_tile<4, kTierCap3>(P, l3, list_cnt + 3, task_ctr + 3, ns, ws.tune.local_ctas_cap, st); break;
      }
    }
    if (te) cudaEventRecord(te->ev[1][1], st);
    if (te) cudaEventRecord(te->ev[2][0], st);
    {
      const int* l4 = ws.loc_list + 4 * L;
      if (ws.tune.local_big_warps == 8) launch_tile<8, kTierCap4>(P, l4, list_cnt + 4, task_ctr + 4, ns, ws.tune.local_ctas_cap, st);
      else launch_tile<4, kTierCap4>(P, l4, list_cnt + 4, task_ctr + 4, ns, ws.tune.local_ctas_cap, st);
    }
    if (te) cudaEventRecord(te->ev[2][1], st);
    k_local_warp<<<(unsigned)ws.loc_ctas, kLocWarps * 32, 0, st>>>(P);
  }
  exclusive_scan<int>(dom_group_cnt, n_domains, dom_group_off, ws.scan_tiles, st);
}

long long local_arena_words(long long cap_items, long long n_warps) { return kArenaWords * cap_items * n_warps; }
int local_warps_per_cta() { return kLocWarps; }

}  // namespace jabba
