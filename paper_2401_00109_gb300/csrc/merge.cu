// merge.cu -- Stage II of the two-stage digitization (Sec. 5): the local
// groups, taken at their centres (or at given points: the starting points of
// the block form at the end of this file), are aggregated once more by the
// same greedy (Sec. 3.2); the result maps every local group to a global
// group, and the dictionary entries are the exact means of their member
// pieces.
//
// The greedy in key order is the lexicographically first maximal set of
// "starts" pairwise farther than alpha apart; every other item joins the
// earliest start within alpha.  It is computed in parallel:
//  1. FP32 centre coordinates: the binary64 centres rounded to nearest
//     (binary64 values are recomputed only for undecided comparisons);
//  2. the exact order: a stable radix sort of the binary64 keys (computed
//     once per item: at 10^7 centres the keys are denser than any FP32
//     interval), ties in compact-index order;
//  3. a uniform grid of cells of side h = alpha/2 (1 + 2^-7): two items in one
//     cell are within alpha, so a cell holds at most one start, and it is the
//     first of its items (in key order) not covered by an earlier start of a
//     neighbouring cell (within 2 cells);
//  4. rounds (one cooperative kernel, bounded grid barriers): each undecided
//     cell skips its items covered by known neighbouring starts; its next item
//     becomes a start once no undecided neighbouring item that precedes it in
//     key order lies within alpha (such an item could still become a start).
//     k_mrounds1 tests coverage on the fly (one barrier per round), k_mrounds
//     marks it between two barriers;
//  5. every item's label is the earliest start within alpha among the starts
//     of its 5 x 5 cell neighbourhood; global ids follow key order.
// If the coordinates span too many cells for the grid, or their error
// exceeds 2^-8 of a cell, a sequential single-CTA greedy on the binary64
// coordinates runs instead (same result).
#include <cooperative_groups.h>

#include "kernels.cuh"

namespace jabba {

// ------------------------------------------------------------------ binary64 definition
struct ExactCentre {
  double X, Y;
};

// Centre (lensum / count, round(inc) / count) normalised by Eq. 4, binary64.
__device__ __forceinline__ ExactCentre exact_centre(const jabba_group& g, double sl, double si, double scl) {
  I192 inc;
  inc.w0 = g.inc[0];
  inc.w1 = g.inc[1];
  inc.w2 = g.inc[2];
  const double cnt = (double)g.count;
  const double c_len = __ddiv_rn((double)g.lensum, cnt);
  const double c_inc = __ddiv_rn(i192_to_double(inc), cnt);
  ExactCentre e;
  e.X = __ddiv_rn(__dmul_rn(scl, c_len), sl);
  e.Y = __ddiv_rn(c_inc, si);
  return e;
}

// The sort key in binary64: X*X + Y*Y, or with the PCA key (pca = 1) the
// projection vx X + vy Y on the axis sigma[2..3].
__device__ __forceinline__ double exact_key(const ExactCentre& e, int pca, const double* sigma) {
  if (pca) return __dadd_rn(__dmul_rn(sigma[2], e.X), __dmul_rn(sigma[3], e.Y));
  return __dadd_rn(__dmul_rn(e.X, e.X), __dmul_rn(e.Y, e.Y));
}

// Order-preserving unsigned image of a binary64 key (negative PCA keys
// included): the sign bit set for non-negative values, every bit flipped for
// negative ones.  -0 is mapped as +0 (the two compare equal, so their order
// is that of equal keys: the compact index).
__device__ __forceinline__ unsigned long long key_image(double k) {
  if (k == 0.0) k = 0.0;
  const unsigned long long u = (unsigned long long)__double_as_longlong(k);
  return (u >> 63) ? ~u : (u | (1ull << 63));
}

__device__ __forceinline__ bool exact_within_c(const ExactCentre& a, const ExactCentre& b, double a2) {
  const double dx = __dsub_rn(b.X, a.X), dy = __dsub_rn(b.Y, a.Y);
  return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) <= a2;
}

struct MergeView {
  const jabba_group* groups;
  const int* rec;       // record of compact index c
  const int* sidx;      // compact index at sorted position a
  const float* sX;      // FP32 coordinates at sorted position a
  const float* sY;
  const double* sigma;  // binary64 sigma_len, sigma_inc
  const double* iX;     // item points by record (null: the records' centres)
  const double* iY;
  double scl, a2;
  float a2lo, a2hi;
};

// Binary64 point of record r: its centre, or the point given for it.
// ------------------------------------------------------------------ binary64 division on the integer units
// This GPU issues binary64 arithmetic at a small fraction of its integer
// rate, and the exact centre of every item takes four correctly rounded
// divisions, so k_mprep divides on the significands.  With a = ma 2^ea and
// b = mb 2^eb (ma, mb in [2^52, 2^53)) and s = [ma < mb], the quotient's
// 53-bit significand is Q = floor(ma 2^(52+s) / mb), rounded to nearest
// (ties to even) by the remainder R = ma 2^(52+s) - Q mb: up when 2R > mb,
// or 2R = mb and Q is odd; a carry out of 53 bits bumps the exponent.  Q is
// estimated as floor(ma v / 2^(64-s)) from v = floor(2^116 / mb), which lies
// below 2^116 / mb by less than 1, so the estimate errs by less than
// ma 2^(52+s) / 2^116 < 1: it is Q or Q - 1, and R (below 2 mb < 2^54) is
// exact in 64-bit arithmetic.  The result equals __ddiv_rn(a, b) wherever
// this path applies (a normal or zero, b positive normal, the quotient
// normal); elsewhere the caller divides in binary64.
struct DivRecip {
  u64 mb;  // the divisor's significand, [2^52, 2^53)
  u64 v;   // floor(2^116 / mb) (2^64 - 1 for mb = 2^52)
  int eb;  // the divisor is mb 2^eb
  int ok;  // the divisor is a positive normal number
};

// v = floor(2^116 / mb) by restoring division, one quotient bit per step
// (2^116 = 2^52 2^64 and 2^52 <= mb: the remainder starts at 2^52).
__device__ __forceinline__ u64 recip116(u64 mb) {
  u64 rem = 1ull << 52, v = 0;
  for (int i = 0; i < 64; ++i) {
    rem <<= 1;
    const u64 bit = rem >= mb ? 1ull : 0ull;
    rem -= bit ? mb : 0ull;
    v = (v << 1) | bit;
  }
  return v;
}

__device__ __forceinline__ DivRecip make_recip(double b) {
  const u64 bb = (u64)__double_as_longlong(b);
  const int be = (int)((bb >> 52) & 0x7FF);
  DivRecip r;
  r.ok = (bb >> 63) == 0 && be != 0 && be != 0x7FF;
  r.mb = (bb & ((1ull << 52) - 1)) | (1ull << 52);
  r.eb = be - 1075;
  r.v = recip116(r.mb);
  return r;
}

// The divisor c = 1 .. kRecipCnt (a member count) from its table entry v.
__device__ __forceinline__ DivRecip count_recip(int c, u64 v) {
  const int top = 31 - __clz(c);
  DivRecip r;
  r.mb = (u64)c << (52 - top);
  r.eb = top - 52;
  r.v = v;
  r.ok = 1;
  return r;
}

// a / b rounded to nearest even; false where the path does not apply.
__device__ __forceinline__ bool div_rn_int(double a, const DivRecip& r, double& q) {
  const u64 ab = (u64)__double_as_longlong(a);
  const u64 sign = ab & (1ull << 63);
  const int ae = (int)((ab >> 52) & 0x7FF);
  if (!r.ok || ae == 0x7FF) return false;
  if (ae == 0) {
    if ((ab << 1) != 0) return false;  // subnormal
    q = __longlong_as_double((long long)sign);  // +-0 / b
    return true;
  }
  const u64 ma = (ab & ((1ull << 52) - 1)) | (1ull << 52);
  const int s = ma < r.mb ? 1 : 0;
  const u64 hi = __umul64hi(ma, r.v), lo = ma * r.v;
  u64 Q = s ? ((hi << 1) | (lo >> 63)) : hi;
  long long R = (long long)((ma << (52 + s)) - Q * r.mb);
  if (R < 0) {
    Q -= 1;
    R += (long long)r.mb;
  } else if (R >= (long long)r.mb) {
    Q += 1;
    R -= (long long)r.mb;
  }
  const u64 R2 = (u64)R << 1;
  if (R2 > r.mb || (R2 == r.mb && (Q & 1ull))) Q += 1;
  int e = (ae - 1075) - r.eb - 52 - s;  // quotient = Q 2^e
  if (Q == (1ull << 53)) {
    Q >>= 1;
    ++e;
  }
  const int be = e + 52 + 1023;
  if (be <= 0 || be >= 0x7FF) return false;
  q = __longlong_as_double((long long)(sign | ((u64)be << 52) | (Q & ((1ull << 52) - 1))));
  return true;
}

// Reciprocals of the member counts 1 .. kRecipCnt (tab[c]) and of the two
// normalisation divisors sigma[0], sigma[1] (sig[0..1]).
__global__ void k_recip_tables(const double* sigma, u64* tab, DivRecip* sig, const int* flags) {
  if (flags[1]) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= 1 && c <= kRecipCnt) {
    const int top = 31 - __clz(c);
    tab[c] = recip116((u64)c << (52 - top));
  }
  if (c < 2) sig[c] = make_recip(sigma[c]);
}

// Self-check of div_rn_int against the binary64 division: counts[0] +=
// quotients the path handled, counts[1] += those that differ in any bit.
// mode 1: b[i] is a member count 1..kRecipCnt, divided through its table
// form (as the exact centres do).
__global__ void k_check_div(const double* a, const double* b, long long n, int mode, long long* counts) {
  long long handled = 0, bad = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    DivRecip r;
    if (mode == 1) {
      const int c = (int)b[i];
      if (!(b[i] >= 1.0 && b[i] <= (double)kRecipCnt) || (double)c != b[i]) continue;
      const int top = 31 - __clz(c);
      r = count_recip(c, recip116((u64)c << (52 - top)));
    } else {
      r = make_recip(b[i]);
    }
    double q;
    if (!div_rn_int(a[i], r, q)) continue;
    ++handled;
    if (__double_as_longlong(q) != __double_as_longlong(__ddiv_rn(a[i], b[i]))) ++bad;
  }
  for (int o = 16; o > 0; o >>= 1) {
    handled += __shfl_xor_sync(0xFFFFFFFFu, handled, o);
    bad += __shfl_xor_sync(0xFFFFFFFFu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd((unsigned long long*)&counts[0], (unsigned long long)handled);
    atomicAdd((unsigned long long*)&counts[1], (unsigned long long)bad);
  }
}

void launch_check_div(const double* a, const double* b, long long n, int mode, long long* counts, int num_sms,
                      cudaStream_t st) {
  cudaMemsetAsync(counts, 0, 2 * sizeof(long long), st);
  if (n > 0) k_check_div<<<(unsigned)(num_sms * 4), 256, 0, st>>>(a, b, n, mode, counts);
}

// exact_centre through div_rn_int: the same binary64 values (every division
// correctly rounded either way); false where a division leaves the path.
__device__ __forceinline__ bool exact_centre_int(const jabba_group& g, const u64* tab, const DivRecip& rsl,
                                                 const DivRecip& rsi, double scl, ExactCentre& e) {
  if (g.count < 1 || g.count > kRecipCnt || g.lensum < 1 || g.lensum >= (1ll << 53)) return false;
  const DivRecip rc = count_recip(g.count, tab[g.count]);
  const u64 L = (u64)g.lensum;  // exact in binary64
  const int top = 63 - __clzll((long long)L);
  const double len_d = __longlong_as_double((long long)(((u64)(top + 1023) << 52) | ((L << (52 - top)) & ((1ull << 52) - 1))));
  I192 inc;
  inc.w0 = g.inc[0];
  inc.w1 = g.inc[1];
  inc.w2 = g.inc[2];
  double c_len, c_inc, X, Y;
  if (!div_rn_int(len_d, rc, c_len) || !div_rn_int(i192_to_double(inc), rc, c_inc)) return false;
  if (!div_rn_int(scl == 1.0 ? c_len : __dmul_rn(scl, c_len), rsl, X) || !div_rn_int(c_inc, rsi, Y)) return false;
  e.X = X;
  e.Y = Y;
  return true;
}

__device__ __forceinline__ ExactCentre item_point(const jabba_group* groups, const double* iX, const double* iY,
                                                  long long r, const double* sigma, double scl) {
  if (iX) {
    ExactCentre e;
    e.X = iX[r];
    e.Y = iY[r];
    return e;
  }
  return exact_centre(groups[r], sigma[0], sigma[1], scl);
}

// 1 = within alpha, 0 = not, decided exactly when the FP32 interval straddles.
__device__ __noinline__ bool exact_within_sorted(const MergeView& V, int a, int b) {
  const ExactCentre ea = item_point(V.groups, V.iX, V.iY, V.rec[V.sidx[a]], V.sigma, V.scl);
  const ExactCentre eb = item_point(V.groups, V.iX, V.iY, V.rec[V.sidx[b]], V.sigma, V.scl);
  return exact_within_c(ea, eb, V.a2);
}

// FP32 filter on the coordinates rounded to nearest from binary64
// (|X32 - X| <= 2^-24 |X|, same for Y): the additive margin is twice the
// coordinate error, the factors cover the FP32 arithmetic here and the
// binary64 rounding of the definition's d^2.
__device__ __forceinline__ int filter_c(float xa, float ya, float xb, float yb, float a2lo, float a2hi) {
  const float dx = fabsf(xb - xa), dy = fabsf(yb - ya);
  const float ex = 0x1p-22f * (fabsf(xa) + fabsf(xb)) + 0x1p-126f;
  const float ey = 0x1p-22f * (fabsf(ya) + fabsf(yb)) + 0x1p-126f;
  const float hx = dx + ex, hy = dy + ey;
  const float lx = fmaxf(dx - ex, 0.f), ly = fmaxf(dy - ey, 0.f);
  const float hi = fmaf(hx, hx, hy * hy) * (1.0f + 0x1p-20f);
  const float lo = fmaf(lx, lx, ly * ly) * (1.0f - 0x1p-20f);
  if (hi < a2lo) return 1;
  if (lo > a2hi) return 0;
  return 2;
}

__device__ __forceinline__ bool within_sorted(const MergeView& V, int a, int b) {
  const int f = filter_c(V.sX[a], V.sY[a], V.sX[b], V.sY[b], V.a2lo, V.a2hi);
  if (f != 2) return f == 1;
  return exact_within_sorted(V, a, b);
}

__device__ __forceinline__ bool maybe_within_sorted(const MergeView& V, int a, int b) {
  return filter_c(V.sX[a], V.sY[a], V.sX[b], V.sY[b], V.a2lo, V.a2hi) != 0;
}

__device__ __forceinline__ long long clamp_groups(const long long* n_p, long long cap) {
  const long long g = *n_p;
  return g < cap ? g : cap;  // past capacity the records were not written (status already set)
}

// ------------------------------------------------------------------ 1. FP32 centres
// flags[0]: use the sequential fallback; bounds: float min/max encoded as ordered ints.
__device__ __forceinline__ int ord_of(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : (int)(0x80000000u - (unsigned)i) ;
}
__device__ __forceinline__ float of_ord(int o) {
  return o >= 0 ? __int_as_float(o) : __int_as_float((int)(0x80000000u - (unsigned)o));
}

__global__ void k_mprep(const jabba_group* groups, const double* iX, const double* iY, const long long* n_p,
                        long long cap, const long long* dom_group_off, const double* sigma, double scl, int pca,
                        unsigned long long* keys, int* vals, int* rec_of, float* X32, float* Y32, int* bounds,
                        const int* flags, const u64* rtab, const DivRecip* rsig) {
  if (flags[1]) return;
  const long long G = clamp_groups(n_p, cap);
  const DivRecip rsl = rsig[0], rsi = rsig[1];
  int mnx = 0x7FFFFFFF, mxx = -0x7FFFFFFF, mny = 0x7FFFFFFF, mxy = -0x7FFFFFFF;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < G; r += (long long)gridDim.x * blockDim.x) {
    const jabba_group g = groups[r];
    const long long c = dom_group_off[g.domain] + g.local_id;
    // the order needs the binary64 key itself (2e7 centres are denser than
    // any FP32 key interval), so every item computes its binary64 centre
    // (4 divisions, once, on the integer units where they apply); the FP32
    // coordinates are that centre rounded to nearest (relative error 2^-24)
    ExactCentre e;
    if (iX || !exact_centre_int(g, rtab, rsl, rsi, scl, e)) e = item_point(groups, iX, iY, r, sigma, scl);
    const float x = __double2float_rn(e.X), y = __double2float_rn(e.Y);
    X32[c] = x;
    Y32[c] = y;
    keys[c] = key_image(exact_key(e, pca, sigma));
    vals[c] = (int)c;
    rec_of[c] = (int)r;
    mnx = min(mnx, ord_of(x));
    mxx = max(mxx, ord_of(x));
    mny = min(mny, ord_of(y));
    mxy = max(mxy, ord_of(y));
  }
  for (int o = 16; o > 0; o >>= 1) {
    mnx = min(mnx, __shfl_xor_sync(0xFFFFFFFFu, mnx, o));
    mxx = max(mxx, __shfl_xor_sync(0xFFFFFFFFu, mxx, o));
    mny = min(mny, __shfl_xor_sync(0xFFFFFFFFu, mny, o));
    mxy = max(mxy, __shfl_xor_sync(0xFFFFFFFFu, mxy, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&bounds[0], mnx);
    atomicMax(&bounds[1], mxx);
    atomicMin(&bounds[2], mny);
    atomicMax(&bounds[3], mxy);
  }
}

// ------------------------------------------------------------------ LSD radix sort (stable)
// 8-bit digits over tiles of kRsTile items, one kernel per pass (the
// decoupled look-back scheme): the CTAs take tiles in increasing order from a
// counter; each counts its tile's digits, publishes the counts, and every
// digit's thread walks back over the earlier tiles' published counts (or
// their inclusive prefixes, once known) to find where the tile's run of that
// digit starts; the global start of each digit comes from one histogram
// kernel per sort that counts all passes' digits at once.  A tile waits only
// on tiles taken before it, so the waits end; every wait is bounded.  The
// tile's items are ranked stably (warp w owns items [w 256, (w+1) 256); ranks
// from ballots on the digit bits), reordered by digit in shared memory and
// written run by run with consecutive threads on consecutive addresses.
//
// Published words (64 bits): tag (31) | state (2: 1 = tile count, 2 =
// inclusive prefix) | value (31; counts are below the group capacity, which
// is below 2^31).  The tag is (sort epoch * 8 + pass), counted from 1, and the
// epoch sits at a fixed place ahead of the status words: a word left by an
// earlier sort or pass (of any size) does not match until the tags wrap after
// 2^28 sorts, so the status array (zeroed when allocated) needs no clearing
// between sorts.
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsPerLane = 8;
constexpr int kRsPerWarp = 32 * kRsPerLane;
constexpr int kRsTile = kRsWarps * kRsPerWarp;  // 2048
constexpr int kRsPasses = 8;

struct RsScratch {
  unsigned long long* status;  // [n_tiles][256]
  unsigned* ghist;             // [kRsPasses][256] digit counts of all items
  unsigned* gbase;             // [kRsPasses][256] exclusive digit starts
  unsigned* tile_ctr;          // [kRsPasses]
  unsigned* epoch;             // [1]
};

template <typename KeyT>
__global__ void __launch_bounds__(256) k_rs_global_hist(const KeyT* keys, const long long* n_p,
                                                       long long cap, int passes, unsigned* ghist,
                                                       const int* flags) {
  __shared__ unsigned h[kRsPasses][256];
  const long long n = flags[1] ? 0 : clamp_groups(n_p, cap);
  for (int i = threadIdx.x; i < kRsPasses * 256; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const KeyT k = keys[i];
    for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(unsigned)(k >> (8 * p)) & 255u], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * 256; i += blockDim.x) {
    const unsigned v = (&h[0][0])[i];
    if (v) atomicAdd(&ghist[i], v);
  }
}

// Exclusive digit starts of every pass (one warp per pass); a new sort epoch.
__global__ void k_rs_bases(const unsigned* ghist, int passes, unsigned* gbase, unsigned* tile_ctr, unsigned* epoch) {
  const int lane = threadIdx.x & 31, p = threadIdx.x >> 5;
  if (p < passes) {
    unsigned carry = 0;
    for (int d0 = 0; d0 < 256; d0 += 32) {
      const unsigned v = ghist[p * 256 + d0 + lane];
      unsigned incl = v;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
      }
      gbase[p * 256 + d0 + lane] = carry + incl - v;
      carry += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
    if (lane == 0) tile_ctr[p] = 0;
  }
  if (threadIdx.x == 0) *epoch += 1;
}

template <typename KeyT>
struct RsSmem {
  KeyT key[kRsTile];
  int val[kRsTile];
  unsigned wh[kRsWarps][256];
  unsigned lstart[256];      // first local position of each digit
  long long gpos[256];       // global position of the tile's first item of each digit
  unsigned wsum[kRsWarps];
  unsigned tile;
  int ok;
};

__device__ __forceinline__ unsigned long long rs_word(unsigned tag, unsigned state, unsigned long long v) {
  return ((unsigned long long)tag << 33) | ((unsigned long long)state << 31) | v;
}

template <typename KeyT>
__global__ void __launch_bounds__(kRsThreads, 4) k_rs_pass(const KeyT* kin, const int* vin,
                                                          KeyT* kout, int* vout, const long long* n_p,
                                                          long long cap, int pass, RsScratch R, long long n_tiles,
                                                          const int* flags, unsigned* status_word) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RsSmem<KeyT>& S = *(RsSmem<KeyT>*)smem_raw;
  // after an error (a look-back of an earlier pass gave up, so the keys no
  // longer match the digit histograms) the remaining passes do nothing
  const long long n = (flags[1] || *(volatile unsigned*)status_word) ? 0 : clamp_groups(n_p, cap);
  const int shift = 8 * pass;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) S.tile = atomicAdd(&R.tile_ctr[pass], 1u);
  __syncthreads();
  const unsigned tile = S.tile;
  const long long base = (long long)tile * kRsTile;
  if (base >= n) return;  // tiles are taken in order: every later tile is empty too
  const unsigned tag = ((*R.epoch) * kRsPasses + (unsigned)pass) & 0x7FFFFFFFu;
  const long long wbase = base + (long long)warp * kRsPerWarp;
  KeyT kr[kRsPerLane];
  int vr[kRsPerLane];
  for (int i = lane; i < 256; i += 32) S.wh[warp][i] = 0;
  __syncwarp();
#pragma unroll
  for (int j = 0; j < kRsPerLane; ++j) {
    const long long k = wbase + j * 32 + lane;
    const bool valid = k < n;
    kr[j] = valid ? kin[k] : (KeyT)0;
    vr[j] = valid ? vin[k] : 0;
    if (valid) atomicAdd(&S.wh[warp][(unsigned)(kr[j] >> shift) & 255u], 1u);
  }
  __syncthreads();
  {
    const int d = threadIdx.x;
    unsigned run = 0;
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) {
      const unsigned c = S.wh[w][d];
      S.wh[w][d] = run;
      run += c;
    }
    // publish this tile's count of digit d, then look back for its prefix
    unsigned long long* mine = R.status + (long long)tile * 256 + d;
    volatile unsigned long long* vs = (volatile unsigned long long*)R.status;
    unsigned long long excl = 0;
    int ok = 1;
    if (tile == 0) {
      *(volatile unsigned long long*)mine = rs_word(tag, 2, run);
    } else {
      *(volatile unsigned long long*)mine = rs_word(tag, 1, run);
      // walk back four tiles per dependent step (their words read together);
      // a tile that has not published yet is polled until it has
      long long t = (long long)tile - 1;
      unsigned spins = 0;
      const unsigned lim = spin_limit(status_word);
      bool done = false;
      while (!done && t >= 0) {
        unsigned long long w4[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) w4[k] = t - k >= 0 ? vs[(t - k) * 256 + d] : 0ull;
        int k = 0;
        for (; k < 4 && t - k >= 0; ++k) {
          const unsigned long long w = w4[k];
          const unsigned wt = (unsigned)(w >> 33), st = (unsigned)(w >> 31) & 3u;
          if (wt != tag || st == 0) break;
          excl += w & 0x7FFFFFFFull;
          if (st == 2) {
            done = true;
            break;
          }
        }
        if (done) break;
        t -= k;
        if (k < 4 && t >= 0) {  // tile t has not published: poll it again
          if (++spins > lim) { ok = 0; break; }
          if (spins > 64) __nanosleep(64);
        }
      }
      __threadfence();
      *(volatile unsigned long long*)mine = rs_word(tag, 2, excl + run);
    }
    if (!ok) set_status(status_word, JABBA_ERR_TIMEOUT);
    // tile-local digit starts
    unsigned incl = run;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) S.wsum[warp] = incl;
    __syncthreads();
    unsigned before = 0;
    for (int w = 0; w < warp; ++w) before += S.wsum[w];
    const unsigned ls = before + incl - run;
    S.lstart[d] = ls;
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) S.wh[w][d] += ls;
    S.gpos[d] = (long long)R.gbase[pass * 256 + d] + (long long)excl;
  }
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int j = 0; j < kRsPerLane; ++j) {
    const long long k = wbase + j * 32 + lane;
    const bool valid = k < n;
    const unsigned dgt = (unsigned)(kr[j] >> shift) & 255u;
    unsigned peers = __ballot_sync(0xFFFFFFFFu, valid);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const unsigned m = __ballot_sync(0xFFFFFFFFu, (dgt >> b) & 1u);
      peers &= ((dgt >> b) & 1u) ? m : ~m;
    }
    const unsigned rank = __popc(peers & lt);
    if (valid) {
      const unsigned pos = S.wh[warp][dgt] + rank;
      S.key[pos] = kr[j];
      S.val[pos] = vr[j];
    }
    __syncwarp();
    if (valid && rank == 0) S.wh[warp][dgt] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  const int in_tile = (int)(n - base < kRsTile ? n - base : kRsTile);
  for (int i = threadIdx.x; i < in_tile; i += kRsThreads) {
    const KeyT key = S.key[i];
    const unsigned dgt = (unsigned)(key >> shift) & 255u;
    const long long pos = S.gpos[dgt] + (i - (long long)S.lstart[dgt]);
    kout[pos] = key;
    vout[pos] = S.val[i];
  }
}

// Scratch words (32-bit) of the sort for cap items: the fixed header
// (2 x kRsPasses x 256 histogram words, 16 tile counters, the epoch, padding
// to 64 words) and one 64-bit status word per (tile, digit).
long long rs_hist_words(long long cap) {
  const long long n_tiles = (cap + kRsTile - 1) / kRsTile + 1;
  return 2 * kRsPasses * 256 + 64 + 2 * 256 * n_tiles;
}

// Stable sort of (keys, vals) by the low `bits` bits of the keys (64-bit
// keys, or 32-bit ones when bits <= 32: fewer bytes moved per pass); the
// result ends in the buffers returned through kres/vres.
template <typename KeyT>
static void radix_sort(KeyT* k0, int* v0, KeyT* k1, int* v1, const long long* n_p,
                       long long cap, int bits, unsigned* hist_words, int num_sms, unsigned* status_word,
                       KeyT** kres, int** vres, const int* flags, cudaStream_t st) {
  const long long n_tiles = (cap + kRsTile - 1) / kRsTile;
  static PerDevice attr;
  attr.get([] {
    cudaFuncSetAttribute(k_rs_pass<KeyT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(RsSmem<KeyT>));
    return 1;
  });
  // Fixed header (histograms, tile counters, epoch) first, status words after
  // it: the layout does not depend on cap, so the epoch persists across sorts
  // of any size and no status word left by an earlier sort carries a live tag.
  RsScratch R;
  R.ghist = hist_words;
  R.gbase = R.ghist + kRsPasses * 256;
  R.tile_ctr = R.gbase + kRsPasses * 256;
  R.epoch = R.tile_ctr + 16;
  R.status = (unsigned long long*)(hist_words + 2 * kRsPasses * 256 + 64);
  const int passes = (bits + 7) / 8;
  KeyT* kin = k0;
  KeyT* kout = k1;
  int* vin = v0;
  int* vout = v1;
  if (n_tiles > 0) {
    cudaMemsetAsync(R.ghist, 0, sizeof(unsigned) * kRsPasses * 256, st);
    k_rs_global_hist<KeyT><<<(unsigned)(num_sms * 4), 256, 0, st>>>(k0, n_p, cap, passes, R.ghist, flags);
    k_rs_bases<<<1, 32 * kRsPasses, 0, st>>>(R.ghist, passes, R.gbase, R.tile_ctr, R.epoch);
  }
  for (int pass = 0; pass < passes && n_tiles > 0; ++pass) {
    k_rs_pass<KeyT><<<(unsigned)n_tiles, kRsThreads, sizeof(RsSmem<KeyT>), st>>>(kin, vin, kout, vout, n_p, cap,
                                                                                 pass, R, n_tiles, flags, status_word);
    KeyT* tk = kin; kin = kout; kout = tk;
    int* tv = vin; vin = vout; vout = tv;
  }
  *kres = kin;
  *vres = vin;
}

// Sorted-order copies of the coordinates, the cell of each item, and checks
// that the grid is usable (else flags[0] = 1: sequential fallback).
struct GridGeom {
  float x0, y0, inv_h, h;
  int ncx, ncy;
};

__global__ void k_mgeom(const int* bounds, double alpha, long long cap_cells, GridGeom* geom, int* flags,
                        const long long* n_p, long long cap) {
  const long long n = clamp_groups(n_p, cap);
  const float xmin = of_ord(bounds[0]), xmax = of_ord(bounds[1]);
  const float ymin = of_ord(bounds[2]), ymax = of_ord(bounds[3]);
  const double h = alpha * 0.5 * (1.0 + 0x1p-7);
  GridGeom g;
  g.x0 = xmin;
  g.y0 = ymin;
  g.inv_h = (float)(1.0 / h);
  g.h = (float)h;
  const double nx = n > 0 ? floor(((double)xmax - xmin) / h) + 1 : 1;
  const double ny = n > 0 ? floor(((double)ymax - ymin) / h) + 1 : 1;
  const double maxc = fmax(fmax(fabs((double)xmin), fabs((double)xmax)), fmax(fabs((double)ymin), fabs((double)ymax)));
  int fb = 0;
  if (!(alpha > 0.0) || !(nx * ny <= (double)cap_cells) || !(maxc * 0x1p-19 <= h * 0x1p-8) || !(h > 1e-30)) fb = 1;
  g.ncx = fb ? 1 : (int)nx;
  g.ncy = fb ? 1 : (int)ny;
  *geom = g;
  flags[0] = flags[1] ? 0 : fb;
}

__device__ __forceinline__ int cell_of(const GridGeom& g, float x, float y) {
  int cx = (int)floorf((x - g.x0) * g.inv_h);
  int cy = (int)floorf((y - g.y0) * g.inv_h);
  cx = min(max(cx, 0), g.ncx - 1);
  cy = min(max(cy, 0), g.ncy - 1);
  return cy * g.ncx + cx;
}

__global__ void k_msorted(const int* sidx, const float* X32, const float* Y32, const long long* n_p, long long cap,
                          const GridGeom* geom, const int* flags, float* sX, float* sY,
                          unsigned* ckey, int* cval) {
  if (flags[1]) return;
  const long long n = clamp_groups(n_p, cap);
  const GridGeom g = *geom;
  const bool fb = flags[0] != 0;
  for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < n; a += (long long)gridDim.x * blockDim.x) {
    const int c = sidx[a];
    const float x = X32[c], y = Y32[c];
    sX[a] = x;
    sY[a] = y;
    ckey[a] = fb ? 0u : (unsigned)cell_of(g, x, y);
    cval[a] = (int)a;
  }
}

// Cell table: cells in id order; cell_of_id[id] = cell index or -1.  Also
// the FP32 coordinates in cell order.
__global__ void k_mcell_heads(const unsigned* ckey_sorted, const int* cord, const float* sX,
                              const float* sY, const long long* n_p, long long cap, const int* flags, int* head,
                              float* cX, float* cY) {
  const long long n = clamp_groups(n_p, cap);
  const bool grid = flags[0] == 0 && flags[1] == 0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < cap; t += (long long)gridDim.x * blockDim.x) {
    head[t] = t < n && grid && (t == 0 || ckey_sorted[t] != ckey_sorted[t - 1]) ? 1 : 0;
    if (t < n && grid) {
      const int a = cord[t];
      cX[t] = sX[a];
      cY[t] = sY[a];
    }
  }
}

__global__ void k_mcell_fill(const unsigned* ckey_sorted, const int* head, const long long* head_off,
                             const long long* n_p, long long cap, int* cell_beg, int* cell_end, int* cell_id,
                             int* cell_of_id, unsigned long long* state, const int* cord, int4* cinfo) {
  const long long n = clamp_groups(n_p, cap);
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    if (!head[t]) continue;
    const long long j = head_off[t];
    cell_beg[j] = (int)t;
    cell_id[j] = (int)ckey_sorted[t];
    cell_of_id[ckey_sorted[t]] = (int)j;
    state[j] = ((unsigned long long)(unsigned)t << 32) | 0xFFFFFFFFull;  // ptr = t, undecided
    cinfo[j].x = 0x7FC00000;  // NaN: no start yet
    cinfo[j].y = 0x7FC00000;
    cinfo[j].z = cord[t];
  }
}

__global__ void k_mcell_end(const int* cell_beg, const long long* n_cells_p, const long long* n_p, long long cap,
                            int* cell_end, int4* cinfo) {
  const long long nc = *n_cells_p;
  const long long n = clamp_groups(n_p, cap);
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < nc; j += (long long)gridDim.x * blockDim.x) {
    const int e = j + 1 < nc ? cell_beg[j + 1] : (int)n;
    cell_end[j] = e;
    cinfo[j].w = e;
  }
}

// A bounded wait of the sort or of the rounds gave up: the kernels after it
// leave the merge outputs alone (flags[1]), as after an earlier error.
__global__ void k_mflag_status(int* flags, const unsigned* status) {
  if (*status != 0u) flags[1] = 1;
}

__global__ void k_clear_i32(int* p, long long n, int v) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) p[i] = v;
}

// ------------------------------------------------------------------ 4. rounds
// state[j] = (ptr << 32) | s, s = 0xFFFFFFFF undecided, 0xFFFFFFFE no start,
// else the sorted position of the cell's start; ptr = first item (cell order)
// not known to be covered.
constexpr unsigned kUndecided = 0xFFFFFFFFu;
constexpr unsigned kNoStart = 0xFFFFFFFEu;
constexpr int kCoverUnit = 128;    // items of one neighbour cell per phase-B work unit (4 per lane)
constexpr int kScanChunks = 4;     // chunks of 32 a blocking scan reads before it waits instead
constexpr unsigned long long kUnitMask = (1ull << 40) - 1;  // packed counter: starts << 40 | units

struct RoundArgs {
  MergeView V;
  const int* cord;          // item (sorted position) at cell-order index t
  const float* cX;          // FP32 coordinates at cell-order index t
  const float* cY;
  const int* cell_end;
  const int* cell_id;
  const int* cell_of_id;
  unsigned long long* state;
  unsigned* cov;            // [t / 32] bit t: item covered by a start; maintained for undecided cells only
  int4* cinfo;              // [cell] FP32 start coordinates (bits; NaN until known), sorted position of the
                            // first item not known covered (a lower bound), end (cell order)
  // the starts created in the current round, in slot order (the order of the
  // packed counter, so s_base is non-decreasing)
  int* s_pos;               // [slots] sorted position of the start
  unsigned* s_base;         // [slots] first coverage unit of the start
  unsigned* s_pre;          // [slots][26] first unit per neighbour k (entry 25: end)
  int* s_q;                 // [slots][25] neighbour cell to cover
  int* s_lo;                // [slots][25] first item (cell order) to test there
  int* chg_list;            // [2][n_cells] cells whose state or coverage changed (by round parity;
                            // k_mrounds1: (cell, grid id) pairs, 2 ints each)
  unsigned* eval_stamp;     // [n_cells] last round + 1 in which the cell was evaluated
  unsigned* chg_stamp;      // [n_cells] last round + 1 in which the cell was listed as changed
  unsigned long long* nctr; // [2] packed new-start counters (by round parity)
  unsigned* chg_cnt;        // [2] changed counts (by round parity)
  const long long* n_cells_p;
  const GridGeom* geom;
  const int* flags;
  unsigned* bar;            // [1] barrier generation, [2] rounds used
  unsigned* bar_sub;        // [32 * (kBarGroups + 1)] barrier arrival counters (one per 128-byte line)
  unsigned* status;
  unsigned max_rounds;
  // one-phase rounds (k_mrounds1)
  unsigned* lcnt;            // [3] sizes of the evaluation lists (by round mod 3)
  unsigned long long* uctr;  // [3] packed new starts << 40 | coverage units (by round mod 3)
  long long slot_stride;     // slots per buffer of s_* (two buffers, by round parity)
  long long item_cap;        // entries of the per-item arrays (cord, cX, cY, cov)
};

__device__ __forceinline__ unsigned long long ld_state(const unsigned long long* p) {
  return *((volatile const unsigned long long*)p);
}

// Bounded grid-wide barrier for a co-resident (cooperative) grid, two-level:
// the CTAs arrive on kBarGroups counters (CTA b on counter b % kBarGroups,
// each on its own 128-byte line); the last arrival of a group arrives on the
// top counter, and the last of those advances the generation that every CTA
// waits on.  bar[1] is the generation; sub[32 g] the group counters and
// sub[32 kBarGroups] the top counter.
constexpr unsigned kBarGroups = 16;

__device__ bool grid_barrier(unsigned* bar, unsigned* sub, unsigned nblocks, unsigned* status) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    int ok = 1;
    const unsigned grp = blockIdx.x % kBarGroups;
    const unsigned gsz = nblocks / kBarGroups + (grp < nblocks % kBarGroups ? 1u : 0u);
    const unsigned ngrp = nblocks < kBarGroups ? nblocks : kBarGroups;
    bool released = false;
    if (atomicAdd(&sub[32 * grp], 1u) == gsz - 1) {
      atomicExch(&sub[32 * grp], 0u);
      if (atomicAdd(&sub[32 * kBarGroups], 1u) == ngrp - 1) {
        atomicExch(&sub[32 * kBarGroups], 0u);
        __threadfence();
        atomicAdd(&bar[1], 1u);
        released = true;
      }
    }
    if (!released) {
      unsigned spins = 0;
      const unsigned lim = spin_limit(status);
      while (*gen == g) {
        if (++spins > lim) { ok = 0; set_status(status, JABBA_ERR_TIMEOUT); break; }
        __nanosleep(32);
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// The same barrier for a caller that counts its barriers (b = 0, 1, ...
// within one launch), on counters that only grow (k_minit zeroes them before
// the launch): barrier b is complete once the group counter of every group
// has reached (b + 1) x its size, i.e. once the top counter, which the last
// arrival of each group advances, reaches (b + 1) x the groups.  Every CTA
// waits on the top counter itself: two dependent atomics and one poll per
// barrier, with no resets.
__device__ bool grid_barrier_n(unsigned* bar, unsigned* sub, unsigned nblocks, unsigned* status, unsigned b) {
  __shared__ int ok_s;
  (void)bar;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* top = sub + 32 * kBarGroups;
    __threadfence();
    int ok = 1;
    const unsigned grp = blockIdx.x % kBarGroups;
    const unsigned gsz = nblocks / kBarGroups + (grp < nblocks % kBarGroups ? 1u : 0u);
    const unsigned ngrp = nblocks < kBarGroups ? nblocks : kBarGroups;
    if (atomicAdd(&sub[32 * grp], 1u) == (b + 1u) * gsz - 1u) {
      __threadfence();
      atomicAdd(&sub[32 * kBarGroups], 1u);
    }
    const unsigned target = (b + 1u) * ngrp;
    unsigned spins = 0;
    const unsigned lim = spin_limit(status);
    while ((int)(*top - target) < 0) {
      if (++spins > lim) { ok = 0; set_status(status, JABBA_ERR_TIMEOUT); break; }
      __nanosleep(32);
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Coverage flags: one bit per item (cell order), set with atomicOr (bits
// only go from 0 to 1), read through L2 (other SMs set them).
__device__ __forceinline__ bool cov_test(const unsigned* cov, int u) { return (__ldcg(&cov[u >> 5]) >> (u & 31)) & 1u; }
__device__ __forceinline__ void cov_set(unsigned* cov, int u) { atomicOr(&cov[u >> 5], 1u << (u & 31)); }

// Bits of the 32 items from `base` that lie in [lo, hi).
__device__ __forceinline__ unsigned range_bits(int base, int lo, int hi) {
  const int a = max(lo - base, 0), b = min(hi - base, 32);
  if (b <= a) return 0u;
  return (b >= 32 ? 0xFFFFFFFFu : ((1u << b) - 1u)) & (0xFFFFFFFFu << a);
}

// First index in [t, end) whose coverage bit is 0, else end (whole warp;
// four 16-byte loads per lane in flight together: 16,384 flags per
// dependent step, so a long covered run in a dense cell costs few trips; the
// bitmap is padded past its last item).
__device__ __forceinline__ int first_uncovered(const unsigned* cov, int t, int end) {
  const int lane = threadIdx.x & 31;
  for (int b = t & ~127; b < end; b += 16384) {
    int hit[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int o = b + k * 4096 + lane * 128;
      hit[k] = -1;
      if (o < end) {
        const uint4 w = __ldcg((const uint4*)(cov + (o >> 5)));
        const unsigned z[4] = {~w.x & range_bits(o, t, end), ~w.y & range_bits(o + 32, t, end),
                               ~w.z & range_bits(o + 64, t, end), ~w.w & range_bits(o + 96, t, end)};
#pragma unroll
        for (int q = 3; q >= 0; --q)
          if (z[q]) hit[k] = o + 32 * q + __ffs(z[q]) - 1;
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const unsigned bal = __ballot_sync(0xFFFFFFFFu, hit[k] >= 0);
      if (bal) return __shfl_sync(0xFFFFFFFFu, hit[k], __ffs(bal) - 1);
    }
  }
  return end;
}

// Evaluate one undecided cell (whole warp): skip its covered items; its first
// uncovered item p becomes the cell's start unless a neighbouring start that
// precedes p covers it (decided in this round, so its coverage is not marked
// yet), or an uncovered item of an undecided neighbouring cell precedes p and
// may lie within alpha (it could still become a start covering p).  Lane k
// (< 25) looks after neighbour k of the 5 x 5 block (geometry, state, the
// start test); the neighbours that need an item scan are then scanned by the
// whole warp, at most kScanChunks chunks each (past that the cell waits).
// A new start takes a slot and lists, for phase B, the undecided neighbours
// within reach with the work units their coverage needs.  Returns whether the
// state changed.
__device__ __forceinline__ bool eval_cell(const RoundArgs& R, const GridGeom& g, long long j,
                                          unsigned long long* nctr) {
  const int lane = threadIdx.x & 31;
  const unsigned long long st = ld_state(&R.state[j]);
  if ((unsigned)st != kUndecided) return false;
  const int end = R.cell_end[j];
  const int t = first_uncovered(R.cov, (int)(st >> 32), end);
  unsigned result = kUndecided;
  int myq = -1, mylo = 0, myhi = 0, p = 0;
  bool need = false;
  if (t >= end) {
    result = kNoStart;
  } else {
    p = R.cord[t];
    const int id = R.cell_id[j];
    const int cx = id % g.ncx, cy = id / g.ncx;
    const float px = R.cX[t], py = R.cY[t];
    // squared distance beyond which a neighbouring cell cannot hold an item
    // within alpha of p (margins cover the FP32 coordinates and cell mapping)
    const float reach = sqrtf(R.V.a2hi) * (1.0f + 0x1p-10f) +
                        0x1p-16f * (fabsf(px) + fabsf(py) + fabsf(g.x0) + fabsf(g.y0) + 4.0f * g.h);
    bool blk = false, scan = false;
    if (lane < 25 && lane != 12) {
      const int xx = cx + lane % 5 - 2, yy = cy + lane / 5 - 2;
      if (xx >= 0 && xx < g.ncx && yy >= 0 && yy < g.ncy) {
        const int q = R.cell_of_id[yy * g.ncx + xx];
        if (q >= 0) {
          const float rx0 = g.x0 + xx * g.h, ry0 = g.y0 + yy * g.h;
          const float ddx = fmaxf(fmaxf(rx0 - px, px - (rx0 + g.h)), 0.f);
          const float ddy = fmaxf(fmaxf(ry0 - py, py - (ry0 + g.h)), 0.f);
          if (!(ddx > reach || ddy > reach || fmaf(ddx, ddx, ddy * ddy) > reach * reach)) {
            const unsigned long long sq = ld_state(&R.state[q]);
            const unsigned sv = (unsigned)sq;
            if (sv < kNoStart) {
              // a start decided this round has not marked its coverage yet
              if ((int)sv < p && within_sorted(R.V, (int)sv, p)) blk = true;
            } else if (sv == kUndecided) {
              myq = q;
              mylo = (int)(sq >> 32);
              myhi = R.cell_end[q];
              need = mylo < myhi;
              scan = need && R.cord[mylo] < p;
            }
          }
        }
      }
    }
    bool blocked = __any_sync(0xFFFFFFFFu, blk);
    unsigned sm = __ballot_sync(0xFFFFFFFFu, scan);
    while (!blocked && sm) {
      const int l = __ffs(sm) - 1;
      sm &= sm - 1;
      const int qe = __shfl_sync(0xFFFFFFFFu, myhi, l);
      int u0 = __shfl_sync(0xFFFFFFFFu, mylo, l);
      for (int ch = 0;; ++ch, u0 += 32) {
        if (u0 >= qe) break;
        if (ch == kScanChunks) { blocked = true; break; }
        const int u = u0 + lane;
        bool past = true, hit = false;
        if (u < qe) {
          const int r = R.cord[u];
          past = r >= p;
          if (!past && !cov_test(R.cov, u) &&
              filter_c(R.cX[u], R.cY[u], px, py, R.V.a2lo, R.V.a2hi) != 0)
            hit = true;
        }
        if (__any_sync(0xFFFFFFFFu, hit)) { blocked = true; break; }
        if (__any_sync(0xFFFFFFFFu, past)) break;
      }
    }
    if (!blocked) result = (unsigned)p;
  }
  const unsigned long long ns = ((unsigned long long)(unsigned)t << 32) | result;
  const bool changed = ns != st;
  if (lane == 0 && changed) atomicExch(&R.state[j], ns);
  if (result < kNoStart) {
    // coverage work of the new start: ceil(items / kCoverUnit) units per neighbour
    const unsigned cnt = need ? (unsigned)((myhi - mylo + kCoverUnit - 1) / kCoverUnit) : 0u;
    unsigned incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += v;
    }
    const unsigned total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    unsigned long long old = 0;
    if (lane == 0) old = atomicAdd(nctr, (1ull << 40) | (unsigned long long)total);
    old = __shfl_sync(0xFFFFFFFFu, old, 0);
    const long long slot = (long long)(old >> 40);
    const unsigned base = (unsigned)(old & kUnitMask);
    if (lane < 25) {
      R.s_q[slot * 25 + lane] = need ? myq : -1;
      R.s_lo[slot * 25 + lane] = mylo;
    }
    if (lane < 26) R.s_pre[slot * 26 + lane] = base + incl - cnt;
    if (lane == 0) {
      R.s_pos[slot] = p;
      R.s_base[slot] = base;
    }
  }
  return changed;
}

// Append cell q to the changed list of this round once (stamp = round + 1).
__device__ __forceinline__ void mark_changed(const RoundArgs& R, long long q, unsigned round, int* chg,
                                             unsigned* n_chg) {
  if (atomicExch(&R.chg_stamp[q], round + 1) != round + 1) chg[atomicAdd(n_chg, 1u)] = (int)q;
}

// Phase B: the coverage units [u, u_end) of this warp (whole warp).  Unit u of
// start s, neighbour k, tests the items [lo + i * kCoverUnit, +kCoverUnit) of
// cell q that follow the start in key order and are not yet covered.
template <bool kMark>
__device__ __forceinline__ void cover_units(const RoundArgs& R, long long soff, unsigned u, unsigned u_end,
                                           unsigned n_new, unsigned round, int* chg, unsigned* n_chg) {
  const int lane = threadIdx.x & 31;
  const unsigned* s_base = R.s_base + soff;
  const unsigned* s_pre = R.s_pre + 26 * soff;
  const int* s_q = R.s_q + 25 * soff;
  const int* s_lo = R.s_lo + 25 * soff;
  const int* s_pos = R.s_pos + soff;
  // the slot holding u: the last one whose first unit is <= u
  // warp-parallel search (s_base is non-decreasing and s_base[0] = 0): each
  // step narrows the range to one of 32 equal parts with one load per lane
  int lo = 0, len = (int)n_new;
  while (len > 32) {
    const int step = (len + 31) / 32;
    const int i = lo + lane * step;
    const unsigned v = lane * step < len ? __ldcg(&s_base[i]) : 0xFFFFFFFFu;
    const int k = 31 - __clz(__ballot_sync(0xFFFFFFFFu, v <= u));
    lo += k * step;
    len = min(step, len - k * step);
  }
  {
    const unsigned v = lane < len ? __ldcg(&s_base[lo + lane]) : 0xFFFFFFFFu;
    lo += 31 - __clz(__ballot_sync(0xFFFFFFFFu, v <= u));
  }
  int s = lo;
  for (;;) {
    const unsigned pre = lane < 26 ? __ldcg(&s_pre[(long long)s * 26 + lane]) : 0xFFFFFFFFu;
    const int q_l = lane < 25 ? __ldcg(&s_q[(long long)s * 25 + lane]) : -1;
    const int lo_l = lane < 25 ? __ldcg(&s_lo[(long long)s * 25 + lane]) : 0;
    const int sp = __ldcg(&s_pos[s]);
    const float spx = R.V.sX[sp], spy = R.V.sY[sp];
    for (;;) {
      const int k = 31 - __clz(__ballot_sync(0xFFFFFFFFu, pre <= u));
      if (k >= 25) break;  // past this slot's units
      const int q = __shfl_sync(0xFFFFFFFFu, q_l, k);
      const unsigned pk = __shfl_sync(0xFFFFFFFFu, pre, k);
      const int t0 = __shfl_sync(0xFFFFFFFFu, lo_l, k) + (int)(u - pk) * kCoverUnit;
      const int t1 = min(t0 + kCoverUnit, R.cell_end[q]);
      int rr[kCoverUnit / 32];
      bool cv[kCoverUnit / 32];
#pragma unroll
      for (int i = 0; i < kCoverUnit / 32; ++i) {
        const int tt = t0 + i * 32 + lane;
        rr[i] = tt < t1 ? __ldg(&R.cord[tt]) : -1;
        cv[i] = tt < t1 ? cov_test(R.cov, tt) : true;
      }
      bool any = false;
#pragma unroll
      for (int i = 0; i < kCoverUnit / 32; ++i) {
        const int tt = t0 + i * 32 + lane;
        if (rr[i] > sp && !cv[i]) {
          int f = filter_c(spx, spy, __ldg(&R.cX[tt]), __ldg(&R.cY[tt]), R.V.a2lo, R.V.a2hi);
          if (f == 2) f = exact_within_sorted(R.V, sp, rr[i]) ? 1 : 0;
          if (f) {
            cov_set(R.cov, tt);
            any = true;
          }
        }
      }
      if constexpr (kMark) {
        if (__any_sync(0xFFFFFFFFu, any) && lane == 0) mark_changed(R, q, round, chg, n_chg);
      }
      if (++u >= u_end) return;
    }
    if (++s >= (int)n_new) return;
  }
}

// Rounds of the cell greedy with worklists: round r evaluates only the
// undecided cells of the 5 x 5 blocks around cells that changed in round r-1
// (their state, or the coverage of their items); a cell whose neighbourhood
// did not change would reach the same verdict.  Phase A evaluates (each cell
// once per round: eval_stamp), phase B marks the coverage of the new starts
// in the undecided cells around them (a decided cell's items are all covered
// and are not read again), split into equal units over all warps.  Items are
// covered only by true starts, and a start is declared only when no undecided
// earlier item can cover it, so the starts are exactly those of the
// sequential greedy.
__global__ void __launch_bounds__(256) k_mrounds(RoundArgs R) {
  if (R.flags[0] || R.flags[1]) return;
  const long long n_cells = *R.n_cells_p;
  const GridGeom g = *R.geom;
  const unsigned nblocks = gridDim.x;
  const int lane = threadIdx.x & 31;
  const long long warp_g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long n_warps = ((long long)gridDim.x * blockDim.x) >> 5;
  const size_t stride = (size_t)(n_cells > 0 ? n_cells : 1);
  for (unsigned round = 0; round < R.max_rounds; ++round) {
    const int par = round & 1;
    int* chg = R.chg_list + (size_t)par * stride;          // cells changed in this round
    const int* prev = R.chg_list + (size_t)(par ^ 1) * stride;
    unsigned long long* nctr = &R.nctr[par];
    unsigned* n_chg = &R.chg_cnt[par];
    const unsigned n_prev = round ? *((volatile unsigned*)&R.chg_cnt[par ^ 1]) : 0u;
    // ---- phase A
    if (round == 0) {
      for (long long j = warp_g; j < n_cells; j += n_warps)
        if (eval_cell(R, g, j, nctr) && lane == 0) mark_changed(R, j, round, chg, n_chg);
    } else {
      for (long long w = warp_g; w < (long long)n_prev * 25; w += n_warps) {
        const int c = __ldcg(&prev[w / 25]);
        const int k = (int)(w % 25);
        const int id = R.cell_id[c];
        const int xx = id % g.ncx + k % 5 - 2, yy = id / g.ncx + k / 5 - 2;
        if (xx < 0 || xx >= g.ncx || yy < 0 || yy >= g.ncy) continue;
        const int q = R.cell_of_id[yy * g.ncx + xx];
        if (q < 0) continue;
        if ((unsigned)ld_state(&R.state[q]) != kUndecided) continue;
        unsigned claim = 0;
        if (lane == 0) claim = atomicExch(&R.eval_stamp[q], round + 1);
        claim = __shfl_sync(0xFFFFFFFFu, claim, 0);
        if (claim == round + 1) continue;                    // already evaluated this round
        if (eval_cell(R, g, q, nctr) && lane == 0) mark_changed(R, q, round, chg, n_chg);
      }
    }
    if (!grid_barrier(R.bar, R.bar_sub, nblocks, R.status)) return;
    // ---- phase B
    // every read of the other parity's counters (n_prev, the previous
    // round's new starts) happened before the barrier; they are written
    // again only after the next barrier
    if (warp_g == 0 && lane == 0) {
      R.nctr[par ^ 1] = 0;
      R.chg_cnt[par ^ 1] = 0;
    }
    {
      const unsigned long long ctr = *((volatile unsigned long long*)nctr);
      const unsigned n_new = (unsigned)(ctr >> 40);
      const unsigned total = (unsigned)(ctr & kUnitMask);
      const unsigned per = (unsigned)(((long long)total + n_warps - 1) / n_warps);
      const unsigned u0 = (unsigned)(warp_g * per);
      if (per && u0 < total) cover_units<true>(R, 0, u0, min(total, u0 + per), n_new, round, chg, n_chg);
    }
    if (!grid_barrier(R.bar, R.bar_sub, nblocks, R.status)) return;
    // nothing changed: a fixed point, where every cell is decided (the
    // earliest undecided candidate always progresses); k_mcheck verifies it
    if (*((volatile unsigned*)n_chg) == 0) {
      if (warp_g == 0 && lane == 0) R.bar[2] = round + 1;  // diagnostics: rounds used
      return;
    }
  }
  if (warp_g == 0 && lane == 0) set_status(R.status, JABBA_ERR_TIMEOUT);
}

// ------------------------------------------------------------------ 4b. rounds, one phase
// The same cell greedy with one grid barrier per round.  Coverage by the
// decided starts is tested on the fly: an evaluation gathers every decided
// start of the 9 x 9 block of cells around its cell (a start within alpha of
// an item of the 5 x 5 block lies there) and tests items against them (FP32
// filter, exact test when it straddles), so it needs no coverage marks.  The
// cov flags become hints, only ever set for items that a decided start
// covers: the coverage units of the starts decided in round r are marked in
// round r + 1 by warps without an evaluation, beside the evaluations, which
// no longer wait for them.  An evaluation that changes its cell lists, for
// the next round, the undecided cells whose verdict may change: the 9 x 9
// block around a new start (its coverage reaches the 5 x 5 block, whose
// items are scanned by the cells of the 9 x 9 block), the 5 x 5 block around
// any other change (the cell itself when it stopped early).  A start is still
// declared only when no undecided earlier item can cover it, so the starts
// are those of the sequential greedy; the cell with the earliest uncovered
// item is listed again after every event that can unblock it, so the rounds
// end only when every cell is decided (k_mcheck verifies it).
constexpr int kOwnSteps = 4;  // 128-item steps an evaluation tests in its own cell before it yields

struct NbScratch {               // one per warp, shared memory
  int sp[81];                    // decided starts of the 9 x 9 block (those of the 5 x 5 block first):
  float sx[81], sy[81];          //   sorted position, FP32 coordinates,
  signed char sdx[81], sdy[81];  //   cell offset from the evaluated cell
  int uq[24], ulo[24], uhi[24];  // undecided cells of the 5 x 5 block: cell, first item not known covered, end
  int ucd[24];                   // and the sorted position of that first item
  signed char udx[24], udy[24];  // and its cell offset
};

// Item (sorted position r, FP32 x, y) covered by a gathered start that
// precedes it, among the gathered starts [0, ns).
__device__ __forceinline__ bool covered_by_starts(const MergeView& V, const NbScratch& W, int ns, int r, float x,
                                                  float y) {
  for (int i = 0; i < ns; ++i) {
    const int s = W.sp[i];
    if (s >= r) continue;
    const int f = filter_c(W.sx[i], W.sy[i], x, y, V.a2lo, V.a2hi);
    if (f == 1) return true;
    if (f == 2 && exact_within_sorted(V, s, r)) return true;
  }
  return false;
}

// The same for an item of the cell at offset (qdx, qdy): only starts within
// two cells of it can lie within alpha (the cell side exceeds alpha / 2, and
// the grid check bounds the coordinates' error by 2^-8 of a cell), so the
// others are skipped before the distance filter.
__device__ __forceinline__ bool covered_by_starts_at(const MergeView& V, const NbScratch& W, int ns, int qdx,
                                                     int qdy, int r, float x, float y) {
  for (int i = 0; i < ns; ++i) {
    const int s = W.sp[i];
    if (s >= r || abs(W.sdx[i] - qdx) > 2 || abs(W.sdy[i] - qdy) > 2) continue;
    const int f = filter_c(W.sx[i], W.sy[i], x, y, V.a2lo, V.a2hi);
    if (f == 1) return true;
    if (f == 2 && exact_within_sorted(V, s, r)) return true;
  }
  return false;
}

// Evaluate undecided cell j (whole warp): its first item p not covered by a
// decided start becomes its start unless an uncovered item of an undecided
// neighbouring cell precedes p and may lie within alpha of it.  Loads that do
// not depend on each other are issued together (the evaluations of a round
// are latency bound).
__device__ void eval_cell1(const RoundArgs& R, const GridGeom& g, int j, int id, unsigned round, NbScratch& W,
                           int2* lnxt, unsigned* lcnt_nxt, unsigned long long* uctr_nxt, long long soff) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  __syncwarp();  // the previous evaluation of this warp is done with W
  const unsigned long long st0 = ld_state(&R.state[j]);
  const int end = R.cell_end[j];
  const int cx = id % g.ncx, cy = id / g.ncx;
  // ---- gather: decided starts of the 9 x 9 block, undecided cells of the 5 x 5
  // block (the neighbour indices are loaded beside the cell's own state)
  int q[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int k = i * 32 + lane;
    const int dx = k % 9 - 4, dy = k / 9 - 4;
    q[i] = -1;
    if (k < 81 && (dx != 0 || dy != 0)) {
      const int xx = cx + dx, yy = cy + dy;
      if (xx >= 0 && xx < g.ncx && yy >= 0 && yy < g.ncy) q[i] = R.cell_of_id[yy * g.ncx + xx];
    }
  }
  const unsigned long long st = __shfl_sync(0xFFFFFFFFu, st0, 0);
  if ((unsigned)st != kUndecided) return;
  unsigned long long sq[3];
  int4 ci[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    sq[i] = q[i] >= 0 ? ld_state(&R.state[q[i]]) : 0ull;
    ci[i] = q[i] >= 0 ? __ldcg(&R.cinfo[q[i]]) : make_int4(0, 0, 0, 0);
  }
  int ns = 0, nu = 0, ns5 = 0;
  bool und[3];  // undecided when gathered (a cell decided since is skipped when evaluated)
  // two passes: the starts of the 5 x 5 block (the only ones that can cover
  // the cell's own items) first, then the rest of the 9 x 9 block
#pragma unroll
  for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int k = i * 32 + lane;
      const int dx = k % 9 - 4, dy = k / 9 - 4;
      const bool inner = dx >= -2 && dx <= 2 && dy >= -2 && dy <= 2;
      const unsigned sv = (unsigned)sq[i];
      const bool is_s = q[i] >= 0 && sv < kNoStart && inner == (pass == 0);
      const unsigned ms = __ballot_sync(0xFFFFFFFFu, is_s);
      if (is_s) {
        const int o = ns + __popc(ms & lt);
        float sx = __int_as_float(ci[i].x), sy = __int_as_float(ci[i].y);
        if (sx != sx || sy != sy) {  // the start's coordinates not visible yet: from the item
          sx = R.V.sX[sv];
          sy = R.V.sY[sv];
        }
        W.sp[o] = (int)sv;
        W.sx[o] = sx;
        W.sy[o] = sy;
        W.sdx[o] = (signed char)dx;
        W.sdy[o] = (signed char)dy;
      }
      ns += __popc(ms);
      if (pass == 1) continue;
      und[i] = q[i] >= 0 && sv == kUndecided;
      const bool is_u = und[i] && inner;
      const unsigned mu = __ballot_sync(0xFFFFFFFFu, is_u);
      if (is_u) {
        const int o = nu + __popc(mu & lt);
        const int lo = (int)(sq[i] >> 32);
        W.uq[o] = q[i];
        W.ulo[o] = lo;
        W.uhi[o] = ci[i].w;
        W.ucd[o] = ci[i].z;  // at most the sorted position of item lo (used only when lo < end)
        W.udx[o] = (signed char)dx;
        W.udy[o] = (signed char)dy;
      }
      nu += __popc(mu);
    }
    if (pass == 0) ns5 = ns;
  }
  __syncwarp();
  // ---- own items: the first one not covered, 128 items per step (four per
  // lane, loads in flight together); the first step from the pointer, later
  // ones after skipping hinted runs
  int t = (int)(st >> 32);
  int tp = end, p = 0;
  float px = 0.f, py = 0.f;
  bool yielded = false;
  for (int steps = 0;; ++steps) {
    if (steps > 0) t = first_uncovered(R.cov, t, end);
    if (t >= end) break;
    if (steps == kOwnSteps) {
      yielded = true;
      break;
    }
    bool h[4];
    int r[4];
    float ux[4], uy[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int u = t + i * 32 + lane;
      h[i] = true;
      r[i] = 0;
      ux[i] = uy[i] = 0.f;
      if (u < end) {
        h[i] = cov_test(R.cov, u);
        r[i] = R.cord[u];
        ux[i] = R.cX[u];
        uy[i] = R.cY[u];
      }
    }
    int found = -1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (found >= 0) continue;
      const int u = t + i * 32 + lane;
      bool unc = false;
      if (!h[i]) {  // also false past the end
        if (covered_by_starts(R.V, W, ns5, r[i], ux[i], uy[i])) cov_set(R.cov, u);  // hint: covered by a decided start
        else unc = true;
      }
      const unsigned b = __ballot_sync(0xFFFFFFFFu, unc);
      if (b) {
        const int first = __ffs(b) - 1;
        found = i * 32 + first;
        p = __shfl_sync(0xFFFFFFFFu, r[i], first);
        px = __shfl_sync(0xFFFFFFFFu, ux[i], first);
        py = __shfl_sync(0xFFFFFFFFu, uy[i], first);
      }
    }
    if (found >= 0) {
      tp = t + found;
      break;
    }
    t += 128;
  }
  // ---- verdict
  unsigned result = kUndecided;
  if (!yielded && tp >= end) {
    result = kNoStart;
  } else if (!yielded) {
    bool need = false;
    int lo = 0, hi = 0;
    if (lane < nu) {
      lo = W.ulo[lane];
      hi = W.uhi[lane];
      need = lo < hi && W.ucd[lane] < p;
    }
    unsigned sm = __ballot_sync(0xFFFFFFFFu, need);
    bool blocked = false;
    // the first chunks of up to four neighbours, their loads in flight together
    unsigned pend = 0;  // neighbours (lane bits) still to scan from their second chunk
    {
      int nl[4], lo4[4], hi4[4], r4[4];
      bool h4[4];
      float x4[4], y4[4];
      bool v4[4];
      unsigned m = sm;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        nl[i] = m ? __ffs(m) - 1 : -1;
        if (m) m &= m - 1;
      }
      const unsigned rest = m;  // beyond four: scanned one by one below
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        lo4[i] = __shfl_sync(0xFFFFFFFFu, lo, nl[i] >= 0 ? nl[i] : 0);
        hi4[i] = __shfl_sync(0xFFFFFFFFu, hi, nl[i] >= 0 ? nl[i] : 0);
        const int u = lo4[i] + lane;
        v4[i] = nl[i] >= 0 && u < hi4[i];
        h4[i] = true;
        r4[i] = 0x7FFFFFFF;
        x4[i] = y4[i] = 0.f;
        if (v4[i]) {
          h4[i] = cov_test(R.cov, u);
          r4[i] = R.cord[u];
          x4[i] = R.cX[u];
          y4[i] = R.cY[u];
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (nl[i] < 0 || blocked) continue;
        const bool past = !v4[i] || r4[i] >= p;  // past the end of the cell counts as past
        const int qn = nl[i] >= 0 ? nl[i] : 0;
        const bool hit = !past && !h4[i] && filter_c(x4[i], y4[i], px, py, R.V.a2lo, R.V.a2hi) != 0 &&
                         !covered_by_starts_at(R.V, W, ns, W.udx[qn], W.udy[qn], r4[i], x4[i], y4[i]);
        if (__any_sync(0xFFFFFFFFu, hit)) blocked = true;
        else if (!__any_sync(0xFFFFFFFFu, past)) pend |= 1u << nl[i];
      }
      if (!blocked) pend |= rest;
    }
    while (!blocked && pend) {
      const int l = __ffs(pend) - 1;
      const bool first_done = __popc(sm & ((1u << l) - 1u)) < 4;  // among the four scanned above
      pend &= pend - 1;
      const int qe = __shfl_sync(0xFFFFFFFFu, hi, l);
      int u0 = __shfl_sync(0xFFFFFFFFu, lo, l) + (first_done ? 32 : 0);
      for (int ch = first_done ? 1 : 0;; ++ch, u0 += 32) {
        if (ch > 0) u0 = first_uncovered(R.cov, u0, qe);
        if (u0 >= qe) break;
        if (ch == kScanChunks) {
          blocked = true;
          break;
        }
        const int u = u0 + lane;
        bool past = true, hit = false;
        if (u < qe) {
          const bool hint = cov_test(R.cov, u);
          const int r = R.cord[u];
          const float ux = R.cX[u], uy = R.cY[u];
          past = r >= p;
          if (!past && !hint && filter_c(ux, uy, px, py, R.V.a2lo, R.V.a2hi) != 0 &&
              !covered_by_starts_at(R.V, W, ns, W.udx[l], W.udy[l], r, ux, uy))
            hit = true;
        }
        if (__any_sync(0xFFFFFFFFu, hit)) {
          blocked = true;
          break;
        }
        if (__any_sync(0xFFFFFFFFu, past)) break;
      }
    }
    if (!blocked) result = (unsigned)p;
  }
  const int tnew = yielded ? t : tp;
  const unsigned long long nsv = ((unsigned long long)(unsigned)tnew << 32) | result;
  if (nsv == st) return;
  const bool start = result < kNoStart;
  if (lane == 0) {
    // the cell's summary first (a reader that sees the new state with an
    // older summary falls back to the items, or scans from an earlier item)
    if (start) {
      R.cinfo[j].x = __float_as_int(px);
      R.cinfo[j].y = __float_as_int(py);
    } else if (!yielded && tp < end) {
      R.cinfo[j].z = p;
    }
    atomicExch(&R.state[j], nsv);
  }
  // ---- coverage units of a new start (marked next round)
  if (start) {
    const unsigned cu = lane < nu ? (unsigned)((W.uhi[lane] - W.ulo[lane] + kCoverUnit - 1) / kCoverUnit) : 0u;
    unsigned incl = cu;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += v;
    }
    const unsigned total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    unsigned long long old = 0;
    if (lane == 0) old = atomicAdd(uctr_nxt, (1ull << 40) | (unsigned long long)total);
    old = __shfl_sync(0xFFFFFFFFu, old, 0);
    const long long slot = soff + (long long)(old >> 40);
    const unsigned base = (unsigned)(old & kUnitMask);
    if (lane < 25) {
      R.s_q[slot * 25 + lane] = lane < nu ? W.uq[lane] : -1;
      R.s_lo[slot * 25 + lane] = lane < nu ? W.ulo[lane] : 0;
    }
    if (lane < 26) R.s_pre[slot * 26 + lane] = base + incl - cu;
    if (lane == 0) {
      R.s_pos[slot] = p;
      R.s_base[slot] = base;
    }
  }
  // ---- list, once each (eval_stamp = round + 2), the cells whose verdict
  // may change: the cells undecided when gathered in the 9 x 9 block of a new
  // start or the 5 x 5 block of another change, and the cell itself when it
  // stopped early.  The gathered cell ids and states serve: a cell decided
  // since then is skipped when evaluated.
  bool c[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int k = i * 32 + lane;
    const int dx = k % 9 - 4, dy = k / 9 - 4;
    c[i] = und[i] && (start || (dx >= -2 && dx <= 2 && dy >= -2 && dy <= 2));
    if (yielded && k == 40) {  // the centre
      q[i] = j;
      c[i] = true;
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
    if (c[i]) c[i] = atomicExch(&R.eval_stamp[q[i]], round + 2) != round + 2;
  const unsigned m0 = __ballot_sync(0xFFFFFFFFu, c[0]), m1 = __ballot_sync(0xFFFFFFFFu, c[1]),
                 m2 = __ballot_sync(0xFFFFFFFFu, c[2]);
  const unsigned n0 = __popc(m0), n1 = __popc(m1), tot = n0 + n1 + __popc(m2);
  if (tot == 0) return;
  unsigned lbase = 0;
  if (lane == 0) lbase = atomicAdd(lcnt_nxt, tot);
  lbase = __shfl_sync(0xFFFFFFFFu, lbase, 0);
  // entries carry the cell's grid id beside its index (one dependent load
  // fewer when the cell is evaluated)
  int gid[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int k = i * 32 + lane;
    gid[i] = k == 40 ? id : (cy + k / 9 - 4) * g.ncx + (cx + k % 9 - 4);
  }
  if (c[0]) lnxt[lbase + __popc(m0 & lt)] = make_int2(q[0], gid[0]);
  if (c[1]) lnxt[lbase + n0 + __popc(m1 & lt)] = make_int2(q[1], gid[1]);
  if (c[2]) lnxt[lbase + n0 + n1 + __popc(m2 & lt)] = make_int2(q[2], gid[2]);
}

template <int kWarps>
__global__ void __launch_bounds__(kWarps * 32) k_mrounds1(RoundArgs R) {
  if (R.flags[0] || R.flags[1]) return;
  __shared__ NbScratch W[kWarps];
  const long long n_cells = *R.n_cells_p;
  const GridGeom g = *R.geom;
  const unsigned nblocks = gridDim.x;
  const int lane = threadIdx.x & 31;
  NbScratch& w = W[threadIdx.x >> 5];
  const long long warp_g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long n_warps = ((long long)gridDim.x * blockDim.x) >> 5;
  const size_t stride = (size_t)(n_cells > 0 ? n_cells : 1);
  // this round's list size, its coverage counter and this warp's first list
  // entry: read together right after the previous round's barrier
  unsigned n_eval = 0;
  unsigned long long ctr = 0;
  int2 j0 = make_int2(0, 0);
  for (unsigned round = 0; round < R.max_rounds; ++round) {
    const int nxt = (round + 1) % 3, old = (round + 2) % 3;
    const int2* lcur = (const int2*)R.chg_list + (size_t)(round & 1) * stride;
    int2* lnxt = (int2*)R.chg_list + (size_t)((round + 1) & 1) * stride;
    // the counters of slot `old` were last read in the previous round
    if (warp_g == 0 && lane == 0) {
      R.lcnt[old] = 0;
      R.uctr[old] = 0;
    }
    // evaluations (warps from the bottom)
    const long long soff_new = (long long)(round & 1) * R.slot_stride;
    if (round == 0) {
      for (long long j = warp_g; j < n_cells; j += n_warps)
        eval_cell1(R, g, (int)j, R.cell_id[j], round, w, lnxt, &R.lcnt[nxt], &R.uctr[nxt], soff_new);
    } else {
      for (long long i = warp_g; i < (long long)n_eval; i += n_warps)
      {
        const int2 e = i == warp_g ? j0 : __ldcg(&lcur[i]);
        eval_cell1(R, g, e.x, e.y, round, w, lnxt, &R.lcnt[nxt], &R.uctr[nxt], soff_new);
      }
      // coverage hints of the previous round's starts (warps from the top)
      const unsigned n_new = (unsigned)(ctr >> 40);
      const unsigned total = (unsigned)(ctr & kUnitMask);
      const unsigned per = (unsigned)(((long long)total + n_warps - 1) / n_warps);
      const unsigned u0 = (unsigned)((n_warps - 1 - warp_g) * per);
      if (per && u0 < total)
        cover_units<false>(R, (long long)((round + 1) & 1) * R.slot_stride, u0, min(total, u0 + per), n_new, round,
                           nullptr, nullptr);
    }
    if (!grid_barrier_n(R.bar, R.bar_sub, nblocks, R.status, round)) return;
    // the next round's list entry is read beside its size (past the size it
    // is a stale entry of the buffer, not used)
    j0 = warp_g < (long long)stride ? __ldcg(&lnxt[warp_g]) : make_int2(0, 0);
    n_eval = *((volatile unsigned*)&R.lcnt[nxt]);
    ctr = *((volatile unsigned long long*)&R.uctr[nxt]);
    if (n_eval == 0) {
      if (warp_g == 0 && lane == 0) R.bar[2] = round + 1;  // diagnostics: rounds used
      return;
    }
  }
  if (warp_g == 0 && lane == 0) set_status(R.status, JABBA_ERR_TIMEOUT);
}

// Count of cells left undecided (0 after a complete run).
__global__ void k_mcheck(const unsigned long long* state, const long long* n_cells_p, const int* flags,
                         unsigned* status) {
  if (flags[0] || flags[1]) return;
  const long long n = *n_cells_p;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
    if ((unsigned)state[j] == kUndecided) set_status(status, JABBA_ERR_TIMEOUT);
}

// ------------------------------------------------------------------ 5. labels
// lab[a] = sorted position of the earliest start within alpha (a itself for a
// start).  Items are visited in cell order, so the lanes of a warp mostly
// share one cell and its 5 x 5 neighbourhood (broadcast loads).
__global__ void __launch_bounds__(256) k_mlabel(MergeView V, const int* cord, const float* cX, const float* cY,
                                               const int* cell_of_id, const unsigned long long* state,
                                               const int4* cinfo, const GridGeom* geom, const int* flags,
                                               const long long* n_p, long long cap, int* lab, int* is_start) {
  if (flags[0] || flags[1]) return;
  const long long n = clamp_groups(n_p, cap);
  const GridGeom g = *geom;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int a = cord[t];
    const float xa = cX[t], ya = cY[t];  // the item's FP32 coordinates (cell order)
    const int id = cell_of(g, xa, ya);
    const int cx = id % g.ncx, cy = id / g.ncx;
    // the 5 x 5 block's cells, then their states and summaries (start
    // coordinates), each level's loads in flight together
    int q[25];
#pragma unroll
    for (int k = 0; k < 25; ++k) {
      const int xx = cx + k % 5 - 2, yy = cy + k / 5 - 2;
      q[k] = xx >= 0 && xx < g.ncx && yy >= 0 && yy < g.ncy ? cell_of_id[yy * g.ncx + xx] : -1;
    }
    unsigned sv[25];
#pragma unroll
    for (int k = 0; k < 25; ++k) sv[k] = q[k] >= 0 ? (unsigned)state[q[k]] : kNoStart;
    int best = 0x7FFFFFFF;
#pragma unroll
    for (int k = 0; k < 25; ++k) {
      const int sp = (int)sv[k];
      if (sv[k] >= kNoStart || sp > a || sp >= best) continue;
      if (sp == a) {
        best = a;
        continue;
      }
      const int4 ci = cinfo[q[k]];
      float sx = __int_as_float(ci.x), sy = __int_as_float(ci.y);
      if (sx != sx || sy != sy) {  // (always written by the rounds; the item's copy otherwise)
        sx = V.sX[sp];
        sy = V.sY[sp];
      }
      int f = filter_c(sx, sy, xa, ya, V.a2lo, V.a2hi);
      if (f == 2) f = exact_within_sorted(V, sp, a) ? 1 : 0;
      if (f) best = sp;
    }
    lab[a] = best;
    is_start[a] = best == a ? 1 : 0;
  }
}

// ------------------------------------------------------------------ fallback: sequential greedy (binary64)
__global__ void k_mexact_prep(const jabba_group* groups, const double* iX, const double* iY, const int* rec_of,
                              const int* sidx, const long long* n_p, long long cap, const double* sigma, double scl,
                              int pca, const int* flags, double* eX, double* eY, double* ekey) {
  if (!flags[0] || flags[1]) return;
  const long long n = clamp_groups(n_p, cap);
  for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < n; a += (long long)gridDim.x * blockDim.x) {
    const ExactCentre e = item_point(groups, iX, iY, rec_of[sidx[a]], sigma, scl);
    eX[a] = e.X;
    eY[a] = e.Y;
    ekey[a] = exact_key(e, pca, sigma);
  }
}

__global__ void __launch_bounds__(1024) k_mexact_greedy(const double* eX, const double* eY, const double* ekey,
                                                       const long long* n_p, long long cap, double alpha, int pca,
                                                       const int* flags, int* lab, int* is_start) {
  if (!flags[0] || flags[1]) return;
  __shared__ int s_next;
  __shared__ int s_stop;
  const long long n = clamp_groups(n_p, cap);
  const int tid = threadIdx.x, nt = blockDim.x;
  const double a2 = __dmul_rn(alpha, alpha);
  for (long long i = tid; i < n; i += nt) lab[i] = -1;
  __syncthreads();
  long long a = 0;
  for (;;) {
    for (;;) {
      if (tid == 0) s_next = 0x7FFFFFFF;
      __syncthreads();
      const long long aa = a + tid;
      if (aa < n && lab[aa] < 0) atomicMin(&s_next, tid);
      __syncthreads();
      const int nx = s_next;
      __syncthreads();
      if (nx != 0x7FFFFFFF) { a += nx; break; }
      a += nt;
      if (a >= n) break;
    }
    if (a >= n) break;
    const double xi = eX[a], yi = eY[a];
    // scan bound (Sec. 5 pruning, lossless): the norm changes by at most the
    // distance, so does a projection on a unit axis
    double T;
    if (pca) {
      T = __dadd_rn(ekey[a], __dmul_rn(alpha, 1.0 + 0x1p-30));
      T = __dadd_rn(T, 0x1p-40 * (fabs(ekey[a]) + fabs(xi) + fabs(yi)));
    } else {
      const double r = __dadd_rn(__dsqrt_rn(ekey[a]), alpha);
      T = __dmul_rn(__dmul_rn(r, r), 1.0 + 0x1p-30);
    }
    if (tid == 0) { lab[a] = (int)a; is_start[a] = 1; }
    for (long long b = a + 1; b < n; b += nt) {
      if (tid == 0) s_stop = 0;
      __syncthreads();
      const long long bb = b + tid;
      if (bb < n) {
        if (ekey[bb] > T) {
          s_stop = 1;
        } else if (lab[bb] < 0) {
          const double dx = __dsub_rn(eX[bb], xi), dy = __dsub_rn(eY[bb], yi);
          if (__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) <= a2) lab[bb] = (int)a;
        }
      } else {
        s_stop = 1;
      }
      __syncthreads();
      const int stop = s_stop;
      __syncthreads();
      if (stop) break;
    }
    ++a;
  }
}

// ------------------------------------------------------------------ ids, map, dictionary
__global__ void k_mids(const int* lab, const long long* start_off, const int* sidx, const int* rec_of,
                       const long long* n_p, long long cap, long long dict_capacity, int* l2g, int2* gr,
                       long long* k_out, unsigned* status, const int* flags) {
  if (flags[1]) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *k_out = 0;
    return;
  }
  const long long n = clamp_groups(n_p, cap);
  for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < n; a += (long long)gridDim.x * blockDim.x) {
    int la = lab[a];
    if (la < 0 || la >= n) {  // unresolved (a bounded wait gave up): status is already set
      set_status(status, JABBA_ERR_TIMEOUT);
      la = 0;
    }
    const int gid = (int)start_off[la];
    const int c = sidx[a];
    l2g[c] = gid;
    gr[a] = make_int2(gid, rec_of[c]);  // for the dictionary sums: global id and record by sorted position
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const long long K = start_off[n];
    *k_out = K;
    if (K > dict_capacity) set_status(status, JABBA_ERR_CAPACITY);
  }
}

// Dictionary sums.  Items are visited in cell order, where neighbours mostly
// share their global group: each warp sums runs of equal ids with a segmented
// scan (count, length sum and the six 32-bit limbs of the increment sum) and
// the last lane of each run adds them to the entry with 64-bit atomics, so
// popular entries see a few atomics per cell instead of one per item.
__global__ void k_dict_clear(const long long* k_p, long long dict_capacity, long long* acc) {
  long long K = *k_p;
  if (K > dict_capacity) K = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < K * 8; i += (long long)gridDim.x * blockDim.x)
    acc[i] = 0;
}

__global__ void __launch_bounds__(256) k_dict_accumulate(const jabba_group* groups, const int* cord,
                                                         const int2* gr, const long long* n_p, long long cap,
                                                         const long long* k_p, long long dict_capacity,
                                                         long long* acc, const int* flags) {
  if (flags[1]) return;
  const long long G = clamp_groups(n_p, cap);
  const long long K = *k_p;
  if (K > dict_capacity) return;
  const int lane = threadIdx.x & 31;
  const long long warp_g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long n_warps = ((long long)gridDim.x * blockDim.x) >> 5;
  // two chunks of 32 items per step, their gathers in flight together
  for (long long base = warp_g * 64; base < G; base += n_warps * 64) {
    int2 q[2];
    jabba_group gg[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const long long t = base + 32 * c + lane;
      q[c] = t < G ? gr[cord[t]] : make_int2(-1, -1);
    }
#pragma unroll
    for (int c = 0; c < 2; ++c)
      if (q[c].y >= 0) gg[c] = groups[q[c].y];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (base + 32 * c >= G) break;
      const bool valid = q[c].y >= 0;
      const int gid = valid ? q[c].x : -1;
      // member count, length sum, and the increment sum in three limbs
      // (bits 0-47 and 48-95 unsigned, bits 96-159 signed: the sums are far
      // below 2^159 in magnitude, and 32 limbs of 48 bits fit a 64-bit
      // word): five words per lane in the scan instead of eight
      long long v[5] = {0, 0, 0, 0, 0};
      if (valid) {
        const jabba_group& g = gg[c];
        v[0] = g.count;
        v[1] = g.lensum;
        v[2] = (long long)(g.inc[0] & 0xFFFFFFFFFFFFull);
        v[3] = (long long)((g.inc[0] >> 48) | ((g.inc[1] & 0xFFFFFFFFull) << 16));
        v[4] = (long long)((g.inc[1] >> 32) | (g.inc[2] << 32));
      }
      const int gprev = __shfl_up_sync(0xFFFFFFFFu, gid, 1);
      const bool head = lane == 0 || gprev != gid;
      bool f = head;
      for (int o = 1; o < 32; o <<= 1) {
        const bool fu = __shfl_up_sync(0xFFFFFFFFu, f, o);
#pragma unroll
        for (int i = 0; i < 5; ++i) {
          const long long vu = __shfl_up_sync(0xFFFFFFFFu, v[i], o);
          if (lane >= o && !f) v[i] += vu;
        }
        if (lane >= o) f = f || fu;
      }
      const bool next_head = __shfl_down_sync(0xFFFFFFFFu, head, 1);
      const bool tail = valid && (lane == 31 || next_head);
      if (tail && gid >= 0 && gid < K) {
        // back to the accumulators' layout: count, length sum, six 32-bit limbs
        I192 w;
        w.w0 = (u64)v[2];
        w.w1 = 0;
        w.w2 = 0;
        add192(w, (u64)v[3] << 48, (u64)v[3] >> 16, 0);
        add192(w, 0, (u64)v[4] << 32, (u64)(v[4] >> 32));
        long long out[8];
        out[0] = v[0];
        out[1] = v[1];
        limbs6(w, out + 2);
        long long* e = acc + (long long)gid * 8;
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (out[i]) atomicAdd((unsigned long long*)&e[i], (unsigned long long)out[i]);
      }
    }
  }
}

__global__ void k_dict_finalize(const long long* acc, const long long* k_p, long long dict_capacity,
                                double* dict_len, double* dict_inc, long long* dict_count) {
  long long K = *k_p;
  if (K > dict_capacity) K = 0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < K; c += (long long)gridDim.x * blockDim.x) {
    const long long* a = acc + c * 8;
    const double cnt = (double)a[0];
    dict_count[c] = a[0];
    dict_len[c] = __ddiv_rn((double)a[1], cnt);
    i64 L[6];
    for (int i = 0; i < 6; ++i) L[i] = a[2 + i];
    dict_inc[c] = __ddiv_rn(i192_to_double(from_limbs6(L)), cnt);
  }
}

__global__ void k_minit(int* bounds, unsigned* bar, unsigned* bar_sub, int* flags, const unsigned* status,
                        const long long* n_p, long long cap) {
  for (unsigned i = 0; i <= kBarGroups; ++i) bar_sub[32 * i] = 0;
  for (int i = 3; i < 16; ++i) bar[i] = 0;  // [2] rounds used, [4..5] changed cells, [8..11] new starts
  flags[0] = 0;
  flags[1] = (*status != 0u || *n_p > cap) ? 1 : 0;  // earlier error: leave the merge outputs alone
  bounds[0] = 0x7FFFFFFF;
  bounds[1] = -0x7FFFFFFF;
  bounds[2] = 0x7FFFFFFF;
  bounds[3] = -0x7FFFFFFF;
  bar[0] = 0;
  bar[1] = 0;
  bar[2] = 0;
}


static float rdown(double v) {
  float f = (float)v;
  if ((double)f > v) f = nextafterf(f, 0.0f);
  return f;
}
static float rup(double v) {
  float f = (float)v;
  if ((double)f < v) f = nextafterf(f, INFINITY);
  return f;
}

void launch_merge(const jabba_group* groups, const double* item_X, const double* item_Y, const long long* n_groups,
                  long long group_capacity, const long long* dom_group_off, const double* sigma, double alpha,
                  double scl, int key_mode, int* l2g, double* dict_len, double* dict_inc, long long* dict_count,
                  long long dict_capacity, long long* k, Scratch& ws, unsigned* status, cudaStream_t st,
                  const Marks& mk) {
  const long long cap = group_capacity;
  const unsigned grid = (unsigned)(ws.num_sms * 8);
  MergeBufs& B = ws.mb;
  k_minit<<<1, 1, 0, st>>>(B.bounds, B.bar, B.bar_sub, B.flags, status, n_groups, cap);
  const u64* rtab = (const u64*)ws.m_recip;
  const DivRecip* rsig = (const DivRecip*)(ws.m_recip + kRecipCnt + 1);
  if (!item_X)
    k_recip_tables<<<(kRecipCnt + 256) / 256, 256, 0, st>>>(sigma, (u64*)ws.m_recip, (DivRecip*)rsig, B.flags);
  k_mprep<<<grid, 256, 0, st>>>(groups, item_X, item_Y, n_groups, cap, dom_group_off, sigma, scl, key_mode, ws.m_k0,
                                ws.m_v0, ws.m_rec, ws.m_X32, ws.m_Y32, B.bounds, B.flags, rtab, rsig);
  unsigned long long* skey;
  int* sidx;
  // the keys' order-preserving images (key_image) sort as the keys; the sort
  // is stable and starts in compact-index order, so ties keep it
  radix_sort(ws.m_k0, ws.m_v0, ws.m_k1, ws.m_v1, n_groups, cap, 64, ws.m_hist, ws.num_sms, status, &skey, &sidx,
             B.flags, st);
  k_mflag_status<<<1, 1, 0, st>>>(B.flags, status);
  k_mgeom<<<1, 1, 0, st>>>(B.bounds, alpha, ws.cap_cells, B.geom, B.flags, n_groups, cap);
  // the cell sort ping-pongs in the buffers the key sort left free
  // (32-bit cell keys in the 64-bit buffers; each buffer still holds the
  // 8 bytes per item that the (global id, record) pairs need later)
  unsigned* ck0 = (unsigned*)(skey == ws.m_k0 ? ws.m_k1 : ws.m_k0);
  int* cv0 = sidx == ws.m_v0 ? ws.m_v1 : ws.m_v0;
  k_msorted<<<grid, 256, 0, st>>>(sidx, ws.m_X32, ws.m_Y32, n_groups, cap, B.geom, B.flags, B.sX, B.sY, ck0, cv0);
  unsigned* ckey;
  int* cord;
  // cell ids are below cap_cells = 2^23: three 8-bit passes over 32-bit keys order them
  radix_sort<unsigned>(ck0, cv0, (unsigned*)B.ck1, B.cv1, n_groups, cap, 24, ws.m_hist, ws.num_sms, status, &ckey,
                       &cord, B.flags, st);
  k_mflag_status<<<1, 1, 0, st>>>(B.flags, status);
  k_mcell_heads<<<grid, 256, 0, st>>>(ckey, cord, B.sX, B.sY, n_groups, cap, B.flags, B.head, B.cX, B.cY);
  exclusive_scan<int>(B.head, cap, B.head_off, ws.scan_tiles, st);  // head_off[cap] = number of cells
  k_clear_i32<<<grid, 256, 0, st>>>(B.cell_of_id, ws.cap_cells, -1);
  cudaMemsetAsync(B.cov, 0, cov_bitmap_bytes(cap), st);
  cudaMemsetAsync(B.eval_stamp, 0, sizeof(unsigned) * (size_t)(cap > 0 ? cap : 1), st);
  cudaMemsetAsync(B.chg_stamp, 0, sizeof(unsigned) * (size_t)(cap > 0 ? cap : 1), st);
  k_mcell_fill<<<grid, 256, 0, st>>>(ckey, B.head, B.head_off, n_groups, cap, B.cell_beg, B.cell_end, B.cell_id,
                                     B.cell_of_id, B.state, cord, B.cinfo);
  k_mcell_end<<<grid, 256, 0, st>>>(B.cell_beg, B.head_off + cap, n_groups, cap, B.cell_end, B.cinfo);
  MergeView V;
  V.groups = groups;
  V.rec = ws.m_rec;
  V.sidx = sidx;
  V.sX = B.sX;
  V.sY = B.sY;
  V.sigma = sigma;
  V.iX = item_X;
  V.iY = item_Y;
  V.scl = scl;
  V.a2 = alpha * alpha;
  V.a2lo = rdown(V.a2 * (1.0 - 0x1p-20));
  V.a2hi = rup(V.a2 * (1.0 + 0x1p-20));
  RoundArgs R;
  R.V = V;
  R.cord = cord;
  R.cX = B.cX;
  R.cY = B.cY;
  R.cell_end = B.cell_end;
  R.cell_id = B.cell_id;
  R.cell_of_id = B.cell_of_id;
  R.state = B.state;
  R.cov = B.cov;
  R.cinfo = B.cinfo;
  R.s_pos = B.s_pos;
  R.s_base = B.s_base;
  R.s_pre = B.s_pre;
  R.s_q = B.s_q;
  R.s_lo = B.s_lo;
  R.chg_list = B.chg_list;
  R.eval_stamp = B.eval_stamp;
  R.chg_stamp = B.chg_stamp;
  R.chg_cnt = B.bar + 4;
  R.nctr = (unsigned long long*)(B.bar + 8);
  R.n_cells_p = B.head_off + cap;
  R.geom = B.geom;
  R.flags = B.flags;
  R.bar = B.bar;
  R.bar_sub = B.bar_sub;
  R.status = status;
  R.max_rounds = 1u << 22;
  {
    // cooperative launch: every block resident, so the bounded grid barrier can complete
    // (the one-phase kernel in CTAs of 4 or 8 warps, jabba_tuning.merge_warps)
    static PerDevice occ[3];  // k_mrounds, k_mrounds1<8>, k_mrounds1<4>
    const int max_per_sm[3] = {
        occ[0].get([] { int b = 0; cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_mrounds, 256, 0); return b < 1 ? 1 : b; }),
        occ[1].get([] { int b = 0; cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_mrounds1<8>, 256, 0); return b < 1 ? 1 : b; }),
        occ[2].get([] { int b = 0; cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_mrounds1<4>, 128, 0); return b < 1 ? 1 : b; })};
    const int form = ws.tune.merge_form == 1 ? (ws.tune.merge_warps == 4 ? 2 : 1) : 0;
    int blocks_per_sm = ws.tune.merge_ctas_per_sm;
    if (blocks_per_sm < 1) blocks_per_sm = 1;
    if (blocks_per_sm > max_per_sm[form]) blocks_per_sm = max_per_sm[form];  // co-residency of the cooperative grid
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ws.num_sms * blocks_per_sm));
    cfg.blockDim = dim3(form == 2 ? 128 : 256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    R.lcnt = B.bar + 4;
    R.uctr = (unsigned long long*)(B.bar + 8);
    R.slot_stride = B.slots;
    R.item_cap = cap > 0 ? cap : 1;
    mark(mk.a0, st);
    if (form == 2) cudaLaunchKernelEx(&cfg, k_mrounds1<4>, R);
    else if (form == 1) cudaLaunchKernelEx(&cfg, k_mrounds1<8>, R);
    else cudaLaunchKernelEx(&cfg, k_mrounds, R);
    mark(mk.a1, st);
  }
  k_mflag_status<<<1, 1, 0, st>>>(B.flags, status);
  k_mcheck<<<grid, 256, 0, st>>>(B.state, B.head_off + cap, B.flags, status);
  k_clear_i32<<<grid, 256, 0, st>>>(B.is_start, cap, 0);
  k_mlabel<<<grid, 256, 0, st>>>(V, cord, B.cX, B.cY, B.cell_of_id, B.state, B.cinfo, B.geom, B.flags, n_groups,
                                 cap, B.lab, B.is_start);
  // sequential fallback (only acts when flags[0] is set)
  k_mexact_prep<<<grid, 256, 0, st>>>(groups, item_X, item_Y, ws.m_rec, sidx, n_groups, cap, sigma, scl, key_mode,
                                      B.flags, B.eX, B.eY, B.ekey);
  k_mexact_greedy<<<1, 1024, 0, st>>>(B.eX, B.eY, B.ekey, n_groups, cap, alpha, key_mode, B.flags, B.lab,
                                      B.is_start);
  exclusive_scan<int>(B.is_start, cap, B.start_off, ws.scan_tiles, st);
  // (global id, record) by sorted position, in the cell keys' buffer (not
  // read after the cells were filled)
  int2* gr = (int2*)ckey;
  k_mids<<<grid, 256, 0, st>>>(B.lab, B.start_off, sidx, ws.m_rec, n_groups, cap, dict_capacity, l2g, gr, k, status,
                               B.flags);
  k_dict_clear<<<grid, 256, 0, st>>>(k, dict_capacity, ws.d_acc);
  k_dict_accumulate<<<grid, 256, 0, st>>>(groups, cord, gr, n_groups, cap, k, dict_capacity, ws.d_acc, B.flags);
  k_dict_finalize<<<grid, 256, 0, st>>>(ws.d_acc, k, dict_capacity, dict_len, dict_inc, dict_count);
}

// ------------------------------------------------------------------ block form of Sec. 5
// The two-stage digitization as the paper states it: one global sort of the
// normalised pieces by rho = X*X + Y*Y (binary64; equal keys in compact-piece
// order), the sorted order cut into contiguous blocks of ceil(N / M) pieces,
// each block aggregated by Stage I (the tile kernels, whose own sort keeps the
// block's order), and Stage II over the local groups' starting points.

// Binary64 key, compact index and compact copies of every piece (warp per domain).
__global__ void k_bf_keys(const int* piece_len, const double* piece_inc, const long long* dom_slot_off,
                          const int* dom_piece_cnt, const long long* dom_piece_off, long long n_domains,
                          const double* sigma, double scl, unsigned long long* keys, int* vals, int* clen,
                          double* cinc) {
  const int lane = threadIdx.x & 31;
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const double sl = sigma[0], si = sigma[1];
  for (long long d = w; d < n_domains; d += nw) {
    const int n = dom_piece_cnt[d];
    const long long s0 = dom_slot_off[d], c0 = dom_piece_off[d];
    for (int j = lane; j < n; j += 32) {
      const int len = piece_len[s0 + j];
      const double inc = piece_inc[s0 + j];
      const double X = __ddiv_rn(__dmul_rn(scl, (double)len), sl);
      const double Y = __ddiv_rn(inc, si);
      const double key = __dadd_rn(__dmul_rn(X, X), __dmul_rn(Y, Y));
      const long long c = c0 + j;
      keys[c] = (unsigned long long)__double_as_longlong(key);
      vals[c] = (int)c;
      clen[c] = len;
      cinc[c] = inc;
    }
  }
}

__global__ void k_bf_count(const long long* dom_piece_off, long long n_domains, long long* n_dev, int* flags) {
  *n_dev = dom_piece_off[n_domains];
  flags[0] = flags[1] = flags[2] = flags[3] = 0;
}

// Pieces in key order (block order) and the blocks' ranges.
__global__ void k_bf_gather(const int* sidx, const int* clen, const double* cinc, long long n, long long B, long long M,
                            int* order, int* blen, double* binc, long long* blk_off, int* blk_cnt,
                            const unsigned* status) {
  const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, step = (long long)gridDim.x * blockDim.x;
  // after an error the sort's output may be incomplete: the identity order
  // keeps every later index in bounds
  const bool err = *status != 0u;
  for (long long i = i0; i < n; i += step) {
    const int c = err ? (int)i : sidx[i];
    order[i] = c;
    blen[i] = clen[c];
    binc[i] = cinc[c];
  }
  for (long long b = i0; b <= M; b += step) {
    const long long lo = b * B < n ? b * B : n;
    blk_off[b] = lo;
    if (b < M) blk_cnt[b] = (int)((lo + B < n ? lo + B : n) - lo);
  }
}

// First piece (block order) of every local group: labels are assigned in
// key order, so the start is the group's smallest position.
__global__ void k_bf_start_init(int* start, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    start[i] = 0x7FFFFFFF;
}
__global__ void k_bf_starts(const int* local_label, const long long* blk_off, const int* blk_cnt,
                            const long long* blk_group_off, long long M, int* start) {
  const int lane = threadIdx.x & 31;
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long b = w; b < M; b += nw) {
    const long long o = blk_off[b], g0 = blk_group_off[b];
    const int n = blk_cnt[b];
    for (int j = lane; j < n; j += 32) atomicMin(&start[g0 + local_label[o + j]], (int)(o + j));
  }
}

// Binary64 point of every group record: its start piece, normalised (Eq. 4).
__global__ void k_bf_items(const jabba_group* groups, const long long* n_groups, long long cap,
                           const long long* blk_group_off, const int* start, const int* blen, const double* binc,
                           long long n_items, const double* sigma, double scl, double* iX, double* iY) {
  const long long G = clamp_groups(n_groups, cap);
  const double sl = sigma[0], si = sigma[1];
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < G; r += (long long)gridDim.x * blockDim.x) {
    const jabba_group g = groups[r];
    const int i = start[blk_group_off[g.domain] + g.local_id];
    if (i < 0 || i >= n_items) {  // a group without a piece: not produced by Stage I
      iX[r] = iY[r] = 0.0;
      continue;
    }
    iX[r] = __ddiv_rn(__dmul_rn(scl, (double)blen[i]), sl);
    iY[r] = __ddiv_rn(binc[i], si);
  }
}

__global__ void k_bf_scatter(const int* order, const int* src, long long n, int* dst) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[order[i]] = src[i];
}

long long bf_hist_words(long long n) { return rs_hist_words(n); }

void launch_block_order(const int* piece_len, const double* piece_inc, const long long* dom_slot_off,
                        const int* dom_piece_cnt, const long long* dom_piece_off, long long n_domains, long long n,
                        long long n_blocks, const double* sigma, double scl, BlockScratch& S, int* order, int* blen,
                        double* binc, long long* blk_off, int* blk_cnt, int num_sms, unsigned* status,
                        cudaStream_t st) {
  const unsigned grid = (unsigned)(num_sms * 8);
  k_bf_count<<<1, 1, 0, st>>>(dom_piece_off, n_domains, S.n_dev, S.flags);
  if (n_domains > 0)
    k_bf_keys<<<grid, 256, 0, st>>>(piece_len, piece_inc, dom_slot_off, dom_piece_cnt, dom_piece_off, n_domains, sigma,
                                    scl, S.k0, S.v0, S.clen, S.cinc);
  unsigned long long* skey = S.k0;
  int* sidx = S.v0;
  if (n > 0)
    radix_sort(S.k0, S.v0, S.k1, S.v1, S.n_dev, n, 64, S.hist, num_sms, status, &skey, &sidx, S.flags, st);
  const long long B = n > 0 ? (n + n_blocks - 1) / n_blocks : 1;
  k_bf_gather<<<grid, 256, 0, st>>>(sidx, S.clen, S.cinc, n, B, n_blocks, order, blen, binc, blk_off, blk_cnt,
                                    status);
}

void launch_block_items(const int* local_label, const long long* blk_off, const int* blk_cnt,
                        const long long* blk_group_off, long long n_blocks, const int* blen, const double* binc,
                        const jabba_group* groups, const long long* n_groups, long long group_capacity,
                        const double* sigma, double scl, int* start, long long n_items, double* item_X,
                        double* item_Y, int num_sms, cudaStream_t st) {
  const unsigned grid = (unsigned)(num_sms * 8);
  k_bf_start_init<<<grid, 256, 0, st>>>(start, group_capacity);
  if (n_blocks > 0)
    k_bf_starts<<<grid, 256, 0, st>>>(local_label, blk_off, blk_cnt, blk_group_off, n_blocks, start);
  k_bf_items<<<grid, 256, 0, st>>>(groups, n_groups, group_capacity, blk_group_off, start, blen, binc, n_items,
                                   sigma, scl, item_X, item_Y);
}

void launch_block_scatter(const int* order, const int* src, long long n, int* dst, int num_sms, cudaStream_t st) {
  if (n > 0) k_bf_scatter<<<(unsigned)(num_sms * 8), 256, 0, st>>>(order, src, n, dst);
}

}  // namespace jabba
