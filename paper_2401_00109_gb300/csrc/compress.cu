// compress.cu -- domain construction (Alg. 1 Phase I, Sec. 4.1.1) and the
// per-domain adaptive polygonal-chain compression (Sec. 3.1 Eq. 1; Alg. 1
// Phase II) of the JABBA path, plus the exact-sum statistics that the
// normalisation (Sec. 3.2 Eq. 4) needs.
#include "kernels.cuh"
#include <cmath>

namespace jabba {

// ------------------------------------------------------------------ domains
__device__ __forceinline__ long long series_domains(long long n_s, int mode, long long value) {
  if (n_s < 2 || value < 1) return 0;
  const long long iv = n_s - 1;
  if (mode == 0) return value < iv ? value : iv;
  return (iv + value - 1) / value;
}

__global__ void k_series_counts(const long long* series_off, long long n_series, int mode, long long value,
                                long long* dom_cnt, long long* slot_cnt) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_series) return;
  const long long n_s = series_off[s + 1] - series_off[s];
  dom_cnt[s] = series_domains(n_s, mode, value);
  slot_cnt[s] = n_s > 1 ? n_s - 1 : 0;
}

// Boundaries b_k of domain k of a series with iv intervals split into M domains.
__device__ __forceinline__ long long domain_bound(long long k, long long M, long long iv, int mode, long long value) {
  if (mode == 0) return (long long)(((unsigned __int128)k * (unsigned long long)iv) / (unsigned long long)M);
  const long long b = k * value;
  return b < iv ? b : iv;
}

__global__ void k_fill_domains(const long long* series_off, long long n_series, int mode, long long value,
                               const long long* series_dom_off, const long long* series_slot_off,
                               long long* dom_begin, long long* dom_end, int* dom_series, long long* dom_slot_off) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_series) return;
  const long long base = series_off[s], n_s = series_off[s + 1] - base;
  const long long M = series_domains(n_s, mode, value), iv = n_s - 1;
  const long long d0 = series_dom_off[s], slot0 = series_slot_off[s];
  for (long long k = 0; k < M; ++k) {
    const long long b0 = domain_bound(k, M, iv, mode, value);
    const long long b1 = domain_bound(k + 1, M, iv, mode, value);
    dom_begin[d0 + k] = base + b0;
    dom_end[d0 + k] = base + b1;
    dom_series[d0 + k] = (int)s;
    dom_slot_off[d0 + k] = slot0 + b0;
  }
}

__global__ void k_copy_scalar(const long long* src, long long* dst) { *dst = *src; }

void launch_build_domains(const long long* series_off, long long n_series, int mode, long long value,
                          long long* series_dom_off, long long* dom_begin, long long* dom_end, int* dom_series,
                          long long* dom_slot_off, long long n_domains, Scratch& ws, cudaStream_t st) {
  long long* dcnt = ws.series_a;
  long long* scnt = ws.series_b;
  long long* slot_off = ws.series_c;
  const unsigned g = (unsigned)((n_series + 255) / 256);
  if (g) k_series_counts<<<g, 256, 0, st>>>(series_off, n_series, mode, value, dcnt, scnt);
  exclusive_scan<long long>(dcnt, n_series, series_dom_off, ws.scan_tiles, st);
  exclusive_scan<long long>(scnt, n_series, slot_off, ws.scan_tiles, st);
  if (g) k_fill_domains<<<g, 256, 0, st>>>(series_off, n_series, mode, value, series_dom_off, slot_off, dom_begin,
                                           dom_end, dom_series, dom_slot_off);
  k_copy_scalar<<<1, 1, 0, st>>>(slot_off + n_series, dom_slot_off + n_domains);
}

// ------------------------------------------------------------------ compression
// One lane compresses one domain; a warp owns 32 domains at a time (work is
// stolen in tasks of 32 domains from a global counter).  The greedy consumes
// exactly one point per step whatever the breakpoints, so the 32 lanes stay
// in lockstep.  Each lane streams its domain through shared memory in chunks
// of kChunk points with a TMA bulk copy (cp.async.bulk) completing on a
// per-warp mbarrier, double-buffered.
//
// Admissibility of the candidate piece (s, e) (Eq. 1 multiplied by L^2,
// L = e - s): with D_i = x_{s+i} - x_s,
//   F(D) = sum_{i=1}^{L-1} (L D_i - i D_L)^2 = L^2 S2 - 2 L D_L SK + D_L^2 K2,
//   S2 = sum D_i^2, SK = sum i D_i, K2 = sum i^2,
// and the piece is admissible when F <= L^2 (L - 1) tol^2.  The lane keeps
// S2, SK, K2 of FP32 copies d_i (truncated conversion of x, FP32 difference)
// and evaluates E ~ F(d) in FP32 per point.  Certified bounds:
//   |E - F(d)| <= A = 2.2 (L + 8) 2^-24 (L^2 S2 + d_L^2 K2)    (rounding; the
//     cross term is bounded by Cauchy-Schwarz),
//   |sqrt F(d) - sqrt F(D)| <= h = 2 tau L sqrt(L - 1),  tau = 2^-20 max|x~|
//     over the piece (conversion and subtraction errors of the d_i, and the
//     binary64 rounding of the definition's own terms, with margin 2).
// Hence, squaring sqrt F +- h against sqrt(L^2 (L-1)) tol,
//   admissible   if E + A < L^2 (L - 1) (tol (1 - 2^-18) - 2^-99 - 2^-19 M)^2,
//   inadmissible if E - A > L^2 (L - 1) (tol (1 + 2^-18) + 2^-99 + 2^-19 M')^2,
// (M = max|x~|, M' = max(M, 2^-40); the 2^-18 slack covers the FP32 roundings
// of the tests themselves and the binary64 roundings of the definition's bound
// and sum, 2^-99 the absolute error of tiny values, and A carries an absolute
// 2^-100 for FP32 underflow).  Domains of 2^24 or more intervals (FP32
// lengths no longer exact) take the exact path at every point.
// Otherwise the whole warp evaluates the binary64 definition for that lane
// (32 terms at a time, exact fixed-point sum): see warp_exact_admissible.
constexpr unsigned kQuickPollLimit = 1024;  // run-time poll limits below this poll without suspending
// Stage size and CTA shape: one bulk copy stages kChunk points of a lane, so
// larger chunks mean fewer copies per point; 48-point chunks in CTAs of 4
// warps (two resident per SM by shared memory) were the fastest of the
// shapes swept on the scale workload (16 to 64 points, 2 to 8 warps).
constexpr int kChunk = 48;                 // points per lane per stage
constexpr int kRow = kChunk + 2;           // doubles per staged row (16-byte multiple, alignment slack)
constexpr int kWarpsPerCta = 4;
constexpr int kStages = 2;
constexpr size_t kStageBytes = sizeof(double) * kWarpsPerCta * kStages * 32 * kRow;  // dynamic shared memory

struct CompressParams {
  const double* x;
  long long n_points;
  const long long* dom_begin;
  const long long* dom_end;
  const long long* dom_slot_off;
  const int* dom_order;  // domains, longest first
  long long n_order;     // entries of dom_order this launch processes
  long long n_domains;
  double tol2;        // tol * tol, binary64
  float tol_lo;       // tol (1 - 2^-18) rounded down
  float tol_hi;       // tol (1 + 2^-18) rounded up
  int* piece_len;
  double* piece_end;  // end value of each piece; turned into increments afterwards
  int* dom_piece_cnt;
  unsigned* status;
  unsigned* task_counter;
  unsigned long long* n_exact;  // number of candidates decided by the exact binary64 path
};

// trunc(v * 2^96) of a finite double v >= 0 with v < 2^95, as 192 bits.
__device__ __forceinline__ I192 fx96(double v) {
  const u64 bits = (u64)__double_as_longlong(v);
  const int e = (int)((bits >> 52) & 0x7FF);
  I192 r = {0, 0, 0};
  if (e == 0) return r;
  const u64 m = (bits & ((1ull << 52) - 1)) | (1ull << 52);
  const int sh = e - 1075 + 96;
  if (sh <= -64) return r;
  if (sh < 0) { r.w0 = m >> (-sh); return r; }
  if (sh < 64) { r.w0 = m << sh; r.w1 = sh ? (m >> (64 - sh)) : 0; return r; }
  if (sh < 128) { const int t = sh - 64; r.w1 = m << t; r.w2 = t ? (m >> (64 - t)) : 0; return r; }
  r.w2 = m << (sh - 128);
  return r;
}

// The binary64 definition (Eq. 1 times L^2) for piece (s, e) of the domain
// starting at xb, evaluated by the whole warp: lane t computes the terms
// k = 1 + t, 33 + t, ... ; the squares are summed exactly (fixed point at
// 2^-96) and rounded once, so the result does not depend on the order.
__device__ __noinline__ bool warp_exact_admissible(const double* xb, int s, int e, double tol2) {
  const int lane = threadIdx.x & 31;
  const int L = e - s;
  const double dL = (double)L;
  const double xs = xb[s];
  const double inc = __dsub_rn(xb[e], xs);
  const double xsL = __dmul_rn(xs, dL);
  I192 acc = {0, 0, 0};
  for (int k = 1 + lane; k < L; k += 32) {
    const double n = __dsub_rn(__dadd_rn(xsL, __dmul_rn(inc, (double)k)), __dmul_rn(xb[s + k], dL));
    const I192 t = fx96(__dmul_rn(n, n));
    add192(acc, t.w0, t.w1, t.w2);
  }
  for (int o = 16; o > 0; o >>= 1) {
    const u64 b0 = __shfl_xor_sync(0xFFFFFFFFu, acc.w0, o);
    const u64 b1 = __shfl_xor_sync(0xFFFFFFFFu, acc.w1, o);
    const u64 b2 = __shfl_xor_sync(0xFFFFFFFFu, acc.w2, o);
    add192(acc, b0, b1, b2);
  }
  const double err_l2 = round_u192(acc.w0, acc.w1, acc.w2, -96, false);
  const double bound = __dmul_rn(__dmul_rn((double)(L - 1), tol2), __dmul_rn(dL, dL));
  return err_l2 <= bound;
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done) : "r"(bar), "r"(parity) : "memory");
  return done != 0;
}
// Non-blocking poll of the phase (returns at once).
__device__ __forceinline__ bool mbar_test_wait(unsigned bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done) : "r"(bar), "r"(parity) : "memory");
  return done != 0;
}
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

struct LaneDomain {
  long long b;      // global index of the domain's first point
  int n_int;        // intervals (points - 1); 0 = inactive lane
};

// Issue the staging copy of chunk c (local points 1 + c*kChunk ...) of this
// lane's domain into its row of buffer `buf`; every lane arrives once.
__device__ __forceinline__ int stage_chunk(const CompressParams& P, const LaneDomain& D, int c, double* row,
                                          unsigned bar) {
  const int p0 = 1 + c * kChunk;
  if (D.n_int <= 0 || p0 > D.n_int) {
    mbar_arrive(bar);
    return 0;
  }
  // 16-byte aligned start at or just below the first needed point (doubles
  // are 8-byte aligned, so at most one extra point is copied in front)
  const double* first = P.x + D.b + p0;
  const double* base = (const double*)((uintptr_t)first & ~(uintptr_t)15);
  const int off = (int)(first - base);
  long long end_needed = D.b + p0 + kChunk;
  if (end_needed > D.b + D.n_int + 1) end_needed = D.b + D.n_int + 1;
  const int cnt = (int)((P.x + end_needed) - base);
  int cnt_even = (cnt + 1) & ~1;
  bool manual = false;
  if (base + cnt_even > P.x + P.n_points) {  // never read past the end of x
    cnt_even = cnt - 1;
    manual = true;
  }
  const unsigned bytes = (unsigned)cnt_even * 8u;
  if (manual) row[cnt - 1] = base[cnt - 1];
  if (bytes) {
    mbar_arrive_tx(bar, bytes);
    bulk_g2s(smem_u32(row), base, bytes, bar);
  } else {
    mbar_arrive(bar);
  }
  return off;
}

// Per-lane state of the greedy on one domain.
struct LaneState {
  double prevd;                 // x at the previous point (end value of a piece)
  float xs, prevf, S2, SK, K2, Lf, M;
  int s;                        // start of the open piece (domain-local index)
  int cnt;                      // pieces written so far
  int* out_len;                 // the domain's first output slot
  double* out_end;
  float tlo, thi;               // tol (1 -+ 2^-18) -+ 2^-99; (-1, inf) forces the exact path
  unsigned amax;
};

// One point p (domain-local) of the lane's domain, value vd.  TAIL: lanes may
// be past their domain end (act = false) and a lane may reach its end.
template <bool TAIL>
__device__ __forceinline__ void step(const CompressParams& P, LaneState& L, const LaneDomain& D, int p, double vd,
                                     unsigned long long* n_exact) {
  const int lane = threadIdx.x & 31;
  const bool act = !TAIL || p <= D.n_int;
  unsigned mh;
  const float v = f64_to_f32_trunc(vd, mh);
  if (!TAIL || act) L.amax = max(L.amax, mh);
  float dd = v - L.xs;
  const float Ln = L.Lf + 1.0f;
  const float L2 = Ln * Ln;
  const float sq = dd * dd;
  const float t3 = sq * L.K2;
  const float cc = (Ln + Ln) * dd;
  const float E = fmaf(L2, L.S2, fmaf(-cc, L.SK, t3));
  const float Pp = fmaf(L2, L.S2, t3);
  const float B0 = L2 * (Ln - 1.0f);
  // rounding bound of E (relative, plus an absolute 2^-100 for FP32 underflow)
  const float A = fmaf(fmaf(Ln, 2.2f * 0x1p-24f, 2.2f * 8.0f * 0x1p-24f), Pp, 0x1p-100f);
  const float Mx = fmaxf(L.M, fabsf(v));
  const float clo = fmaf(-0x1p-19f, Mx, L.tlo);
  // at least 2^-40 in the inadmissibility margin: keeps chi^2 a normal number
  const float chi = fmaf(0x1p-19f, fmaxf(Mx, 0x1p-40f), L.thi);
  bool feas = (E + A < B0 * (clo * clo) && clo > 0.f) || Ln == 1.0f;
  const bool infeas = E - A > B0 * (chi * chi);
  const unsigned amb = __ballot_sync(0xFFFFFFFFu, act && !feas && !infeas);
  if (amb) {
    unsigned m = amb;
    while (m) {
      const int l = __ffs(m) - 1;
      m &= m - 1;
      const long long gb = __shfl_sync(0xFFFFFFFFu, D.b, l);
      const int sl = __shfl_sync(0xFFFFFFFFu, L.s, l);
      const int pl = __shfl_sync(0xFFFFFFFFu, p, l);
      const bool r = warp_exact_admissible(P.x + gb, sl, pl, P.tol2);
      if (lane == l) feas = r;
    }
    if (lane == 0) atomicAdd(n_exact, (unsigned long long)__popc(amb));
  }
  // Branch-free update: on a break (piece (s, p - 1) ends) the open piece
  // restarts at p - 1 with p as its first candidate; otherwise p extends it.
  const bool brk = act && !feas;
  if (brk) {
    L.out_len[L.cnt] = (p - 1) - L.s;
    L.out_end[L.cnt] = L.prevd;
  }
  L.cnt += brk ? 1 : 0;
  L.s = brk ? p - 1 : L.s;
  const float xs_n = brk ? L.prevf : L.xs;
  dd = v - xs_n;
  const float Ln_n = brk ? 1.0f : Ln;
  L.S2 = fmaf(dd, dd, brk ? 0.0f : L.S2);
  L.SK = fmaf(Ln_n, dd, brk ? 0.0f : L.SK);
  L.K2 = fmaf(Ln_n, Ln_n, brk ? 0.0f : L.K2);
  L.Lf = Ln_n;
  L.M = brk ? fmaxf(fabsf(L.prevf), fabsf(v)) : Mx;
  L.xs = xs_n;
  L.prevf = v;
  L.prevd = vd;
  if (TAIL && act && p == D.n_int) {  // domain end: the open piece ends here
    L.out_len[L.cnt] = p - L.s;
    L.out_end[L.cnt] = vd;
    L.cnt += 1;
  }
}

__global__ void __launch_bounds__(kWarpsPerCta * 32, 2) k_compress(CompressParams P) {
  extern __shared__ __align__(16) unsigned char stage_raw[];
  double(*stage)[kStages][32][kRow] = reinterpret_cast<double(*)[kStages][32][kRow]>(stage_raw);
  __shared__ __align__(8) unsigned long long bars[kWarpsPerCta][kStages];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane < kStages) mbar_init(smem_u32(&bars[warp][lane]), 32);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  unsigned phase0 = 0, phase1 = 0;
  const unsigned bar0 = smem_u32(&bars[warp][0]);
  const unsigned bar1 = smem_u32(&bars[warp][1]);
  const long long n_tasks = (P.n_order + 31) / 32;
  LaneState L;
  L.amax = 0;
  const unsigned lim = spin_limit(P.status);

  for (;;) {
    long long task = 0;
    if (lane == 0) task = (long long)atomicAdd(P.task_counter, 1u);
    task = __shfl_sync(0xFFFFFFFFu, task, 0);
    if (task >= n_tasks) break;
    const long long dt = task * 32 + lane;
    const long long d = dt < P.n_order ? (long long)P.dom_order[dt] : P.n_domains;
    LaneDomain D;
    long long slot = 0;
    D.b = 0;
    D.n_int = 0;
    if (d < P.n_domains) {
      D.b = P.dom_begin[d];
      D.n_int = (int)(P.dom_end[d] - D.b);
      slot = P.dom_slot_off[d];
    }
    int max_int = D.n_int, min_int = D.n_int;
    for (int o = 16; o > 0; o >>= 1) {
      max_int = max(max_int, __shfl_xor_sync(0xFFFFFFFFu, max_int, o));
      min_int = min(min_int, __shfl_xor_sync(0xFFFFFFFFu, min_int, o));
    }
    const int n_chunks = (max_int + kChunk - 1) / kChunk;
    const double* xb = P.x + D.b;

    L.out_len = P.piece_len + slot;
    L.out_end = P.piece_end + slot;
    L.cnt = 0;
    // FP32 lengths are exact below 2^24: longer domains take the exact path throughout
    L.tlo = D.n_int < (1 << 24) ? P.tol_lo : -1.0f;
    L.thi = D.n_int < (1 << 24) ? P.tol_hi : INFINITY;
    L.prevd = 0.0;
    L.xs = L.prevf = L.S2 = L.SK = L.K2 = L.Lf = L.M = 0.f;
    L.s = 0;
    if (D.n_int > 0) {
      L.prevd = xb[0];
      unsigned mh;
      L.xs = f64_to_f32_trunc(L.prevd, mh);
      L.amax = max(L.amax, mh);
      L.prevf = L.xs;
      L.M = fabsf(L.xs);
    }
    unsigned long long* n_exact = P.n_exact;

    int off_a = 0, off_b = 0;
    if (n_chunks > 0) off_a = stage_chunk(P, D, 0, stage[warp][0][lane], bar0);
    for (int c = 0; c < n_chunks; ++c) {
      const int buf = c & 1;
      if (c + 1 < n_chunks) {
        __syncwarp();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const int o = stage_chunk(P, D, c + 1, stage[warp][buf ^ 1][lane], buf ? bar0 : bar1);
        if (buf) off_a = o; else off_b = o;
      }
      // wait for this chunk (bounded); on timeout every lane leaves together
      {
        const unsigned bar = buf ? bar1 : bar0;
        const unsigned ph = buf ? phase1 : phase0;
        // try_wait may suspend the thread for a while on each poll; under a
        // small run-time limit (a test of the timeout path) the polls use
        // test_wait, which returns at once, so the limit bounds the wait
        unsigned spins = 0;
        bool ok = true;
        while (!(lim < kQuickPollLimit ? mbar_test_wait(bar, ph) : mbar_try_wait(bar, ph))) {
          if (++spins > lim) { ok = false; break; }
        }
        if (!__all_sync(0xFFFFFFFFu, ok)) {
          set_status(P.status, JABBA_ERR_TIMEOUT);
          // the pieces found so far stay valid (within the domain's slots), so
          // the kernels after this one read in bounds
          if (d < P.n_domains) P.dom_piece_cnt[d] = L.cnt;
          // give the copies still in flight a bounded time (the full limit,
          // whatever the run-time one) to land before the CTA's shared
          // memory is released
          unsigned sp = 0;
          while (!mbar_try_wait(bar0, phase0) && ++sp < kSpinLimit) {}
          sp = 0;
          while (!mbar_try_wait(bar1, phase1) && ++sp < kSpinLimit) {}
          return;
        }
        if (buf) phase1 ^= 1u; else phase0 ^= 1u;
      }
      const double* row = stage[warp][buf][lane] + (buf ? off_b : off_a);
      const int p0 = 1 + c * kChunk;
      if (p0 + kChunk - 1 < min_int) {
        // every lane has all kChunk points and none reaches its domain end
#pragma unroll 2
        for (int j = 0; j < kChunk; ++j) step<false>(P, L, D, p0 + j, row[j], n_exact);
      } else {
#pragma unroll 1
        for (int j = 0; j < kChunk; ++j) step<true>(P, L, D, p0 + j, row[j], n_exact);
      }
    }
    if (d < P.n_domains) P.dom_piece_cnt[d] = L.cnt;
  }
  // range / finiteness of every value this lane read
  if (L.amax >= 0x7FF00000u) set_status(P.status, JABBA_ERR_NONFINITE);
  else if (L.amax >= (1054u << 20)) set_status(P.status, JABBA_ERR_RANGE);
}

// ------------------------------------------------------------------ domain packing
// Domains are handed to warps longest first, 32 of similar length per task,
// so that the lanes of a warp finish together and the longest tasks start
// first.  Counting sort on length buckets of 64 intervals (descending).
constexpr int kLenBuckets = 1 << 16;

__device__ __forceinline__ int len_key(long long n_int) {
  long long b = n_int >> 6;
  if (b > kLenBuckets - 1) b = kLenBuckets - 1;
  return kLenBuckets - 1 - (int)b;  // descending length
}

// Warp-aggregated atomic add on counters[key]; returns this lane's slot.
__device__ __forceinline__ int agg_atomic(int* counters, int key, bool active) {
  const int lane = threadIdx.x & 31;
  const unsigned act = __ballot_sync(0xFFFFFFFFu, active);
  int slot = 0;
  if (active) {
    const unsigned peers = __match_any_sync(act, key);
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    int base = 0;
    if (lane == leader) base = atomicAdd(&counters[key], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    slot = base + rank;
  }
  return slot;
}

__global__ void k_dom_hist(const long long* dom_begin, const long long* dom_end, long long n_domains, int* hist) {
  for (long long d0 = (long long)blockIdx.x * blockDim.x; d0 < n_domains; d0 += (long long)gridDim.x * blockDim.x) {
    const long long d = d0 + threadIdx.x;
    const bool v = d < n_domains;
    const int key = v ? len_key(dom_end[d] - dom_begin[d]) : 0;
    agg_atomic(hist, key, v);
  }
}

__global__ void k_dom_cursor(const long long* off, int* cursor) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kLenBuckets; i += gridDim.x * blockDim.x)
    cursor[i] = (int)off[i];
}

__global__ void k_dom_scatter(const long long* dom_begin, const long long* dom_end, long long n_domains, int* cursor,
                              int* order) {
  for (long long d0 = (long long)blockIdx.x * blockDim.x; d0 < n_domains; d0 += (long long)gridDim.x * blockDim.x) {
    const long long d = d0 + threadIdx.x;
    const bool v = d < n_domains;
    const int key = v ? len_key(dom_end[d] - dom_begin[d]) : 0;
    const int slot = agg_atomic(cursor, key, v);
    if (v) order[slot] = (int)d;
  }
}

void launch_pack_domains(const long long* dom_begin, const long long* dom_end, long long n_domains, Scratch& ws,
                         cudaStream_t st) {
  if (n_domains <= 0) return;
  int* hist = ws.pack_hist;
  long long* off = ws.pack_off;
  cudaMemsetAsync(hist, 0, sizeof(int) * kLenBuckets, st);
  const unsigned g = (unsigned)(ws.num_sms * 4);
  k_dom_hist<<<g, 256, 0, st>>>(dom_begin, dom_end, n_domains, hist);
  exclusive_scan<int>(hist, kLenBuckets, off, ws.scan_tiles, st);
  k_dom_cursor<<<64, 256, 0, st>>>(off, hist);
  k_dom_scatter<<<g, 256, 0, st>>>(dom_begin, dom_end, n_domains, hist, ws.dom_order);
}

long long pack_buckets() { return kLenBuckets; }

// Natural order (no packing): domain d goes to lane d % 32 of task d / 32.
__global__ void k_dom_iota(long long n_domains, int* order) {
  for (long long d = (long long)blockIdx.x * blockDim.x + threadIdx.x; d < n_domains; d += (long long)gridDim.x * blockDim.x)
    order[d] = (int)d;
}

// ------------------------------------------------------------------ increments + statistics
// One warp per domain (grid-stride): turns the end values written by
// k_compress into increments inc_j = x_{e_j} - x_{s_j} (binary64, full-warp
// FP64) and accumulates the exact sums of the normalisation: N, sum len,
// sum len^2 (integers) and sum inc, sum inc^2 (exact squares), the latter two
// as 2^-64 fixed point.  stats layout (int64): [0] N, [1] sum len,
// [2..5] sum len^2 in four 32-bit deferred-carry limbs, [6..11] sum inc and
// [12..17] sum inc^2 in six 32-bit deferred-carry limbs each; with kProd
// (the PCA key) also [18..23] sum len * inc (exact products, each truncated
// toward zero at 2^-64), six limbs.
template <bool kProd>
__global__ void __launch_bounds__(256) k_finish_pieces(const double* x, const long long* dom_begin,
                                                       const long long* dom_slot_off, const int* dom_piece_cnt,
                                                       long long n_domains, const int* piece_len, double* piece_inc,
                                                       long long* stats) {
  const int lane = threadIdx.x & 31;
  const long long warp_g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long n_warps = ((long long)gridDim.x * blockDim.x) >> 5;
  unsigned long long n = 0, s1 = 0;
  U128 s2 = {0, 0};
  I192 a1 = {0, 0, 0}, a2 = {0, 0, 0}, a3 = {0, 0, 0};
  for (long long d = warp_g; d < n_domains; d += n_warps) {
    const int cnt = dom_piece_cnt[d];
    const long long slot = dom_slot_off[d];
    double prev_end = x[dom_begin[d]];
    // four chunks of 32 pieces per group, their loads in flight together
    // (the chunks of a group are then processed in order: each needs the end
    // value of the one before)
    for (int base0 = 0; base0 < cnt; base0 += 128) {
    int lenq[4];
    double endq[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = base0 + 32 * c + lane;
      lenq[c] = j < cnt ? piece_len[slot + j] : 0;
      endq[c] = j < cnt ? piece_inc[slot + j] : 0.0;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int base = base0 + 32 * c;
      if (base >= cnt) break;
      const int j = base + lane;
      const bool valid = j < cnt;
      const int len = lenq[c];
      const double endv = endq[c];
      double startv = __shfl_up_sync(0xFFFFFFFFu, endv, 1);
      if (lane == 0) startv = prev_end;
      const double inc = __dsub_rn(endv, startv);
      const int last = min(31, cnt - 1 - base);
      prev_end = __shfl_sync(0xFFFFFFFFu, endv, last);
      if (valid) {
        piece_inc[slot + j] = inc;
        n += 1;
        s1 += (unsigned long long)len;
        const unsigned long long l2 = (unsigned long long)len * (unsigned long long)len;
        s2.lo += l2;
        s2.hi += (s2.lo < l2) ? 1ull : 0ull;
        bool neg;
        const U128 m = fx_mag(inc, neg);
        acc_signed(a1, m, neg);
        const U128 q = fx_square(inc);
        add192(a2, q.lo, q.hi, 0);
        if (kProd) acc_signed(a3, fx_prod(inc, (unsigned)len), neg);
      }
    }
    }
  }
  // warp reduction of limbs, then one set of atomics per warp
  constexpr int kL = kProd ? 24 : 18;
  i64 L[24];
  L[0] = (i64)n;
  L[1] = (i64)s1;
  L[2] = (i64)(s2.lo & 0xFFFFFFFFull);
  L[3] = (i64)(s2.lo >> 32);
  L[4] = (i64)(s2.hi & 0xFFFFFFFFull);
  L[5] = (i64)(s2.hi >> 32);
  limbs6(a1, L + 6);
  limbs6(a2, L + 12);
  if (kProd) limbs6(a3, L + 18);
#pragma unroll
  for (int i = 0; i < kL; ++i) {
    i64 v = L[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    L[i] = v;
  }
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < kL; ++i)
      if (L[i]) atomicAdd((unsigned long long*)&stats[i], (unsigned long long)L[i]);
  }
}

// sigma_len, sigma_inc from the exact sums (Sec. 3.2 Eq. 4): m = S1 / N,
// v = S2 / N - m * m, sigma = sqrt(v), or 1 when v <= 0 (binary64, IEEE ops).
__device__ double sigma_from(double s1, double s2, double n) {
  const double m = __ddiv_rn(s1, n);
  const double v = __dsub_rn(__ddiv_rn(s2, n), __dmul_rn(m, m));
  if (!(v > 0.0)) return 1.0;
  return __dsqrt_rn(v);
}

// PCA key (Sec. 5 "PCA projection"): the first principal axis of the
// normalised pieces.  Normalising by the population standard deviations makes
// their covariance [[scl^2, scl r], [scl r, 1]] in exact arithmetic (a zero
// variance stays zero), r = cov(len, inc) / (sigma_len sigma_inc) from the
// exact sums; the leading eigenvector by the closed form
//   b = 0: (1, 0) if a >= d else (0, 1); h = (a - d) / 2,
//   lam = (a + d) / 2 + sqrt(h h + b b), v = (lam - d, b) if a >= d else
//   (b, lam - a), normalised, vx > 0 (or vx = 0 and vy > 0);
// binary64 operations in this order.
__device__ void pca_axis(double n, double s1, double s2, double i1, double i2, double li, double scl, double* vx_out,
                         double* vy_out) {
  const double ml = __ddiv_rn(s1, n), mi = __ddiv_rn(i1, n);
  const double vl = __dsub_rn(__ddiv_rn(s2, n), __dmul_rn(ml, ml));
  const double vi = __dsub_rn(__ddiv_rn(i2, n), __dmul_rn(mi, mi));
  const double sl = sigma_from(s1, s2, n), si = sigma_from(i1, i2, n);
  const double c = __dsub_rn(__ddiv_rn(li, n), __dmul_rn(ml, mi));
  const double r = __ddiv_rn(c, __dmul_rn(sl, si));
  const bool var_l = vl > 0.0, var_i = vi > 0.0;
  const double a = var_l ? __dmul_rn(scl, scl) : 0.0;
  const double d = var_i ? 1.0 : 0.0;
  const double b = (var_l && var_i) ? __dmul_rn(scl, r) : 0.0;
  double vx, vy;
  if (b == 0.0) {
    vx = a >= d ? 1.0 : 0.0;
    vy = a >= d ? 0.0 : 1.0;
  } else {
    const double h = __ddiv_rn(__dsub_rn(a, d), 2.0);
    const double lam = __dadd_rn(__ddiv_rn(__dadd_rn(a, d), 2.0), __dsqrt_rn(__dadd_rn(__dmul_rn(h, h), __dmul_rn(b, b))));
    if (a >= d) {
      vx = __dsub_rn(lam, d);
      vy = b;
    } else {
      vx = b;
      vy = __dsub_rn(lam, a);
    }
    const double sn = __dsqrt_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)));
    vx = __ddiv_rn(vx, sn);
    vy = __ddiv_rn(vy, sn);
    if (vx < 0.0 || (vx == 0.0 && vy < 0.0)) {
      vx = -vx;
      vy = -vy;
    }
  }
  *vx_out = vx;
  *vy_out = vy;
}

__global__ void k_sigma(const long long* stats, double* sigma, int key_mode, double scl) {
  const double n = __ll2double_rn(stats[0]);
  const double s1 = __ll2double_rn(stats[1]);
  // sum len^2 from four unsigned 32-bit deferred-carry limbs
  u64 w[4];
  u64 carry = 0;
  for (int i = 0; i < 4; ++i) {
    const u64 v = (u64)stats[2 + i] + carry;
    w[i] = v & 0xFFFFFFFFull;
    carry = v >> 32;
  }
  const u64 lo = w[0] | (w[1] << 32), hi = w[2] | (w[3] << 32);
  const double s2 = round_u192(lo, hi, carry, 0, false);
  i64 L1[6], L2[6];
  for (int i = 0; i < 6; ++i) {
    L1[i] = stats[6 + i];
    L2[i] = stats[12 + i];
  }
  const double i1 = i192_to_double(from_limbs6(L1));
  const double i2 = i192_to_double(from_limbs6(L2));
  sigma[0] = sigma_from(s1, s2, n);
  sigma[1] = sigma_from(i1, i2, n);
  if (key_mode == 1) {  // sigma[2], sigma[3]: the PCA axis
    i64 L3[6];
    for (int i = 0; i < 6; ++i) L3[i] = stats[18 + i];
    const double li = i192_to_double(from_limbs6(L3));
    if (!(n > 0.0)) {
      sigma[2] = 1.0;
      sigma[3] = 0.0;
    } else {
      pca_axis(n, s1, s2, i1, i2, li, scl, &sigma[2], &sigma[3]);
    }
  }
}

void launch_compress(const double* x, long long n_points, const long long* dom_begin, const long long* dom_end,
                     const long long* dom_slot_off, long long n_domains, double tol, int* piece_len,
                     double* piece_inc, int* dom_piece_cnt, long long* dom_piece_off, long long* stats,
                     bool with_products, Scratch& ws, unsigned* status, cudaStream_t st, const Marks& mk) {
  CompressParams P;
  P.x = x;
  P.n_points = n_points;
  P.dom_begin = dom_begin;
  P.dom_end = dom_end;
  P.dom_slot_off = dom_slot_off;
  P.dom_order = ws.dom_order;
  P.n_domains = n_domains;
  P.n_order = n_domains;
  P.tol2 = tol * tol;
  {
    // tau also carries an absolute 2^-100 (conversion of |x| < 2^-126), so the
    // certified margins subtract / add 2^-99 in tol units
    const double lo = tol * (1.0 - 0x1p-18) - 0x1p-99, hi = tol * (1.0 + 0x1p-18) + 0x1p-99;
    P.tol_lo = (float)lo;
    if ((double)P.tol_lo > lo) P.tol_lo = nextafterf(P.tol_lo, 0.0f);
    P.tol_hi = (float)hi;
    if ((double)P.tol_hi < hi) P.tol_hi = nextafterf(P.tol_hi, INFINITY);
    if (!(hi < 3.0e38)) P.tol_hi = INFINITY;
  }
  P.piece_len = piece_len;
  P.piece_end = piece_inc;
  P.dom_piece_cnt = dom_piece_cnt;
  P.status = status;
  P.task_counter = ws.counters;
  P.n_exact = (unsigned long long*)(ws.counters + 2);
  cudaMemsetAsync(ws.counters, 0, 4 * sizeof(unsigned), st);
  cudaMemsetAsync(stats, 0, JABBA_PIECE_STATS_BYTES, st);
  const long long n_tasks = (n_domains + 31) / 32;
  int per_sm = ws.tune.compress_ctas_per_sm;
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 3) per_sm = 3;  // 2 are resident (shared memory); a third CTA per SM waits for a slot
  static PerDevice attr;
  attr.get([] {
    cudaFuncSetAttribute(k_compress, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStageBytes);
    return 1;
  });
  long long ctas = (long long)ws.num_sms * per_sm;
  const long long need = (n_tasks + kWarpsPerCta - 1) / kWarpsPerCta;
  if (ctas > need) ctas = need;
  mark(mk.a0, st);  // the compression time includes the domain packing
  if (ws.tune.per_domain_launch) {
    // the plain form: one launch (one CTA, one active lane) per domain, in order
    if (n_domains > 0) {
      k_dom_iota<<<(unsigned)(ws.num_sms * 4), 256, 0, st>>>(n_domains, ws.dom_order);
      cudaMemsetAsync(ws.plain_ctr, 0, sizeof(unsigned) * (size_t)n_domains, st);
    }
    CompressParams Q = P;
    Q.n_order = 1;
    for (long long d = 0; d < n_domains; ++d) {
      Q.dom_order = ws.dom_order + d;
      Q.task_counter = ws.plain_ctr + d;
      k_compress<<<1, kWarpsPerCta * 32, kStageBytes, st>>>(Q);
    }
  } else {
    if (ws.tune.compress_pack) {
      launch_pack_domains(dom_begin, dom_end, n_domains, ws, st);
    } else if (n_domains > 0) {
      k_dom_iota<<<(unsigned)(ws.num_sms * 4), 256, 0, st>>>(n_domains, ws.dom_order);
    }
    if (ctas > 0) k_compress<<<(unsigned)ctas, kWarpsPerCta * 32, kStageBytes, st>>>(P);
  }
  mark(mk.a1, st);
  mark(mk.b0, st);
  if (n_domains > 0) {
    long long blocks = (n_domains + 7) / 8;
    if (blocks > (long long)ws.num_sms * 16) blocks = (long long)ws.num_sms * 16;
    auto fin = with_products ? k_finish_pieces<true> : k_finish_pieces<false>;
    fin<<<(unsigned)blocks, 256, 0, st>>>(x, dom_begin, dom_slot_off, dom_piece_cnt, n_domains,
                                                      piece_len, piece_inc, stats);
  }
  exclusive_scan<int>(dom_piece_cnt, n_domains, dom_piece_off, ws.scan_tiles, st);
  mark(mk.b1, st);
}

void launch_sigma(const long long* stats, double* sigma, int key_mode, double scl, cudaStream_t st) {
  k_sigma<<<1, 1, 0, st>>>(stats, sigma, key_mode, scl);
}

}  // namespace jabba
