// digitize.cu -- Stage I of the two-stage digitization (Sec. 5): per-domain
// greedy aggregation (Sec. 3.2, fABBA) of the normalised pieces (Eq. 4),
// with exact group sums.
#include "kernels.cuh"

namespace jabba {

constexpr int kLocalThreads = 256;
constexpr int kLocalMax = 4096;  // pieces per domain held in shared memory

struct LocalView {
  double* key;   // [np] squared norms, sorted in place with idx
  double* X;     // [n] normalised length coordinate, by position
  double* Y;     // [n] normalised increment coordinate, by position
  int* idx;      // [np] position of each sorted entry
  int* label;    // [n] local group id by position
  int* gcnt;     // [n] members per group, then running cursor
  int* goff;     // [n + 1] group offsets
  int* members;  // [n] positions grouped by label
};

__device__ __forceinline__ bool kp_greater(double ka, int ia, double kb, int ib) {
  return ka > kb || (ka == kb && ia > ib);
}

// Normalised coordinates (Eq. 4) and the sort key, binary64 with the
// definition's operation order: X = (scl * len) / sigma_len,
// Y = inc / sigma_inc, key = X * X + Y * Y.
__device__ __forceinline__ void coords(int len, double inc, double scl, double sl, double si, double& X, double& Y,
                                       double& key) {
  X = __ddiv_rn(__dmul_rn(scl, (double)len), sl);
  Y = __ddiv_rn(inc, si);
  key = __dadd_rn(__dmul_rn(X, X), __dmul_rn(Y, Y));
}

__device__ __forceinline__ double dist2(double xa, double ya, double xb, double yb) {
  const double dx = __dsub_rn(xb, xa), dy = __dsub_rn(yb, ya);
  return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

// Threshold on the key beyond which no later point can be within alpha of a
// start with key ks: ((sqrt(ks) + alpha)^2) (1 + 2^-30).  Conservative: a
// point whose key exceeds it has norm > norm(start) + alpha (1 + 2^-33), so
// its binary64 distance test would fail (Sec. 5 pruning, made lossless).
__device__ __forceinline__ double gap_threshold(double ks, double alpha) {
  const double r = __dadd_rn(__dsqrt_rn(ks), alpha);
  return __dmul_rn(__dmul_rn(r, r), 1.0 + 0x1p-30);
}

// Whole-CTA aggregation of one domain (n >= 1 pieces).
__device__ void aggregate_domain(const int* plen, const double* pinc, int n, double scl, double sl, double si,
                                 double alpha, LocalView V, int* s_G, long long* s_base, long long domain,
                                 int* local_label, jabba_group* groups, long long group_capacity,
                                 long long* n_groups, unsigned* status) {
  const int tid = threadIdx.x, nt = blockDim.x;
  int np = 1;
  while (np < n) np <<= 1;
  for (int i = tid; i < np; i += nt) {
    if (i < n) {
      double X, Y, key;
      coords(plen[i], pinc[i], scl, sl, si, X, Y, key);
      V.X[i] = X;
      V.Y[i] = Y;
      V.key[i] = key;
      V.idx[i] = i;
      V.label[i] = -1;
    } else {
      V.key[i] = __longlong_as_double(0x7FF0000000000000ll);
      V.idx[i] = 0x7FFFFFFF;
    }
  }
  __syncthreads();
  // bitonic sort of (key, idx) ascending
  for (int k = 2; k <= np; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < np; i += nt) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const double ka = V.key[i], kb = V.key[ixj];
          const int ia = V.idx[i], ib = V.idx[ixj];
          const bool up = (i & k) == 0;
          if (up ? kp_greater(ka, ia, kb, ib) : kp_greater(kb, ib, ka, ia)) {
            V.key[i] = kb;
            V.key[ixj] = ka;
            V.idx[i] = ib;
            V.idx[ixj] = ia;
          }
        }
      }
      __syncthreads();
    }
  }
  // greedy aggregation in key order (warp 0)
  const double a2 = __dmul_rn(alpha, alpha);
  if (tid < 32) {
    const int lane = tid;
    int a = 0, g = 0;
    for (;;) {
      // next unassigned entry at or after a
      for (;;) {
        const int aa = a + lane;
        const bool free_ = aa < n && V.label[V.idx[aa]] < 0;
        const unsigned m = __ballot_sync(0xFFFFFFFFu, free_);
        if (m) { a += __ffs(m) - 1; break; }
        a += 32;
        if (a >= n) break;
      }
      if (a >= n) break;
      const int i = V.idx[a];
      const double xi = V.X[i], yi = V.Y[i];
      const double T = gap_threshold(V.key[a], alpha);
      if (lane == 0) V.label[i] = g;
      for (int b = a + 1; b < n; b += 32) {
        const int bb = b + lane;
        bool stop = true;
        if (bb < n) {
          stop = V.key[bb] > T;
          if (!stop) {
            const int j = V.idx[bb];
            if (V.label[j] < 0 && dist2(xi, yi, V.X[j], V.Y[j]) <= a2) V.label[j] = g;
          }
        }
        if (__any_sync(0xFFFFFFFFu, stop)) break;
      }
      __syncwarp();
      ++g;
      ++a;
    }
    if (lane == 0) *s_G = g;
  }
  __syncthreads();
  const int G = *s_G;
  // group members: count, offsets, scatter
  for (int g = tid; g < G; g += nt) V.gcnt[g] = 0;
  __syncthreads();
  for (int i = tid; i < n; i += nt) atomicAdd(&V.gcnt[V.label[i]], 1);
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int g = 0; g < G; ++g) {
      V.goff[g] = acc;
      acc += V.gcnt[g];
      V.gcnt[g] = 0;
    }
    V.goff[G] = acc;
    const long long base = (long long)atomicAdd((unsigned long long*)n_groups, (unsigned long long)G);
    if (base + G > group_capacity) {
      set_status(status, JABBA_ERR_CAPACITY);
      *s_base = -1;
    } else {
      *s_base = base;
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    const int g = V.label[i];
    const int r = atomicAdd(&V.gcnt[g], 1);
    V.members[V.goff[g] + r] = i;
    local_label[i] = g;
  }
  __syncthreads();
  if (*s_base >= 0) {
    const long long base = *s_base;
    for (int g = tid; g < G; g += nt) {
      I192 acc = {0, 0, 0};
      long long lensum = 0;
      for (int q = V.goff[g]; q < V.goff[g + 1]; ++q) {
        const int i = V.members[q];
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
      rec.count = V.goff[g + 1] - V.goff[g];
      rec.local_id = g;
      rec.domain = (int)domain;
      rec.pad = 0;
      groups[base + g] = rec;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kLocalThreads) k_local_smem(const int* piece_len, const double* piece_inc,
                                                              const long long* dom_slot_off, const int* dom_piece_cnt,
                                                              long long n_domains, const double* sigma, double alpha,
                                                              double scl, int* local_label, int* dom_group_cnt,
                                                              jabba_group* groups, long long group_capacity,
                                                              long long* n_groups, unsigned* status) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_misc[4];
  __shared__ long long s_base;
  LocalView V;
  V.key = (double*)smem;
  V.X = V.key + kLocalMax;
  V.Y = V.X + kLocalMax;
  V.idx = (int*)(V.Y + kLocalMax);
  V.label = V.idx + kLocalMax;
  V.gcnt = V.label + kLocalMax;
  V.goff = V.gcnt + kLocalMax;
  V.members = V.goff + kLocalMax + 1;
  const double sl = sigma[0], si = sigma[1];
  for (long long d = blockIdx.x; d < n_domains; d += gridDim.x) {
    const int n = dom_piece_cnt[d];
    if (n > kLocalMax) continue;  // handled by k_local_big
    if (n == 0) {
      if (threadIdx.x == 0) dom_group_cnt[d] = 0;
      continue;
    }
    const long long slot = dom_slot_off[d];
    aggregate_domain(piece_len + slot, piece_inc + slot, n, scl, sl, si, alpha, V, &s_misc[0], &s_base, d,
                     local_label + slot, groups, group_capacity, n_groups, status);
    if (threadIdx.x == 0) dom_group_cnt[d] = s_misc[0];
  }
}

// Domains with more pieces than the shared-memory tile: one CTA walks them in
// turn with a global-memory view sized by the largest domain.
__global__ void __launch_bounds__(kLocalThreads) k_local_big(const int* piece_len, const double* piece_inc,
                                                             const long long* dom_slot_off, const int* dom_piece_cnt,
                                                             long long n_domains, const double* sigma, double alpha,
                                                             double scl, int* local_label, int* dom_group_cnt,
                                                             jabba_group* groups, long long group_capacity,
                                                             long long* n_groups, unsigned char* scratch,
                                                             long long cap, unsigned* status) {
  __shared__ int s_misc[4];
  __shared__ long long s_base;
  const double sl = sigma[0], si = sigma[1];
  for (long long d = 0; d < n_domains; ++d) {
    const int n = dom_piece_cnt[d];
    if (n <= kLocalMax) continue;
    long long np = 1;
    while (np < n) np <<= 1;
    if (np > cap) {
      if (threadIdx.x == 0) {
        set_status(status, JABBA_ERR_CAPACITY);
        dom_group_cnt[d] = 0;
      }
      continue;
    }
    LocalView V;
    V.key = (double*)scratch;
    V.X = V.key + cap;
    V.Y = V.X + cap;
    V.idx = (int*)(V.Y + cap);
    V.label = V.idx + cap;
    V.gcnt = V.label + cap;
    V.goff = V.gcnt + cap;
    V.members = V.goff + cap + 1;
    const long long slot = dom_slot_off[d];
    aggregate_domain(piece_len + slot, piece_inc + slot, n, scl, sl, si, alpha, V, &s_misc[0], &s_base, d,
                     local_label + slot, groups, group_capacity, n_groups, status);
    if (threadIdx.x == 0) dom_group_cnt[d] = s_misc[0];
    __syncthreads();
  }
}

constexpr size_t kLocalSmem = (size_t)kLocalMax * (8 * 3 + 4 * 5) + 16;

size_t local_big_bytes(long long cap) { return (size_t)cap * (8 * 3 + 4 * 5) + 16; }

void launch_local(const int* piece_len, const double* piece_inc, const long long* dom_slot_off,
                  const int* dom_piece_cnt, long long n_domains, const double* sigma, double alpha, double scl,
                  int* local_label, int* dom_group_cnt, long long* dom_group_off, jabba_group* groups,
                  long long group_capacity, long long* n_groups, Scratch& ws, unsigned* status, cudaStream_t st) {
  cudaMemsetAsync(n_groups, 0, sizeof(long long), st);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_local_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLocalSmem);
    attr_set = true;
  }
  if (n_domains > 0) {
    long long blocks = n_domains;
    if (blocks > (long long)ws.num_sms * 8) blocks = (long long)ws.num_sms * 8;
    k_local_smem<<<(unsigned)blocks, kLocalThreads, kLocalSmem, st>>>(piece_len, piece_inc, dom_slot_off,
                                                                     dom_piece_cnt, n_domains, sigma, alpha, scl,
                                                                     local_label, dom_group_cnt, groups,
                                                                     group_capacity, n_groups, status);
    k_local_big<<<1, kLocalThreads, 0, st>>>(piece_len, piece_inc, dom_slot_off, dom_piece_cnt, n_domains, sigma,
                                             alpha, scl, local_label, dom_group_cnt, groups, group_capacity,
                                             n_groups, ws.big, ws.cap_big, status);
  }
  exclusive_scan<int>(dom_group_cnt, n_domains, dom_group_off, ws.scan_tiles, st);
}

}  // namespace jabba
