// merge.cu -- Stage II of the two-stage digitization (Sec. 5): the local
// groups, taken at their centres, are aggregated once more by the same
// greedy; the result maps every local group to a global group and the
// dictionary entries are the exact means of their member pieces.
#include "kernels.cuh"

namespace jabba {

// ------------------------------------------------------------------ centres, keys
// One thread per group record: compact index c = dom_group_off[domain] +
// local_id, centre (lensum / count, round(inc) / count), normalised point
// X = (scl * c_len) / sigma_len, Y = c_inc / sigma_inc, key X*X + Y*Y.
__device__ __forceinline__ long long clamp_groups(const long long* n_p, long long cap) {
  const long long g = *n_p;
  return g < cap ? g : cap;  // past capacity the records were not written (status already set)
}

__global__ void k_merge_prep(const jabba_group* groups, const long long* n_groups_p, long long cap,
                             const long long* dom_group_off, const double* sigma, double scl, double* X, double* Y,
                             unsigned long long* keys, int* vals, int* rec_of) {
  const long long G = clamp_groups(n_groups_p, cap);
  const double sl = sigma[0], si = sigma[1];
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < G; r += (long long)gridDim.x * blockDim.x) {
    const jabba_group g = groups[r];
    const long long c = dom_group_off[g.domain] + g.local_id;
    I192 inc;
    inc.w0 = g.inc[0];
    inc.w1 = g.inc[1];
    inc.w2 = g.inc[2];
    const double cnt = (double)g.count;
    const double c_len = __ddiv_rn((double)g.lensum, cnt);
    const double c_inc = __ddiv_rn(i192_to_double(inc), cnt);
    const double x = __ddiv_rn(__dmul_rn(scl, c_len), sl);
    const double y = __ddiv_rn(c_inc, si);
    const double key = __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y));
    X[c] = x;
    Y[c] = y;
    keys[c] = (unsigned long long)__double_as_longlong(key);  // key >= 0: bit order = value order
    vals[c] = (int)c;
    rec_of[c] = (int)r;
  }
}

// ------------------------------------------------------------------ LSD radix sort (stable)
// 8-bit digits; per pass: tile histograms, one scan over (digit, tile), and a
// stable scatter in which each warp owns a contiguous run of its tile.
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kSortWarps = kSortThreads / 32;

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const unsigned long long* keys, const long long* n_p,
                                                            long long cap, int shift, unsigned* hist,
                                                            long long n_tiles) {
  __shared__ unsigned h[256];
  const long long n = clamp_groups(n_p, cap);
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kSortTile;
  for (int i = threadIdx.x; i < kSortTile; i += blockDim.x) {
    const long long k = base + i;
    if (k < n) atomicAdd(&h[(keys[k] >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[(long long)i * n_tiles + blockIdx.x] = h[i];
}

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const unsigned long long* kin, const int* vin,
                                                               unsigned long long* kout, int* vout,
                                                               const long long* n_p, long long cap, int shift,
                                                               const long long* offs, long long n_tiles) {
  __shared__ unsigned wh[kSortWarps][256];
  const long long n = clamp_groups(n_p, cap);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long base = (long long)blockIdx.x * kSortTile;
  const int per_warp = kSortTile / kSortWarps;
  const long long wbase = base + (long long)warp * per_warp;
  for (int i = lane; i < 256; i += 32) wh[warp][i] = 0;
  __syncwarp();
  for (int i = lane; i < per_warp; i += 32) {
    const long long k = wbase + i;
    if (k < n) atomicAdd(&wh[warp][(kin[k] >> shift) & 255u], 1u);
  }
  __syncthreads();
  // exclusive prefix over warps per digit, plus the global offset of (digit, tile)
  for (int dgt = threadIdx.x; dgt < 256; dgt += blockDim.x) {
    unsigned run = (unsigned)offs[(long long)dgt * n_tiles + blockIdx.x];
    for (int w = 0; w < kSortWarps; ++w) {
      const unsigned c = wh[w][dgt];
      wh[w][dgt] = run;
      run += c;
    }
  }
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  for (int i0 = 0; i0 < per_warp; i0 += 32) {
    const long long k = wbase + i0 + lane;
    const bool valid = k < n;
    const unsigned long long key = valid ? kin[k] : 0ull;
    const int val = valid ? vin[k] : 0;
    const unsigned dgt = valid ? (unsigned)((key >> shift) & 255u) : 256u + lane;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, dgt);
    const unsigned rank = __popc(peers & lt);
    if (valid) {
      const unsigned pos = wh[warp][dgt] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncwarp();
    if (valid && rank == 0) wh[warp][dgt] += __popc(peers);
    __syncwarp();
  }
}

__global__ void k_u32_to_i64(const unsigned* in, long long n, long long* out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = in[i];
}

// ------------------------------------------------------------------ greedy (one CTA)
// Items in sorted order; each unassigned item starts a global group and
// every later unassigned item within alpha joins it (Sec. 3.2), scanning
// until the conservative key-gap threshold (Sec. 5 pruning).
__device__ __forceinline__ double dist2m(double xa, double ya, double xb, double yb) {
  const double dx = __dsub_rn(xb, xa), dy = __dsub_rn(yb, ya);
  return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

__global__ void __launch_bounds__(1024) k_merge_greedy(const unsigned long long* skeys, const int* sidx,
                                                      const double* X, const double* Y, const long long* n_p,
                                                      long long cap, double alpha, int* label_c, long long* k_out,
                                                      long long dict_capacity, unsigned* status) {
  __shared__ int s_next;
  __shared__ int s_stop;
  const long long n = clamp_groups(n_p, cap);
  const int tid = threadIdx.x, nt = blockDim.x;
  const double a2 = __dmul_rn(alpha, alpha);
  for (long long i = tid; i < n; i += nt) label_c[i] = -1;
  __syncthreads();
  long long a = 0;
  int g = 0;
  for (;;) {
    // next unassigned sorted entry at or after a
    for (;;) {
      if (tid == 0) s_next = 0x7FFFFFFF;
      __syncthreads();
      const long long aa = a + tid;
      if (aa < n && label_c[sidx[aa]] < 0) atomicMin(&s_next, tid);
      __syncthreads();
      const int nx = s_next;
      __syncthreads();
      if (nx != 0x7FFFFFFF) { a += nx; break; }
      a += nt;
      if (a >= n) break;
    }
    if (a >= n) break;
    const int ci = sidx[a];
    const double xi = X[ci], yi = Y[ci];
    const double ks = __longlong_as_double((long long)skeys[a]);
    const double r = __dadd_rn(__dsqrt_rn(ks), alpha);
    const double T = __dmul_rn(__dmul_rn(r, r), 1.0 + 0x1p-30);
    if (tid == 0) label_c[ci] = g;
    for (long long b = a + 1; b < n; b += nt) {
      if (tid == 0) s_stop = 0;
      __syncthreads();
      const long long bb = b + tid;
      if (bb < n) {
        const double kb = __longlong_as_double((long long)skeys[bb]);
        if (kb > T) {
          s_stop = 1;
        } else {
          const int cj = sidx[bb];
          if (label_c[cj] < 0 && dist2m(xi, yi, X[cj], Y[cj]) <= a2) label_c[cj] = g;
        }
      } else {
        s_stop = 1;
      }
      __syncthreads();
      const int stop = s_stop;
      __syncthreads();
      if (stop) break;
    }
    ++g;
    ++a;
  }
  if (tid == 0) {
    *k_out = g;
    if (g > dict_capacity) set_status(status, JABBA_ERR_CAPACITY);
  }
}

// ------------------------------------------------------------------ dictionary
__global__ void k_dict_accumulate(const jabba_group* groups, const int* rec_of, const int* label_c,
                                  const long long* n_p, long long cap, const long long* k_p,
                                  long long dict_capacity, int* l2g, long long* acc) {
  const long long G = clamp_groups(n_p, cap);
  const long long K = *k_p;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < G; c += (long long)gridDim.x * blockDim.x) {
    const int gid = label_c[c];
    l2g[c] = gid;
    if (K > dict_capacity) continue;
    const jabba_group g = groups[rec_of[c]];
    long long* a = acc + (long long)gid * 8;
    atomicAdd((unsigned long long*)&a[0], (unsigned long long)g.count);
    atomicAdd((unsigned long long*)&a[1], (unsigned long long)g.lensum);
    I192 v;
    v.w0 = g.inc[0];
    v.w1 = g.inc[1];
    v.w2 = g.inc[2];
    i64 L[6];
    limbs6(v, L);
    for (int i = 0; i < 6; ++i)
      if (L[i]) atomicAdd((unsigned long long*)&a[2 + i], (unsigned long long)L[i]);
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

void launch_merge(const jabba_group* groups, const long long* n_groups, long long group_capacity,
                  const long long* dom_group_off, const double* sigma, double alpha, double scl, int* l2g,
                  double* dict_len, double* dict_inc, long long* dict_count, long long dict_capacity, long long* k,
                  Scratch& ws, unsigned* status, cudaStream_t st) {
  const long long cap = group_capacity;
  const unsigned grid = (unsigned)(ws.num_sms * 8);
  k_merge_prep<<<grid, 256, 0, st>>>(groups, n_groups, cap, dom_group_off, sigma, scl, ws.m_X, ws.m_Y, ws.m_k0,
                                      ws.m_v0, ws.m_rec);
  // radix sort over the capacity-sized tiling; tiles past n do nothing
  const long long n_tiles = (cap + kSortTile - 1) / kSortTile;
  long long* offs = (long long*)ws.d_acc;  // reused before the dictionary accumulation
  unsigned long long* kin = ws.m_k0;
  unsigned long long* kout = ws.m_k1;
  int* vin = ws.m_v0;
  int* vout = ws.m_v1;
  for (int pass = 0; pass < 8 && n_tiles > 0; ++pass) {
    const int shift = pass * 8;
    k_radix_hist<<<(unsigned)n_tiles, kSortThreads, 0, st>>>(kin, n_groups, cap, shift, ws.m_hist, n_tiles);
    k_u32_to_i64<<<grid, 256, 0, st>>>(ws.m_hist, 256 * n_tiles, offs + 256 * n_tiles + 1);
    exclusive_scan<long long>(offs + 256 * n_tiles + 1, 256 * n_tiles, offs, ws.scan_tiles, st);
    k_radix_scatter<<<(unsigned)n_tiles, kSortThreads, 0, st>>>(kin, vin, kout, vout, n_groups, cap, shift, offs, n_tiles);
    unsigned long long* tk = kin; kin = kout; kout = tk;
    int* tv = vin; vin = vout; vout = tv;
  }
  k_merge_greedy<<<1, 1024, 0, st>>>(kin, vin, ws.m_X, ws.m_Y, n_groups, cap, alpha, ws.m_label, k, dict_capacity,
                                     status);
  cudaMemsetAsync(ws.d_acc, 0, sizeof(long long) * 8 * (size_t)cap, st);
  k_dict_accumulate<<<grid, 256, 0, st>>>(groups, ws.m_rec, ws.m_label, n_groups, cap, k, dict_capacity, l2g, ws.d_acc);
  k_dict_finalize<<<grid, 256, 0, st>>>(ws.d_acc, k, dict_capacity, dict_len, dict_inc, dict_count);
}

}  // namespace jabba
