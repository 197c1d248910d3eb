// reconstruct.cu -- inverse symbolization (Sec. 3.3) and the adjoint of the
// reconstruction MSE with respect to the dictionary increments.
#include "kernels.cuh"

namespace jabba {

// Pieces of series s: [spo[s], spo[s+1]) with spo[s] = dom_piece_off[series_dom_off[s]].
__global__ void k_series_piece_off(const long long* series_dom_off, const long long* dom_piece_off,
                                   long long n_series, long long* spo) {
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s <= n_series;
       s += (long long)gridDim.x * blockDim.x)
    spo[s] = dom_piece_off[series_dom_off[s]];
}

// Sequential pass per series (one thread): quantization with the carry
// v = l~ + e, l^ = round(v), e = v - l^ (Sec. 3.3), and the chain's level and
// position before each piece.  With qlen_in given, the lengths are taken as
// they are (the adjoint holds them fixed).  A non-null `skip` pointing to a
// nonzero word makes the kernel do nothing (the allocation-free entry point's
// device-side bounds check failed).
__global__ void k_recon_seq(const double* x, const long long* series_off, long long n_series, const long long* spo,
                            const int* symbol, const double* dict_len, const double* dict_inc, int round_mode,
                            const int* qlen_in, int* qlen_out, double* level_out, long long* pos_out,
                            long long* tail_pos, double* tail_level, const unsigned* skip) {
  if (skip && *skip) return;
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n_series;
       s += (long long)gridDim.x * blockDim.x) {
    const long long o = series_off[s];
    if (series_off[s + 1] - o <= 0) {
      tail_pos[s] = 0;
      tail_level[s] = 0.0;
      continue;
    }
    double e = 0.0, level = x[o];
    long long pos = 0;
    for (long long j = spo[s]; j < spo[s + 1]; ++j) {
      const int c = symbol[j];
      long long L;
      if (qlen_in) {
        L = qlen_in[j];
      } else {
        const double v = __dadd_rn(dict_len[c], e);
        const double lh = round_mode ? rint(v) : round(v);
        e = __dsub_rn(v, lh);
        L = (long long)lh;
        qlen_out[j] = (int)L;
      }
      level_out[j] = level;
      pos_out[j] = pos;
      level = __dadd_rn(level, dict_inc[c]);
      pos += L;
    }
    tail_pos[s] = pos;
    tail_level[s] = level;
  }
}

__device__ __forceinline__ long long find_series(const long long* spo, long long n_series, long long j) {
  long long lo = 0, hi = n_series - 1;  // largest s with spo[s] <= j
  while (lo < hi) {
    const long long mid = (lo + hi + 1) >> 1;
    if (spo[mid] <= j) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Inverse compression, one thread per piece: xhat[pos + q] = level + (i~ q) / l^.
__global__ void k_recon_fill(const long long* series_off, long long n_series, const long long* spo,
                             const unsigned* skip, const int* symbol, const double* dict_inc, const int* qlen,
                             const double* level, const long long* pos, double* xhat) {
  if (skip && *skip) return;
  const long long N = spo[n_series];
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x) {
    const long long s = find_series(spo, n_series, j);
    const long long o = series_off[s], n_s = series_off[s + 1] - o;
    const int L = qlen[j];
    const double lh = (double)L, inc = dict_inc[symbol[j]], lv = level[j];
    const long long p = pos[j];
    for (int q = 1; q <= L && p + q <= n_s - 1; ++q) xhat[o + p + q] = __dadd_rn(lv, __ddiv_rn(__dmul_rn(inc, (double)q), lh));
  }
}

// t_0 and the tail after the last piece (final level), one warp per series.
__global__ void k_recon_ends(const double* x, const long long* series_off, long long n_series,
                             const long long* tail_pos, const double* tail_level, double* xhat, const unsigned* skip) {
  if (skip && *skip) return;
  const int lane = threadIdx.x & 31;
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long s = w; s < n_series; s += nw) {
    const long long o = series_off[s], n_s = series_off[s + 1] - o;
    if (n_s <= 0) continue;
    if (lane == 0) xhat[o] = x[o];
    for (long long i = tail_pos[s] + 1 + lane; i <= n_s - 1; i += 32) xhat[o + i] = tail_level[s];
  }
}

void launch_reconstruct(const double* x, long long n_points, const long long* series_off, long long n_series,
                        const long long* series_dom_off, const long long* dom_piece_off, const int* symbol,
                        const double* dict_len, const double* dict_inc, int round_mode, int* qlen, double* xhat,
                        Scratch& ws, cudaStream_t st) {
  if (n_series <= 0) return;
  long long* spo = ws.series_a;
  const unsigned g = (unsigned)(ws.num_sms * 8);
  k_series_piece_off<<<g, 256, 0, st>>>(series_dom_off, dom_piece_off, n_series, spo);
  k_recon_seq<<<(unsigned)((n_series + 127) / 128), 128, 0, st>>>(x, series_off, n_series, spo, symbol, dict_len,
                                                                   dict_inc, round_mode, nullptr, qlen, ws.r_level,
                                                                   ws.r_pos, ws.r_tailpos, ws.r_tail_level, nullptr);
  k_recon_fill<<<g, 256, 0, st>>>(series_off, n_series, spo, nullptr, symbol, dict_inc, qlen, ws.r_level, ws.r_pos,
                                  xhat);
  k_recon_ends<<<g, 256, 0, st>>>(x, series_off, n_series, ws.r_tailpos, ws.r_tail_level, xhat, nullptr);
  (void)n_points;
}

// ------------------------------------------------------------------ adjoint
// Per piece j (one thread): recompute xhat on the piece's points and form
// T_j = sum_q r_{pos+q} and U_j = sum_q (q / l^) r_{pos+q}, r = xhat - x.
__global__ void k_grad_piece(const double* x, const long long* series_off, long long n_series, const long long* spo,
                             const int* symbol, const double* dict_inc, const int* qlen, const double* level,
                             const long long* pos, double* T, double* U) {
  const long long N = spo[n_series];
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x) {
    const long long s = find_series(spo, n_series, j);
    const long long o = series_off[s], n_s = series_off[s + 1] - o;
    const int L = qlen[j];
    const double lh = (double)L, inc = dict_inc[symbol[j]], lv = level[j];
    const long long p = pos[j];
    double t = 0.0, u = 0.0;
    for (int q = 1; q <= L && p + q <= n_s - 1; ++q) {
      const double xh = __dadd_rn(lv, __ddiv_rn(__dmul_rn(inc, (double)q), lh));
      const double r = __dsub_rn(xh, x[o + p + q]);
      t = __dadd_rn(t, r);
      u = __dadd_rn(u, __dmul_rn(__ddiv_rn((double)q, lh), r));
    }
    T[j] = t;
    U[j] = u;
  }
}

// Residual sum of the tail (points after the last piece), one warp per series.
__global__ void k_grad_tail(const double* x, const long long* series_off, long long n_series,
                            const long long* tail_pos, const double* tail_level, double* tail_sum) {
  const int lane = threadIdx.x & 31;
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long s = w; s < n_series; s += nw) {
    const long long o = series_off[s], n_s = series_off[s + 1] - o;
    double acc = 0.0;
    if (n_s > 0)
      for (long long i = tail_pos[s] + 1 + lane; i <= n_s - 1; i += 32) acc += tail_level[s] - x[o + i];
    acc = warp_sum(acc);
    if (lane == 0) tail_sum[s] = acc;
  }
}

// Reverse pass per series: grad[a_j] += (2 / n) (U_j + sum_{j' > j} T_j' + tail).
__global__ void k_grad_series(long long n_series, const long long* spo, const int* symbol, const double* T,
                              const double* U, const double* tail_sum, double scale, double* grad) {
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n_series;
       s += (long long)gridDim.x * blockDim.x) {
    double after = tail_sum[s];
    for (long long j = spo[s + 1] - 1; j >= spo[s]; --j) {
      atomicAdd(&grad[symbol[j]], scale * (U[j] + after));
      after += T[j];
    }
  }
}

void launch_reconstruct_backward(const double* x, long long n_points, const long long* series_off,
                                 long long n_series, const long long* series_dom_off,
                                 const long long* dom_piece_off, const int* symbol, const int* qlen,
                                 const double* dict_inc, long long k, double* grad, Scratch& ws, cudaStream_t st) {
  cudaMemsetAsync(grad, 0, sizeof(double) * (size_t)(k > 0 ? k : 0), st);
  if (n_series <= 0 || n_points <= 0) return;
  long long* spo = ws.series_a;
  const unsigned g = (unsigned)(ws.num_sms * 8);
  k_series_piece_off<<<g, 256, 0, st>>>(series_dom_off, dom_piece_off, n_series, spo);
  k_recon_seq<<<(unsigned)((n_series + 127) / 128), 128, 0, st>>>(x, series_off, n_series, spo, symbol, nullptr,
                                                                   dict_inc, 0, qlen, nullptr, ws.r_level, ws.r_pos,
                                                                   ws.r_tailpos, ws.r_tail_level, nullptr);
  k_grad_piece<<<g, 256, 0, st>>>(x, series_off, n_series, spo, symbol, dict_inc, qlen, ws.r_level, ws.r_pos,
                                   ws.r_tsum, ws.r_wsum);
  k_grad_tail<<<g, 256, 0, st>>>(x, series_off, n_series, ws.r_tailpos, ws.r_tail_level, ws.r_tail);
  k_grad_series<<<(unsigned)((n_series + 127) / 128), 128, 0, st>>>(n_series, spo, symbol, ws.r_tsum, ws.r_wsum,
                                                                     ws.r_tail, 2.0 / (double)n_points, grad);
}

}  // namespace jabba

namespace jabba {

// MSE = (1/n) sum (x - xhat)^2 (Sec. 3.3), two fixed-shape passes so the
// summation order (and the result) is the same on every call.
constexpr int kMseBlocks = 512;

__global__ void __launch_bounds__(256) k_mse_partial(const double* x, const double* xhat, long long n,
                                                     double* partial) {
  __shared__ double sw[8];
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double d = x[i] - xhat[i];
    acc = fma(d, d, acc);
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sw[w];
    partial[blockIdx.x] = t;
  }
}

__global__ void k_mse_final(const double* partial, long long n, double* out) {
  __shared__ double sw[8];
  double acc = 0.0;
  for (int i = threadIdx.x; i < kMseBlocks; i += blockDim.x) acc += partial[i];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sw[w];
    *out = n > 0 ? t / (double)n : 0.0;
  }
}

void launch_mse(const double* x, const double* xhat, long long n, double* out, Scratch& ws, cudaStream_t st) {
  double* partial = ws.r_tail;  // >= kMseBlocks doubles is guaranteed by the reservation
  k_mse_partial<<<kMseBlocks, 256, 0, st>>>(x, xhat, n, partial);
  k_mse_final<<<1, 256, 0, st>>>(partial, n, out);
}

}  // namespace jabba


// ------------------------------------------------------------------ allocation-free reconstruction
// Scratch of jabba_reconstruct_noalloc: a file-scope array in the library's
// device memory instead of context memory.  Host code may not use the
// symbol's name as a device address: set-up looks the address up once per
// device (cudaGetSymbolAddress, that device current) and the kernels get it
// as a plain pointer.
#include <mutex>

namespace {

constexpr long long kNaPieces = JABBA_NOALLOC_MAX_PIECES;
constexpr long long kNaSeries = JABBA_NOALLOC_MAX_SERIES;
// layout (8-byte words): level[kNaPieces] | pos[kNaPieces] | spo[kNaSeries + 1] |
// tail_pos[kNaSeries] | tail_level[kNaSeries] | flags (status word of the
// bounds check, sticky until read by jabba_reconstruct_noalloc_status; the
// skip word of the current call)
constexpr long long kNaWords = 2 * kNaPieces + 3 * (kNaSeries + 1) + 1;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNaWords];

constexpr int kMaxDevices = 64;
std::mutex g_na_mutex;
unsigned long long* g_na_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device (set-up on first use).
cudaError_t noalloc_scratch(unsigned long long** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_na_ptr[dev] = (unsigned long long*)p;
  }
  *out = g_na_ptr[dev];
  return cudaSuccess;
}

// Device-side bounds check of one call: every piece offset spo[s] of the
// n_series + 1 series boundaries must lie in [0, n_pieces] (n_pieces <=
// kNaPieces was checked on the host), so that the pieces the kernels visit,
// j in [spo[s], spo[s+1]), index the scratch and qlen in bounds.  Otherwise
// the call's kernels skip all their work and the sticky status word records
// JABBA_ERR_CAPACITY.  One CTA.
__global__ void k_na_guard(const long long* spo, long long n_series, long long n_pieces, unsigned* flags) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (long long s = threadIdx.x; s <= n_series; s += blockDim.x) {
    const long long v = spo[s];
    if (v < 0 || v > n_pieces) bad = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    flags[1] = bad ? 1u : 0u;
    if (bad) atomicCAS(&flags[0], 0u, (unsigned)JABBA_ERR_CAPACITY);
  }
}

}  // namespace

extern "C" jabba_status jabba_reconstruct_noalloc_status(jabba_stream stream) {
  unsigned long long* base = nullptr;
  if (noalloc_scratch(&base) != cudaSuccess) return JABBA_ERR_CUDA;
  unsigned* flags = (unsigned*)(base + kNaWords - 1);
  unsigned h = 0;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return JABBA_ERR_CUDA;
  if (cudaMemcpy(&h, flags, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return JABBA_ERR_CUDA;
  if (h && cudaMemset(flags, 0, sizeof(unsigned)) != cudaSuccess) return JABBA_ERR_CUDA;
  return (jabba_status)h;
}

extern "C" jabba_status jabba_reconstruct_noalloc(const double* x, int64_t n_points, const int64_t* series_off,
                                                  int64_t n_series, const int64_t* series_dom_off,
                                                  const int64_t* dom_piece_off, int64_t n_pieces,
                                                  const int32_t* symbol, const double* dict_len,
                                                  const double* dict_inc, int32_t round_mode, int32_t* qlen,
                                                  double* xhat, jabba_stream stream) {
  using namespace jabba;
  if (n_points < 0 || n_series < 0 || n_pieces < 0 || (round_mode != 0 && round_mode != 1))
    return JABBA_ERR_INVALID_ARG;
  if (n_series > 0 && (!x || !series_off || !series_dom_off || !dom_piece_off || !xhat)) return JABBA_ERR_INVALID_ARG;
  if (n_pieces > 0 && (!symbol || !dict_len || !dict_inc || !qlen)) return JABBA_ERR_INVALID_ARG;
  if (n_pieces > kNaPieces || n_series > kNaSeries) return JABBA_ERR_CAPACITY;
  if (n_series == 0) return JABBA_OK;
  unsigned long long* base = nullptr;
  if (noalloc_scratch(&base) != cudaSuccess) return JABBA_ERR_CUDA;
  double* level = (double*)base;
  long long* pos = (long long*)(base + kNaPieces);
  long long* spo = (long long*)(base + 2 * kNaPieces);
  long long* tail_pos = spo + (kNaSeries + 1);
  double* tail_level = (double*)(tail_pos + kNaSeries);
  unsigned* flags = (unsigned*)(base + kNaWords - 1);
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned g = (unsigned)(sms > 0 ? sms * 8 : 8);
  // every scratch entry these kernels read is written earlier in the same call
  k_series_piece_off<<<g, 256, 0, st>>>((const long long*)series_dom_off, (const long long*)dom_piece_off, n_series,
                                        spo);
  k_na_guard<<<1, 256, 0, st>>>(spo, n_series, n_pieces, flags);
  k_recon_seq<<<(unsigned)((n_series + 127) / 128), 128, 0, st>>>(x, (const long long*)series_off, n_series, spo,
                                                                   symbol, dict_len, dict_inc, round_mode, nullptr,
                                                                   qlen, level, pos, tail_pos, tail_level, flags + 1);
  k_recon_fill<<<g, 256, 0, st>>>((const long long*)series_off, n_series, spo, flags + 1, symbol, dict_inc, qlen,
                                  level, pos, xhat);
  k_recon_ends<<<g, 256, 0, st>>>(x, (const long long*)series_off, n_series, tail_pos, tail_level, xhat, flags + 1);
  // a launch error is reported without being cleared (cudaGetLastError would
  // also consume an error left pending by someone else's earlier work)
  return cudaPeekAtLastError() == cudaSuccess ? JABBA_OK : JABBA_ERR_CUDA;
}
