// api.cu -- the C ABI (include/jabba.h): argument checks, the context and its
// scratch, and the stream-ordered launches of each step.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "kernels.cuh"

using namespace jabba;

constexpr int kProfSlots = 256;
constexpr int kProfStages = 6;

struct jabba_ctx {
  int device = 0;
  int prof_slot = -1;
  cudaEvent_t prof[kProfSlots][kProfStages][2] = {};
  unsigned* status = nullptr;  // device status word
  Scratch ws;
  void* pool = nullptr;        // one allocation backing the scratch
  size_t pool_bytes = 0;
  void* rpool = nullptr;       // per-piece scratch of the reconstruction (allocated on its first use)
  long long cap_recon = 0;
  void* rapool = nullptr;      // scratch of the full reassignment and the SSE (allocated on first use)
  long long cap_ra = -1;
  RaScratch ra;
  void* bfpool = nullptr;      // scratch of the block form (allocated on first use)
  long long cap_bf = -1;
  BlockScratch bf;
  bool tuning = false;         // autotuning mode (jabba_autotune)
};

namespace {

jabba_status cuda_ok(cudaError_t e) { return e == cudaSuccess ? JABBA_OK : JABBA_ERR_CUDA; }

// Event pair of (current slot, stage), created on first use; null when off.
cudaEvent_t prof_event(jabba_ctx* c, int stage, int which) {
  if (c->prof_slot < 0) return nullptr;
  cudaEvent_t& e = c->prof[c->prof_slot][stage][which];
  if (!e && cudaEventCreate(&e) != cudaSuccess) e = nullptr;
  return e;
}

bool params_ok(const jabba_params* p) {
  if (!p) return false;
  if (!(p->tol >= 0.0) || !(p->alpha >= 0.0) || !(p->scl >= 0.0)) return false;  // also rejects NaN
  if (p->tol > 1e300 || p->alpha > 1e150 || p->scl > 1e300) return false;
  if (p->domain_mode != 0 && p->domain_mode != 1) return false;
  if (p->round_mode != 0 && p->round_mode != 1) return false;
  if (p->domain_value < 1) return false;
  if (p->key_mode != 0 && p->key_mode != 1) return false;
  return true;
}

long long series_domains_host(long long n_s, int mode, long long value) {
  if (n_s < 2 || value < 1) return 0;
  const long long iv = n_s - 1;
  if (mode == 0) return value < iv ? value : iv;
  return (iv + value - 1) / value;
}

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

// Carve the scratch out of one pool.  Returns the bytes needed; assigns the
// pointers when `base` is non-null.
size_t layout(Scratch& w, long long S, long long D, long long slots, long long G, long long big,
              unsigned char* base) {
  // big = largest domain in intervals (bounds both piece lengths and pieces per domain)
  const long long cap_len = big > 0 ? big : 1;
  const long long loc_warps = (long long)w.loc_ctas * local_warps_per_cta();
  size_t off = 0;
  auto take = [&](size_t bytes) -> unsigned char* {
    unsigned char* p = base ? base + off : nullptr;
    off += align_up(bytes ? bytes : 1);
    return p;
  };
  long long scan_n = scan_scratch_elems((S > D ? S : D) + 1);
  if (scan_scratch_elems(pack_buckets() + 1) > scan_n) scan_n = scan_scratch_elems(pack_buckets() + 1);
  {
    const long long a = scan_scratch_elems(256 * ((G + 4095) / 4096) + 1), b = scan_scratch_elems(G + 1);
    if (a > scan_n) scan_n = a;
    if (b > scan_n) scan_n = b;
    scan_n += 8;
  }
  w.series_a = (long long*)take(8 * (S + 1));
  w.series_b = (long long*)take(8 * (S + 1));
  w.series_c = (long long*)take(8 * (S + 1));
  w.scan_tiles = (long long*)take(8 * scan_n);
  w.counters = (unsigned*)take(64);
  w.dom_order = (int*)take(4 * (D > 0 ? D : 1));
  w.loc_list = (int*)take(24 * (D > 0 ? D : 1));
  w.loc_ctr = (unsigned*)take(64);
  w.plain_ctr = (unsigned*)take(4 * (D > 0 ? D : 1) + 16);
  if (base) w.loc_stride = D > 0 ? D : 1;
  w.pack_hist = (int*)take(4 * pack_buckets());
  w.pack_off = (long long*)take(8 * (pack_buckets() + 1));
  w.big = nullptr;
  w.arena = (unsigned*)take(4 * (size_t)local_arena_words(cap_len, loc_warps));
  w.xtab64 = (double*)take(8 * (cap_len + 1));
  w.xtab32 = (float*)take(4 * (cap_len + 1));
  w.rinv32 = (float*)take(16);
  if (base) {
    w.cap_len = cap_len;
    w.cap_items = cap_len;
  }
  w.m_k0 = (unsigned long long*)take(8 * G);
  w.m_k1 = (unsigned long long*)take(8 * G);
  w.m_v0 = (int*)take(4 * G);
  w.m_v1 = (int*)take(4 * G);
  w.m_rec = (int*)take(4 * G);
  w.m_recip = (unsigned long long*)take(8 * (kRecipCnt + 1 + 8));
  w.m_hist = (unsigned*)take(4 * (size_t)rs_hist_words(G));
  w.m_X32 = (float*)take(4 * G);
  w.m_Y32 = (float*)take(4 * G);
  {
    const long long cells = G > 0 ? (1ll << 23) : 1;
    if (base) w.cap_cells = cells;
    MergeBufs& B = w.mb;
    B.bounds = (int*)take(16);
    B.bar = (unsigned*)take(64);
    B.bar_sub = (unsigned*)take(4 * 32 * 17);
    B.geom = (struct GridGeom*)take(64);
    B.flags = (int*)take(16);
    B.sX = (float*)take(4 * G);
    B.sY = (float*)take(4 * G);
    B.ck1 = (unsigned long long*)take(8 * G);
    B.cv1 = (int*)take(4 * G);
    B.head = (int*)take(4 * G);
    B.head_off = (long long*)take(8 * (G + 1));
    B.cell_of_id = (int*)take(4 * cells);
    B.cell_beg = (int*)take(4 * G);
    B.cell_end = (int*)take(4 * G);
    B.cell_id = (int*)take(4 * G);
    B.state = (unsigned long long*)take(8 * G);
    // a round creates at most one start per non-empty cell
    const long long slots = (G < cells ? G : cells) + 1;
    B.cX = (float*)take(4 * G);
    B.cY = (float*)take(4 * G);
    B.cov = (unsigned*)take(cov_bitmap_bytes(G));
    B.cinfo = (int4*)take(16 * (G > 0 ? G : 1));
    B.chg_list = (int*)take(16 * (G > 0 ? G : 1));
    // two buffers: the one-phase rounds mark a round's starts in the next round
    if (base) B.slots = slots;
    B.s_pos = (int*)take(4 * 2 * slots);
    B.s_base = (unsigned*)take(4 * 2 * slots);
    B.s_pre = (unsigned*)take(4 * 2 * 26 * slots);
    B.s_q = (int*)take(4 * 2 * 25 * slots);
    B.s_lo = (int*)take(4 * 2 * 25 * slots);
    B.eval_stamp = (unsigned*)take(4 * (G > 0 ? G : 1));
    B.chg_stamp = (unsigned*)take(4 * (G > 0 ? G : 1));
    B.lab = (int*)take(4 * G);
    B.is_start = (int*)take(4 * G);
    B.start_off = (long long*)take(8 * (G + 1));
    B.eX = (double*)take(8 * G);
    B.eY = (double*)take(8 * G);
    B.ekey = (double*)take(8 * G);
  }
  {
    const long long tiles = (G + 4095) / 4096;
    const long long acc_elems = 8 * (G > 1 ? G : 1);
    const long long off_elems = 512 * tiles + 2;
    w.d_acc = (long long*)take(8 * (acc_elems > off_elems ? acc_elems : off_elems) + 64);
  }
  w.r_tail = (double*)take(8 * (S + 1 > 512 ? S + 1 : 512));
  w.r_tailpos = (long long*)take(8 * (S + 1));
  w.r_tail_level = (double*)take(8 * (S + 1));
  return off;
}

jabba_status ensure(jabba_ctx* c, long long S, long long D, long long slots, long long G, long long big,
                    cudaStream_t st) {
  Scratch& w = c->ws;
  if (S <= w.cap_series && D <= w.cap_domains && slots <= w.cap_slots && G <= w.cap_groups && big <= w.cap_big)
    return JABBA_OK;
  if (st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs != cudaStreamCaptureStatusNone) return JABBA_ERR_STATE;  // no allocation during capture
  }
  S = S > w.cap_series ? S : w.cap_series;
  D = D > w.cap_domains ? D : w.cap_domains;
  slots = slots > w.cap_slots ? slots : w.cap_slots;
  G = G > w.cap_groups ? G : w.cap_groups;
  big = big > w.cap_big ? big : w.cap_big;
  Scratch tmp = w;
  const size_t bytes = layout(tmp, S, D, slots, G, big, nullptr);
  if (cudaDeviceSynchronize() != cudaSuccess) return JABBA_ERR_CUDA;
  if (c->pool) cudaFree(c->pool);
  c->pool = nullptr;
  if (cudaMalloc(&c->pool, bytes) != cudaSuccess) {
    c->pool_bytes = 0;
    w.cap_series = w.cap_domains = w.cap_slots = w.cap_groups = w.cap_big = 0;
    return JABBA_ERR_CUDA;
  }
  c->pool_bytes = bytes;
  layout(w, S, D, slots, G, big, (unsigned char*)c->pool);
  // the merge sort's look-back status words must start without a valid tag
  if (cudaMemset(w.m_hist, 0, 4 * (size_t)rs_hist_words(G)) != cudaSuccess) return JABBA_ERR_CUDA;
  w.cap_series = S;
  w.cap_domains = D;
  w.cap_slots = slots;
  w.cap_groups = G;
  w.cap_big = big;
  return JABBA_OK;
}

bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  return cs != cudaStreamCaptureStatusNone;
}

// Milliseconds between two events already recorded on a stream (synchronizes).
float elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) return 3.0e38f;
  return ms;
}

bool tuning_ok(const jabba_tuning* t) {
  if (!t) return false;
  if (t->compress_ctas_per_sm < 1 || t->compress_ctas_per_sm > 3) return false;
  if (t->compress_pack != 0 && t->compress_pack != 1) return false;
  if (t->local_k_warps != 1 && t->local_k_warps != 4) return false;
  if (t->local_mid_warps != 1 && t->local_mid_warps != 2 && t->local_mid_warps != 4 && t->local_mid_warps != 8)
    return false;
  if (t->local_big_warps != 4 && t->local_big_warps != 8) return false;
  if (t->merge_ctas_per_sm != 1 && t->merge_ctas_per_sm != 2 && t->merge_ctas_per_sm != 4) return false;
  if (t->per_domain_launch != 0 && t->per_domain_launch != 1) return false;
  if (t->local_ctas_cap < 0 || t->local_ctas_cap > 16) return false;
  if (t->merge_form != 0 && t->merge_form != 1) return false;
  if (t->merge_warps != 4 && t->merge_warps != 8) return false;
  return true;
}

// Per-piece scratch of the reconstruction and its adjoint (level, position,
// two residual sums per piece), kept apart from the forward path's pool and
// allocated by the first reconstruction call that needs it (never during
// graph capture).
jabba_status ensure_recon(jabba_ctx* c, long long pieces, cudaStream_t st) {
  if (pieces <= c->cap_recon) return JABBA_OK;
  if (st && capturing(st)) return JABBA_ERR_STATE;
  if (cudaDeviceSynchronize() != cudaSuccess) return JABBA_ERR_CUDA;
  if (c->rpool) cudaFree(c->rpool);
  c->rpool = nullptr;
  c->cap_recon = 0;
  const size_t per = align_up(8 * (size_t)(pieces > 0 ? pieces : 1));
  if (cudaMalloc(&c->rpool, 4 * per) != cudaSuccess) return JABBA_ERR_CUDA;
  unsigned char* b = (unsigned char*)c->rpool;
  c->ws.r_level = (double*)b;
  c->ws.r_pos = (long long*)(b + per);
  c->ws.r_tsum = (double*)(b + 2 * per);
  c->ws.r_wsum = (double*)(b + 3 * per);
  c->cap_recon = pieces;
  return JABBA_OK;
}

// Scratch of jabba_reassign / jabba_sse for dictionaries of up to `entries`
// entries (allocated by the first call that needs it, never during capture).
jabba_status ensure_ra(jabba_ctx* c, long long entries, cudaStream_t st) {
  if (entries <= c->cap_ra) return JABBA_OK;
  if (st && capturing(st)) return JABBA_ERR_STATE;
  if (cudaDeviceSynchronize() != cudaSuccess) return JABBA_ERR_CUDA;
  if (c->rapool) cudaFree(c->rapool);
  c->rapool = nullptr;
  c->cap_ra = -1;
  const long long e = entries > 0 ? entries : 1;
  const long long cells = ra_cells_max() + 1;
  size_t off = 0;
  size_t sz[13] = {8 * (size_t)e, 8 * (size_t)e, 4 * (size_t)e, 4 * (size_t)e, 4 * (size_t)e, 4 * (size_t)e,
                   4 * (size_t)e, 4 * (size_t)cells, 8 * (size_t)cells, 8 * (size_t)scan_scratch_elems(cells), 64,
                   16, 64};
  size_t at[13];
  for (int i = 0; i < 13; ++i) {
    at[i] = off;
    off += align_up(sz[i]);
  }
  if (cudaMalloc(&c->rapool, off) != cudaSuccess) return JABBA_ERR_CUDA;
  unsigned char* b = (unsigned char*)c->rapool;
  RaScratch& R = c->ra;
  R.X64 = (double*)(b + at[0]);
  R.Y64 = (double*)(b + at[1]);
  R.X32 = (float*)(b + at[2]);
  R.Y32 = (float*)(b + at[3]);
  R.eX = (float*)(b + at[4]);
  R.eY = (float*)(b + at[5]);
  R.ent = (int*)(b + at[6]);
  R.cnt = (int*)(b + at[7]);
  R.off = (long long*)(b + at[8]);
  R.scan = (long long*)(b + at[9]);
  R.geom = (struct RaGeom*)(b + at[10]);
  R.bounds = (int*)(b + at[11]);
  R.acc = (unsigned long long*)(b + at[12]);
  c->cap_ra = entries;
  return JABBA_OK;
}

jabba_status ensure_bf(jabba_ctx* c, long long n, cudaStream_t st) {
  if (n <= c->cap_bf) return JABBA_OK;
  if (st && capturing(st)) return JABBA_ERR_STATE;
  if (cudaDeviceSynchronize() != cudaSuccess) return JABBA_ERR_CUDA;
  if (c->bfpool) cudaFree(c->bfpool);
  c->bfpool = nullptr;
  c->cap_bf = -1;
  const long long e = n > 0 ? n : 1;
  size_t sz[10] = {8 * (size_t)e, 8 * (size_t)e, 4 * (size_t)e, 4 * (size_t)e, 4 * (size_t)e, 8 * (size_t)e,
                   4 * (size_t)bf_hist_words(e), 64, 64, 4 * (size_t)e};
  size_t at[10], off = 0;
  for (int i = 0; i < 10; ++i) {
    at[i] = off;
    off += align_up(sz[i]);
  }
  if (cudaMalloc(&c->bfpool, off) != cudaSuccess) return JABBA_ERR_CUDA;
  unsigned char* b = (unsigned char*)c->bfpool;
  // the sort's look-back status words must start without a valid tag
  if (cudaMemset(b + at[6], 0, sz[6]) != cudaSuccess) return JABBA_ERR_CUDA;
  BlockScratch& S = c->bf;
  S.k0 = (unsigned long long*)(b + at[0]);
  S.k1 = (unsigned long long*)(b + at[1]);
  S.v0 = (int*)(b + at[2]);
  S.v1 = (int*)(b + at[3]);
  S.clen = (int*)(b + at[4]);
  S.cinc = (double*)(b + at[5]);
  S.hist = (unsigned*)(b + at[6]);
  S.n_dev = (long long*)(b + at[7]);
  S.flags = (int*)(b + at[8]);
  S.start = (int*)(b + at[9]);
  c->cap_bf = n;
  return JABBA_OK;
}

}  // namespace

extern "C" {

const char* jabba_version(void) { return "jabba-gb300 0.1 (sm_103a)"; }

const char* jabba_status_string(jabba_status s) {
  switch (s) {
    case JABBA_OK: return "ok";
    case JABBA_ERR_INVALID_ARG: return "invalid argument";
    case JABBA_ERR_CAPACITY: return "capacity exceeded";
    case JABBA_ERR_NONFINITE: return "non-finite input value";
    case JABBA_ERR_CUDA: return "CUDA runtime error";
    case JABBA_ERR_TIMEOUT: return "bounded device wait timed out";
    case JABBA_ERR_STATE: return "call out of order or allocation needed during graph capture";
    case JABBA_ERR_RANGE: return "input value out of range (|x| >= 2^31)";
  }
  return "unknown status";
}

jabba_status jabba_create(jabba_ctx** out, int device) {
  if (!out) return JABBA_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return JABBA_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return JABBA_ERR_CUDA;
  jabba_ctx* c = new (std::nothrow) jabba_ctx();
  if (!c) return JABBA_ERR_CUDA;
  c->device = device;
  // status word and the poll limit of the bounded waits (0 = the default)
  if (cudaMalloc(&c->status, 2 * sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(c->status, 0, 2 * sizeof(unsigned)) != cudaSuccess) {
    delete c;
    return JABBA_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&c->ws.num_sms, cudaDevAttrMultiProcessorCount, device);
  if (c->ws.num_sms <= 0) c->ws.num_sms = 1;
  c->ws.loc_ctas = c->ws.num_sms * 2;
  *out = c;
  return JABBA_OK;
}

void jabba_destroy(jabba_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  for (int i = 0; i < kProfSlots; ++i)
    for (int j = 0; j < kProfStages; ++j)
      for (int k = 0; k < 2; ++k)
        if (c->prof[i][j][k]) cudaEventDestroy(c->prof[i][j][k]);
  if (c->pool) cudaFree(c->pool);
  if (c->rpool) cudaFree(c->rpool);
  if (c->rapool) cudaFree(c->rapool);
  if (c->bfpool) cudaFree(c->bfpool);
  if (c->status) cudaFree(c->status);
  delete c;
}

jabba_status jabba_sync_status(jabba_ctx* c, jabba_stream stream) {
  if (!c) return JABBA_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  unsigned h = 0;
  if (cudaStreamSynchronize(st) != cudaSuccess) return JABBA_ERR_CUDA;
  if (cudaMemcpy(&h, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return JABBA_ERR_CUDA;
  if (cudaMemset(c->status, 0, sizeof(unsigned)) != cudaSuccess) return JABBA_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return JABBA_ERR_CUDA;
  return (jabba_status)h;
}

jabba_status jabba_set_spin_limit(jabba_ctx* c, uint32_t polls) {
  if (!c) return JABBA_ERR_INVALID_ARG;
  if (cudaSetDevice(c->device) != cudaSuccess) return JABBA_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return JABBA_ERR_CUDA;
  if (cudaMemcpy(c->status + 1, &polls, sizeof(unsigned), cudaMemcpyHostToDevice) != cudaSuccess) return JABBA_ERR_CUDA;
  return JABBA_OK;
}

jabba_status jabba_plan(const int64_t* series_off_host, int64_t n_series, const jabba_params* p,
                        int64_t* n_domains, int64_t* n_slots, int64_t* max_dom_intervals) {
  if (!series_off_host || n_series < 0 || !params_ok(p) || !n_domains || !n_slots) return JABBA_ERR_INVALID_ARG;
  if (series_off_host[0] != 0) return JABBA_ERR_INVALID_ARG;
  long long D = 0, slots = 0, mx = 0;
  for (long long s = 0; s < n_series; ++s) {
    const long long n_s = series_off_host[s + 1] - series_off_host[s];
    if (n_s < 0) return JABBA_ERR_INVALID_ARG;
    if (n_s > 0x7FFFFFFFll) return JABBA_ERR_RANGE;
    const long long M = series_domains_host(n_s, p->domain_mode, p->domain_value);
    D += M;
    slots += n_s > 1 ? n_s - 1 : 0;
    if (M > 0) {
      const long long iv = n_s - 1;
      const long long longest = p->domain_mode == 0 ? (iv + M - 1) / M : (p->domain_value < iv ? p->domain_value : iv);
      if (longest > mx) mx = longest;
    }
  }
  *n_domains = D;
  *n_slots = slots;
  if (max_dom_intervals) *max_dom_intervals = mx;
  return JABBA_OK;
}

jabba_status jabba_reserve(jabba_ctx* c, int64_t n_points, int64_t n_series, int64_t n_domains, int64_t n_slots,
                           int64_t group_capacity, int64_t max_dom_intervals) {
  if (!c || n_points < 0 || n_series < 0 || n_domains < 0 || n_slots < 0 || group_capacity < 0 ||
      max_dom_intervals < 0)
    return JABBA_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  c->ws.cap_points = n_points > c->ws.cap_points ? n_points : c->ws.cap_points;
  return ensure(c, n_series, n_domains, n_slots > n_points ? n_slots : n_points, group_capacity, max_dom_intervals,
                nullptr);
}

jabba_status jabba_compress(jabba_ctx* c, const double* x, int64_t n_points, const int64_t* series_off,
                            int64_t n_series, const jabba_params* p, int64_t n_domains, int64_t n_slots,
                            int64_t* dom_begin, int64_t* dom_end, int32_t* dom_series, int64_t* series_dom_off,
                            int64_t* dom_slot_off, int32_t* piece_len, double* piece_inc, int32_t* dom_piece_cnt,
                            int64_t* dom_piece_off, void* piece_stats, jabba_stream stream) {
  if (!c || !params_ok(p) || n_points < 0 || n_series < 0 || n_domains < 0 || n_slots < 0) return JABBA_ERR_INVALID_ARG;
  if (!series_off || !series_dom_off || !dom_slot_off || !dom_piece_off || !piece_stats) return JABBA_ERR_INVALID_ARG;
  if (n_domains > 0 && (!x || !dom_begin || !dom_end || !dom_series || !dom_piece_cnt)) return JABBA_ERR_INVALID_ARG;
  if (n_slots > 0 && (!piece_len || !piece_inc)) return JABBA_ERR_INVALID_ARG;
  if (n_slots > 0x7FFFFFFFll * 64) return JABBA_ERR_RANGE;
  cudaSetDevice(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  jabba_status r = ensure(c, n_series, n_domains, c->ws.cap_slots, c->ws.cap_groups, c->ws.cap_big, st);
  if (r != JABBA_OK) return r;
  launch_build_domains((const long long*)series_off, n_series, p->domain_mode, p->domain_value,
                       (long long*)series_dom_off, (long long*)dom_begin, (long long*)dom_end, dom_series,
                       (long long*)dom_slot_off, n_domains, c->ws, st);
  Marks mk;
  mk.a0 = prof_event(c, 0, 0);
  mk.a1 = prof_event(c, 0, 1);
  mk.b0 = prof_event(c, 1, 0);
  mk.b1 = prof_event(c, 1, 1);
  auto run = [&](const Marks& m) {
    launch_compress(x, n_points, (const long long*)dom_begin, (const long long*)dom_end,
                    (const long long*)dom_slot_off, n_domains, p->tol, piece_len, piece_inc, dom_piece_cnt,
                    (long long*)dom_piece_off, (long long*)piece_stats, p->key_mode == 1, c->ws, c->status, st, m);
  };
  if (c->ws.tune.per_domain_launch && (capturing(st) || c->tuning)) return JABBA_ERR_STATE;
  if (c->tuning) {
    // every candidate once on these inputs; the packing and the kernel are timed together
    if (capturing(st)) return JABBA_ERR_STATE;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return JABBA_ERR_CUDA;
    Tuning best = c->ws.tune;
    float best_ms = 3.0e38f;
    for (int pack = 0; pack <= 1; ++pack) {
      for (int per_sm = 1; per_sm <= 3; ++per_sm) {
        c->ws.tune.compress_pack = pack;
        c->ws.tune.compress_ctas_per_sm = per_sm;
        Marks m;
        m.a0 = e0;
        m.a1 = e1;
        run(m);
        const float ms = elapsed_ms(e0, e1);
        if (ms < best_ms) {
          best_ms = ms;
          best = c->ws.tune;
        }
      }
    }
    c->ws.tune = best;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return cuda_ok(cudaGetLastError());
  }
  run(mk);
  return cuda_ok(cudaGetLastError());
}

jabba_status jabba_digitize_local(jabba_ctx* c, const int32_t* piece_len, const double* piece_inc,
                                  const int64_t* dom_slot_off, const int32_t* dom_piece_cnt, int64_t n_domains,
                                  const void* piece_stats, const jabba_params* p, double* sigma,
                                  int32_t* local_label, int32_t* dom_group_cnt, int64_t* dom_group_off,
                                  jabba_group* groups, int64_t group_capacity, int64_t* n_groups,
                                  jabba_stream stream) {
  if (!c || !params_ok(p) || n_domains < 0 || group_capacity < 0) return JABBA_ERR_INVALID_ARG;
  if (!piece_stats || !sigma || !dom_group_off || !n_groups) return JABBA_ERR_INVALID_ARG;
  if (n_domains > 0 && (!piece_len || !piece_inc || !dom_slot_off || !dom_piece_cnt || !local_label ||
                        !dom_group_cnt || (group_capacity > 0 && !groups)))
    return JABBA_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  // domains above the shared-memory tile use the scratch sized by jabba_reserve
  jabba_status r = ensure(c, c->ws.cap_series, n_domains, c->ws.cap_slots, c->ws.cap_groups, c->ws.cap_big, st);
  if (r != JABBA_OK) return r;
  auto run = [&]() {
    launch_sigma((const long long*)piece_stats, sigma, p->key_mode, p->scl, st);
    launch_local(piece_len, piece_inc, (const long long*)dom_slot_off, dom_piece_cnt, n_domains, sigma, p->alpha,
                 p->scl, p->key_mode, local_label, dom_group_cnt, (long long*)dom_group_off, groups, group_capacity,
                 (long long*)n_groups, c->ws, c->status, st);
  };
  if (c->ws.tune.per_domain_launch && (capturing(st) || c->tuning)) return JABBA_ERR_STATE;
  if (c->tuning) {
    // four runs cover every tile variant: (k, mid, big) warps = (1, 1, 4), (4, 2, 8), (1, 4, 4), (4, 8, 8);
    // each variable tile kernel is timed on its own
    if (capturing(st)) return JABBA_ERR_STATE;
    TierEvents te;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 2; ++j)
        if (cudaEventCreate(&te.ev[i][j]) != cudaSuccess) return JABBA_ERR_CUDA;
    const int ks[4] = {1, 4, 1, 4}, mids[4] = {1, 2, 4, 8}, bigs[4] = {4, 8, 4, 8};
    float k_ms[4], mid_ms[4], big_ms[4];
    c->ws.tier_ev = &te;
    for (int r = 0; r < 4; ++r) {
      c->ws.tune.local_k_warps = ks[r];
      c->ws.tune.local_mid_warps = mids[r];
      c->ws.tune.local_big_warps = bigs[r];
      run();
      k_ms[r] = elapsed_ms(te.ev[0][0], te.ev[0][1]);
      mid_ms[r] = elapsed_ms(te.ev[1][0], te.ev[1][1]);
      big_ms[r] = elapsed_ms(te.ev[2][0], te.ev[2][1]);
    }
    c->ws.tier_ev = nullptr;
    int bm = 0;
    for (int r = 1; r < 4; ++r)
      if (mid_ms[r] < mid_ms[bm]) bm = r;
    c->ws.tune.local_mid_warps = mids[bm];
    c->ws.tune.local_k_warps = fminf(k_ms[1], k_ms[3]) < fminf(k_ms[0], k_ms[2]) ? 4 : 1;
    c->ws.tune.local_big_warps = fminf(big_ms[1], big_ms[3]) < fminf(big_ms[0], big_ms[2]) ? 8 : 4;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 2; ++j) cudaEventDestroy(te.ev[i][j]);
    return cuda_ok(cudaGetLastError());
  }
  mark(prof_event(c, 2, 0), st);
  run();
  mark(prof_event(c, 2, 1), st);
  return cuda_ok(cudaGetLastError());
}

}  // extern "C"

namespace {
jabba_status merge_impl(jabba_ctx* c, const jabba_group* groups, const double* item_X, const double* item_Y,
                        const int64_t* n_groups, int64_t group_capacity, const int64_t* dom_group_off,
                        const double* sigma, const jabba_params* p, int32_t* l2g, double* dict_len, double* dict_inc,
                        int64_t* dict_count, int64_t dict_capacity, int64_t* k, jabba_stream stream) {
  if (!c || !params_ok(p) || group_capacity < 0 || dict_capacity < 0) return JABBA_ERR_INVALID_ARG;
  if (!n_groups || !dom_group_off || !sigma || !k) return JABBA_ERR_INVALID_ARG;
  if (group_capacity > 0 && (!groups || !l2g)) return JABBA_ERR_INVALID_ARG;
  if (dict_capacity > 0 && (!dict_len || !dict_inc || !dict_count)) return JABBA_ERR_INVALID_ARG;
  if (group_capacity >= 0x7FFFFFFFll) return JABBA_ERR_RANGE;
  cudaSetDevice(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  jabba_status r = ensure(c, c->ws.cap_series, c->ws.cap_domains, c->ws.cap_slots, group_capacity, c->ws.cap_big, st);
  if (r != JABBA_OK) return r;
  auto run = [&]() {
    Marks mk;
    if (!c->tuning) {
      mk.a0 = prof_event(c, 5, 0);
      mk.a1 = prof_event(c, 5, 1);
    }
    launch_merge(groups, item_X, item_Y, (const long long*)n_groups, group_capacity,
                 (const long long*)dom_group_off, sigma, p->alpha, p->scl, p->key_mode, l2g, dict_len, dict_inc,
                 (long long*)dict_count, dict_capacity, (long long*)k, c->ws, c->status, st, mk);
  };
  if (c->tuning) {
    if (capturing(st)) return JABBA_ERR_STATE;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return JABBA_ERR_CUDA;
    // CTAs per SM {1, 2, 4} x (one-barrier form) warps per CTA {8, 4}
    const int cand[3] = {1, 2, 4};
    const int nw = c->ws.tune.merge_form == 1 ? 2 : 1;
    int best = c->ws.tune.merge_ctas_per_sm, best_w = c->ws.tune.merge_warps;
    float best_ms = 3.0e38f;
    for (int r = 0; r < 3; ++r) {
      for (int w = 0; w < nw; ++w) {
        c->ws.tune.merge_ctas_per_sm = cand[r];
        c->ws.tune.merge_warps = w ? 4 : 8;
        cudaEventRecord(e0, st);
        run();
        cudaEventRecord(e1, st);
        const float ms = elapsed_ms(e0, e1);
        if (ms < best_ms) {
          best_ms = ms;
          best = cand[r];
          best_w = c->ws.tune.merge_warps;
        }
      }
    }
    c->ws.tune.merge_ctas_per_sm = best;
    c->ws.tune.merge_warps = best_w;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return cuda_ok(cudaGetLastError());
  }
  mark(prof_event(c, 3, 0), st);
  run();
  mark(prof_event(c, 3, 1), st);
  return cuda_ok(cudaGetLastError());
}

}  // namespace

extern "C" {

jabba_status jabba_merge_global(jabba_ctx* c, const jabba_group* groups, const int64_t* n_groups,
                                int64_t group_capacity, const int64_t* dom_group_off, const double* sigma,
                                const jabba_params* p, int32_t* l2g, double* dict_len, double* dict_inc,
                                int64_t* dict_count, int64_t dict_capacity, int64_t* k, jabba_stream stream) {
  return merge_impl(c, groups, nullptr, nullptr, n_groups, group_capacity, dom_group_off, sigma, p, l2g, dict_len,
                    dict_inc, dict_count, dict_capacity, k, stream);
}

jabba_status jabba_merge_global_points(jabba_ctx* c, const jabba_group* groups, const double* item_X,
                                       const double* item_Y, const int64_t* n_groups, int64_t group_capacity,
                                       const int64_t* dom_group_off, const double* sigma, const jabba_params* p,
                                       int32_t* l2g, double* dict_len, double* dict_inc, int64_t* dict_count,
                                       int64_t dict_capacity, int64_t* k, jabba_stream stream) {
  if (group_capacity > 0 && (!item_X || !item_Y)) return JABBA_ERR_INVALID_ARG;
  return merge_impl(c, groups, item_X, item_Y, n_groups, group_capacity, dom_group_off, sigma, p, l2g, dict_len,
                    dict_inc, dict_count, dict_capacity, k, stream);
}

jabba_status jabba_block_order(jabba_ctx* c, const int32_t* piece_len, const double* piece_inc,
                               const int64_t* dom_slot_off, const int32_t* dom_piece_cnt, const int64_t* dom_piece_off,
                               int64_t n_domains, int64_t n_pieces, const void* piece_stats, const jabba_params* p,
                               int64_t n_blocks, double* sigma, int32_t* order, int32_t* blk_len, double* blk_inc,
                               int64_t* blk_slot_off, int32_t* blk_piece_cnt, jabba_stream stream) {
  if (!c || !params_ok(p) || n_domains < 0 || n_pieces < 0 || n_blocks < 1) return JABBA_ERR_INVALID_ARG;
  if (p->key_mode != 0) return JABBA_ERR_INVALID_ARG;  // the block form sorts by the norm key
  if (n_pieces >= 0x7FFFFFFFll) return JABBA_ERR_RANGE;
  if (!piece_stats || !sigma || !dom_piece_off || !blk_slot_off || !blk_piece_cnt) return JABBA_ERR_INVALID_ARG;
  if (n_domains > 0 && (!piece_len || !piece_inc || !dom_slot_off || !dom_piece_cnt)) return JABBA_ERR_INVALID_ARG;
  if (n_pieces > 0 && (!order || !blk_len || !blk_inc)) return JABBA_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  // the blocks are the domains of the next jabba_digitize_local: size its
  // per-domain scratch and the arena for blocks above the tile size
  const long long B = n_pieces > 0 ? (n_pieces + n_blocks - 1) / n_blocks : 1;
  jabba_status r = ensure(c, c->ws.cap_series, n_blocks, c->ws.cap_slots > n_pieces ? c->ws.cap_slots : n_pieces,
                          c->ws.cap_groups, c->ws.cap_big > B ? c->ws.cap_big : B, st);
  if (r != JABBA_OK) return r;
  r = ensure_bf(c, n_pieces, st);
  if (r != JABBA_OK) return r;
  launch_sigma((const long long*)piece_stats, sigma, 0, p->scl, st);
  launch_block_order(piece_len, piece_inc, (const long long*)dom_slot_off, dom_piece_cnt,
                     (const long long*)dom_piece_off, n_domains, n_pieces, n_blocks, sigma, p->scl, c->bf, order,
                     blk_len, blk_inc, (long long*)blk_slot_off, blk_piece_cnt, c->ws.num_sms, c->status, st);
  return cuda_ok(cudaGetLastError());
}

jabba_status jabba_block_items(jabba_ctx* c, const int32_t* local_label, const int64_t* blk_slot_off,
                               const int32_t* blk_piece_cnt, const int64_t* blk_group_off, int64_t n_blocks,
                               const int32_t* blk_len, const double* blk_inc, const jabba_group* groups,
                               const int64_t* n_groups, int64_t group_capacity, const double* sigma,
                               const jabba_params* p, double* item_X, double* item_Y, jabba_stream stream) {
  if (!c || !params_ok(p) || n_blocks < 0 || group_capacity < 0) return JABBA_ERR_INVALID_ARG;
  if (!n_groups || !sigma || !blk_group_off) return JABBA_ERR_INVALID_ARG;
  if (n_blocks > 0 && (!local_label || !blk_slot_off || !blk_piece_cnt || !blk_len || !blk_inc))
    return JABBA_ERR_INVALID_ARG;
  if (group_capacity > 0 && (!groups || !item_X || !item_Y)) return JABBA_ERR_INVALID_ARG;
  if (c->cap_bf < 0) return JABBA_ERR_STATE;  // jabba_block_order first
  cudaSetDevice(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  // every local group holds a piece, so at most cap_bf groups have a start
  const long long gcap = group_capacity < c->cap_bf ? group_capacity : (c->cap_bf > 0 ? c->cap_bf : 1);
  launch_block_items(local_label, (const long long*)blk_slot_off, blk_piece_cnt, (const long long*)blk_group_off,
                     n_blocks, blk_len, blk_inc, groups, (const long long*)n_groups, gcap, sigma, p->scl, c->bf.start,
                     c->cap_bf, item_X, item_Y, c->ws.num_sms, st);
  return cuda_ok(cudaGetLastError());
}

jabba_status jabba_block_scatter(jabba_ctx* c, const int32_t* order, const int32_t* src, int64_t n, int32_t* dst,
                                 jabba_stream stream) {
  if (!c || n < 0 || (n > 0 && (!order || !src || !dst))) return JABBA_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  launch_block_scatter(order, src, n, dst, c->ws.num_sms, (cudaStream_t)stream);
  return cuda_ok(cudaGetLastError());
}

jabba_status jabba_symbolize(jabba_ctx* c, const int32_t* local_label, const int64_t* dom_slot_off,
                             const int32_t* dom_piece_cnt, const int64_t* dom_piece_off,
                             const int64_t* dom_group_off, int64_t n_domains, const int32_t* l2g,
                             int32_t* symbol, jabba_stream stream) {
  if (!c || n_domains < 0) return JABBA_ERR_INVALID_ARG;
  if (n_domains > 0 && (!local_label || !dom_slot_off || !dom_piece_cnt || !dom_piece_off || !dom_group_off ||
                        !l2g || !symbol))
    return JABBA_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  mark(prof_event(c, 4, 0), (cudaStream_t)stream);
  launch_symbolize(local_label, (const long long*)dom_slot_off, dom_piece_cnt, (const long long*)dom_piece_off,
                   (const long long*)dom_group_off, n_domains, l2g, symbol, c->ws, (cudaStream_t)stream);
  mark(prof_event(c, 4, 1), (cudaStream_t)stream);
  return cuda_ok(cudaGetLastError());
}

jabba_status jabba_reconstruct(jabba_ctx* c, const double* x, int64_t n_points, const int64_t* series_off,
                               int64_t n_series, const int64_t* series_dom_off, const int64_t* dom_piece_off,
                               const int32_t* symbol, const double* dict_len, const double* dict_inc,
                               const jabba_params* p, int32_t* qlen, double* xhat, jabba_stream stream) {
  if (!c || !params_ok(p) || n_points < 0 || n_series < 0) return JABBA_ERR_INVALID_ARG;
  if (n_series > 0 && (!x || !series_off || !series_dom_off || !dom_piece_off || !xhat)) return JABBA_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  // pieces never outnumber the slots (intervals), which are fewer than the points
  jabba_status r = ensure(c, n_series, c->ws.cap_domains, c->ws.cap_slots, c->ws.cap_groups, c->ws.cap_big, st);
  if (r != JABBA_OK) return r;
  r = ensure_recon(c, n_points, st);
  if (r != JABBA_OK) return r;
  launch_reconstruct(x, n_points, (const long long*)series_off, n_series, (const long long*)series_dom_off,
                     (const long long*)dom_piece_off, symbol, dict_len, dict_inc, p->round_mode, qlen, xhat, c->ws,
                     st);
  return cuda_ok(cudaGetLastError());
}

jabba_status jabba_reconstruct_backward(jabba_ctx* c, const double* x, int64_t n_points,
                                        const int64_t* series_off, int64_t n_series,
                                        const int64_t* series_dom_off, const int64_t* dom_piece_off,
                                        const int32_t* symbol, const int32_t* qlen, const double* dict_inc,
                                        int64_t k, double* grad_dict_inc, jabba_stream stream) {
  if (!c || n_points < 0 || n_series < 0 || k < 0) return JABBA_ERR_INVALID_ARG;
  if (k > 0 && !grad_dict_inc) return JABBA_ERR_INVALID_ARG;
  if (n_series > 0 && (!x || !series_off || !series_dom_off || !dom_piece_off)) return JABBA_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  jabba_status r = ensure(c, n_series, c->ws.cap_domains, c->ws.cap_slots, c->ws.cap_groups, c->ws.cap_big, st);
  if (r != JABBA_OK) return r;
  r = ensure_recon(c, n_points, st);
  if (r != JABBA_OK) return r;
  launch_reconstruct_backward(x, n_points, (const long long*)series_off, n_series, (const long long*)series_dom_off,
                              (const long long*)dom_piece_off, symbol, qlen, dict_inc, k, grad_dict_inc, c->ws, st);
  return cuda_ok(cudaGetLastError());
}

jabba_status jabba_diagnostics(jabba_ctx* c, int64_t* out, int n) {
  if (!c || !out || n < 0) return JABBA_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  for (int i = 0; i < n; ++i) out[i] = 0;
  if (!c->ws.counters || n == 0) return JABBA_OK;
  if (cudaDeviceSynchronize() != cudaSuccess) return JABBA_ERR_CUDA;
  unsigned long long v = 0;
  if (cudaMemcpy(&v, c->ws.counters + 2, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess) return JABBA_ERR_CUDA;
  out[0] = (int64_t)v;
  if (n > 1 && c->ws.mb.bar) {
    unsigned r = 0;
    if (cudaMemcpy(&r, c->ws.mb.bar + 2, sizeof r, cudaMemcpyDeviceToHost) != cudaSuccess) return JABBA_ERR_CUDA;
    out[1] = (int64_t)r;
  }
  return JABBA_OK;
}

jabba_status jabba_profile_slot(jabba_ctx* c, int slot) {
  if (!c || slot < -1 || slot >= kProfSlots) return JABBA_ERR_INVALID_ARG;
  c->prof_slot = slot;
  return JABBA_OK;
}

jabba_status jabba_profile_elapsed(jabba_ctx* c, int slot, int stage, float* ms) {
  if (!c || !ms || slot < 0 || slot >= kProfSlots || stage < 0 || stage >= kProfStages) return JABBA_ERR_INVALID_ARG;
  cudaEvent_t a = c->prof[slot][stage][0], b = c->prof[slot][stage][1];
  if (!a || !b) return JABBA_ERR_STATE;
  cudaSetDevice(c->device);
  if (cudaEventSynchronize(b) != cudaSuccess) return JABBA_ERR_CUDA;
  return cuda_ok(cudaEventElapsedTime(ms, a, b));
}

jabba_status jabba_reassign(jabba_ctx* c, const int32_t* piece_len, const double* piece_inc,
                            const int64_t* dom_slot_off, const int32_t* dom_piece_cnt, const int64_t* dom_piece_off,
                            int64_t n_domains, const double* sigma, const double* dict_len, const double* dict_inc,
                            const int64_t* k, int64_t dict_capacity, const jabba_params* p, int32_t* symbol,
                            jabba_stream stream) {
  if (!c || !params_ok(p) || n_domains < 0 || dict_capacity < 1 || dict_capacity >= 0x7FFFFFFFll)
    return JABBA_ERR_INVALID_ARG;
  if (!sigma || !dict_len || !dict_inc || !k) return JABBA_ERR_INVALID_ARG;
  if (n_domains > 0 && (!piece_len || !piece_inc || !dom_slot_off || !dom_piece_cnt || !dom_piece_off || !symbol))
    return JABBA_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  jabba_status r = ensure(c, c->ws.cap_series, c->ws.cap_domains, c->ws.cap_slots, c->ws.cap_groups, c->ws.cap_big, st);
  if (r != JABBA_OK) return r;
  r = ensure_ra(c, dict_capacity, st);
  if (r != JABBA_OK) return r;
  launch_reassign(piece_len, piece_inc, (const long long*)dom_slot_off, dom_piece_cnt, (const long long*)dom_piece_off,
                  n_domains, sigma, dict_len, dict_inc, (const long long*)k, dict_capacity, p->scl, p->alpha, symbol,
                  c->ra, c->ws, st);
  return cuda_ok(cudaGetLastError());
}

jabba_status jabba_sse(jabba_ctx* c, const int32_t* piece_len, const double* piece_inc, const int64_t* dom_slot_off,
                       const int32_t* dom_piece_cnt, const int64_t* dom_piece_off, int64_t n_domains,
                       const double* sigma, const double* dict_len, const double* dict_inc, const int32_t* symbol,
                       const jabba_params* p, double* sse, jabba_stream stream) {
  if (!c || !params_ok(p) || n_domains < 0 || !sigma || !sse) return JABBA_ERR_INVALID_ARG;
  if (n_domains > 0 && (!piece_len || !piece_inc || !dom_slot_off || !dom_piece_cnt || !dom_piece_off || !symbol ||
                        !dict_len || !dict_inc))
    return JABBA_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  jabba_status r = ensure(c, c->ws.cap_series, c->ws.cap_domains, c->ws.cap_slots, c->ws.cap_groups, c->ws.cap_big, st);
  if (r != JABBA_OK) return r;
  r = ensure_ra(c, c->cap_ra > 0 ? c->cap_ra : 1, st);
  if (r != JABBA_OK) return r;
  launch_sse(piece_len, piece_inc, (const long long*)dom_slot_off, dom_piece_cnt, (const long long*)dom_piece_off,
             n_domains, sigma, dict_len, dict_inc, symbol, p->scl, sse, c->ra, c->ws, st);
  return cuda_ok(cudaGetLastError());
}

jabba_status jabba_autotune(jabba_ctx* c, int enable) {
  if (!c || (enable != 0 && enable != 1)) return JABBA_ERR_INVALID_ARG;
  c->tuning = enable != 0;
  return JABBA_OK;
}

jabba_status jabba_get_tuning(jabba_ctx* c, jabba_tuning* out) {
  if (!c || !out) return JABBA_ERR_INVALID_ARG;
  const Tuning& t = c->ws.tune;
  out->compress_ctas_per_sm = t.compress_ctas_per_sm;
  out->compress_pack = t.compress_pack;
  out->local_mid_warps = t.local_mid_warps;
  out->local_big_warps = t.local_big_warps;
  out->merge_ctas_per_sm = t.merge_ctas_per_sm;
  out->per_domain_launch = t.per_domain_launch;
  out->local_k_warps = t.local_k_warps;
  out->local_ctas_cap = t.local_ctas_cap;
  out->merge_form = t.merge_form;
  out->merge_warps = t.merge_warps;
  return JABBA_OK;
}

jabba_status jabba_set_tuning(jabba_ctx* c, const jabba_tuning* in) {
  if (!c || !tuning_ok(in)) return JABBA_ERR_INVALID_ARG;
  Tuning& t = c->ws.tune;
  t.compress_ctas_per_sm = in->compress_ctas_per_sm;
  t.compress_pack = in->compress_pack;
  t.local_mid_warps = in->local_mid_warps;
  t.local_big_warps = in->local_big_warps;
  t.merge_ctas_per_sm = in->merge_ctas_per_sm;
  t.per_domain_launch = in->per_domain_launch;
  t.local_k_warps = in->local_k_warps;
  t.local_ctas_cap = in->local_ctas_cap;
  t.merge_form = in->merge_form;
  t.merge_warps = in->merge_warps;
  return JABBA_OK;
}

jabba_status jabba_check_division(jabba_ctx* c, const double* a, const double* b, int64_t n, int mode,
                                  int64_t* counts, jabba_stream stream) {
  if (!c || n < 0 || !counts || (mode != 0 && mode != 1) || (n > 0 && (!a || !b))) return JABBA_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  launch_check_div(a, b, n, mode, (long long*)counts, c->ws.num_sms, (cudaStream_t)stream);
  return cuda_ok(cudaGetLastError());
}

jabba_status jabba_mse(jabba_ctx* c, const double* x, const double* xhat, int64_t n_points, double* out,
                       jabba_stream stream) {
  if (!c || n_points < 0 || !out || (n_points > 0 && (!x || !xhat))) return JABBA_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  jabba_status r = ensure(c, c->ws.cap_series, c->ws.cap_domains, c->ws.cap_slots, c->ws.cap_groups, c->ws.cap_big, st);
  if (r != JABBA_OK) return r;
  if (!c->ws.r_tail) {
    r = ensure(c, 1, c->ws.cap_domains, c->ws.cap_slots, c->ws.cap_groups, c->ws.cap_big, st);
    if (r != JABBA_OK) return r;
  }
  launch_mse(x, xhat, n_points, out, c->ws, st);
  return cuda_ok(cudaGetLastError());
}

}  // extern "C"
