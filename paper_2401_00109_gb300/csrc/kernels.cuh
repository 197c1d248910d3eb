// kernels.cuh -- launch interfaces between the C ABI (api.cu) and the CUDA
// kernels of the JABBA path.
#pragma once
#include <mutex>

#include "jabba_dev.cuh"
#include "scan.cuh"

namespace jabba {

// Per-device, thread-safe one-time set-up of a kernel's launch attributes
// (dynamic shared-memory limit, occupancy): get(f) runs f() the first time it
// is reached with a device current and returns f()'s value for that device
// on every later call.
struct PerDevice {
  std::mutex m;
  unsigned long long done = 0;  // bit d: device d is set up
  int value[64] = {};
  template <class F>
  int get(F f) {
    int dev = 0;
    cudaGetDevice(&dev);
    dev &= 63;
    std::lock_guard<std::mutex> lock(m);
    if (!(done >> dev & 1ull)) {
      value[dev] = f();
      done |= 1ull << dev;
    }
    return value[dev];
  }
};

// Buffers of the global merge (sizes: cap = group capacity, cells = grid cells).
// Member counts up to this have tabulated reciprocals for the exact centres.
constexpr int kRecipCnt = 4096;

// Bytes of the merge's coverage bitmap for cap items: whole 16-byte groups
// of words (128 items each) plus one group of padding (a warp's 16-byte
// loads may read past the last item).
inline size_t cov_bitmap_bytes(long long cap) { return (size_t)(((cap > 0 ? cap : 1) + 127) / 128 + 1) * 16; }

struct MergeBufs {
  int* bounds = nullptr;             // [4] ordered-int min/max of the FP32 coordinates
  unsigned* bar = nullptr;           // [16] grid barrier generation and round counters
  unsigned* bar_sub = nullptr;       // [32 * 17] grid barrier arrival counters
  struct GridGeom* geom = nullptr;   // grid geometry (device)
  int* flags = nullptr;              // [4] [0] = sequential fallback
  float* sX = nullptr;               // [cap] FP32 coordinates in key order
  float* sY = nullptr;
  unsigned long long* ck1 = nullptr; // [cap] cell sort ping-pong
  int* cv1 = nullptr;
  int* head = nullptr;               // [cap]
  long long* head_off = nullptr;     // [cap + 1]
  int* cell_of_id = nullptr;         // [cells]
  int* cell_beg = nullptr;           // [cap]
  int* cell_end = nullptr;
  int* cell_id = nullptr;
  unsigned long long* state = nullptr;  // [cap]
  float* cX = nullptr;               // [cap] FP32 coordinates in cell order
  float* cY = nullptr;
  unsigned* cov = nullptr;           // covered flags (cell order), one bit per item
  int4* cinfo = nullptr;             // [cap] per cell: start coordinates, first-item bound, end
  int* chg_list = nullptr;           // [2 * cap] cells that changed (per round parity)
  long long slots = 0;               // slots of one buffer of s_* (two buffers)
  int* s_pos = nullptr;              // [2 * slots] new starts of a round: sorted position
  unsigned* s_base = nullptr;        // [2 * slots] first coverage unit
  unsigned* s_pre = nullptr;         // [2 * 26 * slots] coverage units per neighbour
  int* s_q = nullptr;                // [2 * 25 * slots] neighbour cells to cover
  int* s_lo = nullptr;               // [2 * 25 * slots] first item to test there
  unsigned* eval_stamp = nullptr;    // [cap]
  unsigned* chg_stamp = nullptr;     // [cap]
  int* lab = nullptr;                // [cap]
  int* is_start = nullptr;           // [cap]
  long long* start_off = nullptr;    // [cap + 1]
  double* eX = nullptr;              // [cap] binary64 coordinates (fallback only)
  double* eY = nullptr;
  double* ekey = nullptr;
};

// Launch configuration of the batched kernels (chosen by the autotuner of
// api.cu, or set by the caller).  Every choice computes the same result.
struct Tuning {
  int compress_ctas_per_sm = 2;  // resident CTAs per SM of the persistent compression kernel (1..3)
  int compress_pack = 1;         // 1: domains handed to warps longest first; 0: natural order
  int local_k_warps = 1;         // warps per domain of 513..1024 pieces (1 or 4)
  int local_mid_warps = 4;       // warps per domain of 1025..2048 pieces (1, 2, 4 or 8)
  int local_big_warps = 4;       // warps per domain of 2049..4096 pieces (4 or 8)
  int merge_ctas_per_sm = 4;     // CTAs per SM of the cooperative merge-rounds kernel (1, 2 or 4)
  int per_domain_launch = 0;     // 1: the plain form, one launch per domain for compression and Stage I
  int local_ctas_cap = 0;        // at most this many resident CTAs per SM per local kernel (0: all that fit)
  int merge_form = 1;            // merge rounds: 1 = one barrier per round (coverage tested on the fly), 0 = two
  int merge_warps = 8;           // warps per CTA of the one-barrier rounds kernel (4 or 8)
};

// Events around the local-aggregation kernels of the tiles (tuning only).
struct TierEvents {
  cudaEvent_t ev[3][2] = {};
};

// Scratch owned by a context (device memory).  Sized by jabba_reserve().
struct Scratch {
  int num_sms = 0;
  Tuning tune;
  TierEvents* tier_ev = nullptr;  // non-null while the autotuner times the tiles
  long long cap_series = 0, cap_domains = 0, cap_slots = 0, cap_groups = 0, cap_points = 0;
  long long cap_big = 0;          // elements of the big-domain aggregation scratch
  long long* series_a = nullptr;  // [cap_series + 1]
  long long* series_b = nullptr;
  long long* series_c = nullptr;
  long long* scan_tiles = nullptr;
  unsigned* counters = nullptr;   // [16]: task counters, diagnostics
  int* dom_order = nullptr;       // [cap_domains] domains, longest first
  unsigned* plain_ctr = nullptr;  // [cap_domains] task counters of the per-domain launches (plain form)
  int* pack_hist = nullptr;       // [65536] length buckets
  long long* pack_off = nullptr;  // [65537]
  // local aggregation: per-warp arenas and the FP32 normalisation tables
  long long cap_len = 0;          // largest piece length covered by the X table
  long long cap_items = 0;        // largest domain (pieces) an arena holds
  int loc_ctas = 0;               // CTAs of the arena local-aggregation kernel
  int* loc_list = nullptr;        // [6 * loc_stride] domains routed to each local-aggregation tier
  unsigned* loc_ctr = nullptr;    // [16] list sizes and task counters of the tiers
  long long loc_stride = 0;
  unsigned* arena = nullptr;
  double* xtab64 = nullptr;
  float* xtab32 = nullptr;
  float* rinv32 = nullptr;
  unsigned char* big = nullptr;
  // merge
  unsigned long long* m_k0 = nullptr;  // radix sort ping-pong
  unsigned long long* m_k1 = nullptr;
  int* m_v0 = nullptr;
  int* m_v1 = nullptr;
  float* m_X32 = nullptr;         // [cap_groups] FP32 centre coordinates (compact index)
  float* m_Y32 = nullptr;
  long long cap_cells = 0;        // grid cells of the merge
  MergeBufs mb;
  int* m_rec = nullptr;           // [cap_groups] record of each compact index
  unsigned long long* m_recip = nullptr;  // [kRecipCnt + 1 + 8] reciprocal tables of the exact centres
  unsigned* m_hist = nullptr;     // radix histograms
  long long* d_acc = nullptr;     // [cap_groups * 8] dictionary accumulators
  // reconstruction
  double* r_level = nullptr;      // [cap_slots] level before each piece (compact)
  long long* r_pos = nullptr;     // [cap_slots] position of each piece in its series
  double* r_tsum = nullptr;       // [cap_slots] per-piece residual sums (backward)
  double* r_wsum = nullptr;
  double* r_tail = nullptr;       // [cap_series]
  long long* r_tailpos = nullptr; // [cap_series]
  double* r_tail_level = nullptr; // [cap_series]
};

void launch_build_domains(const long long* series_off, long long n_series, int mode, long long value,
                          long long* series_dom_off, long long* dom_begin, long long* dom_end, int* dom_series,
                          long long* dom_slot_off, long long n_domains, Scratch& ws, cudaStream_t st);

// Optional event pairs recorded around kernels (benchmark timing).
struct Marks {
  cudaEvent_t a0 = nullptr, a1 = nullptr;  // around the compression kernel
  cudaEvent_t b0 = nullptr, b1 = nullptr;  // around increments + exact sums
};

long long pack_buckets();
void launch_pack_domains(const long long* dom_begin, const long long* dom_end, long long n_domains, Scratch& ws,
                         cudaStream_t st);

void launch_compress(const double* x, long long n_points, const long long* dom_begin, const long long* dom_end,
                     const long long* dom_slot_off, long long n_domains, double tol, int* piece_len,
                     double* piece_inc, int* dom_piece_cnt, long long* dom_piece_off, long long* stats,
                     bool with_products, Scratch& ws, unsigned* status, cudaStream_t st, const Marks& mk);

// Records an event on `st`; inside stream capture the record becomes a graph
// node (external record) so that replays time the same kernels.
inline void mark(cudaEvent_t e, cudaStream_t st) {
  if (!e) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
  else cudaEventRecord(e, st);
}

// sigma[0..1]; with key_mode 1 (PCA key) also the axis sigma[2..3].
void launch_sigma(const long long* stats, double* sigma, int key_mode, double scl, cudaStream_t st);

long long local_arena_words(long long cap_items, long long n_warps);
int local_warps_per_cta();

void launch_local(const int* piece_len, const double* piece_inc, const long long* dom_slot_off,
                  const int* dom_piece_cnt, long long n_domains, const double* sigma, double alpha, double scl,
                  int key_mode, int* local_label, int* dom_group_cnt, long long* dom_group_off, jabba_group* groups,
                  long long group_capacity, long long* n_groups, Scratch& ws, unsigned* status, cudaStream_t st);

long long rs_hist_words(long long cap);  // radix-sort histogram words for cap items

// Scratch of the full reassignment and of the SSE (reassign.cu), allocated
// by their first call for a dictionary capacity.
struct RaScratch {
  double* X64 = nullptr;   // [cap] entry coordinates, binary64
  double* Y64 = nullptr;
  float* X32 = nullptr;    // [cap] FP32
  float* Y32 = nullptr;
  float* eX = nullptr;     // [cap] FP32 coordinates in cell order
  float* eY = nullptr;
  int* ent = nullptr;      // [cap] entry index in cell order
  int* cnt = nullptr;      // [cells + 1]
  long long* off = nullptr;  // [cells + 1]
  long long* scan = nullptr; // scan scratch for cells + 1 elements
  struct RaGeom* geom = nullptr;
  int* bounds = nullptr;   // [4]
  unsigned long long* acc = nullptr;  // [8]
};
long long ra_cells_max();

void launch_reassign(const int* piece_len, const double* piece_inc, const long long* dom_slot_off,
                     const int* dom_piece_cnt, const long long* dom_piece_off, long long n_domains,
                     const double* sigma, const double* dict_len, const double* dict_inc, const long long* k,
                     long long dict_capacity, double scl, double alpha, int* symbol, RaScratch& R, Scratch& ws,
                     cudaStream_t st);
void launch_sse(const int* piece_len, const double* piece_inc, const long long* dom_slot_off,
                const int* dom_piece_cnt, const long long* dom_piece_off, long long n_domains, const double* sigma,
                const double* dict_len, const double* dict_inc, const int* symbol, double scl, double* out,
                RaScratch& R, Scratch& ws, cudaStream_t st);

// item_X / item_Y (nullable): binary64 points of the group records to merge
// (the block form's starting points); null merges the records' centres.
// Self-check of the integer-unit division of the exact centres (merge.cu).
void launch_check_div(const double* a, const double* b, long long n, int mode, long long* counts, int num_sms,
                      cudaStream_t st);
void launch_merge(const jabba_group* groups, const double* item_X, const double* item_Y, const long long* n_groups,
                  long long group_capacity, const long long* dom_group_off, const double* sigma, double alpha,
                  double scl, int key_mode, int* l2g, double* dict_len, double* dict_inc, long long* dict_count,
                  long long dict_capacity, long long* k, Scratch& ws, unsigned* status, cudaStream_t st,
                  const Marks& mk);

// Block form of Sec. 5 (global key sort, contiguous sorted blocks, merge of
// starting points): scratch for N pieces.
struct BlockScratch {
  unsigned long long* k0 = nullptr;  // [N] keys, sort ping-pong
  unsigned long long* k1 = nullptr;
  int* v0 = nullptr;                 // [N] compact indices, sort ping-pong
  int* v1 = nullptr;
  int* clen = nullptr;               // [N] compact copies of the pieces
  double* cinc = nullptr;
  unsigned* hist = nullptr;          // radix sort scratch for N items
  long long* n_dev = nullptr;        // [1] N on the device
  int* flags = nullptr;              // [4] zero (the sort's skip flags)
  int* start = nullptr;              // [N] first piece of every local group
};
long long bf_hist_words(long long n);
void launch_block_order(const int* piece_len, const double* piece_inc, const long long* dom_slot_off,
                        const int* dom_piece_cnt, const long long* dom_piece_off, long long n_domains, long long n,
                        long long n_blocks, const double* sigma, double scl, BlockScratch& S, int* order, int* blen,
                        double* binc, long long* blk_off, int* blk_cnt, int num_sms, unsigned* status,
                        cudaStream_t st);
void launch_block_items(const int* local_label, const long long* blk_off, const int* blk_cnt,
                        const long long* blk_group_off, long long n_blocks, const int* blen, const double* binc,
                        const jabba_group* groups, const long long* n_groups, long long group_capacity,
                        const double* sigma, double scl, int* start, long long n_items, double* item_X,
                        double* item_Y, int num_sms, cudaStream_t st);
void launch_block_scatter(const int* order, const int* src, long long n, int* dst, int num_sms, cudaStream_t st);

void launch_symbolize(const int* local_label, const long long* dom_slot_off, const int* dom_piece_cnt,
                      const long long* dom_piece_off, const long long* dom_group_off, long long n_domains,
                      const int* l2g, int* symbol, Scratch& ws, cudaStream_t st);

void launch_reconstruct(const double* x, long long n_points, const long long* series_off, long long n_series,
                        const long long* series_dom_off, const long long* dom_piece_off, const int* symbol,
                        const double* dict_len, const double* dict_inc, int round_mode, int* qlen, double* xhat,
                        Scratch& ws, cudaStream_t st);

void launch_reconstruct_backward(const double* x, long long n_points, const long long* series_off,
                                 long long n_series, const long long* series_dom_off,
                                 const long long* dom_piece_off, const int* symbol, const int* qlen,
                                 const double* dict_inc, long long k, double* grad, Scratch& ws, cudaStream_t st);

void launch_mse(const double* x, const double* xhat, long long n, double* out, Scratch& ws, cudaStream_t st);

}  // namespace jabba
