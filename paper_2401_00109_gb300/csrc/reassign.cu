// reassign.cu -- full-reassignment digitization (Alg. 1, Digitize(P^(m), D);
// the argmin of Sec. 3.2): every piece takes its nearest dictionary entry in
// normalised coordinates, ties to the smaller entry index -- the O(N k) pass
// that Sec. 5's label propagation replaces -- and the exact sum of squared
// errors of an assignment (the quantity whose ratio Table 2 reports).
//
// The entries are binned into a uniform grid of side alpha.  A piece
// searches rings of cells around its own (FP32 coordinates with the error
// bounds of the Stage I filter) until no farther ring can beat the best upper
// bound found; the entries whose lower bound reaches that upper bound are then
// compared in binary64 by the definition (dx*dx + dy*dy, no fused operations),
// ties to the smaller index.
#include "kernels.cuh"

namespace jabba {

constexpr long long kRaMaxCells = 1ll << 22;

struct RaGeom {
  float x0, y0, inv_h, h;
  int ncx, ncy;
};

__device__ __forceinline__ int ra_ord(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : (int)(0x80000000u - (unsigned)i);
}
__device__ __forceinline__ float ra_unord(int o) {
  return o >= 0 ? __int_as_float(o) : __int_as_float((int)(0x80000000u - (unsigned)o));
}

__device__ __forceinline__ long long ra_k(const long long* k_p, long long cap) {
  const long long k = *k_p;
  return k < cap ? (k < 0 ? 0 : k) : cap;
}

// Entry coordinates (binary64 by the definition, FP32 rounded) and the FP32
// bounding box (ordered-int min/max in bounds[0..3]).
__global__ void k_ra_entries(const double* dict_len, const double* dict_inc, const long long* k_p, long long cap,
                             const double* sigma, double scl, double* X64, double* Y64, float* X32, float* Y32,
                             int* bounds) {
  const long long k = ra_k(k_p, cap);
  const double sl = sigma[0], si = sigma[1];
  int mnx = 0x7FFFFFFF, mxx = -0x7FFFFFFF, mny = 0x7FFFFFFF, mxy = -0x7FFFFFFF;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < k; c += (long long)gridDim.x * blockDim.x) {
    const double X = __ddiv_rn(__dmul_rn(scl, dict_len[c]), sl);
    const double Y = __ddiv_rn(dict_inc[c], si);
    X64[c] = X;
    Y64[c] = Y;
    const float x = __double2float_rn(X), y = __double2float_rn(Y);
    X32[c] = x;
    Y32[c] = y;
    mnx = min(mnx, ra_ord(x));
    mxx = max(mxx, ra_ord(x));
    mny = min(mny, ra_ord(y));
    mxy = max(mxy, ra_ord(y));
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

__global__ void k_ra_init(int* bounds, unsigned long long* acc) {
  bounds[0] = 0x7FFFFFFF;
  bounds[1] = -0x7FFFFFFF;
  bounds[2] = 0x7FFFFFFF;
  bounds[3] = -0x7FFFFFFF;
  for (int i = 0; i < 8; ++i) acc[i] = 0;
}

// Cell side h = alpha: every piece lies within about 2 alpha of the entry of
// its own group (the entries come from starts more than alpha apart), so a few
// rings of cells settle it; a uniform side from the area (about four entries
// per cell) when alpha = 0; grown until the grid has at most kRaMaxCells cells.
__global__ void k_ra_geom(const int* bounds, const long long* k_p, long long cap, double alpha, RaGeom* geom) {
  const long long k = ra_k(k_p, cap);
  RaGeom g;
  if (k == 0) {
    g.x0 = g.y0 = 0.f;
    g.h = 1.f;
    g.inv_h = 1.f;
    g.ncx = g.ncy = 1;
    *geom = g;
    return;
  }
  const double xmin = ra_unord(bounds[0]), xmax = ra_unord(bounds[1]);
  const double ymin = ra_unord(bounds[2]), ymax = ra_unord(bounds[3]);
  const double w = fmax(xmax - xmin, 1e-30), hh = fmax(ymax - ymin, 1e-30);
  double h = alpha > 0.0 ? alpha : sqrt(w * hh * 4.0 / (double)k);
  if (!(h > 1e-30)) h = fmax(w, hh);
  for (;;) {
    const double nx = floor(w / h) + 1, ny = floor(hh / h) + 1;
    if (nx * ny <= (double)kRaMaxCells) {
      g.ncx = (int)nx;
      g.ncy = (int)ny;
      break;
    }
    h *= 1.5;
  }
  g.x0 = (float)xmin;
  g.y0 = (float)ymin;
  g.h = (float)h;
  g.inv_h = (float)(1.0 / h);
  *geom = g;
}

__device__ __forceinline__ void ra_cell(const RaGeom& g, float x, float y, int& cx, int& cy) {
  cx = (int)floorf((x - g.x0) * g.inv_h);
  cy = (int)floorf((y - g.y0) * g.inv_h);
  cx = min(max(cx, 0), g.ncx - 1);
  cy = min(max(cy, 0), g.ncy - 1);
}

__global__ void k_ra_count(const float* X32, const float* Y32, const long long* k_p, long long cap,
                           const RaGeom* geom, int* cnt) {
  const long long k = ra_k(k_p, cap);
  const RaGeom g = *geom;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < k; c += (long long)gridDim.x * blockDim.x) {
    int cx, cy;
    ra_cell(g, X32[c], Y32[c], cx, cy);
    atomicAdd(&cnt[cy * g.ncx + cx], 1);
  }
}

// Entries in cell order (order within a cell arbitrary: ties are settled by index).
__global__ void k_ra_fill(const float* X32, const float* Y32, const long long* k_p, long long cap,
                          const RaGeom* geom, const long long* off, int* cursor, float* eX, float* eY, int* ent) {
  const long long k = ra_k(k_p, cap);
  const RaGeom g = *geom;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < k; c += (long long)gridDim.x * blockDim.x) {
    int cx, cy;
    ra_cell(g, X32[c], Y32[c], cx, cy);
    const int cell = cy * g.ncx + cx;
    const long long pos = off[cell] + atomicAdd(&cursor[cell], 1);
    eX[pos] = X32[c];
    eY[pos] = Y32[c];
    ent[pos] = (int)c;
  }
}

// Bounds of the squared distance between (xa, ya) and (xb, yb) in binary64
// from their FP32 images (the Stage I filter's error model).
__device__ __forceinline__ void ra_bounds(float xa, float ya, float xb, float yb, float& lo, float& hi) {
  const float dx = fabsf(xb - xa), dy = fabsf(yb - ya);
  const float ex = 0x1p-23f * (fabsf(xa) + fabsf(xb)) + 0x1p-126f;
  const float ey = 0x1p-20f * (fabsf(ya) + fabsf(yb)) + 0x1p-126f;
  const float hx = dx + ex, hy = dy + ey;
  const float lx = fmaxf(dx - ex, 0.f), ly = fmaxf(dy - ey, 0.f);
  hi = fmaf(hx, hx, hy * hy) * (1.0f + 0x1p-21f);
  lo = fmaf(lx, lx, ly * ly) * (1.0f - 0x1p-21f);
}

struct RaArgs {
  const int* piece_len;
  const double* piece_inc;
  const long long* dom_slot_off;
  const int* dom_piece_cnt;
  const long long* dom_piece_off;
  long long n_domains;
  const double* sigma;
  double scl;
  const RaGeom* geom;
  const long long* off;   // [cells + 1] first entry of each cell (cell order)
  const float* eX;        // entry FP32 coordinates in cell order
  const float* eY;
  const int* ent;         // entry index in cell order
  const double* X64;      // entry binary64 coordinates by index
  const double* Y64;
  int* symbol;            // compact output
};

// One lane per piece (a warp per domain).  Pass 1 walks rings of cells until
// ring r, whose points lie at least (r - 2) h away in FP32 coordinates (one
// ring of slack covers the rounding of the cell mapping), cannot beat the
// best upper bound; pass 2 revisits those rings and compares every entry whose
// lower bound reaches it in binary64.
__global__ void __launch_bounds__(256) k_ra_assign(RaArgs A) {
  const int lane = threadIdx.x & 31;
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const RaGeom g = *A.geom;
  const double sl = A.sigma[0], si = A.sigma[1];
  const float rinv = __double2float_rn(__ddiv_rn(1.0, si));
  for (long long d = w; d < A.n_domains; d += nw) {
    const int n = A.dom_piece_cnt[d];
    const long long slot = A.dom_slot_off[d], po = A.dom_piece_off[d];
    for (int j = lane; j < n; j += 32) {
      const int len = A.piece_len[slot + j];
      const double inc = A.piece_inc[slot + j];
      const double X = __ddiv_rn(__dmul_rn(A.scl, (double)len), sl);
      const float x = __double2float_rn(X);
      unsigned mh;
      const float y = f64_to_f32_trunc(inc, mh) * rinv;
      int cx, cy;
      ra_cell(g, x, y, cx, cy);
      // pass 1: the best upper bound
      float best = INFINITY;
      int rmax = 0;
      const float slack = 0x1p-16f * (fabsf(x) + fabsf(y) + fabsf(g.x0) + fabsf(g.y0) + 4.0f * g.h);
      const int rlim = max(g.ncx, g.ncy);
      for (int r = 0; r <= rlim; ++r) {
        if (r >= 2 && (float)(r - 2) * g.h > sqrtf(best) * (1.0f + 0x1p-10f) + slack) break;
        rmax = r;
        for (int yy = cy - r; yy <= cy + r; ++yy) {
          if (yy < 0 || yy >= g.ncy) continue;
          const bool edge_row = yy == cy - r || yy == cy + r;
          for (int xx = cx - r; xx <= cx + r; xx += edge_row ? 1 : 2 * r) {
            if (xx >= 0 && xx < g.ncx) {
              const int cell = yy * g.ncx + xx;
              for (long long e = A.off[cell]; e < A.off[cell + 1]; ++e) {
                float lo, hi;
                ra_bounds(x, y, A.eX[e], A.eY[e], lo, hi);
                best = fminf(best, hi);
              }
            }
            if (r == 0) break;
          }
        }
      }
      // pass 2: exact comparison of the entries that can still be nearest
      int bi = -1;
      double bd = 0.0;
      const double Y = __ddiv_rn(inc, si);
      for (int r = 0; r <= rmax; ++r) {
        for (int yy = cy - r; yy <= cy + r; ++yy) {
          if (yy < 0 || yy >= g.ncy) continue;
          const bool edge_row = yy == cy - r || yy == cy + r;
          for (int xx = cx - r; xx <= cx + r; xx += edge_row ? 1 : 2 * r) {
            if (xx >= 0 && xx < g.ncx) {
              const int cell = yy * g.ncx + xx;
              for (long long e = A.off[cell]; e < A.off[cell + 1]; ++e) {
                float lo, hi;
                ra_bounds(x, y, A.eX[e], A.eY[e], lo, hi);
                if (lo > best) continue;
                const int c = A.ent[e];
                const double dx = __dsub_rn(X, A.X64[c]), dy = __dsub_rn(Y, A.Y64[c]);
                const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
                if (bi < 0 || d2 < bd || (d2 == bd && c < bi)) {
                  bd = d2;
                  bi = c;
                }
              }
            }
            if (r == 0) break;
          }
        }
      }
      A.symbol[po + j] = bi;
    }
  }
}

// Exact SSE of an assignment: per piece the binary64 d2 to its entry (the
// definition's operations), truncated to 2^-64 fixed point, summed in 32-bit
// deferred-carry limbs (acc[0..5]).
__global__ void __launch_bounds__(256) k_ra_sse(const int* piece_len, const double* piece_inc,
                                                const long long* dom_slot_off, const int* dom_piece_cnt,
                                                const long long* dom_piece_off, long long n_domains,
                                                const double* sigma, double scl, const double* dict_len,
                                                const double* dict_inc, const int* symbol,
                                                unsigned long long* acc) {
  const int lane = threadIdx.x & 31;
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const double sl = sigma[0], si = sigma[1];
  I192 s = {0, 0, 0};
  for (long long d = w; d < n_domains; d += nw) {
    const int n = dom_piece_cnt[d];
    const long long slot = dom_slot_off[d], po = dom_piece_off[d];
    for (int j = lane; j < n; j += 32) {
      const int c = symbol[po + j];
      const double dx = __dsub_rn(__ddiv_rn(__dmul_rn(scl, (double)piece_len[slot + j]), sl),
                                  __ddiv_rn(__dmul_rn(scl, dict_len[c]), sl));
      const double dy = __dsub_rn(__ddiv_rn(piece_inc[slot + j], si), __ddiv_rn(dict_inc[c], si));
      const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
      bool neg;
      const U128 m = fx_mag(d2, neg);
      add192(s, m.lo, m.hi, 0);
    }
  }
  i64 L[6];
  limbs6(s, L);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    i64 v = L[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if (lane == 0 && v) atomicAdd(&acc[i], (unsigned long long)v);
  }
}

__global__ void k_ra_sse_final(const unsigned long long* acc, double* out) {
  i64 L[6];
  for (int i = 0; i < 6; ++i) L[i] = (i64)acc[i];
  *out = i192_to_double(from_limbs6(L));
}

static unsigned ra_grid(const Scratch& ws, long long n, int per_block) {
  long long b = (n + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > (long long)ws.num_sms * 16) b = (long long)ws.num_sms * 16;
  return (unsigned)b;
}

void launch_reassign(const int* piece_len, const double* piece_inc, const long long* dom_slot_off,
                     const int* dom_piece_cnt, const long long* dom_piece_off, long long n_domains,
                     const double* sigma, const double* dict_len, const double* dict_inc, const long long* k,
                     long long dict_capacity, double scl, double alpha, int* symbol, RaScratch& R, Scratch& ws,
                     cudaStream_t st) {
  k_ra_init<<<1, 1, 0, st>>>(R.bounds, R.acc);
  const unsigned gk = ra_grid(ws, dict_capacity, 256);
  k_ra_entries<<<gk, 256, 0, st>>>(dict_len, dict_inc, k, dict_capacity, sigma, scl, R.X64, R.Y64, R.X32, R.Y32,
                                   R.bounds);
  k_ra_geom<<<1, 1, 0, st>>>(R.bounds, k, dict_capacity, alpha, R.geom);
  cudaMemsetAsync(R.cnt, 0, sizeof(int) * (size_t)(kRaMaxCells + 1), st);
  k_ra_count<<<gk, 256, 0, st>>>(R.X32, R.Y32, k, dict_capacity, R.geom, R.cnt);
  exclusive_scan<int>(R.cnt, kRaMaxCells, R.off, R.scan, st);
  cudaMemsetAsync(R.cnt, 0, sizeof(int) * (size_t)(kRaMaxCells + 1), st);
  k_ra_fill<<<gk, 256, 0, st>>>(R.X32, R.Y32, k, dict_capacity, R.geom, R.off, R.cnt, R.eX, R.eY, R.ent);
  if (n_domains > 0) {
    RaArgs A;
    A.piece_len = piece_len;
    A.piece_inc = piece_inc;
    A.dom_slot_off = dom_slot_off;
    A.dom_piece_cnt = dom_piece_cnt;
    A.dom_piece_off = dom_piece_off;
    A.n_domains = n_domains;
    A.sigma = sigma;
    A.scl = scl;
    A.geom = R.geom;
    A.off = R.off;
    A.eX = R.eX;
    A.eY = R.eY;
    A.ent = R.ent;
    A.X64 = R.X64;
    A.Y64 = R.Y64;
    A.symbol = symbol;
    k_ra_assign<<<ra_grid(ws, n_domains, 8), 256, 0, st>>>(A);
  }
}

void launch_sse(const int* piece_len, const double* piece_inc, const long long* dom_slot_off,
                const int* dom_piece_cnt, const long long* dom_piece_off, long long n_domains, const double* sigma,
                const double* dict_len, const double* dict_inc, const int* symbol, double scl, double* out,
                RaScratch& R, Scratch& ws, cudaStream_t st) {
  cudaMemsetAsync(R.acc, 0, 8 * sizeof(unsigned long long), st);
  if (n_domains > 0)
    k_ra_sse<<<ra_grid(ws, n_domains, 8), 256, 0, st>>>(piece_len, piece_inc, dom_slot_off, dom_piece_cnt,
                                                        dom_piece_off, n_domains, sigma, scl, dict_len, dict_inc,
                                                        symbol, R.acc);
  k_ra_sse_final<<<1, 1, 0, st>>>(R.acc, out);
}

long long ra_cells_max() { return kRaMaxCells; }

}  // namespace jabba
