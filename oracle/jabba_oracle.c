/*
 * jabba_oracle.c -- plain, slow, FP64 CPU oracle of the JABBA symbolization
 * path (arXiv 2401.00109).  TEST INFRASTRUCTURE ONLY: the tests, the smoke
 * check and the CPU-baseline leg of the benchmark call it; the product path
 * never does.  It shares no code with the CUDA library.
 *
 * Every function states the passage it follows.  Where the paper is silent or
 * ambiguous the reading taken is stated beside the code.  Build with
 *   gcc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC
 * so that every floating-point expression is evaluated exactly as written
 * (IEEE double, round to nearest even, no fused multiply-add).
 *
 * Index base: series are 0-based, x[0..n_s-1] (the paper uses both t_1..t_n,
 * Sec. 3, and t_0..t_n, Table 1).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Exact fixed-point accumulator (order-independent sums of doubles).        */
/* A value v is represented by the integer trunc(v * 2^64) (truncation       */
/* toward zero) held in 256-bit two's complement (4 little-endian 64-bit     */
/* limbs).  Sums of such integers are exact, so any summation order gives   */
/* the same total; the total is rounded once to double (nearest, ties to    */
/* even).  Range contract: |v| < 2^120 per term (callers guarantee far less).*/
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t w[4]; } jo_fx;

static void fx_zero(jo_fx* a) { memset(a, 0, sizeof *a); }

static void fx_add_fx(jo_fx* a, const jo_fx* b) {
  unsigned __int128 c = 0;
  for (int i = 0; i < 4; ++i) {
    c += (unsigned __int128)a->w[i] + b->w[i];
    a->w[i] = (uint64_t)c;
    c >>= 64;
  }
}

static void fx_neg(jo_fx* a) {
  unsigned __int128 c = 1;
  for (int i = 0; i < 4; ++i) {
    c += (uint64_t)~a->w[i];
    a->w[i] = (uint64_t)c;
    c >>= 64;
  }
}

/* out = (neg ? -1 : 1) * trunc(mag * 2^sh), mag < 2^110. */
static void fx_from_scaled(jo_fx* out, unsigned __int128 mag, int sh, int neg) {
  fx_zero(out);
  if (sh < 0) {
    if (sh <= -128) return;
    mag >>= -sh;                               /* truncate toward zero */
    sh = 0;
  }
  if (!mag) return;
  for (int i = 0; i < 4; ++i) {                /* place mag << sh into 256 bits */
    int lo = 64 * i;
    unsigned __int128 part;
    if (sh >= lo + 64) part = 0;
    else if (sh >= lo) part = mag << (sh - lo);
    else part = (sh - lo) <= -128 ? 0 : mag >> (lo - sh);
    out->w[i] = (uint64_t)part;
  }
  if (neg) fx_neg(out);
}

/* v = m * 2^E with m an integer of at most 53 bits. */
static void split_double(double v, uint64_t* m, int* E) {
  int e;
  double f = frexp(fabs(v), &e);               /* |v| = f * 2^e, f in [0.5, 1) */
  *m = (uint64_t)ldexp(f, 53);
  *E = e - 53;
}

/* Fixed-point image of v: trunc(v * 2^64). */
static void fx_from_double(jo_fx* out, double v) {
  if (v == 0.0) { fx_zero(out); return; }
  uint64_t m;
  int E;
  split_double(v, &m, &E);
  fx_from_scaled(out, m, E + 64, v < 0);
}

/* Fixed-point image of the EXACT square of v: trunc(v^2 * 2^64). */
static void fx_from_square(jo_fx* out, double v) {
  if (v == 0.0) { fx_zero(out); return; }
  uint64_t m;
  int E;
  split_double(v, &m, &E);
  fx_from_scaled(out, (unsigned __int128)m * m, 2 * E + 64, 0);
}

static void fx_add_double(jo_fx* a, double v) {
  jo_fx t;
  fx_from_double(&t, v);
  fx_add_fx(a, &t);
}

/* Bit b of the 256-bit magnitude. */
static int fx_bit(const jo_fx* m, int b) { return (int)((m->w[b / 64] >> (b % 64)) & 1u); }

/* Round the 256-bit integer to double (nearest, ties to even), then scale by
 * 2^-64 (exact: results here are far from the subnormal range). */
static double fx_to_double(const jo_fx* a) {
  jo_fx m = *a;
  int neg = (int)(m.w[3] >> 63);
  if (neg) fx_neg(&m);
  int top = -1;
  for (int i = 3; i >= 0 && top < 0; --i)
    if (m.w[i]) top = i * 64 + 63 - __builtin_clzll(m.w[i]);
  if (top < 0) return 0.0;
  double r;
  if (top <= 52) {
    r = ldexp((double)m.w[0], -64);              /* fewer than 54 bits: exact */
  } else {
    int lo = top - 52;                            /* keep bits lo..top         */
    uint64_t sig = 0;
    for (int b = top; b >= lo; --b) sig = (sig << 1) | (uint64_t)fx_bit(&m, b);
    int rb = fx_bit(&m, lo - 1), sticky = 0;
    for (int b = lo - 2; b >= 0 && !sticky; --b) sticky = fx_bit(&m, b);
    if (rb && (sticky || (sig & 1u))) sig += 1;   /* 2^53 is still exact       */
    r = ldexp((double)sig, lo - 64);
  }
  return neg ? -r : r;
}

/* Exposed for the tests: fixed-point round trip of a list of doubles. */
double jo_fx_sum(const double* v, int64_t n) {
  jo_fx a;
  fx_zero(&a);
  for (int64_t i = 0; i < n; ++i) fx_add_double(&a, v[i]);
  return fx_to_double(&a);
}

/* Exposed for the tests: the 4 limbs of the fixed-point image of v. */
void jo_fx_of(double v, uint64_t* limbs) {
  jo_fx a;
  fx_from_double(&a, v);
  memcpy(limbs, a.w, 32);
}

/* Exposed for the tests: round 4 limbs to double. */
double jo_fx_round(const uint64_t* limbs) {
  jo_fx a;
  memcpy(a.w, limbs, 32);
  return fx_to_double(&a);
}

/* Correctly rounded conversion of an unsigned 128-bit integer. */
static double u128_to_double(unsigned __int128 v) { return (double)v; }

/* ------------------------------------------------------------------------ */
/* Phase I: domain construction (Alg. 1 Phase I; Sec. 4.1.1).                */
/* Domains are consecutive, share endpoints (s_{k+1} = e_k) and never cross  */
/* a series boundary.  Reading of "split uniformly":                         */
/*   EQUAL_COUNT M: M_s = min(M, n_s - 1) domains, b_k = floor(k (n_s-1)/M_s)*/
/*   FIXED_LEN   D: ceil((n_s-1)/D) domains, b_k = min(k D, n_s - 1)        */
/* (D counts intervals, so a full domain holds D+1 points).  A series with   */
/* fewer than 2 points has no domain.                                        */
/* ------------------------------------------------------------------------ */
static int64_t series_domains(int64_t n_s, int mode, int64_t value) {
  if (n_s < 2 || value < 1) return 0;
  int64_t iv = n_s - 1;
  if (mode == 0) return value < iv ? value : iv;
  return (iv + value - 1) / value;
}

int64_t jo_count_domains(const int64_t* series_off, int64_t n_series, int mode, int64_t value) {
  int64_t d = 0;
  for (int64_t s = 0; s < n_series; ++s) d += series_domains(series_off[s + 1] - series_off[s], mode, value);
  return d;
}

int64_t jo_build_domains(const int64_t* series_off, int64_t n_series, int mode, int64_t value,
                         int64_t* dom_begin, int64_t* dom_end, int32_t* dom_series) {
  int64_t d = 0;
  for (int64_t s = 0; s < n_series; ++s) {
    int64_t base = series_off[s], n_s = series_off[s + 1] - base;
    int64_t M = series_domains(n_s, mode, value), iv = n_s - 1;
    for (int64_t k = 0; k < M; ++k) {
      int64_t b0, b1;
      if (mode == 0) {
        b0 = (int64_t)(((unsigned __int128)k * (uint64_t)iv) / (uint64_t)M);
        b1 = (int64_t)(((unsigned __int128)(k + 1) * (uint64_t)iv) / (uint64_t)M);
      } else {
        b0 = k * value < iv ? k * value : iv;
        b1 = (k + 1) * value < iv ? (k + 1) * value : iv;
      }
      dom_begin[d] = base + b0;
      dom_end[d] = base + b1;
      dom_series[d] = (int32_t)s;
      ++d;
    }
  }
  return d;
}

/* ------------------------------------------------------------------------ */
/* Phase II: compression of one domain (Sec. 3.1, Eq. 1).                    */
/* Piece (s, e) is admissible when the squared distance of the interior      */
/* points from the chord through (s, x_s) and (e, x_e) is at most            */
/* (e - s - 1) tol^2.  Readings:                                             */
/*  - greedy: from s, extend e while the next end is admissible, stop at the */
/*    first inadmissible end ("largest possible i_j" read as the largest     */
/*    end reached by extension, which keeps the method linear);              */
/*  - the sum runs over interior points only (the endpoint residuals are     */
/*    zero in exact arithmetic);                                             */
/*  - Eq. 1 is used multiplied through by L^2 (L = e - s > 0; form 0, the    */
/*    default; the plain form 1 follows below), which leaves                 */
/*    the criterion unchanged in exact arithmetic and needs no division:     */
/*      sum_{k=1}^{L-1} n_k^2 <= ((L - 1) tol^2) L^2,                         */
/*      n_k = (x_s L + inc k) - x_{s+k} L,  inc = x_e - x_s,                  */
/*    every n_k and n_k^2 evaluated in binary64 in that order, the squares   */
/*    summed exactly (fixed point, resolution 2^-96, each term truncated)    */
/*    and the total rounded once, so the sum has no order;                  */
/*  - no slack on "<=".                                                      */
/* ------------------------------------------------------------------------ */

/* Exact sum of non-negative doubles at resolution 2^-96, rounded once. */
static double exact_sum96(const double* v, int64_t n) {
  jo_fx a;
  fx_zero(&a);
  for (int64_t i = 0; i < n; ++i) {
    if (v[i] == 0.0) continue;
    uint64_t m;
    int E;
    split_double(v[i], &m, &E);
    jo_fx t;
    fx_from_scaled(&t, m, E + 96, 0);
    fx_add_fx(&a, &t);
  }
  return ldexp(fx_to_double(&a), -32);   /* fx_to_double scales by 2^-64; 2^-96 in total */
}

/* L^2 times the Eq. 1 error of piece (s, e). */
double jo_piece_error_l2(const double* x, int64_t s, int64_t e) {
  int64_t L = e - s;
  if (L < 2) return 0.0;
  double dL = (double)L;
  double inc = x[e] - x[s];
  double xsL = x[s] * dL;
  double* sq = (double*)malloc(sizeof(double) * (size_t)(L - 1));
  for (int64_t k = 1; k < L; ++k) {
    double n = (xsL + inc * (double)k) - x[s + k] * dL;
    sq[k - 1] = n * n;
  }
  double r = exact_sum96(sq, L - 1);
  free(sq);
  return r;
}

/* The Eq. 1 error itself (reporting and tests). */
double jo_piece_error(const double* x, int64_t s, int64_t e) {
  double dL = (double)(e - s);
  return jo_piece_error_l2(x, s, e) / (dL * dL);
}

int jo_piece_admissible(const double* x, int64_t s, int64_t e, double tol) {
  double dL = (double)(e - s);
  return jo_piece_error_l2(x, s, e) <= ((double)(e - s - 1) * (tol * tol)) * (dL * dL);
}

/* ------------------------------------------------------------------------ */
/* Eq. 1 in its plain form, the formula read as printed: the residual of     */
/* interior point s+k from the chord is r_k = (x_s + (inc * k) / L) - x_{s+k} */
/* (binary64, in that order, no fused operations), the squares are summed    */
/* sequentially in ascending k, and the piece is admissible when the sum is  */
/* at most (L - 1) * (tol * tol).  This is the second reading of Eq. 1 kept  */
/* beside the L^2-scaled exact form above: the two agree in exact arithmetic */
/* and may differ only where the error lies within rounding of the bound (a  */
/* "breakpoint flip"; the tests count them and check how close they are).   */
/* ------------------------------------------------------------------------ */
double jo_piece_error_plain(const double* x, int64_t s, int64_t e) {
  int64_t L = e - s;
  if (L < 2) return 0.0;
  double dL = (double)L;
  double inc = x[e] - x[s];
  double err = 0.0;
  for (int64_t k = 1; k < L; ++k) {
    double r = (x[s] + (inc * (double)k) / dL) - x[s + k];
    err = err + r * r;
  }
  return err;
}

int jo_piece_admissible_plain(const double* x, int64_t s, int64_t e, double tol) {
  return jo_piece_error_plain(x, s, e) <= (double)(e - s - 1) * (tol * tol);
}

/* Admissibility in the chosen reading: form 0 = L^2-scaled exact sum,
 * form 1 = plain sequential sum. */
static int admissible_form(const double* x, int64_t s, int64_t e, double tol, int form) {
  return form ? jo_piece_admissible_plain(x, s, e, tol) : jo_piece_admissible(x, s, e, tol);
}

/* End of the greedy piece that starts at s in a domain ending at e_dom. */
int64_t jo_piece_end(const double* x, int64_t s, int64_t e_dom, double tol, int form) {
  int64_t e = s + 1;                           /* a one-interval piece is always admissible */
  while (e + 1 <= e_dom && admissible_form(x, s, e + 1, tol, form)) ++e;
  return e;
}

int64_t jo_compress_domain(const double* x, int64_t b, int64_t e_dom, double tol, int form,
                           int32_t* len_out, double* inc_out) {
  int64_t n = 0, s = b;
  while (s < e_dom) {
    int64_t e = jo_piece_end(x, s, e_dom, tol, form);
    len_out[n] = (int32_t)(e - s);
    inc_out[n] = x[e] - x[s];
    ++n;
    s = e;
  }
  return n;
}

/* Compress every domain; domain d writes its pieces at slot dom_cap_off[d]
 * (capacity = its interval count) and its count to dom_count[d].  Domains
 * are independent (Alg. 1 Phase II "in parallel"); n_threads > 1 splits them
 * over POSIX threads exactly as the paper's multicore compression does. */
typedef struct {
  const double* x; const int64_t* b; const int64_t* e; const int64_t* cap_off;
  double tol; int form; int32_t* len; double* inc; int64_t* count; int64_t d0, d1;
} jo_cjob;

static void* compress_worker(void* p) {
  jo_cjob* j = (jo_cjob*)p;
  for (int64_t d = j->d0; d < j->d1; ++d)
    j->count[d] = jo_compress_domain(j->x, j->b[d], j->e[d], j->tol, j->form, j->len + j->cap_off[d],
                                     j->inc + j->cap_off[d]);
  return NULL;
}

void jo_compress_all(const double* x, const int64_t* dom_begin, const int64_t* dom_end, int64_t n_domains,
                     const int64_t* dom_cap_off, double tol, int form, int32_t* len, double* inc,
                     int64_t* dom_count, int n_threads) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  jo_cjob jobs[256];
  for (int t = 0; t < n_threads; ++t) {
    jobs[t] = (jo_cjob){x, dom_begin, dom_end, dom_cap_off, tol, form, len, inc, dom_count,
                        n_domains * t / n_threads, n_domains * (t + 1) / n_threads};
    if (n_threads == 1) compress_worker(&jobs[t]);
    else pthread_create(&th[t], NULL, compress_worker, &jobs[t]);
  }
  if (n_threads > 1)
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
}

/* End reached from each of n given piece starts (starts[i] in a domain that
 * ends at dom_ends[i]) by the greedy of the given form; the check of another
 * implementation's breakpoints against either reading of Eq. 1.  Pieces are
 * dealt to the threads round robin (their costs differ widely). */
typedef struct {
  const double* x; const int64_t* s; const int64_t* e; int64_t n; double tol; int form; int64_t* out;
  int t, nt;
} jo_ejob;

static void* ends_worker(void* p) {
  jo_ejob* j = (jo_ejob*)p;
  for (int64_t i = j->t; i < j->n; i += j->nt) j->out[i] = jo_piece_end(j->x, j->s[i], j->e[i], j->tol, j->form);
  return NULL;
}

void jo_piece_ends(const double* x, const int64_t* starts, const int64_t* dom_ends, int64_t n, double tol,
                   int form, int64_t* out, int n_threads) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  jo_ejob jobs[256];
  for (int t = 0; t < n_threads; ++t) {
    jobs[t] = (jo_ejob){x, starts, dom_ends, n, tol, form, out, t, n_threads};
    if (n_threads == 1) ends_worker(&jobs[t]);
    else pthread_create(&th[t], NULL, ends_worker, &jobs[t]);
  }
  if (n_threads > 1)
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------------ */
/* Normalisation (Sec. 3.2, Eq. 4): sigma_len, sigma_inc are the population  */
/* standard deviations of all pieces of all domains (the dictionary is       */
/* shared).  Sums are exact (integers for len; fixed point, of inc and of    */
/* the exact square of inc, for inc), so the result does not depend on      */
/* summation order; then, in FP64,                                          */
/*   m = S1 / N;  v = S2 / N - m * m;  sigma = sqrt(v), or 1 when v <= 0.     */
/* ------------------------------------------------------------------------ */
static double sigma_from(double s1, double s2, double n) {
  double m = s1 / n;
  double v = s2 / n - m * m;
  if (!(v > 0.0)) return 1.0;
  return sqrt(v);
}

void jo_sigma(const int32_t* len, const double* inc, int64_t n, double* sigma_len, double* sigma_inc) {
  int64_t s1 = 0;
  unsigned __int128 s2 = 0;
  jo_fx i1, i2;
  fx_zero(&i1);
  fx_zero(&i2);
  for (int64_t j = 0; j < n; ++j) {
    s1 += len[j];
    s2 += (unsigned __int128)((int64_t)len[j] * (int64_t)len[j]);
    fx_add_double(&i1, inc[j]);
    jo_fx sq;
    fx_from_square(&sq, inc[j]);
    fx_add_fx(&i2, &sq);
  }
  double dn = (double)n;
  *sigma_len = sigma_from((double)s1, u128_to_double(s2), dn);
  *sigma_inc = sigma_from(fx_to_double(&i1), fx_to_double(&i2), dn);
}

/* ------------------------------------------------------------------------ */
/* PCA key (Sec. 5: the sort key is "norm or PCA projection").  The first    */
/* principal axis of the normalised pieces X = (scl len) / sigma_len,        */
/* Y = inc / sigma_inc.  Normalising by the population standard deviations   */
/* makes their covariance, in exact arithmetic,                             */
/*     [[scl^2, scl r], [scl r, 1]],  r = cov(len, inc) / (sigma_len sigma_inc) */
/* (a variance that is 0 stays 0).  Reading: r comes from the same exact     */
/* order-independent sums as the standard deviations plus the exact sum of   */
/* the products len * inc (each truncated toward zero at 2^-64), all rounded */
/* once; in binary64, in this order:                                        */
/*     m_l = S_l / N, m_i = S_i / N, c = S_li / N - m_l * m_i,                */
/*     r = c / (sigma_len * sigma_inc),                                      */
/*     a = scl * scl (0 when var len = 0), d = 1 (0 when var inc = 0),        */
/*     b = scl * r (0 when either variance is 0);                            */
/* the leading eigenvector of [[a, b], [b, d]] by the closed form            */
/*     b = 0: (1, 0) if a >= d else (0, 1);                                   */
/*     h = (a - d) / 2, lam = (a + d) / 2 + sqrt(h * h + b * b),              */
/*     v = (lam - d, b) if a >= d else (b, lam - a), v /= sqrt(vx^2 + vy^2),  */
/* with the sign that makes vx > 0 (or vx = 0 and vy > 0).                   */
/* ------------------------------------------------------------------------ */
void jo_pca_axis(const int32_t* len, const double* inc, int64_t n, double scl, double* out /* vx, vy, r */) {
  out[0] = 1.0;
  out[1] = 0.0;
  out[2] = 0.0;
  if (n <= 0) return;
  int64_t s1 = 0;
  unsigned __int128 s2 = 0;
  jo_fx i1, i2, li;
  fx_zero(&i1);
  fx_zero(&i2);
  fx_zero(&li);
  for (int64_t j = 0; j < n; ++j) {
    s1 += len[j];
    s2 += (unsigned __int128)((int64_t)len[j] * (int64_t)len[j]);
    fx_add_double(&i1, inc[j]);
    jo_fx t;
    fx_from_square(&t, inc[j]);
    fx_add_fx(&i2, &t);
    if (inc[j] != 0.0) {                       /* exact product len * inc, truncated at 2^-64 */
      uint64_t m;
      int E;
      split_double(inc[j], &m, &E);
      fx_from_scaled(&t, (unsigned __int128)m * (uint64_t)len[j], E + 64, inc[j] < 0);
      fx_add_fx(&li, &t);
    }
  }
  const double dn = (double)n;
  const double ml = (double)s1 / dn, mi = fx_to_double(&i1) / dn;
  const double vl = u128_to_double(s2) / dn - ml * ml;
  const double vi = fx_to_double(&i2) / dn - mi * mi;
  const double sl = sigma_from((double)s1, u128_to_double(s2), dn);
  const double si = sigma_from(fx_to_double(&i1), fx_to_double(&i2), dn);
  const double c = fx_to_double(&li) / dn - ml * mi;
  const double r = c / (sl * si);
  const int var_l = vl > 0.0, var_i = vi > 0.0;
  const double a = var_l ? scl * scl : 0.0;
  const double d = var_i ? 1.0 : 0.0;
  const double b = (var_l && var_i) ? scl * r : 0.0;
  out[2] = (var_l && var_i) ? r : 0.0;
  if (b == 0.0) {
    out[0] = a >= d ? 1.0 : 0.0;
    out[1] = a >= d ? 0.0 : 1.0;
    return;
  }
  const double h = (a - d) / 2.0;
  const double lam = (a + d) / 2.0 + sqrt(h * h + b * b);
  double vx, vy;
  if (a >= d) {
    vx = lam - d;
    vy = b;
  } else {
    vx = b;
    vy = lam - a;
  }
  const double sn = sqrt(vx * vx + vy * vy);
  vx = vx / sn;
  vy = vy / sn;
  if (vx < 0.0 || (vx == 0.0 && vy < 0.0)) {
    vx = -vx;
    vy = -vy;
  }
  out[0] = vx;
  out[1] = vy;
}

/* ------------------------------------------------------------------------ */
/* Greedy aggregation (Sec. 3.2, fABBA; pruning rule of Sec. 5).             */
/* Points p = (X, Y): X = (scl * len) / sigma_len, Y = inc / sigma_inc        */
/* (Eq. 4).  Sort key: the squared norm X*X + Y*Y (orders exactly as the     */
/* norm).  Order: key ascending, ties by position.  In that order each       */
/* unassigned point starts a new group; every later unassigned point q with  */
/* (X_q - X_p)^2 + (Y_q - Y_p)^2 <= alpha^2 joins it.  The scan of later     */
/* points stops once norm(q) - norm(p) exceeds alpha (Sec. 5 pruning); the   */
/* stop test carries a 2^-40 relative margin so that, despite rounding, it   */
/* never skips a point that the distance test would accept: the result is   */
/* that of the unpruned greedy (checked in the tests).                       */
/* ------------------------------------------------------------------------ */
typedef struct { double key; int64_t pos; } jo_kp;

static int kp_cmp(const void* a, const void* b) {
  const jo_kp* u = (const jo_kp*)a;
  const jo_kp* v = (const jo_kp*)b;
  if (u->key < v->key) return -1;
  if (u->key > v->key) return 1;
  return (u->pos > v->pos) - (u->pos < v->pos);
}

static double dist2(double xa, double ya, double xb, double yb) {
  double dx = xb - xa, dy = yb - ya;
  return dx * dx + dy * dy;
}

/* Generic greedy over n points (X[], Y[]); labels[i] receives the group id in
 * creation order; returns the number of groups; starts[g] = first point.
 * prune = 0 gives the unpruned greedy (used only by the tests).
 * mode 0: the squared-norm key above.  mode 1 (the PCA key of Sec. 5): the
 * projection key vx * X + vy * Y on a unit axis (vx, vy); a projection on a
 * unit vector changes by at most the distance, so the scan stops once the key
 * gap exceeds alpha (margin 2^-40 of the coordinates' size for rounding). */
static int64_t greedy_core(const double* X, const double* Y, int64_t n, double alpha, int prune, int mode,
                           double vx, double vy, int64_t* labels, int64_t* starts) {
  jo_kp* o = (jo_kp*)malloc(sizeof(jo_kp) * (size_t)(n ? n : 1));
  for (int64_t i = 0; i < n; ++i) {
    o[i].key = mode ? vx * X[i] + vy * Y[i] : X[i] * X[i] + Y[i] * Y[i];
    o[i].pos = i;
    labels[i] = -1;
  }
  qsort(o, (size_t)n, sizeof(jo_kp), kp_cmp);
  double a2 = alpha * alpha;
  int64_t g = 0;
  for (int64_t a = 0; a < n; ++a) {
    int64_t i = o[a].pos;
    if (labels[i] >= 0) continue;
    labels[i] = g;
    if (starts) starts[g] = i;
    double ri = mode ? o[a].key : sqrt(o[a].key);
    for (int64_t b = a + 1; b < n; ++b) {
      int64_t j = o[b].pos;
      if (prune) {
        if (mode) {
          double m = 0x1p-40 * (alpha + fabs(X[i]) + fabs(Y[i]) + fabs(X[j]) + fabs(Y[j]));
          if (o[b].key - ri > alpha + m) break;
        } else {
          double rj = sqrt(o[b].key);
          if (rj - ri > alpha + 0x1p-40 * (alpha + rj)) break;
        }
      }
      if (labels[j] < 0 && dist2(X[i], Y[i], X[j], Y[j]) <= a2) labels[j] = g;
    }
    ++g;
  }
  free(o);
  return g;
}

int64_t jo_greedy(const double* X, const double* Y, int64_t n, double alpha, int prune,
                  int64_t* labels, int64_t* starts) {
  return greedy_core(X, Y, n, alpha, prune, 0, 0.0, 0.0, labels, starts);
}

int64_t jo_greedy_proj(const double* X, const double* Y, int64_t n, double alpha, double vx, double vy, int prune,
                       int64_t* labels, int64_t* starts) {
  return greedy_core(X, Y, n, alpha, prune, 1, vx, vy, labels, starts);
}

/* Exact sums of the groups given by labels[i] in [0, G): count, lensum,
 * incacc (fixed point, 4 limbs per group). */
void jo_group_sums(const int32_t* len, const double* inc, int64_t n, const int64_t* labels, int64_t G,
                   int64_t* grp_count, int64_t* grp_lensum, uint64_t* grp_incacc) {
  for (int64_t g = 0; g < G; ++g) {
    grp_count[g] = 0;
    grp_lensum[g] = 0;
    memset(grp_incacc + 4 * g, 0, 32);
  }
  for (int64_t i = 0; i < n; ++i) {
    int64_t g = labels[i];
    grp_count[g] += 1;
    grp_lensum[g] += len[i];
    fx_add_double((jo_fx*)(grp_incacc + 4 * g), inc[i]);
  }
}

/* Normalised coordinates of a piece (Eq. 4). */
static double norm_len(double len, double scl, double sigma_len) { return (scl * len) / sigma_len; }
static double norm_inc(double inc, double sigma_inc) { return inc / sigma_inc; }

/* Stage I, per domain (Sec. 5; per-domain blocks): aggregate the pieces of one
 * domain.  Group sums: count, lensum (exact int), incacc (exact fixed point).
 * Returns the number of local groups. */
int64_t jo_local_aggregate(const int32_t* len, const double* inc, int64_t n, double sigma_len,
                           double sigma_inc, double alpha, double scl, int32_t* label,
                           int64_t* grp_count, int64_t* grp_lensum, uint64_t* grp_incacc /* 4 limbs/group */) {
  double* X = (double*)malloc(sizeof(double) * (size_t)(n ? n : 1));
  double* Y = (double*)malloc(sizeof(double) * (size_t)(n ? n : 1));
  int64_t* lab = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
  for (int64_t i = 0; i < n; ++i) {
    X[i] = norm_len((double)len[i], scl, sigma_len);
    Y[i] = norm_inc(inc[i], sigma_inc);
  }
  int64_t G = jo_greedy(X, Y, n, alpha, 1, lab, NULL);
  for (int64_t g = 0; g < G; ++g) {
    grp_count[g] = 0;
    grp_lensum[g] = 0;
    memset(grp_incacc + 4 * g, 0, 32);
  }
  for (int64_t i = 0; i < n; ++i) {
    int64_t g = lab[i];
    label[i] = (int32_t)g;
    grp_count[g] += 1;
    grp_lensum[g] += len[i];
    fx_add_double((jo_fx*)(grp_incacc + 4 * g), inc[i]);
  }
  free(X);
  free(Y);
  free(lab);
  return G;
}

/* Centre of a group in original units: (lensum / count, round(incacc) / count). */
void jo_centre(int64_t count, int64_t lensum, const uint64_t* incacc, double* c_len, double* c_inc) {
  *c_len = (double)lensum / (double)count;
  *c_inc = fx_to_double((const jo_fx*)incacc) / (double)count;
}

/* Stage II (Sec. 5 "global merging"): the same greedy over all local groups
 * taken as points at their normalised centres, in (domain, local id) order.
 * Reading: the weighted local centres are merged (membership unweighted, the
 * weights enter the merged centres through the exact sums).  l2g[g] = global
 * group (creation order); dictionary entry = exact mean of its pieces. */
int64_t jo_merge(const int64_t* grp_count, const int64_t* grp_lensum, const uint64_t* grp_incacc, int64_t G,
                 double sigma_len, double sigma_inc, double alpha, double scl, int32_t* l2g,
                 double* dict_len, double* dict_inc, int64_t* dict_count) {
  double* X = (double*)malloc(sizeof(double) * (size_t)(G ? G : 1));
  double* Y = (double*)malloc(sizeof(double) * (size_t)(G ? G : 1));
  int64_t* lab = (int64_t*)malloc(sizeof(int64_t) * (size_t)(G ? G : 1));
  for (int64_t g = 0; g < G; ++g) {
    double cl, ci;
    jo_centre(grp_count[g], grp_lensum[g], grp_incacc + 4 * g, &cl, &ci);
    X[g] = norm_len(cl, scl, sigma_len);
    Y[g] = norm_inc(ci, sigma_inc);
  }
  int64_t k = jo_greedy(X, Y, G, alpha, 1, lab, NULL);
  int64_t* cnt = (int64_t*)calloc((size_t)(k ? k : 1), sizeof(int64_t));
  int64_t* ls = (int64_t*)calloc((size_t)(k ? k : 1), sizeof(int64_t));
  jo_fx* ia = (jo_fx*)calloc((size_t)(k ? k : 1), sizeof(jo_fx));
  for (int64_t g = 0; g < G; ++g) {
    int64_t c = lab[g];
    l2g[g] = (int32_t)c;
    cnt[c] += grp_count[g];
    ls[c] += grp_lensum[g];
    fx_add_fx(&ia[c], (const jo_fx*)(grp_incacc + 4 * g));
  }
  for (int64_t c = 0; c < k; ++c) {
    jo_centre(cnt[c], ls[c], ia[c].w, &dict_len[c], &dict_inc[c]);
    dict_count[c] = cnt[c];
  }
  free(X);
  free(Y);
  free(lab);
  free(cnt);
  free(ls);
  free(ia);
  return k;
}

/* Stage II over given points (Sec. 5 as the paper states it: the local
 * starting points are merged): the same pruned greedy over the points
 * (X[g], Y[g]) of the G local groups (key by mode as in greedy_core), in
 * index order for equal keys;
 * l2g[g] = global group (creation order); the dictionary entry of a global
 * group is the exact mean of the pieces of its local groups (their exact
 * sums), as in jo_merge.  Returns k. */
int64_t jo_merge_points(const double* X, const double* Y, const int64_t* grp_count, const int64_t* grp_lensum,
                        const uint64_t* grp_incacc, int64_t G, double alpha, int mode, double vx, double vy,
                        int32_t* l2g, double* dict_len, double* dict_inc, int64_t* dict_count) {
  int64_t* lab = (int64_t*)malloc(sizeof(int64_t) * (size_t)(G ? G : 1));
  int64_t k = greedy_core(X, Y, G, alpha, 1, mode, vx, vy, lab, NULL);
  int64_t* cnt = (int64_t*)calloc((size_t)(k ? k : 1), sizeof(int64_t));
  int64_t* ls = (int64_t*)calloc((size_t)(k ? k : 1), sizeof(int64_t));
  jo_fx* ia = (jo_fx*)calloc((size_t)(k ? k : 1), sizeof(jo_fx));
  for (int64_t g = 0; g < G; ++g) {
    int64_t c = lab[g];
    l2g[g] = (int32_t)c;
    cnt[c] += grp_count[g];
    ls[c] += grp_lensum[g];
    fx_add_fx(&ia[c], (const jo_fx*)(grp_incacc + 4 * g));
  }
  for (int64_t c = 0; c < k; ++c) {
    jo_centre(cnt[c], ls[c], ia[c].w, &dict_len[c], &dict_inc[c]);
    dict_count[c] = cnt[c];
  }
  free(lab);
  free(cnt);
  free(ls);
  free(ia);
  return k;
}

/* Label propagation (Sec. 5): l_i = l~_g for a piece in local group g. */
void jo_symbolize(const int32_t* local_label, const int64_t* dom_piece_off, const int64_t* dom_group_off,
                  int64_t n_domains, const int32_t* l2g, int32_t* symbol) {
  for (int64_t d = 0; d < n_domains; ++d)
    for (int64_t p = dom_piece_off[d]; p < dom_piece_off[d + 1]; ++p)
      symbol[p] = l2g[dom_group_off[d] + local_label[p]];
}

/* ------------------------------------------------------------------------ */
/* Full-reassignment digitization (Alg. 1, Digitize(P^(m), D); the argmin of */
/* Sec. 3.2): each piece takes the dictionary entry nearest to it in         */
/* normalised coordinates, d2 = dx*dx + dy*dy with dx = X_p - X_c and        */
/* dy = Y_p - Y_c (binary64, in that order), X = (scl len) / sigma_len and   */
/* Y = inc / sigma_inc for pieces and entries alike; a tie goes to the       */
/* smaller entry index.  Plain O(N k) scan.  The two-stage scheme of Sec. 5  */
/* replaces this pass by label propagation.                                  */
/* ------------------------------------------------------------------------ */
void jo_reassign(const int32_t* len, const double* inc, int64_t n, double sigma_len, double sigma_inc, double scl,
                 const double* dict_len, const double* dict_inc, int64_t k, int32_t* symbol) {
  double* Xc = (double*)malloc(sizeof(double) * (size_t)(k ? k : 1));
  double* Yc = (double*)malloc(sizeof(double) * (size_t)(k ? k : 1));
  for (int64_t c = 0; c < k; ++c) {
    Xc[c] = norm_len(dict_len[c], scl, sigma_len);
    Yc[c] = norm_inc(dict_inc[c], sigma_inc);
  }
  for (int64_t i = 0; i < n; ++i) {
    const double X = norm_len((double)len[i], scl, sigma_len), Y = norm_inc(inc[i], sigma_inc);
    double best = 0.0;
    int64_t bi = -1;
    for (int64_t c = 0; c < k; ++c) {
      const double dx = X - Xc[c], dy = Y - Yc[c];
      const double d2 = dx * dx + dy * dy;
      if (bi < 0 || d2 < best) {
        best = d2;
        bi = c;
      }
    }
    symbol[i] = (int32_t)bi;
  }
  free(Xc);
  free(Yc);
}

/* Sum of squared errors of an assignment in normalised units (Sec. 3.2; the */
/* quantity whose ratio Table 2 reports): sum over pieces of d2(piece, entry */
/* of its symbol), d2 as in jo_reassign, summed exactly (fixed point 2^-64,  */
/* each term truncated toward zero) and rounded once.                        */
double jo_sse(const int32_t* len, const double* inc, int64_t n, double sigma_len, double sigma_inc, double scl,
              const double* dict_len, const double* dict_inc, const int32_t* symbol) {
  jo_fx acc;
  fx_zero(&acc);
  for (int64_t i = 0; i < n; ++i) {
    const int32_t c = symbol[i];
    const double dx = norm_len((double)len[i], scl, sigma_len) - norm_len(dict_len[c], scl, sigma_len);
    const double dy = norm_inc(inc[i], sigma_inc) - norm_inc(dict_inc[c], sigma_inc);
    fx_add_double(&acc, dx * dx + dy * dy);
  }
  return fx_to_double(&acc);
}

/* ------------------------------------------------------------------------ */
/* Inverse symbolization of one series (Sec. 3.3).                          */
/* inverse digitization: (l~, i~) = dictionary entry of each symbol;         */
/* quantization: v = l~_j + e; l^_j = round(v); e = v - l^_j (e_0 = 0)        */
/*   (the consistent sign of the carry; round_mode 0 = half away from zero,  */
/*   1 = half to even);                                                      */
/* inverse compression from t_0: x^_{pos+q} = level + (i~_j * q) / l^_j,      */
/*   q = 1..l^_j; level += i~_j; pos += l^_j.  Points past the series end are */
/*   dropped; a short chain leaves the tail at the final level.               */
/* qlen receives l^_j.                                                        */
/* ------------------------------------------------------------------------ */
/* round_mode 1: nearest, ties to even (rint in the default rounding mode).
 * round_mode 0 (the default) is C's round(): nearest, ties away from zero. */
static double round_half_even(double v) { return rint(v); }

void jo_reconstruct_series(const int32_t* symbol, int64_t n_pieces, const double* dict_len, const double* dict_inc,
                           double x0, int64_t n_s, int round_mode, int32_t* qlen, double* xhat) {
  if (n_s <= 0) return;
  xhat[0] = x0;
  double e = 0.0, level = x0;
  int64_t pos = 0;
  for (int64_t j = 0; j < n_pieces; ++j) {
    double lt = dict_len[symbol[j]];
    double it = dict_inc[symbol[j]];
    double v = lt + e;
    double lh = round_mode ? round_half_even(v) : round(v);
    e = v - lh;
    int64_t L = (int64_t)lh;
    qlen[j] = (int32_t)L;
    for (int64_t q = 1; q <= L && pos + q <= n_s - 1; ++q) xhat[pos + q] = level + (it * (double)q) / lh;
    level = level + it;
    pos += L;
  }
  for (int64_t i = pos + 1; i <= n_s - 1; ++i) xhat[i] = level;
}

/* Reconstruction MSE over all series (Sec. 3.3): sum of squared differences
 * over all points divided by the total number of points. */
double jo_mse(const double* x, const double* xhat, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double d = x[i] - xhat[i];
    s = s + d * d;
  }
  return s / (double)n;
}

/* Gradient of the MSE with respect to dict_inc, with the quantized lengths
 * held fixed (x^ is then affine in dict_inc).  For piece j of a series with
 * start pos_j and length l^_j, d x^_{pos_j+q} / d i~_{a_j} = q / l^_j for
 * q <= l^_j and 1 for every later point of the series.  Accumulates
 * (2 / n_total) * sum_i (x^_i - x_i) * d x^_i / d i~ into grad. */
void jo_reconstruct_grad_series(const double* x, const double* xhat, const int32_t* symbol, const int32_t* qlen,
                                int64_t n_pieces, int64_t n_s, double n_total, double* grad) {
  /* suffix[i] = sum_{i' >= i} r_i' */
  double* suffix = (double*)malloc(sizeof(double) * (size_t)(n_s + 1));
  suffix[n_s] = 0.0;
  for (int64_t i = n_s - 1; i >= 0; --i) suffix[i] = suffix[i + 1] + (xhat[i] - x[i]);
  int64_t pos = 0;
  for (int64_t j = 0; j < n_pieces; ++j) {
    int64_t L = qlen[j];
    double acc = 0.0;
    for (int64_t q = 1; q <= L && pos + q <= n_s - 1; ++q) acc = acc + ((double)q / (double)L) * (xhat[pos + q] - x[pos + q]);
    int64_t after = pos + L + 1;
    if (after <= n_s - 1) acc = acc + suffix[after];
    grad[symbol[j]] += (2.0 / n_total) * acc;
    pos += L;
  }
  free(suffix);
}
