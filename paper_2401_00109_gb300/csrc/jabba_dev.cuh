// jabba_dev.cuh -- device helpers shared by the CUDA kernels of the JABBA
// symbolization library (arXiv 2401.00109).  sm_103a only.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/jabba.h"

namespace jabba {

typedef unsigned long long u64;
typedef long long i64;

// ---------------------------------------------------------------- status word
// First error wins; read back by jabba_sync_status.
__device__ __forceinline__ void set_status(unsigned* st, unsigned code) { atomicCAS(st, 0u, code); }

// Bounded spin limit for every device-side wait (mbarrier phases, flags).
constexpr unsigned kSpinLimit = 1u << 26;

// The context's status word is followed by the poll limit of its bounded
// waits (jabba_set_spin_limit; 0 = kSpinLimit).  Kernels that wait read it
// once at their start.
__device__ __forceinline__ unsigned spin_limit(const unsigned* status) {
  const unsigned v = ((volatile const unsigned*)status)[1];
  return v ? v : kSpinLimit;
}

// ---------------------------------------------------------------- f64 -> f32 by integer ops
// Truncating conversion of a binary64 value to binary32 using integer
// instructions only (this GPU's FP64 and F2F pipes run at ~1/64 of FP32).
// Valid for |v| < 2^127; |v| < 2^-126 (including 0) maps to a value of the
// same sign with magnitude in [2^-126, 2^-125).  Error: |r - v| <= 2^-23 |v| +
// 2^-125.  Also returns the magnitude's high word for range checks.
__device__ __forceinline__ float f64_to_f32_trunc(double v, unsigned& mag_hi) {
  const unsigned hi = (unsigned)__double2hiint(v);
  const unsigned lo = (unsigned)__double2loint(v);
  const unsigned a = hi & 0x7FFFFFFFu;
  mag_hi = a;
  const unsigned ac = max(a, 897u << 20);            // clamp tiny magnitudes to 2^-126 range
  const unsigned f = __funnelshift_l(lo, ac, 3);     // exponent bits 7..0 and 23 mantissa bits
  // re-bias the exponent: (e - 896) mod 256 == (e + 128) mod 256 -> flip bit 30
  const unsigned r = ((f & 0x7FFFFFFFu) ^ 0x40000000u) | (hi & 0x80000000u);
  return __uint_as_float(r);
}

// ---------------------------------------------------------------- 128/192-bit integers
struct U128 { u64 lo, hi; };
struct I192 { u64 w0, w1, w2; };  // two's complement

__device__ __forceinline__ U128 shl128(u64 m, int s) {  // m << s, 0 <= s < 128
  U128 r;
  if (s >= 64) { r.lo = 0; r.hi = m << (s - 64); }
  else if (s > 0) { r.lo = m << s; r.hi = m >> (64 - s); }
  else { r.lo = m; r.hi = 0; }
  return r;
}

__device__ __forceinline__ U128 shr128(U128 v, int s) {  // v >> s, s >= 0 (truncating)
  U128 r;
  if (s >= 128) { r.lo = 0; r.hi = 0; }
  else if (s >= 64) { r.lo = v.hi >> (s - 64); r.hi = 0; }
  else if (s > 0) { r.lo = (v.lo >> s) | (v.hi << (64 - s)); r.hi = v.hi >> s; }
  else r = v;
  return r;
}

__device__ __forceinline__ void add192(I192& a, u64 b0, u64 b1, u64 b2) {
  asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, %4;\n\taddc.u64 %2, %2, %5;"
      : "+l"(a.w0), "+l"(a.w1), "+l"(a.w2) : "l"(b0), "l"(b1), "l"(b2));
}

__device__ __forceinline__ void sub192(I192& a, u64 b0, u64 b1, u64 b2) {
  asm("sub.cc.u64 %0, %0, %3;\n\tsubc.cc.u64 %1, %1, %4;\n\tsubc.u64 %2, %2, %5;"
      : "+l"(a.w0), "+l"(a.w1), "+l"(a.w2) : "l"(b0), "l"(b1), "l"(b2));
}

// Fixed-point image trunc(|v| * 2^64) of a finite double with |v| < 2^64, as
// an unsigned 128-bit magnitude; the sign is returned separately.
__device__ __forceinline__ U128 fx_mag(double v, bool& neg) {
  const u64 bits = (u64)__double_as_longlong(v);
  neg = (bits >> 63) != 0;
  const int e = (int)((bits >> 52) & 0x7FF);
  U128 z = {0, 0};
  if (e == 0) return z;                                  // zero or subnormal: below 2^-64
  const u64 m = (bits & ((1ull << 52) - 1)) | (1ull << 52);
  const int s = e - 1011;                                // |v| * 2^64 = m * 2^(e - 1075 + 64)
  if (s >= 0) return shl128(m, s);
  if (s <= -64) return z;
  z.lo = m >> (-s);
  return z;
}

// trunc(v^2 * 2^64) for the EXACT square of a finite double, |v| < 2^32.
__device__ __forceinline__ U128 fx_square(double v) {
  const u64 bits = (u64)__double_as_longlong(v);
  const int e = (int)((bits >> 52) & 0x7FF);
  U128 z = {0, 0};
  if (e == 0) return z;
  const u64 m = (bits & ((1ull << 52) - 1)) | (1ull << 52);
  U128 sq;
  sq.lo = m * m;
  sq.hi = __umul64hi(m, m);                              // m^2 < 2^106
  const int s = 2 * (e - 1075) + 64;                     // v^2 * 2^64 = m^2 * 2^s
  if (s >= 0) {                                          // s <= 22 under the range contract
    if (s == 0) return sq;
    U128 r;
    r.lo = sq.lo << s;
    r.hi = (sq.hi << s) | (sq.lo >> (64 - s));
    return r;
  }
  return shr128(sq, -s);
}

// trunc(|v| * L * 2^64) for the EXACT product of a finite double v,
// |v| < 2^32, and an integer 0 <= L < 2^32 (the product is below 2^128).
__device__ __forceinline__ U128 fx_prod(double v, unsigned L) {
  const u64 bits = (u64)__double_as_longlong(v);
  const int e = (int)((bits >> 52) & 0x7FF);
  U128 z = {0, 0};
  if (e == 0 || L == 0) return z;
  const u64 m = (bits & ((1ull << 52) - 1)) | (1ull << 52);
  U128 p;
  p.lo = m * (u64)L;
  p.hi = __umul64hi(m, (u64)L);                          // m L < 2^85
  const int s = e - 1011;                                // |v| L 2^64 = m L 2^s
  if (s >= 0) {
    if (s == 0) return p;
    U128 r;                                              // s <= 42 under the range contract
    r.lo = p.lo << s;
    r.hi = (p.hi << s) | (p.lo >> (64 - s));
    return r;
  }
  return shr128(p, -s);
}

// Signed add of a magnitude into a 192-bit accumulator.
__device__ __forceinline__ void acc_signed(I192& a, U128 m, bool neg) {
  if (neg) sub192(a, m.lo, m.hi, 0); else add192(a, m.lo, m.hi, 0);
}

// Split a 192-bit two's-complement value into six 32-bit limbs for
// deferred-carry accumulation with 64-bit atomics: the top limb is signed.
__device__ __forceinline__ void limbs6(const I192& a, i64 out[6]) {
  out[0] = (i64)(a.w0 & 0xFFFFFFFFull);
  out[1] = (i64)(a.w0 >> 32);
  out[2] = (i64)(a.w1 & 0xFFFFFFFFull);
  out[3] = (i64)(a.w1 >> 32);
  out[4] = (i64)(a.w2 & 0xFFFFFFFFull);
  out[5] = (i64)(int)(unsigned)(a.w2 >> 32);           // sign-extended top limb
}

// Normalize six deferred-carry limbs (sum_i L_i 2^(32 i)) into 192 bits.
__device__ __forceinline__ I192 from_limbs6(const i64 L[6]) {
  u64 w[6];
  i64 carry = 0;
  for (int i = 0; i < 6; ++i) {
    const i64 v = L[i] + carry;
    w[i] = (u64)v & 0xFFFFFFFFull;
    carry = v >> 32;                                     // arithmetic shift keeps the sign
  }
  I192 r;
  r.w0 = w[0] | (w[1] << 32);
  r.w1 = w[2] | (w[3] << 32);
  r.w2 = w[4] | (w[5] << 32);
  return r;
}

// Build the binary64 value sig * 2^exp2 for 2^52 <= sig <= 2^53 (exact).
__device__ __forceinline__ double make_double(u64 sig, int exp2, bool neg) {
  if (sig == (1ull << 53)) { sig >>= 1; ++exp2; }
  const int be = exp2 + 52 + 1023;                       // normal range assumed
  const u64 bits = ((u64)neg << 63) | ((u64)be << 52) | (sig & ((1ull << 52) - 1));
  return __longlong_as_double((i64)bits);
}

// Low 64 bits of (w2:w1:w0) >> s, 0 <= s < 192.
__device__ __forceinline__ u64 shr192_lo(u64 w0, u64 w1, u64 w2, int s) {
  if (s >= 128) return w2 >> (s - 128);
  if (s >= 64) {
    const int t = s - 64;
    return t ? ((w1 >> t) | (w2 << (64 - t))) : w1;
  }
  return s ? ((w0 >> s) | (w1 << (64 - s))) : w0;
}

// Whether any of the bits [0, p) of (w2:w1:w0) is set, 0 <= p <= 192.
__device__ __forceinline__ bool any_below(u64 w0, u64 w1, u64 w2, int p) {
  u64 m0 = 0, m1 = 0, m2 = 0;
  if (p >= 128) { m0 = ~0ull; m1 = ~0ull; m2 = (p - 128) ? ((1ull << (p - 128)) - 1) : 0; if (p == 192) m2 = ~0ull; }
  else if (p >= 64) { m0 = ~0ull; m1 = (p - 64) ? ((1ull << (p - 64)) - 1) : 0; }
  else { m0 = p ? ((1ull << p) - 1) : 0; }
  return ((w0 & m0) | (w1 & m1) | (w2 & m2)) != 0;
}

// Round an unsigned integer held in up to 192 bits (w2:w1:w0) to binary64
// (nearest, ties to even), times 2^scale2 (result assumed in normal range).
__device__ __forceinline__ double round_u192(u64 w0, u64 w1, u64 w2, int scale2, bool neg) {
  int top;
  if (w2) top = 128 + 63 - __clzll((i64)w2);
  else if (w1) top = 64 + 63 - __clzll((i64)w1);
  else if (w0) top = 63 - __clzll((i64)w0);
  else return neg ? -0.0 : 0.0;
  if (top <= 52) {                                       // exact
    const int sh = 52 - top;
    return make_double(w0 << sh, scale2 - sh, neg);
  }
  const int lo = top - 52;                               // keep bits lo..top
  u64 sig = shr192_lo(w0, w1, w2, lo);
  const int rb = (int)(shr192_lo(w0, w1, w2, lo - 1) & 1ull);
  const bool sticky = any_below(w0, w1, w2, lo - 1);
  if (rb && (sticky || (sig & 1ull))) sig += 1;
  return make_double(sig, lo + scale2, neg);
}

// Signed 192-bit fixed point (units 2^-64) -> binary64, nearest-even.
__device__ __forceinline__ double i192_to_double(I192 a) {
  const bool neg = (i64)a.w2 < 0;
  if (neg) {
    a.w0 = ~a.w0; a.w1 = ~a.w1; a.w2 = ~a.w2;
    add192(a, 1, 0, 0);
  }
  return round_u192(a.w0, a.w1, a.w2, -64, neg);
}

// ---------------------------------------------------------------- small utilities
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

}  // namespace jabba
