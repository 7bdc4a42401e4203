// Device evaluation of compiled count tables (see pm_table.h for the format).
//
// A table holds the piecewise quasi-polynomial properties p_i(n) of one kernel
// (Sec. 2: "cheaply reevaluated for changed values of the parameter vector n").
// Evaluation is exact: atoms with 32-bit magic-number division, piece selection
// with 64-bit condition sums, monomials in 64-bit two's-complement arithmetic
// (exact whenever the final count fits in int64, which the compiler checks on
// the declared parameter box).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"
#include "pm_table.h"

namespace pmd {

// Granlund & Montgomery (1994), Fig. 4.1: q = floor(x / c) for unsigned 32-bit x.
__device__ __forceinline__ uint32_t udiv_magic(uint32_t x, uint32_t m, uint32_t sh2) {
  uint32_t t = __umulhi(m, x);
  return (t + ((x - t) >> 1)) >> sh2;
}

// Mathematical floor(num / c), c >= 2.
__device__ __forceinline__ int32_t floor_div(int32_t num, uint32_t c, uint32_t m, uint32_t sh2, bool mayneg) {
  if (!mayneg) return (int32_t)udiv_magic((uint32_t)num, m, sh2);
  bool neg = num < 0;
  uint32_t x = neg ? (uint32_t)(-num) + c - 1u : (uint32_t)num;
  int32_t q = (int32_t)udiv_magic(x, m, sh2);
  return neg ? -q : q;
}

__device__ __forceinline__ int64_t ld64(const uint32_t *p) {
  return (int64_t)((uint64_t)p[0] | ((uint64_t)p[1] << 32));
}

// Evaluate table T at point n (int32, already known to lie in T's box) for the
// calling thread.  slots: this thread's pmt::MAX_SLOTS int64 slots (stride ss, shared
// memory).  emit(col, value) is called once per non-empty column of the selected
// piece, post(col, value) once per post-op.  Returns false on a malformed table.
template <class Emit, class Post>
__device__ __forceinline__ bool eval_table(const uint32_t *__restrict__ T, const int32_t *n, int64_t *slots, int ss,
                                           Emit &&emit, Post &&post) {
  const int P = (int)T[pmt::H_NPARAMS];
  const int A = (int)T[pmt::H_NATOMS];
  const int NC = (int)T[pmt::H_NCONDS];
  if (P > 4 || P + A > pmt::MAX_VALUES || NC > pmt::MAX_CONDS) return false;
#pragma unroll
  for (int p = 0; p < 4; p++) {
    if (p < P) slots[p * ss] = n[p];
    slots[(pmt::HOLD_SLOT + p) * ss] = 0;  // post-op inputs a piece does not produce are zero
  }
  slots[pmt::CONST_SLOT * ss] = 1;
  const uint32_t *at = T + T[pmt::H_OFF_ATOMS];
  for (int a = 0; a < A; a++, at += pmt::ATOM_WORDS) {
    const uint4 q0 = *(const uint4 *)at, q1 = *(const uint4 *)(at + 4);
    int32_t num = (int32_t)q1.x;
    num += (int32_t)q0.x * n[0];
    if (P > 1) num += (int32_t)q0.y * n[1];
    if (P > 2) num += (int32_t)q0.z * n[2];
    if (P > 3) num += (int32_t)q0.w * n[3];
    slots[(P + a) * ss] = floor_div(num, q1.y, q1.z, (q1.w >> 8) & 0xFF, (q1.w >> 16) & 1);
  }
  uint32_t bits = 0;
  const uint32_t *cd = T + T[pmt::H_OFF_CONDS];
  for (int c = 0; c < NC; c++) {
    const int nt = (int)cd[0];
    int64_t s = ld64(cd + 1);
    for (int t = 0; t < nt; t++) s += (int64_t)(int32_t)cd[4 + 2 * t] * slots[min(cd[3 + 2 * t], (uint32_t)pmt::MAX_SLOTS - 1) * ss];
    bits |= (uint32_t)(s >= 0) << c;
    cd += 3 + 2 * nt;
  }
  const uint32_t *lut = T + T[pmt::H_OFF_LUT];
  const uint32_t piece = (lut[bits >> 2] >> (8 * (bits & 3))) & 0xFF;
  if (piece >= T[pmt::H_NPIECES]) return false;
  const uint4 pc = *(const uint4 *)(T + T[pmt::H_OFF_PIECES] + 4 * piece);
  if (P + A + pc.y > (uint32_t)pmt::MAX_PRODS) return false;
  const uint32_t *pr = T + T[pmt::H_OFF_PRODS] + pc.x;
  int64_t *dst = slots + (P + A) * ss;
  for (uint32_t j = 0; j < pc.y; j++, dst += ss) {
    const uint32_t w = pr[j];
    *dst = (int64_t)((uint64_t)slots[min(w & 0xFF, (uint32_t)pmt::MAX_SLOTS - 1) * ss] *
                     (uint64_t)slots[min((w >> 8) & 0xFF, (uint32_t)pmt::MAX_SLOTS - 1) * ss]);
  }
  const uint4 *en = (const uint4 *)(T + T[pmt::H_OFF_ENTRIES]) + pc.z;
  // exact division by the table's denominator (D * count < 2^62, so no wrap before it)
  const bool den = T[pmt::H_DEN] != 1;
  const uint32_t den_sh = T[pmt::H_DEN_SHIFT] & 63;
  const uint64_t den_inv = ld64(T + pmt::H_DEN_INV);
  uint64_t acc = 0;
  for (uint32_t e = 0; e < pc.w; e++) {
    const uint4 E = en[e];
    const uint32_t sl = (E.z >> 8) & 0xFF;
    const uint64_t coef = (uint64_t)E.x | ((uint64_t)E.y << 32);
    acc += coef * (uint64_t)slots[min(sl, (uint32_t)pmt::MAX_SLOTS - 1) * ss];
    if (E.z & pmt::ENTRY_LAST) {
      const int64_t val = den ? (int64_t)((uint64_t)((int64_t)acc >> den_sh) * den_inv) : (int64_t)acc;
      const uint32_t hold = (E.z >> 16) & 0xF;
      if (hold) slots[(pmt::HOLD_SLOT + hold - 1) * ss] = val;
      emit((int)(E.z & 0xFF), val);
      acc = 0;
    }
  }
  const uint32_t npost = T[pmt::H_NPOST];
  const uint32_t *po = T + T[pmt::H_OFF_POST];
  for (uint32_t q = 0; q < npost; q++) {
    const uint32_t w = po[q];
    const int64_t va = slots[(pmt::HOLD_SLOT + ((w >> 8) & 3)) * ss];
    const int64_t vb = slots[(pmt::HOLD_SLOT + ((w >> 16) & 3)) * ss];
    post((int)(w & 0xFF), va < vb ? va : vb);
  }
  return true;
}

// Load a point (int64 [4] or [P]) and check it against T's box; writes int32 n.
__device__ __forceinline__ bool point_in_box(const uint32_t *T, const int64_t *pt, int P, int32_t *n) {
  bool ok = true;
#pragma unroll
  for (int p = 0; p < 4; p++) {
    if (p < P) {
      int64_t x = pt[p];
      int64_t lo = (int32_t)T[pmt::H_BOX_LO + p], hi = (int32_t)T[pmt::H_BOX_HI + p];
      ok = ok && x >= lo && x <= hi;
      n[p] = (int32_t)x;
    } else {
      n[p] = 0;
    }
  }
  return ok;
}

// ---- Exact fixed-point prediction on the integer pipes.
// Weights become integers W = round(w * 2^E) with one E per weight vector, the largest
// for which sum_i |W_i| <= 2^62 (weight_exponent).  Any counts |v_i| <= 2^63 then give
// |sum_i v_i W_i| < 2^126, so the exact sum S = sum_i v_i W_i never wraps its 128 bits,
// and T = S * 2^-E differs from sum_i v_i w_i by at most 2^-(E+1) sum_i |v_i|, i.e. by
// at most 2^-62 (sum_i |w_i| / min_i |w_i|) of sum_i |v_i w_i|: 4e-11 for weights with
// the spread of the paper's fitted set (Table 2: 1.29e-4 s next to 3.91e-13 s).
struct Acc128 {
  uint64_t lo, hi;  // two's complement
  __device__ __forceinline__ void zero() { lo = hi = 0; }
};

// A fixed-point weight W (|W| <= 2^62) as three limbs: W = w2 2^56 + w1 2^28 + w0 with
// w0, w1 in [0, 2^28) and w2 signed (|w2| <= 2^6).
struct Limbs3 { uint32_t w0, w1; int32_t w2; };
__host__ __device__ __forceinline__ Limbs3 to_limbs3(int64_t W) {
  return Limbs3{(uint32_t)(W & 0x0FFFFFFF), (uint32_t)((W >> 28) & 0x0FFFFFFF), (int32_t)(W >> 56)};
}

// Exact sum of count x weight products in five 64-bit limb accumulators.  A count
// v (0 <= v < 2^62) is split into 28-bit limbs v0, v1 and the top bits v2 (< 2^6);
// each limb pair is one 32 x 32 -> 64-bit multiply-add into the accumulator of its
// power of 2^28.  Every partial product is below 2^56 in magnitude, at most three
// meet in one accumulator per term, so 34 terms never overflow.
struct LimbAcc {
  uint64_t l0;
  int64_t l1, l2, l3, l4;
  __device__ __forceinline__ void zero() { l0 = 0; l1 = l2 = l3 = l4 = 0; }
  __device__ __forceinline__ void add(uint64_t v, Limbs3 w) {
    const uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
    const uint32_t v0 = lo & 0x0FFFFFFFu;
    const uint32_t v1 = __funnelshift_r(lo, hi, 28) & 0x0FFFFFFFu;
    const uint32_t v2 = hi >> 24;
    asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(l0) : "r"(v0), "r"(w.w0));
    asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(l1) : "r"(v0), "r"(w.w1));
    asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(l1) : "r"(v1), "r"(w.w0));
    asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(l2) : "r"(v0), "r"(w.w2));
    asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(l2) : "r"(v1), "r"(w.w1));
    asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(l2) : "r"(v2), "r"(w.w0));
    asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(l3) : "r"(v1), "r"(w.w2));
    asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(l3) : "r"(v2), "r"(w.w1));
    asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(l4) : "r"(v2), "r"(w.w2));
  }
  __device__ __forceinline__ Acc128 sum() const {
    // S = l0 + l1 2^28 + l2 2^56 + l3 2^84 + l4 2^112 (mod 2^128, two's complement)
    const uint64_t a1 = (uint64_t)l1 << 28, a2 = (uint64_t)l2 << 56;
    const uint64_t h1 = (uint64_t)(l1 >> 36), h2 = (uint64_t)(l2 >> 8), h3 = (uint64_t)l3 << 20,
                   h4 = (uint64_t)l4 << 48;
    uint64_t lo = l0 + a1;
    uint64_t hi = h1 + h2 + h3 + h4 + (lo < a1 ? 1ull : 0ull);
    const uint64_t lo2 = lo + a2;
    hi += lo2 < a2 ? 1ull : 0ull;
    return Acc128{lo2, hi};
  }
};

// signed 128-bit a < b
__device__ __forceinline__ bool acc_less(const Acc128 &a, const Acc128 &b) {
  return (int64_t)a.hi < (int64_t)b.hi || (a.hi == b.hi && a.lo < b.lo);
}

// Monotone 64-bit key of a 128-bit signed value: sign, 7-bit exponent and the 56 bits
// below the leading one (a float with a 56-bit mantissa; equal values give equal keys).
__device__ __forceinline__ int64_t acc_key(const Acc128 &a) {
  const bool neg = (int64_t)a.hi < 0;
  uint64_t ml = neg ? ~a.lo + 1ull : a.lo;
  uint64_t mh = neg ? ~a.hi + (a.lo == 0 ? 1ull : 0ull) : a.hi;
  if ((mh | ml) == 0) return 0;
  const int lz = mh ? __clzll((long long)mh) : 64 + __clzll((long long)ml);
  // normalise so that bit 127 is the leading one
  if (lz >= 64) { mh = ml << (lz - 64); ml = 0; }
  else if (lz > 0) { mh = (mh << lz) | (ml >> (64 - lz)); ml <<= lz; }
  const int64_t e = 127 - lz;                       // 0..126
  const int64_t k = ((e + 1) << 56) | (int64_t)((mh >> 7) & ((1ull << 56) - 1));
  return neg ? -k : k;
}

// For a positive key k: the smallest 128-bit S with acc_key(S) >= k, so that
// acc_key(S) < k  <=>  S < key_floor(k).  (Used to test candidates without a key.)
__device__ __forceinline__ Acc128 key_floor(int64_t k) {
  Acc128 r;
  const int e = (int)(k >> 56) - 1;                 // exponent of the leading one
  const uint64_t m = (1ull << 56) | ((uint64_t)k & ((1ull << 56) - 1));  // 57 bits
  if (e >= 56) {
    const int sh = e - 56;                          // 0..70
    if (sh == 0) { r.lo = m; r.hi = 0; }
    else if (sh < 64) { r.lo = m << sh; r.hi = m >> (64 - sh); }
    else { r.lo = 0; r.hi = m << (sh - 64); }
  } else {
    const int sh = 56 - e;                          // 1..56: round the mantissa up
    r.lo = (m + (1ull << sh) - 1) >> sh;
    r.hi = 0;
  }
  return r;
}

// Inverse of acc_key times 2^-E, for output: the value (1 + f 2^-56) 2^(e - E) with its
// 56-bit fraction f rounded once to FP64's 52 bits (to nearest, ties to even).  The
// double is assembled from its bit fields with integer operations (this GPU's FP64 pipe
// is narrow); values outside FP64's normal range take ldexp of the same significand.
__device__ __forceinline__ double key_value(int64_t k, int E) {
  if (k == 0) return 0.0;
  const bool neg = k < 0;
  const uint64_t a = (uint64_t)(neg ? -k : k);
  const int e = (int)(a >> 56) - 1;
  const uint64_t f = a & ((1ull << 56) - 1);
  const uint64_t rest = f & 15;
  uint64_t g = (f >> 4) + ((rest > 8 || (rest == 8 && ((f >> 4) & 1))) ? 1 : 0);
  int x = e - E + 1023;                               // biased exponent
  if (g >> 52) {                                      // rounded up to 2: next binade
    g = 0;
    x++;
  }
  if (x >= 1 && x <= 2046)
    return __longlong_as_double((long long)(((uint64_t)neg << 63) | ((uint64_t)x << 52) | g));
  const double v = ldexp((double)((1ull << 52) | g), x - 1023 - 52);
  return neg ? -v : v;
}

// Exponent E of the fixed-point weights W_i = round(w_i 2^E): the largest with
// sum_i |w_i| 2^E <= 2^62 (the sum is rounded up by 2^-40 relative to cover its own
// rounding), so that sum_i |W_i| <= 2^62 + k/2.  Every kernel that ranks or converts
// with E calls this same serial loop, so all of them agree on E bit for bit.
__device__ __forceinline__ int weight_exponent(const double *w, int k) {
  double s = 0;
  for (int c = 0; c < k; c++) s += fabs(w[c]);
  s *= 1.0 + 0x1p-40;
  int e = 0;
  if (s > 0) frexp(s, &e);  // s in [2^(e-1), 2^e)
  return 62 - e;
}

}  // namespace pmd
