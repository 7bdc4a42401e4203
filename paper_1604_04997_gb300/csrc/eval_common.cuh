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
// calling thread.  vals: this thread's value slots (int32, stride vs); prods: its
// product slots (int64, stride ps), both in shared memory.  emit(col, value) is
// called once per non-empty column of the selected piece, post(col, value) once
// per post-op.  Returns false on a malformed table.
template <class Emit, class Post>
__device__ __forceinline__ bool eval_table(const uint32_t *__restrict__ T, const int32_t *n, int32_t *vals, int vs,
                                           int64_t *prods, int ps, Emit &&emit, Post &&post) {
  const int P = (int)T[pmt::H_NPARAMS];
  const int A = (int)T[pmt::H_NATOMS];
  const int NC = (int)T[pmt::H_NCONDS];
  if (P > 4 || P + A > pmt::MAX_VALUES || NC > pmt::MAX_CONDS) return false;
#pragma unroll
  for (int p = 0; p < 4; p++)
    if (p < P) vals[p * vs] = n[p];
  const uint32_t *at = T + T[pmt::H_OFF_ATOMS];
  for (int a = 0; a < A; a++, at += pmt::ATOM_WORDS) {
    const uint4 q0 = *(const uint4 *)at, q1 = *(const uint4 *)(at + 4);
    int32_t num = (int32_t)q1.x;
    num += (int32_t)q0.x * n[0];
    if (P > 1) num += (int32_t)q0.y * n[1];
    if (P > 2) num += (int32_t)q0.z * n[2];
    if (P > 3) num += (int32_t)q0.w * n[3];
    vals[(P + a) * vs] = floor_div(num, q1.y, q1.z, (q1.w >> 8) & 0xFF, (q1.w >> 16) & 1);
  }
  uint32_t bits = 0;
  const uint32_t *cd = T + T[pmt::H_OFF_CONDS];
  for (int c = 0; c < NC; c++) {
    int nt = (int)cd[0];
    int64_t s = ld64(cd + 1);
    for (int t = 0; t < nt; t++) s += (int64_t)(int32_t)cd[4 + 2 * t] * (int64_t)vals[cd[3 + 2 * t] * vs];
    bits |= (uint32_t)(s >= 0) << c;
    cd += 3 + 2 * nt;
  }
  const uint32_t *lut = T + T[pmt::H_OFF_LUT];
  const uint32_t piece = (lut[bits >> 2] >> (8 * (bits & 3))) & 0xFF;
  if (piece >= T[pmt::H_NPIECES]) return false;
  const uint4 pc = *(const uint4 *)(T + T[pmt::H_OFF_PIECES] + 4 * piece);
  if (pc.y > (uint32_t)pmt::MAX_PRODS) return false;
  const uint32_t *pr = T + T[pmt::H_OFF_PRODS] + pc.x;
  for (uint32_t j = 0; j < pc.y; j++) {
    const uint32_t w = pr[j];
    const uint32_t src = w & 0xFF;
    const int64_t v = (int64_t)vals[((w >> 8) & 0xFF) * vs];
    prods[j * ps] = src == 0xFF ? v : (int64_t)((uint64_t)prods[src * ps] * (uint64_t)v);
  }
  const uint4 *en = (const uint4 *)(T + T[pmt::H_OFF_ENTRIES]) + pc.z;
  int64_t h0 = 0, h1 = 0, h2 = 0, h3 = 0;
  uint64_t acc = 0;
  for (uint32_t e = 0; e < pc.w; e++) {
    const uint4 E = en[e];
    const uint32_t p = (E.z >> 8) & 0xFF;
    const uint64_t coef = (uint64_t)E.x | ((uint64_t)E.y << 32);
    acc += p == 0xFF ? coef : coef * (uint64_t)prods[p * ps];
    if (E.z & pmt::ENTRY_LAST) {
      const int64_t val = (int64_t)acc;
      const uint32_t hold = (E.z >> 16) & 0xF;
      if (hold == 1) h0 = val;
      else if (hold == 2) h1 = val;
      else if (hold == 3) h2 = val;
      else if (hold == 4) h3 = val;
      emit((int)(E.z & 0xFF), val);
      acc = 0;
    }
  }
  const uint32_t npost = T[pmt::H_NPOST];
  const uint32_t *po = T + T[pmt::H_OFF_POST];
  for (uint32_t q = 0; q < npost; q++) {
    uint32_t w = po[q];
    uint32_t a = (w >> 8) & 0xFF, b = (w >> 16) & 0xFF;
    int64_t va = a == 0 ? h0 : a == 1 ? h1 : a == 2 ? h2 : h3;
    int64_t vb = b == 0 ? h0 : b == 1 ? h1 : b == 2 ? h2 : h3;
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

// ---- FP64-accurate accumulation on FP32 pipes (Ogita, Rump & Oishi 2005, Dot2).
// An exact int64 count v is split as vh + vl (vh = rn(v), vl = rn(v - vh)); the
// weight w as wh + wl.  Each product's leading term is made error-free with an
// FMA (TwoProduct) and summed error-free (TwoSum); the small cross terms and all
// error terms go to a compensation accumulator.
struct FF { float hi, lo; };

__device__ __forceinline__ FF split_weight(double w) {
  float h = __double2float_rn(w);
  return FF{h, __double2float_rn(w - (double)h)};
}

// The _rn intrinsics keep the compiler from contracting these steps into FMAs,
// which would break the error-free transformations.
__device__ __forceinline__ void two_sum_acc(float &s, float &c, float p, float pe) {
  float t = __fadd_rn(s, p);
  float z = __fsub_rn(t, s);
  float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(e, pe));
}

__device__ __forceinline__ void dot2_term(float &s, float &c, float vh, float vl, float wh, float wl) {
  float p = __fmul_rn(vh, wh);
  float pe = __fmaf_rn(vh, wh, -p);
  pe = __fmaf_rn(vh, wl, pe);
  pe = __fmaf_rn(vl, wh, pe);
  two_sum_acc(s, c, p, pe);
}

__device__ __forceinline__ void dot2_add(float &s, float &c, int64_t v, float wh, float wl) {
  float vh = __ll2float_rn(v);
  float vl = __ll2float_rn(v - (int64_t)vh);
  dot2_term(s, c, vh, vl, wh, wl);
}

}  // namespace pmd
