// Device helpers shared by the single-instance round kernels (dp_kernels.cu)
// and the batched-node kernels (dp_batch.cu): IEEE bit tests, the
// order-preserving binary64 <-> int64 key map used by the bound atomics,
// directed binary32 conversions, the binary32 screen, and the per-row
// decisions of Step 2 (arXiv 2009.07785, Sec. 1.1).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cfloat>

#include "dp_internal.h"

namespace dp {

// ---------------------------------------------------------------- helpers --

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ float f_inf() { return __uint_as_float(0x7F800000u); }

// The two 32-bit halves of a binary64 value through an opaque register move,
// so that the tests below stay integer operations.  Written as plain bit
// tests on the 64-bit pattern, some of them are recognised by the compiler
// as binary64 comparisons (class tests), which issue on the binary64 pipe:
// one per test, i.e. as many as the activity FMAs in the activity loop.
__device__ __forceinline__ void dsplit(double x, unsigned &lo, unsigned &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(x));
}

// Sign change of a binary64 value on the integer pipe (exact).
__device__ __forceinline__ double d_neg(double x) {
  unsigned lo, hi;
  dsplit(x, lo, hi);
  double r;
  asm("mov.b64 %0, {%1, %2};" : "=d"(r) : "r"(lo), "r"(hi ^ 0x80000000u));
  return r;
}
// The 64-bit pattern of a binary64 value, assembled from its halves so that
// sign flips, masks and zero tests on it stay integer operations.
__device__ __forceinline__ unsigned long long dbits(double x) {
  unsigned lo, hi;
  dsplit(x, lo, hi);
  return ((unsigned long long)hi << 32) | lo;
}
__device__ __forceinline__ bool d_isinf(double x) {
  unsigned lo, hi;
  dsplit(x, lo, hi);
  return ((hi & 0x7FFFFFFFu) == 0x7FF00000u) & (lo == 0u);
}
__device__ __forceinline__ bool d_isfinite(double x) {
  unsigned lo, hi;
  dsplit(x, lo, hi);
  return (hi & 0x7FF00000u) != 0x7FF00000u;
}
__device__ __forceinline__ bool d_isnan(double x) {
  unsigned lo, hi;
  dsplit(x, lo, hi);
  const unsigned h = hi & 0x7FFFFFFFu;
  return (h > 0x7FF00000u) | ((h == 0x7FF00000u) & (lo != 0u));
}
__device__ __forceinline__ bool d_is_neginf(double x) {
  unsigned lo, hi;
  dsplit(x, lo, hi);
  return (hi == 0xFFF00000u) & (lo == 0u);
}
__device__ __forceinline__ bool d_is_posinf(double x) {
  unsigned lo, hi;
  dsplit(x, lo, hi);
  return (hi == 0x7FF00000u) & (lo == 0u);
}
// The binary64 value of a nonzero integer v with |v| <= 127, assembled on
// the integer pipe from the IEEE 754 fields: sign, exponent 1023 + e with
// e = floor(log2|v|), and the bits of |v| below its leading one shifted to
// the top of the 52-bit fraction.  Exact.
__device__ __forceinline__ double small_int_to_double(int v) {
  const unsigned long long s = v < 0 ? 1ull : 0ull;
  const unsigned m = (unsigned)(v < 0 ? -v : v);
  const int e = 31 - __clz(m);
  const unsigned long long frac = (unsigned long long)(m - (1u << e)) << (52 - e);
  return __longlong_as_double(
      (long long)((s << 63) | ((unsigned long long)(1023 + e) << 52) | frac));
}
// Coefficient at element `off` of the sliced layout: from the int8 copy
// when the matrix has one (1 byte per value instead of 8), streamed.
__device__ __forceinline__ double ld_coef(const DevMatrix &M, int64_t off) {
  if (M.val8) return small_int_to_double((int)__ldcs(M.val8 + off));
  return __ldcs(M.val + off);
}

// coefficient sign without a binary64 comparison (coefficients are nonzero)
__device__ __forceinline__ bool d_pos(double a) {
  unsigned lo, hi;
  dsplit(a, lo, hi);
  return (int)hi >= 0;
}

// Order-preserving map between binary64 values and signed 64-bit keys, so
// that integer atomicMax/atomicMin implement max/min of doubles.
// (Built from the two 32-bit halves: sign and zero tests on the 64-bit
// pattern of a binary64 value can be turned into binary64 comparisons.)
__device__ __forceinline__ long long key_of(double x) {
  unsigned lo, hi;
  dsplit(x, lo, hi);
  const unsigned m = (unsigned)((int)hi >> 31);  // all ones for a negative value
  return (long long)(((unsigned long long)(hi ^ (m >> 1)) << 32) | (lo ^ m));
}
__device__ __forceinline__ double val_of_key(long long k) {
  return __longlong_as_double(k >= 0 ? k : (k ^ 0x7FFFFFFFFFFFFFFFll));
}

// Exact floor / ceil of a binary64 value computed on the integer pipe from
// the IEEE 754 binary64 layout (1 sign, 11 exponent, 52 fraction bits):
// clear the fraction bits below the binary point; a negative value with a
// nonzero cleared part moves one unit away from zero (a carry out of the
// fraction field correctly bumps the exponent).  Keeps binary64 pipe time for
// the arithmetic that needs it.
__device__ __forceinline__ double d_floor_int(double x) {
  const unsigned long long b = dbits(x);
  const int e = (int)((b >> 52) & 0x7FFull) - 1023;
  const bool neg = (b >> 63) != 0ull;
  if (e >= 52) return x;  // integral, infinite or NaN
  if (e < 0) {            // |x| < 1
    if (!neg) return 0.0;
    return ((b << 1) == 0ull) ? x : -1.0;  // -0 stays -0
  }
  const unsigned long long unit = 1ull << (52 - e);
  const unsigned long long frac = unit - 1ull;
  if ((b & frac) == 0ull) return x;
  unsigned long long t = b & ~frac;
  if (neg) t += unit;
  return __longlong_as_double((long long)t);
}
__device__ __forceinline__ double d_ceil_int(double x) {
  return d_neg(d_floor_int(d_neg(x)));
}
// x > y for non-NaN binary64 values, on the integer pipe: order-preserving
// keys with -0 folded onto +0 (IEEE comparison treats them as equal).
__device__ __forceinline__ long long cmp_key(double x) {
  unsigned lo, hi;
  dsplit(x, lo, hi);
  if (((hi << 1) | lo) == 0u) hi = 0u;  // -0 -> +0
  const unsigned m = (unsigned)((int)hi >> 31);
  return (long long)(((unsigned long long)(hi ^ (m >> 1)) << 32) | (lo ^ m));
}
// |x| < t for a positive (possibly infinite) t; false for NaN x.
__device__ __forceinline__ bool d_abs_lt(double x, double t) {
  return (dbits(x) & 0x7FFFFFFFFFFFFFFFull) < dbits(t);
}
// max(1, |x|) for non-NaN x, by selection.
__device__ __forceinline__ double d_max1abs(double x) {
  unsigned lo, hi;
  dsplit(x, lo, hi);
  hi &= 0x7FFFFFFFu;  // |x| >= 1 iff its high word is at least that of 1.0
  double a;
  asm("mov.b64 %0, {%1, %2};" : "=d"(a) : "r"(lo), "r"(hi));
  return hi >= 0x3FF00000u ? a : 1.0;
}

// A binary32 value >= x, from the bit pattern b of x (IEEE 754 field
// layout), with no binary64-pipe work.  Truncates the significand toward
// zero and steps one unit up when bits were dropped from a positive value.
// Sign changes and absolute values are applied to the bit pattern (never to
// a binary64 value, which would cost a binary64-pipe instruction).
__device__ __forceinline__ float f32_up_bits(unsigned long long b) {
  unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  unsigned mh = hi & 0x7FFFFFFFu;
  bool neg = (hi >> 31) != 0;
  unsigned e = mh >> 20;
  if (e == 0x7FFu) return __uint_as_float((hi & 0x80000000u) | 0x7F800000u);
  if (e >= 1151u) return neg ? -FLT_MAX : f_inf();
  if (e < 897u) {
    if (neg) return -0.0f;
    return (mh | lo) ? FLT_MIN : 0.0f;
  }
  unsigned t = ((mh << 3) | (lo >> 29)) - (896u << 23);
  bool exact = (lo & 0x1FFFFFFFu) == 0u;
  if (!neg) return __uint_as_float(exact ? t : t + 1u);
  return -__uint_as_float(t);
}
constexpr unsigned long long kSign64 = 0x8000000000000000ull;
__device__ __forceinline__ float f32_up(double x) { return f32_up_bits(dbits(x)); }
// a binary32 value <= x
__device__ __forceinline__ float f32_dn(double x) { return -f32_up_bits(dbits(x) ^ kSign64); }
// binary32 bounds of |x| from above and below
__device__ __forceinline__ float f32_up_abs(double x) { return f32_up_bits(dbits(x) & ~kSign64); }
__device__ __forceinline__ float f32_dn_abs(double x) { return -f32_up_bits(dbits(x) | kSign64); }

// Upper bound on |a| as binary32, exact when |a| is a binary32 value, for
// |a| in [2^-126, 2^127); rows holding a coefficient outside [2^-120, 2^120]
// are flagged on the host and never use this value.
__device__ __forceinline__ float absup_fast(double a) {
  unsigned long long b = (unsigned long long)__double_as_longlong(a);
  unsigned mh = (unsigned)(b >> 32) & 0x7FFFFFFFu, lo = (unsigned)b;
  unsigned t = ((mh << 3) | (lo >> 29)) - (896u << 23);
  return __uint_as_float(t + ((lo & 0x1FFFFFFFu) != 0u));
}
// Lower bound on |a| as binary32 (truncated significand), same range.
__device__ __forceinline__ float absdn_fast(double a) {
  unsigned lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(a));
  const unsigned mh = hi & 0x7FFFFFFFu;
  return __uint_as_float(((mh << 3) | (lo >> 29)) - (896u << 23));
}
// Upper bound on |a| * W from |a| in [ad, au] and an upper bound W of the
// width (either sign).
__device__ __forceinline__ float screen_prod(float au, float ad, float W) {
  return __fmul_ru(W >= 0.0f ? au : ad, W);
}

// ---- the binary32 screen ---------------------------------------------------
//
// For a > 0 the upper-bound candidate of x_j from the right-hand side is, in
// exact arithmetic, L_j + s/a with s = rhs - minact; it is applied only if
// it lies below U_j - tau*max(1,|U_j|) (continuous) or, after rounding,
// below U_j (integer: L_j + s/a < U_j - eps_int).  So it can only be applied
// if  s < |a| WU_j  with  WU_j = U_j - L_j - tau*max(1,|U_j|)  (continuous)
// or  U_j - L_j - eps_int  (integer).  The three other sign/side cases give
// the same form with WL_j (lower candidates use max(1,|L_j|)):
//   right-hand side: a > 0 -> upper (WU), a < 0 -> lower (WL)
//   left-hand side:  a > 0 -> lower (WL), a < 0 -> upper (WU)
// The record stores binary32 upper bounds of WU, WL enlarged by
// 2^-40 (|L|+|U|); a row side stores a binary32 lower bound thr of
// s - 2^-39 (|side| + |activity|).  These margins exceed the rounding of
// every binary64 operation of the candidate formula and of the acceptance
// threshold, so  upper(|a| W) <= thr  proves that the nonzero's candidate
// from that side is not applied.  W may be negative (a fixed variable, or
// bounds closer than the threshold): then |a| W <= lower(|a|) * upper(W),
// which keeps the candidates of fixed variables in tight rows (zero slack,
// e.g. set partitioning rows at the fixed point) out of the exact path.

__device__ __forceinline__ void screen_widths(double L, double U, bool isint, float tau_dn,
                                              float eps_dn, float &WU, float &WL) {
  float base = __fsub_ru(f32_up(U), f32_dn(L));
  if (!(base <= FLT_MAX)) {  // an infinite (or unrepresentable) width
    WU = WL = f_inf();
    return;
  }
  float absorb = __fmul_ru(0x1p-40f, __fadd_ru(f32_up_abs(L), f32_up_abs(U)));
  float cu, cl;
  if (isint) {
    cu = cl = eps_dn;
  } else {
    cu = __fmul_rd(tau_dn, fmaxf(1.0f, f32_dn_abs(U)));
    cl = __fmul_rd(tau_dn, fmaxf(1.0f, f32_dn_abs(L)));
  }
  WU = __fadd_ru(__fsub_ru(base, cu), absorb);
  WL = __fadd_ru(__fsub_ru(base, cl), absorb);
  if (!(WU == WU)) WU = f_inf();  // never NaN (inf - inf on invalid input)
  if (!(WL == WL)) WL = f_inf();
}

__device__ __forceinline__ void ld_rec(const VarRec *p, double &L, double &U, float &WU,
                                       float &WL, uint32_t &flags) {
  double d2, d3;
  asm("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];"
      : "=d"(L), "=d"(U), "=d"(d2), "=d"(d3)
      : "l"(p));
  long long w = __double_as_longlong(d2);
  WU = __int_as_float((int)(w & 0xFFFFFFFFll));
  WL = __int_as_float((int)((unsigned long long)w >> 32));
  flags = (uint32_t)((unsigned long long)__double_as_longlong(d3) & 0xFFFFFFFFull);
}
// ld_rec through L2 (coherent with the stores of the same launch), for the
// persistent loops, which rewrite the records between their phases; the
// read-only path of ld_rec is only valid where a kernel never sees a record
// change.
__device__ __forceinline__ void ld_rec_cg(const VarRec *p, double &L, double &U, float &WU,
                                          float &WL, uint32_t &flags) {
  const double2 *q = reinterpret_cast<const double2 *>(p);
  const double2 lu = __ldcg(q), wf = __ldcg(q + 1);
  L = lu.x;
  U = lu.y;
  const double d3 = wf.y;
  long long w = __double_as_longlong(wf.x);
  WU = __int_as_float((int)(w & 0xFFFFFFFFll));
  WL = __int_as_float((int)((unsigned long long)w >> 32));
  flags = (uint32_t)((unsigned long long)__double_as_longlong(d3) & 0xFFFFFFFFull);
}
template <bool kCo>
__device__ __forceinline__ void ld_rec_t(const VarRec *p, double &L, double &U, float &WU,
                                         float &WL, uint32_t &flags) {
  if (kCo) ld_rec_cg(p, L, U, WU, WL, flags);
  else ld_rec(p, L, U, WU, WL, flags);
}

__device__ __forceinline__ void st_rec(VarRec *p, double L, double U, float WU, float WL,
                                       uint32_t flags) {
  long long w = (long long)(((unsigned long long)__float_as_uint(WL) << 32) |
                            (unsigned long long)__float_as_uint(WU));
  double d2 = __longlong_as_double(w);
  double d3 = __longlong_as_double((long long)flags);
  asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(L), "d"(U), "d"(d2),
               "d"(d3)
               : "memory");
}

__device__ __forceinline__ void write_var(VarRec *p, double L, double U, uint32_t vt,
                                          float tau_dn, float eps_dn) {
  float WU, WL;
  screen_widths(L, U, vt != 0u, tau_dn, eps_dn, WU, WL);
  st_rec(p, L, U, WU, WL, vt);
}

__device__ __forceinline__ void set_flag(int32_t *f) {
  atomicExch(f, 1);
  __threadfence();
}

// ------------------------------------------------------- per-row decisions --

// What the candidate step needs to know about one row (kept in shared
// memory so that any lane of the warp can process any lane's nonzeros).
struct RowView {
  double minfin, maxfin, lhs, rhs;
  int32_t mininf, maxinf;
  float thr_r, thr_l;
  int32_t exact;
  int32_t act;  // some nonzero of the row may yield an accepted candidate
};

// Step 2 of Sec. 1.1 for both sides of a row, and the screen thresholds.
__device__ __forceinline__ bool row_sides_eval(RowView &rv, float Tr, float Tl,
                                               double eps_feas) {
  bool infeas = false;
  bool act_r = false, act_l = false;
  rv.thr_r = f_inf();
  rv.thr_l = f_inf();
  if (d_isfinite(rv.rhs) && rv.mininf <= 1) {
    if (rv.mininf == 1) {
      act_r = true;  // only the nonzero with the infinite contribution
    } else {
      double s = rv.rhs - rv.minfin;
      if (__double2hiint(s) < 0) {  // s < 0 (or -0, harmless)
        double thr = rv.rhs + eps_feas * d_max1abs(rv.rhs);
        if (rv.minfin > thr) infeas = true;
      }
      float mg = __fmul_ru(0x1p-39f, __fadd_ru(f32_up_abs(rv.rhs), f32_up_abs(rv.minfin)));
      rv.thr_r = __fsub_rd(f32_dn(s), mg);
      act_r = Tr > rv.thr_r;
    }
  }
  if (d_isfinite(rv.lhs) && rv.maxinf <= 1) {
    if (rv.maxinf == 1) {
      act_l = true;
    } else {
      double s = rv.maxfin - rv.lhs;
      if (__double2hiint(s) < 0) {
        double thr = rv.lhs - eps_feas * d_max1abs(rv.lhs);
        if (rv.maxfin < thr) infeas = true;
      }
      float mg = __fmul_ru(0x1p-39f, __fadd_ru(f32_up_abs(rv.lhs), f32_up_abs(rv.maxfin)));
      rv.thr_l = __fsub_rd(f32_dn(s), mg);
      act_l = Tl > rv.thr_l;
    }
  }
  rv.act = (act_r || act_l) ? 1 : 0;
  return infeas;
}
__device__ __forceinline__ void row_sides(RowView &rv, float Tr, float Tl, double eps_feas,
                                          int32_t *infeasible_flag) {
  if (row_sides_eval(rv, Tr, Tl, eps_feas)) set_flag(infeasible_flag);
}

// One bound candidate of one nonzero from one side of its row (Eq. 3a/3b in
// the residual form of Eq. 5a/5b, with the exactly-one-infinity rule of
// Sec. 3.4), its integer rounding (Step 3), the infinity threshold and the
// acceptance test against the start-of-round bound (Sec. 3.5).  The
// right-hand side gives an upper candidate for a > 0 and a lower one for
// a < 0; the left-hand side the reverse.  The steps are written once, for
// upper candidates: a lower candidate c is processed as the upper candidate
// -c of -x (ceil(c - eps) = -floor(-c + eps), and c > L + t(L) iff
// -c < -L - t(-L), all exact under negation), so that a warp whose lanes mix
// sides and signs issues one division, not one per case.
struct SideCand {
  double v;    // the candidate (rounded for integers)
  bool upper;  // an upper bound candidate (else lower)
  bool apply;  // it passes the threshold and the acceptance test
};

__device__ __forceinline__ SideCand side_candidate(double a, double L, double U, bool isint,
                                                   bool use_rhs, const RowView &rv,
                                                   double eps_int, double tau_rel,
                                                   double inf_thr) {
  SideCand c;
  c.v = 0.0;
  c.apply = false;
  const bool pos = d_pos(a);
  c.upper = use_rhs == pos;
  const int32_t ninf = use_rhs ? rv.mininf : rv.maxinf;
  const double fin = use_rhs ? rv.minfin : rv.maxfin;
  const double bnd = c.upper ? L : U;  // this nonzero's term in that activity
  const double res = (ninf == 0) ? fma(-a, bnd, fin) : fin;
  if (!d_isfinite(res)) return c;
  const double q = ((use_rhs ? rv.rhs : rv.lhs) - res) / a;
  const double x = c.upper ? q : d_neg(q);
  const double B = c.upper ? U : d_neg(L);
  const double xr = isint ? d_floor_int(x + eps_int) : x;
  if (!d_abs_lt(xr, inf_thr)) return c;
  if (d_is_posinf(B)) c.apply = true;
  else if (isint) c.apply = cmp_key(xr) < cmp_key(B);
  else c.apply = cmp_key(xr) < cmp_key(B - tau_rel * d_max1abs(B));
  c.v = c.upper ? xr : d_neg(xr);
  return c;
}

// Which sides of one nonzero survive the screen (bit 0: right-hand side,
// bit 1: left-hand side).
__device__ __forceinline__ unsigned nnz_sides(double a, double L, double U, float WU,
                                              float WL, const RowView &rv) {
  bool pos = d_pos(a);
  double bmin = pos ? L : U;
  double bmax = pos ? U : L;
  float au = absup_fast(a), ad = absdn_fast(a);
  float tr = rv.exact ? f_inf() : screen_prod(au, ad, pos ? WU : WL);
  float tl = rv.exact ? f_inf() : screen_prod(au, ad, pos ? WL : WU);
  bool r = d_isfinite(rv.rhs) &&
           ((rv.mininf == 0 && tr > rv.thr_r) || (rv.mininf == 1 && d_isinf(bmin)));
  bool l = d_isfinite(rv.lhs) &&
           ((rv.maxinf == 0 && tl > rv.thr_l) || (rv.maxinf == 1 && d_isinf(bmax)));
  return (r ? 1u : 0u) | (l ? 2u : 0u);
}

}  // namespace dp
