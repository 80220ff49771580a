// ac_df64.cuh -- binary64 values handled on the FP32 and integer pipes.
//
// GB300 executes FP64 arithmetic, and every conversion to or from binary64,
// at about 1/64 of its FP32 rate.  The mixed form's defect correction
// therefore reads the stored binary64 phase field and right-hand side
// through integer operations on their bit patterns (IEEE 754-2008, 3.4:
// sign, 11-bit biased exponent, 52-bit trailing significand) and computes
// in double-float arithmetic: a value is the unevaluated sum h + l of two
// floats, combined by error-free transformations -- Knuth's two-sum (TAOCP
// vol. 2, 4.2.2, Theorem B), Dekker's fast two-sum (Numer. Math. 18, 1971)
// for |a| >= |b|, and the exact product a b = p + e with e = fma(a, b, -p).
//
// Everything here is host- and device-callable so that the host build can
// check it against exact rational arithmetic.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define AC_HD __host__ __device__ __forceinline__
#else
#define AC_HD inline
#endif

namespace ac {

AC_HD uint32_t f32_bits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
#endif
}

AC_HD float bits_f32(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, 4);
  return f;
#endif
}

// The two 32-bit words of a binary64 value (register moves on the device).
AC_HD void f64_words(double d, uint32_t &hi, uint32_t &lo) {
#ifdef __CUDA_ARCH__
  hi = (uint32_t)__double2hiint(d);
  lo = (uint32_t)__double2loint(d);
#else
  uint64_t u;
  std::memcpy(&u, &d, 8);
  hi = (uint32_t)(u >> 32);
  lo = (uint32_t)u;
#endif
}

AC_HD double words_f64(uint32_t hi, uint32_t lo) {
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  const uint64_t u = ((uint64_t)hi << 32) | lo;
  double d;
  std::memcpy(&d, &u, 8);
  return d;
#endif
}

AC_HD float fma_f32(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fmaf(a, b, c);
#endif
}

AC_HD bool f64_isnan(double d) {
  uint32_t hi, lo;
  f64_words(d, hi, lo);
  const uint32_t ah = hi & 0x7FFFFFFFu;
  return ah > 0x7FF00000u || (ah == 0x7FF00000u && lo != 0u);
}

// Binary64 -> binary32 rounded to nearest, ties to even, for magnitudes in
// the binary32 normal range; below it the result is a signed zero (no
// subnormals), above it an infinity, and NaN stays NaN.  The binary64
// exponent e (bias 1023) maps to e - 896 (bias 127); the 52-bit significand
// keeps its top 23 bits, the 29 dropped bits decide the rounding.
AC_HD float f64_to_f32_rn(double d) {
  uint32_t hi, lo;
  f64_words(d, hi, lo);
  const uint32_t sign = hi & 0x80000000u, ah = hi & 0x7FFFFFFFu;
  uint32_t t = ((ah - 0x38000000u) << 3) | (lo >> 29);
  const uint32_t round_bit = (lo >> 28) & 1u, sticky = (lo & 0x0FFFFFFFu) != 0u ? 1u : 0u;
  t += round_bit & (sticky | (t & 1u));  // a carry out of the significand bumps the exponent
  t = ah < 0x38100000u ? 0u : t;          // |d| < 2^-126
  t = ah >= 0x47F00000u ? 0x7F800000u : t;  // |d| >= 2^128 (and infinities)
  t = (ah > 0x7FF00000u || (ah == 0x7FF00000u && lo != 0u)) ? 0x7FC00000u : t;
  return bits_f32(sign | t);
}

// Binary32 -> binary64, exact for normal values; subnormal inputs give a
// signed zero, infinities and NaN carry over.
AC_HD double f32_to_f64(float f) {
  const uint32_t b = f32_bits(f);
  const uint32_t sign = b & 0x80000000u, ab = b & 0x7FFFFFFFu;
  uint32_t hi = ((ab >> 3) + 0x38000000u), lo = ab << 29;
  if (ab < 0x00800000u) {
    hi = 0u;
    lo = 0u;
  }
  if (ab >= 0x7F800000u) {
    hi = 0x7FF00000u | ((ab & 0x007FFFFFu) ? 0x00080000u : 0u);
    lo = 0u;
  }
  return words_f64(sign | hi, lo);
}

// d = h + l with h the binary64 significand truncated to 24 bits and l the
// remaining 29 bits rounded to a float (same sign as h):
// |d - (h + l)| <= 2^-47 |d|.  For |d| < 2^-97 the tail is dropped (l = 0)
// and for |d| < 2^-126 also the head; NaN and infinities give (d, 0).
// The tail's 29 bits m = a 2^6 + c are turned into floats by the
// exponent-bias device: the float with exponent field E and significand
// field a is 2^(E-127) + a 2^(E-150), so subtracting 2^(E-127) leaves
// a 2^(E-150) exactly.
AC_HD void split_f64(double d, float &h, float &l) {
  uint32_t hi, lo;
  f64_words(d, hi, lo);
  const uint32_t sign = hi & 0x80000000u, ah = hi & 0x7FFFFFFFu;
  uint32_t t = ((ah - 0x38000000u) << 3) | (lo >> 29);  // |h|, exponent field e - 896
  const uint32_t eh = t & 0x7F800000u;
  const uint32_t ba = eh - (23u << 23), bc = eh - (29u << 23);  // weights 2^6 and 2^0 of the tail's ulp
  const uint32_t m = lo & 0x1FFFFFFFu;
  const float ta = bits_f32(ba | (m >> 6)) - bits_f32(ba);
  const float tc = bits_f32(bc | (m & 63u)) - bits_f32(bc);
  uint32_t tl = f32_bits(ta + tc);
  const bool normal = ah >= 0x38100000u && ah < 0x47F00000u;
  tl = (normal && ah >= 0x39E00000u) ? tl : 0u;  // tail kept for |d| >= 2^-97
  if (!normal) {
    t = ah < 0x38100000u ? 0u : 0x7F800000u;
    if (ah > 0x7FF00000u || (ah == 0x7FF00000u && lo != 0u)) t = 0x7FC00000u;
  }
  h = bits_f32(sign | t);
  l = bits_f32(sign | tl);
}

// The binary64 significand of d truncated to 24 bits, as a float (the head
// of split_f64, integer pipe): |d - head| <= 2^-23 |d|; 0 (signed) for
// |d| < 2^-126; NaN for |d| >= 2^128, infinities and NaN.  The pixel-label
// filter sums these heads of phase values in [0, 1] in float.
AC_HD float f64_head(double d) {
  uint32_t hi, lo;
  f64_words(d, hi, lo);
  const uint32_t sign = hi & 0x80000000u, ah = hi & 0x7FFFFFFFu;
  uint32_t t = ah < 0x38100000u ? 0u : (((ah - 0x38000000u) << 3) | (lo >> 29));
  t = ah >= 0x47F00000u ? 0x7FC00000u : t;
  return bits_f32(sign | t);
}

// Double-float value h + l.
struct f2 {
  float h, l;
};

// a + b = s + e exactly (Knuth).
AC_HD f2 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

// a + b = s + e exactly when |a| >= |b| or a = 0 (Dekker).
AC_HD f2 fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

// (ah + al)(bh + bl) to double-float accuracy, the al bl term dropped; the
// result is not renormalised.
AC_HD f2 mul_f2(float ah, float al, float bh, float bl) {
  const float p = ah * bh;
  const float e = fma_f32(ah, bh, -p);
  return {p, e + (ah * bl + al * bh)};
}

// (a.h + a.l) + (bh + bl): one two-sum on the heads, the tails added in
// float, renormalised (Dekker's add); the error is about 2^-46 (|a| + |b|).
AC_HD f2 add_f2(f2 a, float bh, float bl) {
  const f2 s = two_sum(a.h, bh);
  return fast_two_sum(s.h, s.l + (a.l + bl));
}

AC_HD int popcount_hd(unsigned m) {
#ifdef __CUDA_ARCH__
  return __popc(m);
#else
  return __builtin_popcount(m);
#endif
}

// 1/k for the kept-component counts 1..8 (exact for 1, 2, 4, 8; rounded
// otherwise), without a division.
template <typename T>
AC_HD T rcp_count(int k) {
  return k == 1 ? T(1) : k == 2 ? T(0.5) : k == 3 ? T(1.0 / 3.0) : k == 4 ? T(0.25)
       : k == 5 ? T(0.2) : k == 6 ? T(1.0 / 6.0) : k == 7 ? T(1.0 / 7.0) : T(0.125);
}

// The mixed form's update of one node of the binary64 phase field,
// u <- P_G(u + delta) (Sec. 3.3's simplex projection, the FP32 correction
// delta added in binary64):
//  - the float solve's obstacle is u's truncated head (f64_head: the
//    significand cut to 24 bits, so 0 <= head <= u and u + delta >= 0 on the
//    float solve's feasible set); a component it put on its bound
//    (delta_i == -head(u_i)) is set to exactly 0 -- u_i + delta_i would leave
//    the residue u_i - head(u_i) -- so that exact zeros (the active set) are
//    the same as in the FP64 form; the others are v_i = u_i + delta_i in
//    binary64;
//  - Michelot's iteration on the kept components (target sum 1):
//    theta = (sum of the kept v - 1)/|kept|, components at or below theta
//    leave, repeat; then u_i = v_i - theta on the kept set, 0 elsewhere.
// Binary64 arithmetic is slow on GB300, so the kept set is found by the
// iteration on the heads of v, theta computed once in binary64 on that set,
// and the set's conditions (kept v_i > theta, the others at or below it)
// checked on the heads with a margin of 2^-21 (|v_i| + |theta|) + 2^-120.
// Truncation is monotone and within 2^-23 of its argument, so a float gap
// that large (the absolute term covers the flush below 2^-126) proves the
// binary64 inequality with a gap far above the binary64 rounding of the
// iteration's intermediate thetas.  Where the conditions hold, the binary64
// iteration from the full set ends on the same set -- its theta does not
// exceed the final one, so it drops no component above it, and it cannot
// stop on a larger set -- and sums it in the same order, so the result is
// bit-identical to that iteration's.  Elsewhere (near ties), and always
// with FP64_ONLY, the binary64 iteration runs.
// any_or(m) returns the OR of m over the lanes that run together (the
// identity on the host): a binary64 operation on component i is skipped
// when no lane needs it.  Returns 0 (float set accepted), 1 (binary64
// iteration) or 2 (no kept component, which a feasible correction cannot
// give: u is then zero and the caller projects it).
template <int N, bool FP64_ONLY = false, typename AnyOr>
AC_HD int outer_update_node(double (&uk)[N], const float (&dk)[N], AnyOr any_or) {
  unsigned keep0 = 0;
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (!(dk[i] == -f64_head(uk[i]))) keep0 |= 1u << i;
  const unsigned any0 = any_or(keep0);
  const int cnt = popcount_hd(keep0);
  float vf[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    vf[i] = 0.f;
    if (((any0 >> i) & 1u) && ((keep0 >> i) & 1u)) {
      uk[i] += f32_to_f64(dk[i]);
      vf[i] = f64_head(uk[i]);
    } else {
      uk[i] = 0.0;
    }
  }
  if (cnt == 0) return 2;
  unsigned keep = keep0;
  double theta = 0.0;
  bool ok = !FP64_ONLY;
  if (!FP64_ONLY) {
    float sf = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i)
      if ((keep >> i) & 1u) sf += vf[i];
    float tf = (sf - 1.f) * rcp_count<float>(cnt);
#pragma unroll 1
    for (int pass = 1; pass < N; ++pass) {
      unsigned drop = 0;
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (((keep >> i) & 1u) && vf[i] <= tf) drop |= 1u << i;
      if (!drop || drop == keep) break;
      keep &= ~drop;
      sf = 0.f;
#pragma unroll
      for (int i = 0; i < N; ++i)
        if ((keep >> i) & 1u) sf += vf[i];
      tf = (sf - 1.f) * rcp_count<float>(popcount_hd(keep));
    }
    const unsigned anyk = any_or(keep);
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (((anyk >> i) & 1u) && ((keep >> i) & 1u)) s += uk[i];
    theta = (s - 1.0) * rcp_count<double>(popcount_hd(keep));
    const float t32 = f64_head(theta);
#pragma unroll
    for (int i = 0; i < N; ++i)
      if ((keep0 >> i) & 1u) {
        const float d = vf[i] - t32, m = (fabsf(vf[i]) + fabsf(t32)) * 0x1.0p-21f + 0x1.0p-120f;
        ok = ok && (((keep >> i) & 1u) ? d > m : d < -m);
      }
  }
  if (!ok) {
    keep = keep0;
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (((any0 >> i) & 1u) && ((keep >> i) & 1u)) s += uk[i];
    theta = (s - 1.0) * rcp_count<double>(cnt);
#pragma unroll 1
    for (int pass = 1; pass < N; ++pass) {
      unsigned drop = 0;
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (((any0 >> i) & 1u) && ((keep >> i) & 1u) && uk[i] <= theta) drop |= 1u << i;
      if (!drop || drop == keep) break;
      keep &= ~drop;
      s = 0.0;
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (((any0 >> i) & 1u) && ((keep >> i) & 1u)) s += uk[i];
      theta = (s - 1.0) * rcp_count<double>(popcount_hd(keep));
    }
  }
  const unsigned anyf = any_or(keep);
#pragma unroll
  for (int i = 0; i < N; ++i)
    uk[i] = (((anyf >> i) & 1u) && ((keep >> i) & 1u)) ? uk[i] - theta : 0.0;
  return ok ? 0 : 1;
}

}  // namespace ac
