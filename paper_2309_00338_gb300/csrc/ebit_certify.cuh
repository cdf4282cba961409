// Certified circle fit of the FP32 form on the FP32 pipe (Sec. 2.2).
//
// The FP32 form keeps a new unaligned marker as the float nearest to the
// crossing that the circle fit computes in double (the fit's solve stays in
// FP64 precision: its result is what counts).  GB300's FP64 pipe runs at
// 1/64 of its FP32 rate, and the fits are the busiest part of a sweep.  So a
// candidate's fit is first evaluated in double-float arithmetic (a value is
// an unevaluated sum of two floats, about 44 significant bits) on the FP32
// pipe, following the double evaluation operation by operation, and every
// intermediate carries a bound e on its distance from the value that the
// double evaluation produces at that point (the same operations, each
// rounded to double).  Where every decision the fit takes (separation of the
// points, sign of the discriminant, which root, the band of the edge) is
// certain under those bounds, and the whole interval around the crossing
// rounds to one float, that float is the double evaluation's result bit for
// bit.  Otherwise the candidate is left to the FP64 pass (the double
// evaluation itself).
//
// Bounds.  For double values a_d, b_d within e_a, e_b of the double-float
// values a, b, with A >= |a_d|, |a| and B >= |b_d|, |b|:
//   round_d(a_d + b_d) is within e_a + e_b + 2^-53 (A + B) of a + b, and the
//     double-float sum is within 2^-45 (A + B) of a + b;
//   round_d(a_d b_d) is within A e_b + B e_a + 2^-53 A B of a b, and the
//     double-float product within 2^-45 A B;
//   quotients and square roots likewise (below).
// K = 2^-42 covers the double rounding, the double-float rounding and the
// use of float magnitudes; bounds are computed in float and multiplied by
// kSafe = 1 + 2^-20, which covers the few roundings of each bound update.
// The bounds hold for finite values; anything non-finite is uncertain.
#pragma once
#include <cmath>
#include <cstdint>

#ifdef __CUDACC__
#define CERT_FN __host__ __device__ __forceinline__
#else
#define CERT_FN inline
#endif

namespace ebit {
namespace cert {

constexpr float kK = 2.2737367544323206e-13f;  // 2^-42
constexpr float kSafe = 1.00000095367431640625f;  // 1 + 2^-20

CERT_FN float fma_(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fmaf(a, b, c);
#endif
}
CERT_FN float fabs_(float a) { return a < 0.0f ? -a : a; }
CERT_FN bool finite_(float a) { return a - a == 0.0f; }

// A double-float value hi + lo with |lo| <= ulp(hi)/2 and the bound e.
struct Df {
  float hi, lo, e;
};

CERT_FN void two_sum(float a, float b, float* s, float* t) {
  const float x = a + b;
  const float bb = x - a;
  *s = x;
  *t = (a - (x - bb)) + (b - bb);
}
CERT_FN void fast_two_sum(float a, float b, float* s, float* t) {  // |a| >= |b| or a == 0
  const float x = a + b;
  *s = x;
  *t = b - (x - a);
}
CERT_FN float mag(const Df& a) { return fabs_(a.hi) + fabs_(a.lo) + a.e; }

// n + f exactly (n a small integer, f a float): the points of the FP32 form.
CERT_FN Df exact_nf(int n, float f) {
  Df r;
  two_sum((float)n, f, &r.hi, &r.lo);
  r.e = 0.0f;
  return r;
}
CERT_FN Df constant(float hi, float lo) { return Df{hi, lo, 0.0f}; }
CERT_FN Df neg(const Df& a) { return Df{-a.hi, -a.lo, a.e}; }
// times a power of two (exact in both arithmetics, away from under/overflow)
CERT_FN Df scale2(const Df& a, float p) { return Df{a.hi * p, a.lo * p, a.e * fabs_(p)}; }

CERT_FN Df add(const Df& a, const Df& b) {
  float s, t, hi, lo;
  two_sum(a.hi, b.hi, &s, &t);
  t = t + (a.lo + b.lo);
  fast_two_sum(s, t, &hi, &lo);
  const float A = mag(a), B = mag(b);
  return Df{hi, lo, ((a.e + b.e) + kK * (A + B)) * kSafe};
}
CERT_FN Df sub(const Df& a, const Df& b) { return add(a, neg(b)); }

CERT_FN Df mul(const Df& a, const Df& b) {
  const float p = a.hi * b.hi;
  float t = fma_(a.hi, b.hi, -p);
  t = t + (a.hi * b.lo + a.lo * b.hi);
  float hi, lo;
  fast_two_sum(p, t, &hi, &lo);
  const float A = mag(a), B = mag(b);
  return Df{hi, lo, ((A * b.e + B * a.e) + kK * (A * B)) * kSafe};
}

// a / b, b certainly nonzero (else ok = false): the double quotient of values
// within e_a, e_b of a, b lies within (e_a + |q| e_b) / (|b| - e_b) of a / b.
CERT_FN Df div(const Df& a, const Df& b, bool* ok) {
  const float bmin = (fabs_(b.hi) - fabs_(b.lo) - b.e) * (1.0f - 9.5367431640625e-07f);
  if (!(bmin > 0.0f)) {
    *ok = false;
    return Df{0.0f, 0.0f, 0.0f};
  }
  const float q0 = a.hi / b.hi;
  // remainder a - q0 b in double-float
  const float p = q0 * b.hi;
  const float pe = fma_(q0, b.hi, -p);
  float r = (a.hi - p);
  r = r + (a.lo - (pe + q0 * b.lo));
  const float q1 = r / b.hi;
  float hi, lo;
  fast_two_sum(q0, q1, &hi, &lo);
  const float Q = fabs_(hi) + fabs_(lo);
  const float e = ((a.e + Q * b.e) / bmin + kK * (Q + fabs_(a.hi) / bmin)) * kSafe;
  if (!finite_(hi) || !finite_(e)) *ok = false;
  return Df{hi, lo, e};
}

// sqrt(a), a certainly positive (else ok = false): the double square root of
// a value within e_a of a lies within e_a / sqrt(a - e_a) of sqrt(a).
CERT_FN Df sqrt_(const Df& a, bool* ok) {
  const float amin = (a.hi - fabs_(a.lo) - a.e) * (1.0f - 9.5367431640625e-07f);
  if (!(amin > 0.0f)) {
    *ok = false;
    return Df{0.0f, 0.0f, 0.0f};
  }
  const float s0 = sqrtf(a.hi);
  const float p = s0 * s0;
  const float pe = fma_(s0, s0, -p);
  const float r = ((a.hi - p) - pe) + a.lo;
  const float s1 = r / (2.0f * s0);
  float hi, lo;
  fast_two_sum(s0, s1, &hi, &lo);
  const float S = fabs_(hi) + fabs_(lo);
  const float e = (a.e / sqrtf(amin) + kK * S * 4.0f) * kSafe;
  return Df{hi, lo, e};
}

// Certain signs of the double value: +1 / -1, 0 when uncertain.
CERT_FN int sign(const Df& a) {
  const float slack = (a.e + fabs_(a.lo)) * kSafe;
  if (a.hi > slack) return 1;
  if (a.hi < -slack) return -1;
  return 0;
}

// The float nearest to the double value (round to nearest even), when the
// whole interval rounds to it: returns true and writes it.
CERT_FN bool round_to_float(const Df& a, float* out) {
  if (!finite_(a.hi) || !finite_(a.e)) return false;
  float f = a.hi + a.lo;  // the float nearest to hi + lo
  // distance of hi + lo from f, exactly: (hi - f) is exact (Sterbenz, or 0),
  // then add lo
  const float d = (a.hi - f) + a.lo;
  // the rounding cell of f: half the gaps to its neighbours
#ifdef __CUDA_ARCH__
  const float up = __int_as_float(__float_as_int(f) + 1) - f;
  const float dn = f - __int_as_float(__float_as_int(f) - 1);
#else
  const float up = std::nextafter(f, INFINITY) - f;
  const float dn = f - std::nextafter(f, -INFINITY);
#endif
  if (!(f > 0.0f)) return false;  // crossings are positive fractions here
  const float slack = (a.e + fabs_(d) * 9.5367431640625e-07f) * kSafe;
  if (d + slack < 0.5f * fabs_(up) && d - slack > -0.5f * fabs_(dn)) {
    *out = f;
    return true;
  }
  return false;
}

// One circle of a candidate (the double evaluation is circle_cross_r):
// points in cells relative to vertex (k, j), q = B - A, q2 = |q|^2,
// (rx, ry) = T - A, r2 = |T - A|^2.  Returns 1 with *y when the circle
// certainly gives a crossing, 0 when it certainly gives none, -1 when
// uncertain.  t_far: T is at least the minimum separation away from B (a
// certain decision made by the caller).
CERT_FN int circle(const Df& Ay, const Df& x0, const Df& qx, const Df& qy, const Df& q2,
                   const Df& rx, const Df& ry, const Df& r2, const Df& sep, Df* y) {
  bool ok = true;
  // d_below_sep(r2): r2 < kMinSep2
  const int s_r2 = sign(sub(r2, sep));
  if (s_r2 == 0) return -1;
  if (s_r2 < 0) return 0;
  const Df kap = sub(mul(qx, ry), mul(qy, rx));
  const Df al = sub(mul(r2, qy), mul(q2, ry));
  const Df be = sub(mul(q2, rx), mul(r2, qx));
  const Df c0 = mul(x0, add(mul(kap, x0), al));
  const Df disc = sub(mul(be, be), mul(scale2(kap, 4.0f), c0));
  const int s_disc = sign(disc);
  if (s_disc == 0) return -1;
  if (s_disc < 0) return 0;  // the circle misses the grid line
  const Df sq = sqrt_(disc, &ok);
  if (!ok) return -1;
  const int s_be = sign(be);
  if (s_be == 0) return -1;
  const Df h = scale2(add(be, s_be > 0 ? sq : neg(sq)), -0.5f);
  if (sign(h) == 0) return -1;  // h == 0 cannot be excluded
  const Df ya = div(c0, h, &ok);
  if (!ok) return -1;
  Df yrel = ya;
  const int s_kap = sign(kap);
  if (s_kap == 0) {
    // kap == 0 exactly takes the near root; a tiny kap of either sign could
    // take the far one: settle only the case where the near root is not on
    // T's side for either sign, i.e. sa == 0 ... leave it to FP64
    return -1;
  }
  const Df sa = sub(mul(qx, ya), mul(qy, x0));
  const int s_sa = sign(sa);
  if (s_sa == 0) return -1;
  if (s_sa == s_kap) {  // the near root lies on T's side: the far root, if not
    const Df yb = div(h, kap, &ok);
    if (!ok) return -1;
    const Df sb = sub(mul(qx, yb), mul(qy, x0));
    const int s_sb = sign(sb);
    if (s_sb == 0) return -1;
    if (s_sb != s_kap) yrel = yb;
  }
  const Df best = add(Ay, yrel);
  const int lo_in = sign(best);
  const int hi_in = sign(sub(constant(1.0f, 0.0f), best));
  if (lo_in == 0 || hi_in == 0) return -1;
  if (lo_in < 0 || hi_in < 0) return 0;  // outside the band
  *y = best;
  return 1;
}

}  // namespace cert
}  // namespace ebit
