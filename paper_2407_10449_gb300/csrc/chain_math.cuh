// chain_math.cuh -- per-row arithmetic shared by the chain-step kernels:
// the closed-form roots of App. B with the Sec. 3.2 edge cases, and the cheap
// approximate arcs used only to decide which arcs the sort can skip.
#pragma once

#include <cfloat>
#include <cmath>

#include "ess_common.cuh"

namespace ess {
namespace chainmath {

constexpr unsigned kFull = 0xffffffffu;

template <typename T> struct Lim;
template <> struct Lim<float> {
  __device__ static float inf() { return INFINITY; }
  __device__ static float two_pi() { return kTwoPiF; }
};
template <> struct Lim<double> {
  __device__ static double inf() { return INFINITY; }
  __device__ static double two_pi() { return kTwoPi; }
};

// ---- roots (App. B, Sec. 3.2) ------------------------------------------
__device__ __forceinline__ bool roots_dp(double p, double q, double b, double& al, double& be,
                                         bool& infeasible) {
  double r = sqrt(p * p + q * q);
  if (r == 0.0) {
    infeasible = b < 0.0;
    return false;
  }
  double ratio = b / r;
  if (ratio >= 1.0) return false;
  if (ratio < -1.0) ratio = -1.0;
  double tau = atan2(q, p);
  if (tau < 0.0) tau += kTwoPi;
  double h = acos(ratio);
  al = fmax(0.0, tau - h);
  be = fmin(kTwoPi, tau + h);
  return true;
}

__device__ __forceinline__ bool roots(double p, double q, double b, double b64, double,
                                      double& al, double& be, bool& infeasible, int& tangent) {
  (void)b;
  (void)tangent;
  return roots_dp(p, q, b64, al, be, infeasible);
}

__device__ __forceinline__ bool roots(float p, float q, float b, double b64, double thresh,
                                      float& al, float& be, bool& infeasible, int& tangent) {
  float r2 = fmaf(p, p, q * q);
  if (r2 == 0.0f) {
    infeasible = b64 < 0.0;
    return false;
  }
  float ratio = b / sqrtf(r2);
  if (ratio >= (float)(1.0 + thresh)) return false;  // clearly no root
  if (fabsf(ratio) > (float)(1.0 - thresh)) {
    // near tangency: the arccos argument and the angles in double
    ++tangent;
    double ad, bd;
    bool has = roots_dp((double)p, (double)q, b64, ad, bd, infeasible);
    if (has) {
      al = (float)ad;
      be = fminf((float)bd, kTwoPiF);
    }
    return has;
  }
  float tau = atan2f(q, p);
  if (tau < 0.0f) tau += kTwoPiF;
  float h = acosf(ratio);
  al = fmaxf(0.0f, tau - h);
  be = fminf(kTwoPiF, tau + h);
  return true;
}

// ---- approximate arcs for the domination prune -------------------------------
// Cheap polynomial forms of atan and arccos (coefficients fitted for this
// kernel by least squares on Chebyshev nodes).  In FP32 they stay within
// 1.3e-5 rad (atan2) and 4.4e-5 rad (arccos) of the exact functions on their
// whole domain (checked on 2e7 random and 4e6 grid points); the prune below
// only trusts them up to kPruneMargin = 1e-3 rad.  They decide nothing but
// which arcs may be dropped: every kept arc gets exact roots.
constexpr float kPruneMargin = 1e-3f;

__device__ __forceinline__ float atan01_poly(float z) {  // atan(z), z in [0, 1]
  const float z2 = z * z;
  return z * fmaf(z2, fmaf(z2, fmaf(z2, fmaf(z2, 0.020931812f, -0.085408308f), 0.18041268f),
                           -0.33040557f),
                  0.99987874f);
}

__device__ __forceinline__ float atan2_poly(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
  float a = mx > 0.f ? atan01_poly(__fdividef(mn, mx)) : 0.f;
  if (ay > ax) a = 1.5707964f - a;
  if (x < 0.f) a = 3.1415927f - a;
  return y < 0.f ? -a : a;
}

__device__ __forceinline__ float acos_poly(float x) {  // x in [-1, 1]
  const float ax = fabsf(x);
  const float v = sqrtf(fmaxf(0.f, 1.f - ax)) *
                  fmaf(ax, fmaf(ax, fmaf(ax, -0.020585312f, 0.076513453f), -0.21275975f), 1.5707535f);
  return x < 0.f ? 3.1415927f - v : v;
}

// A double rounded to float by integer operations on its two halves, so that
// the FP64 chains' classification (three conversions per row) leaves the
// narrow FP64 pipe to the FP64 work proper.  Values in float's normal range
// are rounded to nearest (ties away from zero: error at most half an ulp,
// 2^-24 relative); values below it become zero, finite values above it
// become infinity, and NaN stays NaN.  The classification keeps rows whose
// float p, q or b is zero or non-finite where that decides the class (r = 0 or
// a non-finite r^2).
__device__ __forceinline__ float dbl_to_flt_bits(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u;
  const unsigned dexp = (hi >> 20) & 0x7FFu;
  const int e = (int)dexp - 896;  // float exponent field for normal values
  const unsigned mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  unsigned bits = (sign | ((unsigned)e << 23) | mant) + ((lo >> 28) & 1u);
  bits = e <= 0 ? sign : bits;
  bits = e >= 255 ? (sign | 0x7F800000u) : bits;
  bits = dexp == 0x7FFu && ((hi & 0xFFFFFu) | lo) != 0u ? 0x7FC00000u : bits;
  return __uint_as_float(bits);
}

// Row classification of the prune: the has-root decision is exactly the one
// roots() takes; rows near tangency (where arccos is ill-conditioned) or with
// tau close to the 0 / 2 pi cut are never dropped.
enum : int { kRowNone = 0, kRowApprox = 1, kRowKeep = 2 };

template <typename T>
__device__ __forceinline__ int classify_row(T p, T q, T b, double b64, T tlo, T thi, float& a_ap,
                                            float& b_ap, bool& infeasible) {
  float pf, qf, ratio;
  if constexpr (sizeof(T) == 4) {
    pf = p;
    qf = q;
    const float r2 = fmaf(p, p, q * q);
    if (r2 == 0.0f) {
      infeasible = b64 < 0.0;
      return kRowNone;
    }
    // b / r from the reciprocal square root (relative error < 1e-6): only
    // decisions that hold with that slack are taken here; rows inside the
    // slack are kept and get the exact test in roots()
    ratio = b * rsqrtf(r2);
    if (ratio >= thi * 1.000001f) return kRowNone;
    if (fabsf(ratio) > tlo * 0.999999f) return kRowKeep;
  } else {
    // FP64 chains: the same float decisions on p, q, b rounded by integer
    // operations (no FP64 instruction; the rounding adds at most 2^-23 to the
    // error of b / r, well inside the 1e-6 slack).  Rows whose r^2 leaves
    // [1e-30, 1e30] in float -- including r = 0, decided by the exact roots --
    // are kept.
    pf = dbl_to_flt_bits(p);
    qf = dbl_to_flt_bits(q);
    const float r2 = fmaf(pf, pf, qf * qf);
    if (!(r2 >= 1e-30f && r2 <= 1e30f)) return kRowKeep;
    ratio = dbl_to_flt_bits(b) * rsqrtf(r2);
    if (ratio >= (float)thi * 1.000001f) return kRowNone;
    if (fabsf(ratio) > (float)tlo * 0.999999f) return kRowKeep;
  }
  float tau = atan2_poly(qf, pf);
  if (tau < 0.f) tau += kTwoPiF;
  // (written so that a NaN angle keeps the row)
  if (!(tau >= 0.02f && tau <= kTwoPiF - 0.02f)) return kRowKeep;
  const float h = acos_poly(ratio);
  a_ap = fmaxf(0.f, tau - h);
  b_ap = fminf(kTwoPiF, tau + h);
  return kRowApprox;
}


// Pseudo-angle of a nonzero vector (x, y): a non-decreasing function of its
// polar angle in [0, 2 pi), with values in [0, 4], computed without
// trigonometry.  With xn = x / (|x| + |y|) (in [-1, 1], decreasing in the
// angle on [0, pi] and increasing on [pi, 2 pi]):
//   y >= 0:  1 - xn   (0 at angle 0, 1 at pi / 2, 2 at pi)
//   y <  0:  3 + xn   (2 at pi, 3 at 3 pi / 2, 4 at 2 pi)
// i.e. 2 - copysign(1 + xn, y).  Comparisons of pseudo-angles are
// comparisons of angles; its slope lies between 1/2 and 1 per radian.
// inv is 1 / (|x| + |y|).
__device__ __forceinline__ float pseudo_angle(float x, float y, float inv) {
  return 2.f - copysignf(fmaf(x, inv, 1.f), y);
}

// Pseudo-angles of the two roots: with w = sqrt(r^2 - b^2), the points of the
// ellipse on the hyperplane sit at the angles of
//   u_alpha = (p b + q w, q b - p w)   (= r^2 (cos(tau - h), sin(tau - h)))
//   u_beta  = (p b - q w, q b + p w)   (= r^2 (cos(tau + h), sin(tau + h)))
// (App. B: cos tau = p / r, sin tau = q / r, cos h = b / r, sin h = w / r).
__device__ __forceinline__ void root_pseudo_angles(float p, float q, float b, float w, float& pa,
                                                   float& pb) {
  const float pbv = p * b, qbv = q * b;
  const float ax = fmaf(q, w, pbv), ay = fmaf(-p, w, qbv);
  const float bx = fmaf(-q, w, pbv), by = fmaf(p, w, qbv);
  pa = pseudo_angle(ax, ay, __fdividef(1.f, fabsf(ax) + fabsf(ay)));
  pb = pseudo_angle(bx, by, __fdividef(1.f, fabsf(bx) + fabsf(by)));
}

// Row classes of the prune for FP64 chains, taken in FP32 (GB300's FP64 pipe
// is narrow): the float classification of the rounded p, q, b keeps every row
// whose no-root or near-tangent decision lies within its slack, and the rows
// it cannot classify (r = 0 or non-finite in float: underflow or overflow of
// the rounding) are kept too; every kept row gets the exact FP64 roots.
// Non-finite doubles are detected from their exponent bits.
__device__ __forceinline__ int classify_phi_d(double p, double q, double b, float tlo2,
                                              float thi2, float& pa, float& pb,
                                              bool& nonfinite);

// Row classes of the prune (float chains), branch-free so that the rows of a
// batch interleave.  The no-root and near-tangent decisions compare b^2 with
// r^2 times the squared thresholds, which carry a 1e-6 relative slack beyond
// the ones roots() applies to b / r: only decisions that hold with that slack
// are taken here, rows inside it are kept and get the exact test in roots().
//   tlo2 = ((1 - thresh) (1 - 1e-6))^2,  thi2 = ((1 + thresh) (1 + 1e-6))^2.
// pa and pb are meaningful only for kRowApprox.  A row with r = 0 has no
// root; it sets *zero, and the caller decides infeasibility from the exact b_i
// (b_i < 0) outside the hot loop.
__device__ __forceinline__ int classify_phi_nb(float p, float q, float b, float tlo2, float thi2,
                                               float& pa, float& pb, bool& zero,
                                               bool& nonfinite) {
  const float r2 = fmaf(p, p, q * q);
  nonfinite |= !(r2 <= FLT_MAX);  // NaN or Inf in p or q
  const float b2 = b * b;
  const float w2 = fmaf(-b, b, r2);
  root_pseudo_angles(p, q, b, w2 * rsqrtf(fmaxf(w2, FLT_MIN)), pa, pb);
  int cls = pa < pb ? kRowApprox : kRowKeep;
  cls = w2 > 0.f ? cls : kRowKeep;
  cls = b2 > tlo2 * r2 ? kRowKeep : cls;                 // |b / r| > 1 - thresh (with slack)
  cls = b >= 0.f && b2 >= thi2 * r2 ? kRowNone : cls;    // b / r >= 1 + thresh (with slack)
  zero = r2 == 0.0f;
  return zero ? kRowNone : cls;
}

// The row classes of classify_phi_nb with fewer operations, for the streamed
// warp kernel:
//   no root   : b >= 0 and b^2 >= thi2 r^2 (this also takes r = 0 with b >= 0);
//   keep      : otherwise, if b^2 > tlo2 r^2 (near tangency; it includes
//               w^2 <= 0 and r = 0 with b < 0, which the exact roots then
//               report as infeasible) or the pseudo-angles do not increase
//               (an arc through the 0 / 2 pi cut, or NaN);
//   arc       : otherwise, placed by its pseudo-angles pa < pb.
// nf accumulates r^2 * 0: it turns NaN once p or q is non-finite (or r^2
// overflows), so one test after the rows finds non-finite input.
__device__ __forceinline__ int classify_lean(float p, float q, float b, float tlo2, float thi2,
                                             float& pa, float& pb, float& nf) {
  const float r2 = fmaf(p, p, q * q);
  nf = fmaf(r2, 0.f, nf);
  const float w2 = fmaf(-b, b, r2);
  root_pseudo_angles(p, q, b, w2 * rsqrtf(fmaxf(w2, FLT_MIN)), pa, pb);
  const float b2 = b * b;
  const bool none = b >= 0.f && b2 >= thi2 * r2;
  const bool keep = b2 > tlo2 * r2 || !(pa < pb);
  return none ? kRowNone : keep ? kRowKeep : kRowApprox;
}

__device__ __forceinline__ int classify_phi_d(double p, double q, double b, float tlo2,
                                              float thi2, float& pa, float& pb,
                                              bool& nonfinite) {
  nonfinite |= (__double2hiint(p) & 0x7FF00000) == 0x7FF00000 ||
               (__double2hiint(q) & 0x7FF00000) == 0x7FF00000;
  bool zero = false, nf = false;
  const int cls = classify_phi_nb(dbl_to_flt_bits(p), dbl_to_flt_bits(q), dbl_to_flt_bits(b),
                                  tlo2, thi2, pa, pb, zero, nf);
  return zero || nf ? kRowKeep : cls;
}

}  // namespace chainmath
}  // namespace ess
