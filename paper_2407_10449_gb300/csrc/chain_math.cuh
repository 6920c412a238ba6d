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

// Row classification of the prune: the has-root decision is exactly the one
// roots() takes; rows near tangency (where arccos is ill-conditioned) or with
// tau close to the 0 / 2 pi cut are never dropped.
enum : int { kRowNone = 0, kRowApprox = 1, kRowKeep = 2 };

template <typename T>
__device__ __forceinline__ int classify_row(T p, T q, T b, double b64, T tlo, T thi, float& a_ap,
                                            float& b_ap, bool& infeasible) {
  T ratio;
  if constexpr (sizeof(T) == 4) {
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
    const double r = sqrt(p * p + q * q);
    if (r == 0.0) {
      infeasible = b64 < 0.0;
      return kRowNone;
    }
    ratio = b64 / r;
    if (ratio >= 1.0) return kRowNone;
    if (fabs(ratio) > tlo || r < 1e-30) return kRowKeep;
  }
  float tau = atan2_poly((float)q, (float)p);
  if (tau < 0.f) tau += kTwoPiF;
  if (tau < 0.02f || tau > kTwoPiF - 0.02f) return kRowKeep;
  const float h = acos_poly((float)ratio);
  a_ap = fmaxf(0.f, tau - h);
  b_ap = fminf(kTwoPiF, tau + h);
  return kRowApprox;
}


// Pseudo-angle of a nonzero vector (x, y): a strictly increasing function of
// its polar angle in [0, 2 pi), with values in [0, 4) ("diamond angle", one
// unit per quadrant).  Comparisons of pseudo-angles are comparisons of angles.
// With yn = y / (|x| + |y|): quadrant I gives yn, II and III give 2 - yn,
// IV gives 4 + yn (continuous across the quadrant boundaries).
__device__ __forceinline__ float diamond_angle(float x, float y) {
  const float yn = __fdividef(y, fabsf(x) + fabsf(y));
  return x >= 0.f ? (y >= 0.f ? yn : 4.f + yn) : 2.f - yn;
}

// Pseudo-angles of the two roots: with w = sqrt(r^2 - b^2), the points of the
// ellipse on the hyperplane sit at the angles of
//   u_alpha = (p b + q w, q b - p w)   (= r^2 (cos(tau - h), sin(tau - h)))
//   u_beta  = (p b - q w, q b + p w)   (= r^2 (cos(tau + h), sin(tau + h)))
// (App. B: cos tau = p / r, sin tau = q / r, cos h = b / r, sin h = w / r).
// The row classes match roots(): the no-root and near-tangent decisions are
// taken only outside a 1e-6 relative slack of the b/r computed here, and rows
// whose arc would wrap through 0 (boundary points) are always kept.  b64
// points at the exact b_i (read only when r = 0); nonfinite is set when p or
// q is NaN or infinite (r^2 is then not finite).
template <typename T>
__device__ __forceinline__ int classify_phi(T p, T q, T b, const double* b64, T tlo, T thi,
                                            float& pa, float& pb, bool& infeasible,
                                            bool& nonfinite) {
  const float pf = (float)p, qf = (float)q, bf = (float)b;
  if constexpr (sizeof(T) == 4) {
    const float r2 = fmaf(p, p, q * q);
    nonfinite |= !(r2 <= FLT_MAX);  // NaN or Inf in p or q
    if (r2 == 0.0f) {
      infeasible = *b64 < 0.0;
      return kRowNone;
    }
    const float ratio = b * rsqrtf(r2);
    if (ratio >= thi * 1.000001f) return kRowNone;
    if (fabsf(ratio) > tlo * 0.999999f) return kRowKeep;
  } else {
    const double r2 = p * p + q * q;
    nonfinite |= !(r2 <= DBL_MAX);
    const double r = sqrt(r2);
    if (r == 0.0) {
      infeasible = b < 0.0;
      return kRowNone;
    }
    const double rd = b / r;
    if (rd >= 1.0) return kRowNone;
    if (fabs(rd) > tlo || r < 1e-30 || r > 1e30) return kRowKeep;
  }
  const float r2f = fmaf(pf, pf, qf * qf);
  const float w2 = fmaf(-bf, bf, r2f);
  if (!(w2 > 0.f)) return kRowKeep;
  const float w = w2 * rsqrtf(w2);
  pa = diamond_angle(fmaf(pf, bf, qf * w), fmaf(qf, bf, -pf * w));
  pb = diamond_angle(fmaf(pf, bf, -qf * w), fmaf(qf, bf, pf * w));
  return pa < pb ? kRowApprox : kRowKeep;
}

// Branch-free float form of classify_phi (same classes and pseudo-angles):
// every quantity is computed and the class picked by selects, so the rows of a
// batch are straight-line code that the compiler can interleave.  pa and pb
// are meaningful only for kRowApprox.
__device__ __forceinline__ int classify_phi_nb(float p, float q, float b, const double* b64,
                                               float tlo, float thi, float& pa, float& pb,
                                               bool& infeasible, bool& nonfinite) {
  const float r2 = fmaf(p, p, q * q);
  nonfinite |= !(r2 <= FLT_MAX);  // NaN or Inf in p or q
  const float ratio = b * rsqrtf(r2);
  const float w2 = fmaf(-b, b, r2);
  const float w = w2 * rsqrtf(fmaxf(w2, FLT_MIN));
  pa = diamond_angle(fmaf(p, b, q * w), fmaf(q, b, -p * w));
  pb = diamond_angle(fmaf(p, b, -q * w), fmaf(q, b, p * w));
  int cls = pa < pb ? kRowApprox : kRowKeep;
  cls = w2 > 0.f ? cls : kRowKeep;
  cls = fabsf(ratio) > tlo * 0.999999f ? kRowKeep : cls;
  cls = ratio >= thi * 1.000001f ? kRowNone : cls;
  if (r2 == 0.0f) {  // rare: read the exact b only here
    infeasible = *b64 < 0.0;
    cls = kRowNone;
  }
  return cls;
}

}  // namespace chainmath
}  // namespace ess
