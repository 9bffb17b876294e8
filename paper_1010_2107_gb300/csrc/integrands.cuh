// integrands.cuh -- step 3 (Sec. 2.1) on the device: the integrand registry.
//
// Each integrand reads its constants from shared memory (`P`, already in the
// kernel precision T) as prepared on the host by derive_params() in abi.cu,
// and takes the mapped point x[0..d) in registers.  DM is the compile-time
// bound on d (loops are unrolled to DM with a guard on the runtime d).
#pragma once

#include "common.cuh"

namespace gv {

// exp of a non-positive Gaussian exponent: the special-function unit for
// FP32 (relative error ~2^-21 over the range that matters), libm for FP64.
__device__ __forceinline__ float gexp(float x) { return __expf(x); }
__device__ __forceinline__ double gexp(double x) { return exp(x); }

// t^e for t > 0: FP32 as exp(e ln t) on the quick forms, FP64 the library.
__device__ __forceinline__ float qpow_pos(float t, float e) { return __expf(e * __logf(t)); }
__device__ __forceinline__ double qpow_pos(double t, double e) { return pow(t, e); }

// cos of a moderate argument: FP32 reduces to [-pi, pi] by r = t - k 2pi
// with 2pi split in two floats (Cody and Waite): the fused multiply-add
// subtracts k 2pi_hi with one rounding and k (2pi - 2pi_hi) corrects it,
// before the quick form; FP64 the library.
__device__ __forceinline__ float qcos_any(float t) {
  const float k = rintf(t * 0.159154943091895336f);  // t / (2 pi)
  // 2pi_hi = 6.28318548f exceeds 2pi by 1.7484555e-7
  const float r = fmaf(k, 1.7484555e-7f, fmaf(-k, 6.28318548f, t));
  return __cosf(r);
}
__device__ __forceinline__ double qcos_any(double t) { return cos(t); }

// Derived-constant slots.  Genz / Gaussian: a-like values at [0, d),
// u-like values at [kMaxDim, kMaxDim + d), raw a_i at [2 kMaxDim, ...),
// scalars from kScalar on.
constexpr int kScalar = 3 * kMaxDim;

// Integrands with an analytic parameter gradient define
//   static T grad(x, d, P, g)  ->  f(x), with g[t] = df/dtheta_t
// in the units of the integrand's own (dimensionless) value; NT is the
// largest number of parameters for a compile-time bound DM.

// ----------------------------------------------------------------- Genz
// f = exp(-sum a_i^2 (x_i - u_i)^2).  P[i] = a_i^2, P[kMaxDim+i] = u_i.
// FP32 pairs of consecutive axes for the paired FP32 instructions: x[a],
// x[a+1] (the second replaced by `pad` past d) and the constants P[o + a],
// P[o + a + 1] (8-byte aligned: o and a even).
template <int DM>
__device__ __forceinline__ float2 xpair(const float (&x)[DM], int a, int d, float pad) {
  return make_float2(x[a], a + 1 < d ? x[a + 1] : pad);
}
__device__ __forceinline__ float2 ppair(const float* P, int i) { return *reinterpret_cast<const float2*>(P + i); }

template <typename T, int DM>
struct GenzGaussian {
  static __device__ __forceinline__ T eval(const T (&x)[DM], int d, const T* P) {
    T q = T(0);
    if constexpr (std::is_same<T, float>::value && DM % 2 == 0) {
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int a = 0; a < DM; a += 2)
        if (a < d) {
          const float2 u = ppair(P, kMaxDim + a);
          const float2 t = __fadd2_rn(xpair(x, a, d, u.y), make_float2(-u.x, -u.y));
          s = __ffma2_rn(__fmul2_rn(ppair(P, a), t), t, s);
        }
      q = s.x + s.y;
    } else {
#pragma unroll
      for (int a = 0; a < DM; ++a)
        if (a < d) {
          const T t = x[a] - P[kMaxDim + a];
          q = vfma(P[a] * t, t, q);
        }
    }
    return gexp(-q);
  }
  // theta = (u_1..u_d, a_1..a_d): df/du_i = 2 a_i^2 (x_i - u_i) f,
  // df/da_i = -2 a_i (x_i - u_i)^2 f.
  static constexpr int NT = 2 * DM;
  static __device__ __forceinline__ T grad(const T (&x)[DM], int d, const T* P, T* g) {
    const T f = eval(x, d, P);
#pragma unroll
    for (int a = 0; a < DM; ++a)
      if (a < d) {
        const T t = x[a] - P[kMaxDim + a];
        g[a] = T(2) * P[a] * t * f;
        g[DM + a] = T(-2) * P[2 * kMaxDim + a] * t * t * f;
      }
    return f;
  }
};

// f = prod (a_i^-2 + (x_i - u_i)^2)^-1.  P[i] = a_i^-2, P[kMaxDim+i] = u_i.
template <typename T, int DM>
struct GenzProductPeak {
  static __device__ __forceinline__ T eval(const T (&x)[DM], int d, const T* P) {
    T den = T(1);
    if constexpr (std::is_same<T, float>::value && DM % 2 == 0) {
      float2 dd = make_float2(1.f, 1.f);
#pragma unroll
      for (int a = 0; a < DM; a += 2)
        if (a < d) {
          const float2 u = ppair(P, kMaxDim + a), c = ppair(P, a);
          // past d: t = 0 and the factor c.y replaced by 1
          const float2 t = __fadd2_rn(xpair(x, a, d, u.y), make_float2(-u.x, -u.y));
          dd = __fmul2_rn(dd, __ffma2_rn(t, t, make_float2(c.x, a + 1 < d ? c.y : 1.f)));
        }
      den = dd.x * dd.y;
    } else {
#pragma unroll
      for (int a = 0; a < DM; ++a)
        if (a < d) {
          const T t = x[a] - P[kMaxDim + a];
          den *= vfma(t, t, P[a]);
        }
    }
    return qdiv(T(1), den);
  }
};

// f = (1 + sum a_i x_i)^-(d+1).  P[i] = a_i, P[kScalar] = -(d+1).
template <typename T, int DM>
struct GenzCornerPeak {
  static __device__ __forceinline__ T eval(const T (&x)[DM], int d, const T* P) {
    T t = T(1);
    if constexpr (std::is_same<T, float>::value && DM % 2 == 0) {
      float2 s = make_float2(1.f, 0.f);
#pragma unroll
      for (int a = 0; a < DM; a += 2)
        if (a < d) s = __ffma2_rn(ppair(P, a), xpair(x, a, d, 0.f), s);
      t = s.x + s.y;
    } else {
#pragma unroll
      for (int a = 0; a < DM; ++a)
        if (a < d) t = vfma(P[a], x[a], t);
    }
    return qpow_pos(t, P[kScalar]);
  }
};

// f = cos(2 pi u1 + sum a_i x_i).  P[i] = a_i, P[kScalar] = 2 pi u1.
template <typename T, int DM>
struct GenzOscillatory {
  static __device__ __forceinline__ T eval(const T (&x)[DM], int d, const T* P) {
    T t = P[kScalar];
    if constexpr (std::is_same<T, float>::value && DM % 2 == 0) {
      float2 s = make_float2(P[kScalar], 0.f);
#pragma unroll
      for (int a = 0; a < DM; a += 2)
        if (a < d) s = __ffma2_rn(ppair(P, a), xpair(x, a, d, 0.f), s);
      t = s.x + s.y;
    } else {
#pragma unroll
      for (int a = 0; a < DM; ++a)
        if (a < d) t = vfma(P[a], x[a], t);
    }
    return qcos_any(t);
  }
};

// f = exp(-sum a_i |x_i - u_i|) (Genz "continuous").  P[i] = a_i,
// P[kMaxDim+i] = u_i.
template <typename T, int DM>
struct GenzContinuous {
  static __device__ __forceinline__ T eval(const T (&x)[DM], int d, const T* P) {
    T q = T(0);
#pragma unroll
    for (int a = 0; a < DM; ++a)
      if (a < d) q = vfma(P[a], fabs(x[a] - P[kMaxDim + a]), q);
    return gexp(-q);
  }
};

// f = exp(sum a_i x_i) where x_1 <= u_1 and x_2 <= u_2, else 0 (Genz
// "discontinuous"; only x_1 for d = 1).  P[i] = a_i, P[kScalar], P[kScalar+1]
// = u_1, u_2 (u_2 = 2 when d = 1: never binding).
template <typename T, int DM>
struct GenzDiscontinuous {
  static __device__ __forceinline__ T eval(const T (&x)[DM], int d, const T* P) {
    static_assert(DM >= 2, "compiled bounds start at 4 axes");
    if (x[0] > P[kScalar] || (d > 1 && x[1] > P[kScalar + 1])) return T(0);
    T t = T(0);
#pragma unroll
    for (int a = 0; a < DM; ++a)
      if (a < d) t = vfma(P[a], x[a], t);
    return qexp(t);
  }
};

// Two Gaussian peaks (Lepage's test shape), normalised to unit integral over
// R^d: f = K/2 (exp(-|x - c1|^2 / w^2) + exp(-|x - c2|^2 / w^2)).
// P[kScalar + 0..3] = c1, c2, 1/w^2, K/2 with K = (w sqrt pi)^-d.
template <typename T, int DM>
struct DoubleGaussian {
  static __device__ __forceinline__ T eval(const T (&x)[DM], int d, const T* P) {
    const T c1 = P[kScalar], c2 = P[kScalar + 1];
    T q1 = T(0), q2 = T(0);
#pragma unroll
    for (int a = 0; a < DM; ++a)
      if (a < d) {
        const T t1 = x[a] - c1, t2 = x[a] - c2;
        q1 = vfma(t1, t1, q1);
        q2 = vfma(t2, t2, q2);
      }
    const T iw2 = P[kScalar + 2];
    return P[kScalar + 3] * (gexp(-q1 * iw2) + gexp(-q2 * iw2));
  }
  // theta = (c1, c2, w): df/dc_k = K/2 E_k 2 sum_i (x_i - c_k) / w^2,
  // df/dw = K/2 sum_k E_k (2 q_k / w^3 - d / w), q_k = sum_i (x_i - c_k)^2.
  static constexpr int NT = 3;
  static __device__ __forceinline__ T grad(const T (&x)[DM], int d, const T* P, T* g) {
    const T c1 = P[kScalar], c2 = P[kScalar + 1], iw2 = P[kScalar + 2], K2 = P[kScalar + 3];
    const T w = P[kScalar + 4];
    T q1 = T(0), q2 = T(0), l1 = T(0), l2 = T(0);
#pragma unroll
    for (int a = 0; a < DM; ++a)
      if (a < d) {
        const T t1 = x[a] - c1, t2 = x[a] - c2;
        q1 = vfma(t1, t1, q1);
        q2 = vfma(t2, t2, q2);
        l1 += t1;
        l2 += t2;
      }
    const T e1 = K2 * gexp(-q1 * iw2), e2 = K2 * gexp(-q2 * iw2);
    g[0] = e1 * T(2) * l1 * iw2;
    g[1] = e2 * T(2) * l2 * iw2;
    const T iw = T(1) / w;
    g[2] = e1 * (T(2) * q1 * iw2 * iw - T(d) * iw) + e2 * (T(2) * q2 * iw2 * iw - T(d) * iw);
    return e1 + e2;
  }
};

// ----------------------------------------------------------------- RAMBO
// Massless n-body phase space (Kleiss, Stirling, Ellis 1986) in units of
// sqrt(s), with the integrand of include/gvegas.h evaluated dimensionless:
//   returns  cut * [mu_g / ((s12 - mu)^2 + mu_g^2)] * prod_i 1/s_{i,i+1}
// (s_ij in units of s, mu = M^2/s, mu_g = M Gamma / s); the host multiplies
// every sum by the constant V_n s^-3 (or the observable's own scale).
// The invariants come from the isotropic momenta q_i of RAMBO's first step,
// before its boost: with n_i the unit direction of q_i, 2 q_i.q_j =
// q0_i q0_j |n_i - n_j|^2, the total mass is M^2 = sum_{i<j} 2 q_i.q_j, and
// the boost and scaling that follow leave s_ij / s = 2 q_i.q_j / M^2.  Every
// term is non-negative, so nothing cancels however strongly the system of
// q's is boosted (forming M^2 = Q0^2 - |Q|^2 or s_ij from the boosted momenta
// loses about gamma^2 of the precision, which in FP32 biased the estimate;
// the Breit-Wigner amplifies an error of s12 by up to M / Gamma).  For two
// partons s12 = s exactly.  The boosted momenta give pT, eta and the
// transverse direction u for the cuts (|u_i - u_j| = 2 sin(dphi/2), no
// atan2).
// The FP32 kernels use the quick forms of common.cuh; FP64 the library.
enum {
  RB_N = kScalar, RB_MU, RB_MUG, RB_MUG2, RB_PTMIN, RB_DR2, RB_CUT, RB_T,
  RB_INVWC, RB_OBS,
  RB_DMU_DM,    // d mu / dM = 2 M / s            (per GeV)
  RB_DMUG_DM,   // d mu_g / dM = Gamma / s        (per GeV)
  RB_DMUG_DG,   // d mu_g / dGamma = M / s        (per GeV)
  RB_INVWC_GEV  // 1 / w_c                        (per GeV)
};

template <typename T, int DM>
struct RamboBW {
  static constexpr int NM = DM / 4;

  struct Event {
    T pt[NM], eta[NM], ux[NM], uy[NM];
    T s[NM];  // s_{i, i+1 mod n} / s
  };

  // Momenta -> (pT, eta, transverse direction) and the cyclic invariants.
  // Returns false for a zero-weight point.
  static __device__ __forceinline__ bool kinematics(const T (&x)[DM], int n, Event& ev) {
    T E[NM], nx[NM], ny[NM], nz[NM];
    T Q0 = T(0), Qx = T(0), Qy = T(0), Qz = T(0);
#pragma unroll
    for (int i = 0; i < NM; ++i)
      if (i < n) {
        const T r1 = x[4 * i], r2 = x[4 * i + 1], r3 = x[4 * i + 2], r4 = x[4 * i + 3];
        if (!(r1 > T(0) && r2 > T(0))) return false;
        const T q0 = -qlog_rel(r1 * r2);  // energy density q0 e^{-q0}: one logarithm
        const T sn = T(2) * qsqrt(r3 * (T(1) - r3));
        T sp, cp;
        qsincos2pi(r4, &sp, &cp);
        E[i] = q0;
        nx[i] = sn * cp;
        ny[i] = sn * sp;
        nz[i] = T(2) * r3 - T(1);
        Q0 += q0;
        Qx = vfma(q0, nx[i], Qx);
        Qy = vfma(q0, ny[i], Qy);
        Qz = vfma(q0, nz[i], Qz);
      }
    // pair masses m_ij = 2 q_i.q_j, their sum M^2 and the cyclic ones
    T M2 = T(0), cyc[NM];
#pragma unroll
    for (int i = 0; i < NM; ++i)
#pragma unroll
      for (int j = i + 1; j < NM; ++j)
        if (j < n) {
          const T dx = nx[i] - nx[j], dy = ny[i] - ny[j], dz = nz[i] - nz[j];
          const T m = E[i] * E[j] * vfma(dx, dx, vfma(dy, dy, dz * dz));
          M2 += m;
          if (j == i + 1) cyc[i] = m;
          if (i == 0 && j == n - 1) cyc[j] = m;  // (n-1, 0); for n = 2 the same pair twice
        }
    const T iM2 = qdiv(T(1), M2);
#pragma unroll
    for (int i = 0; i < NM; ++i)
      if (i < n) ev.s[i] = cyc[i] * iM2;
    const T MQ = qsqrt(M2);
    const T iM = qdiv(T(1), MQ);
    const T bx = -Qx * iM, by = -Qy * iM, bz = -Qz * iM;
    const T gam = Q0 * iM;
    const T A = qdiv(T(1), T(1) + gam);
#pragma unroll
    for (int i = 0; i < NM; ++i)
      if (i < n) {
        const T px = E[i] * nx[i], py = E[i] * ny[i], pz = E[i] * nz[i];
        const T bq = bx * px + by * py + bz * pz;
        const T ab = A * bq + E[i];
        const T qx = iM * vfma(ab, bx, px);
        const T qy = iM * vfma(ab, by, py);
        const T qz = iM * vfma(ab, bz, pz);
        const T pt2 = qx * qx + qy * qy;
        const T pt = qsqrt(pt2);
        const T pa = qsqrt(vfma(qz, qz, pt2));
        const T ipt = qdiv(T(1), pt);
        ev.pt[i] = pt;
        // (the rapidities feed only the Delta R cut: the quick logarithm)
        ev.eta[i] = vcopysign(qlog((fabs(qz) + pa) * ipt), qz);
        ev.ux[i] = qx * ipt;
        ev.uy[i] = qy * ipt;
      }
    return true;
  }

  // |u_i - u_j|^2 = 4 sin^2(dphi / 2)
  static __device__ __forceinline__ T chord2(const Event& ev, int i, int j) {
    const T dx = ev.ux[i] - ev.ux[j], dy = ev.uy[i] - ev.uy[j];
    return vfma(dx, dx, dy * dy);
  }

  static __device__ __forceinline__ T bw(T s12, const T* P) {
    const T t = s12 - P[RB_MU];
    return qdiv(P[RB_MUG], vfma(t, t, P[RB_MUG2]));
  }

  // Delta R > R (pseudorapidity, dphi wrapped to [-pi, pi]): with
  // t = R^2 - deta^2 > 0 the pair needs |dphi| > sqrt(t), i.e. sqrt(t) < pi
  // and a chord |u_i - u_j| = 2 sin(|dphi|/2) beyond 2 sin(sqrt(t)/2).  In
  // FP32 with R^2 <= 1/4 the squared bound 4 sin^2(sqrt(t)/2) = 2 (1 - cos
  // sqrt(t)) is its Taylor series t - t^2/12 + t^3/360 - t^4/20160
  // (truncation below 2e-9 relative for t <= 1/4): no root and no sine.
  static __device__ __forceinline__ bool dr_pass(const Event& ev, int i, int j, const T* P) {
    const T de = ev.eta[i] - ev.eta[j];
    const T t = P[RB_DR2] - de * de;
    if (!(t > T(0))) return true;
    if constexpr (std::is_same<T, float>::value) {
      if (P[RB_DR2] <= T(0.25)) {
        const T b = t * vfma(-t * T(1.0 / 12.0), vfma(-t * T(1.0 / 30.0), vfma(-t, T(1.0 / 56.0), T(1)), T(1)), T(1));
        return chord2(ev, i, j) > b;
      }
    }
    const T th = qsqrt(t);
    if (!(th < T(3.14159265358979323846))) return false;
    const T h = qsin(T(0.5) * th);
    return chord2(ev, i, j) > T(4) * h * h;
  }

  static __device__ __forceinline__ T eval(const T (&x)[DM], int d, const T* P) {
    const int obs = (int)P[RB_OBS];
    if (obs == 1) return T(1);
    const int n = d >> 2;
    Event ev;
    if (!kinematics(x, n, ev)) return T(0);
    const int cut = (int)P[RB_CUT];
    T cw = T(1);
    if (obs == 0 && cut == 0) {
#pragma unroll
      for (int i = 0; i < NM; ++i)
        if (i < n && !(ev.pt[i] > P[RB_PTMIN])) return T(0);
    } else if (obs == 0 && cut == 1) {
#pragma unroll
      for (int i = 0; i < NM; ++i)
        if (i < n) cw *= qdiv(T(1), T(1) + qexp(-(ev.pt[i] - P[RB_T]) * P[RB_INVWC]));
    }
    if (obs == 0 && cut != 2) {
#pragma unroll
      for (int i = 0; i < NM; ++i)
#pragma unroll
        for (int j = i + 1; j < NM; ++j)
          if (j < n && !dr_pass(ev, i, j, P)) return T(0);
    }
    const T s12 = ev.s[0];
    if (obs == 2) return s12;
    const T b = bw(s12, P);
    if (obs == 3) return b;
    T den = s12;
#pragma unroll
    for (int i = 1; i < NM; ++i)
      if (i < n) den *= ev.s[i];
    return qdiv(cw * b, den);
  }

  // theta = (M, Gamma, T) in GeV for the full integrand (obs 0).  The Breit-
  // Wigner factor b = mu_g / ((s12 - mu)^2 + mu_g^2) depends on M through mu
  // and mu_g and on Gamma through mu_g; the sigmoid cut gives
  // d ln(cut)/dT = -sum_i (1 - sigma_i) / w_c; the hard cut has dT = 0.
  static constexpr int NT = 3;
  static __device__ __forceinline__ T grad(const T (&x)[DM], int d, const T* P, T* g) {
    g[0] = g[1] = g[2] = T(0);
    const int obs = (int)P[RB_OBS];
    if (obs != 0) return eval(x, d, P);
    const int n = d >> 2;
    Event ev;
    if (!kinematics(x, n, ev)) return T(0);
    const int cut = (int)P[RB_CUT];
    T cw = T(1), dlc = T(0);
    if (cut == 0) {
#pragma unroll
      for (int i = 0; i < NM; ++i)
        if (i < n && !(ev.pt[i] > P[RB_PTMIN])) return T(0);
    } else if (cut == 1) {
#pragma unroll
      for (int i = 0; i < NM; ++i)
        if (i < n) {
          const T sg = qdiv(T(1), T(1) + qexp(-(ev.pt[i] - P[RB_T]) * P[RB_INVWC]));
          cw *= sg;
          dlc -= (T(1) - sg) * P[RB_INVWC_GEV];
        }
    }
    if (cut != 2) {
#pragma unroll
      for (int i = 0; i < NM; ++i)
#pragma unroll
        for (int j = i + 1; j < NM; ++j)
          if (j < n && !dr_pass(ev, i, j, P)) return T(0);
    }
    const T s12 = ev.s[0];
    T den = s12;
#pragma unroll
    for (int i = 1; i < NM; ++i)
      if (i < n) den *= ev.s[i];
    const T t = s12 - P[RB_MU], mug = P[RB_MUG];
    const T D = vfma(t, t, P[RB_MUG2]);
    const T iD = qdiv(T(1), D);
    const T b = mug * iD;
    const T pre = qdiv(cw, den);
    // db/dM = (mug' D - mug D') / D^2 with D' = -2 t mu' + 2 mug mug', whose
    // numerator is mug' (t - mug)(t + mug) + 2 mug t mu' (no cancellation
    // between mug' D and 2 mug^2 mug'); d/dGamma has mu' = 0.
    const T tm = (t - mug) * (t + mug);
    g[0] = pre * vfma(P[RB_DMUG_DM], tm, T(2) * mug * t * P[RB_DMU_DM]) * iD * iD;
    g[1] = pre * (P[RB_DMUG_DG] * tm) * iD * iD;
    const T f = pre * b;
    g[2] = f * dlc;
    return f;
  }
};

// --------------------------------------------------- u dbar -> W+ -> mu+ nu
// Sec. 4's process with n = 0 gluons and the mu+ cuts, five variables
// (Breit-Wigner shat, W rapidity, cos theta and azimuth of the mu+, the
// helicity combination; the slot layout of VG_W_MUNU in gvegas.h).  Only
// u(-) dbar(+) -> nu(-) mu+(+) couples, so the other 15 helicity cells
// return 0 at once.  With shat = M^2 + M Gamma tan(rho) the Breit-Wigner
// denominator cancels against dshat/drho = M Gamma sec^2(rho), and the
// product of flux, phase space, averaged |M|^2 and Jacobians reduces to
//   f = K exp(a_u ln x1 + b_u ln(1 - x1) + a_d ln x2 + b_d ln(1 - x2)) L shat (1 - c)^2
// with L = -ln tau, ln x1,2 = -L/2 +- y_W, c = cos theta, and
// K = A_u A_d Delta rho g^4 |V_ud|^2 (pb GeV^2) / (48 pi S M Gamma).
enum {
  W_RLO = kScalar, W_DRHO, W_M2, W_MG, W_INVS, W_PT2, W_ETA, W_CUTS, W_K, W_ALU, W_BU, W_ALD, W_BD
};
constexpr int kWHelicity = 0 | 2 | 0 | 8;  // bits u, dbar, nu, mu+ (1 = positive)

template <typename T, int DM>
struct WMuNu {
  static __device__ __forceinline__ T eval(const T (&x)[DM], int d, const T* P) {
    const int h = (int)(x[4] * T(16));  // x < 1: the cell floor(16 y5)
    if ((h < 15 ? h : 15) != kWHelicity) return T(0);
    T sn, cs;
    const T rho = vfma(P[W_DRHO], x[0], P[W_RLO]);
    if constexpr (std::is_same<T, float>::value)
      __sincosf(rho, &sn, &cs);
    else
      sincos(rho, &sn, &cs);
    const T shat = vfma(P[W_MG], qdiv(sn, cs), P[W_M2]);
    const T L = -qlog_rel(shat * P[W_INVS]);
    const T yw = (x[1] - T(0.5)) * L;
    const T lx1 = vfma(T(-0.5), L, yw), lx2 = vfma(T(-0.5), L, -yw);
    const T x1 = qexp(lx1), x2 = qexp(lx2);
    if (!(x1 < T(1) && x2 < T(1) && L > T(0))) return T(0);
    const T c = vfma(T(2), x[2], T(-1));
    if (P[W_CUTS] != T(0)) {
      if (!(shat * (T(1) - c) * (T(1) + c) > P[W_PT2])) return T(0);
      const T eta = vfma(T(0.5), qlog(qdiv(T(1) + c, T(1) - c)), yw);
      if (!(fabs(eta) < P[W_ETA])) return T(0);
    }
    const T e = P[W_ALU] * lx1 + P[W_BU] * qlog_rel(T(1) - x1) + P[W_ALD] * lx2 + P[W_BD] * qlog_rel(T(1) - x2);
    const T omc = T(1) - c;
    return P[W_K] * qexp(e) * L * shat * omc * omc;
  }
};

}  // namespace gv
