// Pointwise pieces shared by the SIMT and tensor-core step kernels: the
// reaction terms g^u, g^v and one direction of the tridiagonal Kronecker-sum
// action (Sec. 2, Eq. 6, with the finite-difference rows of Sec. 4).
#pragma once

#include <stdint.h>

#include "adr_internal.h"

namespace adr {

template <typename T>
__device__ __forceinline__ void react(const ReactionT<T>& rx, T u, T v, T& gu, T& gv) {
  switch (rx.model) {
    case ADR_SCHNAKENBERG: {
      const T g = rx.p[0], a = rx.p[1], b = rx.p[2];
      const T u2v = u * u * v;
      gu = g * (a - u + u2v);
      gv = g * (b - u2v);
    } break;
    case ADR_FHN: {
      const T e = rx.p[0], a1 = rx.p[1], a0 = rx.p[2];
      gu = u - u * u * u - v;
      gv = e * (u - a1 * v - a0);
    } break;
    case ADR_BRUSSELATOR: {
      const T a = rx.p[0], b = rx.p[1];
      const T u2v = u * u * v;
      gu = a - (b + (T)1) * u + u2v;
      gv = b * u - u2v;
    } break;
    case ADR_FHN_RHO: {
      const T rho = rx.p[0], a1 = rx.p[1], a2 = rx.p[2];
      gu = rho * (u - u * u * u - v);
      gv = rho * a1 * (u - a2 * v);
    } break;
    case ADR_DIB: {
      const T rho = rx.p[0], a1u = rx.p[1], a2u = rx.p[2], a3u = rx.p[3], a4u = rx.p[4];
      const T a1v = rx.p[5], a2v = rx.p[6], a3v = rx.p[7], a4v = rx.p[8], a5v = rx.p[9];
      const T one = (T)1;
      gu = rho * (a1u * (one - v) * u - a2u * u * u * u - a3u * (v - a4u));
      gv = rho * (a1v * (one + a2v * u) * (one - v) * (one - a3v * (one - v)) -
                  a4v * v * (one + a5v * u) * (one + a3v * v));
    } break;
    default:
      gu = (T)0;
      gv = (T)0;
  }
}

// One direction of the tridiagonal action at one point, in difference form
// (the rows sum to zero): interior lo (x_{i-1} - x_i) + up (x_{i+1} - x_i),
// Neumann rows b0 (x_1 - x_0) and bn (x_{n-2} - x_{n-1}).
// Double-float numbers: a value is h + l with two FP32 words (about 48
// significant bits).  Sums use Knuth's TwoSum and products the exact FMA
// residual (Dekker's TwoProduct with a fused multiply-add), so a reaction
// polynomial whose terms cancel (the Brusselator's a - (b + 1) u + u^2 v
// at u, v of a few units, say) keeps the digits an FP32 evaluation loses.
// The pairs are left unrenormalised: a sum is the TwoSum of the high words
// with the low words added to its error, a product the rounded high product
// with its exact residual and the cross terms, and neither ends with the
// TwoSum that would make l at most half an ulp of h.  Every operation still
// errs by a few units of 2^-47 of its operands' size (the low words stay
// about 2^-23 of the values they refine, or are themselves the result after
// a cancellation), which is what the normalised pair guarantees, and the
// single rounding to FP32 at the end dominates; each sum costs 8 FP32
// operations instead of 14 and each product 4 instead of 10.
// The _rn intrinsics keep the compiler from contracting or reordering the
// error terms.
struct dfloat {
  float h, l;
  __device__ __forceinline__ dfloat() : h(0.f), l(0.f) {}
  __device__ __forceinline__ dfloat(float x) : h(x), l(0.f) {}
  __device__ __forceinline__ dfloat(float x, float y) : h(x), l(y) {}
};

__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return dfloat(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  const dfloat s = df_two_sum(a.h, b.h);
  return dfloat(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.h, -a.l); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
  const float p = __fmul_rn(a.h, b.h);
  const float e = __fmaf_rn(a.h, b.h, -p);  // exact: a.h b.h = p + e
  return dfloat(p, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e)));
}

// The reaction of Eq. 1 evaluated in double-float from single-precision
// state values (parameters as p + plo).
__device__ __forceinline__ void react_dfd(const ReactionT<float>& rx, float u, float v, dfloat& gu,
                                          dfloat& gv) {
  ReactionT<dfloat> r;
  r.model = rx.model;
#pragma unroll
  for (int i = 0; i < 16; ++i) r.p[i] = dfloat(rx.p[i], rx.plo[i]);
  react<dfloat>(r, dfloat(u), dfloat(v), gu, gv);
}

// The same, rounded once to FP32.
__device__ __forceinline__ void react_df(const ReactionT<float>& rx, float u, float v, float& gu,
                                         float& gv) {
  dfloat a, b;
  react_dfd(rx, u, v, a, b);
  gu = __fadd_rn(a.h, a.l);
  gv = __fadd_rn(b.h, b.l);
}

// x - y exactly, as a double-float.
__device__ __forceinline__ dfloat df_diff(float x, float y) { return df_two_sum(x, -y); }

// One direction of the stencil of Eq. 6 in double-float, coefficients as
// hi + lo (the FP64 operator): interior rows lo (x- - x) + up (x+ - x),
// Neumann rows b0 (x+ - x) and bn (x- - x).  The stencil's terms can be
// large next to their sum (delta / h^2 of 10^5 on fine grids), so the
// accurate mode sums them without intermediate rounding.
__device__ __forceinline__ dfloat dtri_in(float xm, float xc, float xp, dfloat lo, dfloat up) {
  return lo * df_diff(xm, xc) + up * df_diff(xp, xc);
}
__device__ __forceinline__ dfloat dtri_dir(float xm, float xc, float xp, int i, int n, dfloat lo,
                                           dfloat up, dfloat b0, dfloat bn) {
  if (i == 0) return b0 * df_diff(xp, xc);
  if (i == n - 1) return bn * df_diff(xm, xc);
  return dtri_in(xm, xc, xp, lo, up);
}
__device__ __forceinline__ dfloat dtri_x4(int j, float xm, float xc, float xp, int i, int n,
                                          dfloat lo, dfloat up, dfloat b0, dfloat bn) {
  if (j == 0 && i == 0) return b0 * df_diff(xp, xc);
  if (j == 3 && i == n - 1) return bn * df_diff(xm, xc);
  return dtri_in(xm, xc, xp, lo, up);
}

// The tridiagonal coefficients of one component on one axis as double-floats.
struct CoefDF {
  dfloat lo, up, b0, bn;
};
__device__ __forceinline__ CoefDF coef_df(const TridiagT<float>& A, const TridiagT<float>& Al) {
  return CoefDF{dfloat(A.lo, Al.lo), dfloat(A.up, Al.up), dfloat(A.b0, Al.b0), dfloat(A.bn, Al.bn)};
}

// Round a double-float to FP32.
__device__ __forceinline__ float df_round(dfloat x) { return __fadd_rn(x.h, x.l); }

// D = G(u2, v2) - G(u0, v0), the stage-2 reaction difference of Eq. 11, in
// increment form: with du = u2 - u0 and dv = v2 - v0 (a single rounding,
// relative to the increment), every polynomial difference is expanded by
// d(AB) = dA B2 + A dB, e.g. d(u^2 v) = (u0 + u2) du v2 + u0^2 dv and
// d(u^3) = (u2^2 + u2 u0 + u0^2) du.  The terms are of the size of D itself,
// so the rounding is relative to D and not to the reactions, whose
// difference cancels most of their digits when the step is small.
template <typename T>
__device__ __forceinline__ void react_diff(const ReactionT<T>& rx, T u0, T v0, T u2, T v2, T& du,
                                           T& dv) {
  const T eu = u2 - u0, ev = v2 - v0;
  switch (rx.model) {
    case ADR_SCHNAKENBERG: {
      const T g = rx.p[0];
      const T d = (u0 + u2) * eu * v2 + u0 * u0 * ev;  // d(u^2 v)
      du = g * (d - eu);
      dv = -g * d;
    } break;
    case ADR_FHN: {
      const T e = rx.p[0], a1 = rx.p[1];
      const T d3 = (u2 * u2 + u2 * u0 + u0 * u0) * eu;  // d(u^3)
      du = eu - d3 - ev;
      dv = e * (eu - a1 * ev);
    } break;
    case ADR_BRUSSELATOR: {
      const T b = rx.p[1];
      const T d = (u0 + u2) * eu * v2 + u0 * u0 * ev;
      du = d - (b + (T)1) * eu;
      dv = b * eu - d;
    } break;
    case ADR_FHN_RHO: {
      const T rho = rx.p[0], a1 = rx.p[1], a2 = rx.p[2];
      const T d3 = (u2 * u2 + u2 * u0 + u0 * u0) * eu;
      du = rho * (eu - d3 - ev);
      dv = rho * a1 * (eu - a2 * ev);
    } break;
    case ADR_DIB: {
      const T rho = rx.p[0], a1u = rx.p[1], a2u = rx.p[2], a3u = rx.p[3];
      const T a1v = rx.p[5], a2v = rx.p[6], a3v = rx.p[7], a4v = rx.p[8], a5v = rx.p[9];
      const T one = (T)1;
      // g^u: a1u (1 - v) u - a2u u^3 - a3u (v - a4u);  d((1 - v) u) = du - (v2 du + u0 dv)
      const T d3 = (u2 * u2 + u2 * u0 + u0 * u0) * eu;
      du = rho * (a1u * (eu - (v2 * eu + u0 * ev)) - a2u * d3 - a3u * ev);
      // g^v: a1v P(u) Q(v) - a4v R(v) S(u) with P = 1 + a2v u, Q = w (1 - a3v w),
      // w = 1 - v, R = v (1 + a3v v), S = 1 + a5v u
      const T w0 = one - v0, w2 = one - v2;
      const T q2 = w2 * (one - a3v * w2);
      const T dq = -ev * (one - a3v * (w0 + w2));
      const T r0 = v0 * (one + a3v * v0);
      const T dr = ev * (one + a3v * (v0 + v2));
      const T d1 = a2v * eu * q2 + (one + a2v * u0) * dq;
      const T d2 = dr * (one + a5v * u2) + r0 * (a5v * eu);
      dv = rho * (a1v * d1 - a4v * d2);
    } break;
    default:
      du = (T)0;
      dv = (T)0;
  }
}

template <typename T>
__device__ __forceinline__ T stencil_dir(const T* __restrict__ x, int64_t idx, int64_t stride,
                                         int i, int n, const TridiagT<T>& A) {
  const T xc = x[idx];
  if (i == 0) return A.b0 * (x[idx + stride] - xc);
  if (i == n - 1) return A.bn * (x[idx - stride] - xc);
  return A.lo * (x[idx - stride] - xc) + A.up * (x[idx + stride] - xc);
}

// W^c = sum_mu (A_mu^c U^c) + G^c(U, V) at the point with coordinates
// (i1, i2, i3) and linear index idx; writes both components.
template <typename T>
__device__ __forceinline__ void rhs_point(const PointwiseArgsT<T>& a, const T* __restrict__ u,
                                          const T* __restrict__ v, int64_t idx, int i1, int i2,
                                          int i3, T& wu, T& wv) {
  const int n1 = (int)a.n[0], n2 = (int)a.n[1];
  T ku = stencil_dir(u, idx, 1, i1, n1, a.A[0][0]) +
         stencil_dir(u, idx, (int64_t)n1, i2, n2, a.A[0][1]);
  T kv = stencil_dir(v, idx, 1, i1, n1, a.A[1][0]) +
         stencil_dir(v, idx, (int64_t)n1, i2, n2, a.A[1][1]);
  if (a.d == 3) {
    const int n3 = (int)a.n[2];
    ku += stencil_dir(u, idx, (int64_t)n1 * n2, i3, n3, a.A[0][2]);
    kv += stencil_dir(v, idx, (int64_t)n1 * n2, i3, n3, a.A[1][2]);
  }
  T gu, gv;
  react<T>(a.rx, u[idx], v[idx], gu, gv);
  wu = ku + gu;
  wv = kv + gv;
}

}  // namespace adr
