// Device arithmetic of the Lagrange-flux scheme (arXiv:1607.08710):
// equation of state (eq. 1), slope limiter (eq. "sweby"), Lagrangian HLL /
// acoustic interface solver (eqs. 13-14) and upwind Lagrange flux (eq. 12),
// with NF = 4 + nspecies fields per cell: the transported mass fractions of
// Sec. 5 ride on the same upwind flux as (rho, rho u, rho v, rho E).
//
// FP64 uses IEEE division and square root throughout.  FP32 uses the
// hardware approximate reciprocal and reciprocal square root (__fdividef,
// rsqrtf): each is within a few ulp, far inside the FP32 error budget of the
// scheme, and keeps the special-function unit off the critical path.
#pragma once

#include <cuda_runtime.h>
#include "lf_internal.h"

namespace lf {

template <typename T> struct Ar;

template <> struct Ar<double> {
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  // a = sqrt(x) and 1/a
  static __device__ __forceinline__ void sqrt_and_rsqrt(double x, double& a, double& ia) {
    a = sqrt(x);
    ia = 1.0 / a;
  }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
};

template <> struct Ar<float> {
  static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
  static __device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
  static __device__ __forceinline__ void sqrt_and_rsqrt(float x, float& a, float& ia) {
    ia = rsqrtf(x);
    a = x * ia;
  }
  static __device__ __forceinline__ float sqrt_(float x) { return x * rsqrtf(x); }
};

// Rounding is pinned: the kernels are compiled with -fmad=false, so a
// product and a sum are fused only where fma_ is written.  Every inlined copy
// of an expression (e.g. the first face of a row tile in its prologue and the
// same face inside the previous tile's march) then rounds identically, which
// makes results independent of the tile height and of the launch shape.
__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }

// Physics constants of one launch, in the kernel's precision.
template <typename T>
struct Phys {
  T gamma, gm1, inv_gm1, beta, rdx, rdy;
  int riemann;
  __device__ __forceinline__ explicit Phys(const MeshDesc& m)
      : gamma(T(m.gamma)), gm1(T(m.gamma - 1.0)), inv_gm1(T(1) / gm1), beta(T(m.beta)),
        rdx(T(m.rdx)), rdy(T(m.rdy)), riemann(m.riemann) {}
};

// Conservative (rho, rho u, rho v, rho E, rho y_k) -> primitive
// (rho, u, v, p, y_k), eq. (1); y_k = (rho y_k) / rho.
template <typename T, int NF = 4>
__device__ __forceinline__ void to_prim(const Phys<T>& P, const T U[NF], T q[NF]) {
  T ir = Ar<T>::rcp(U[0]);
  T u = U[1] * ir, v = U[2] * ir;
  q[0] = U[0];
  q[1] = u;
  q[2] = v;
  q[3] = P.gm1 * fma_(T(-0.5), fma_(U[1], u, U[2] * v), U[3]);
#pragma unroll
  for (int k = 4; k < NF; ++k) q[k] = U[k] * ir;
}

// Half of the limited slope, phi(a,b)/2, so that the face states are
// q +/- limiter_half: eq. (sweby) for LIM_MINMOD / LIM_SWEBY, and van Leer's
// limiter (ab>0) 2ab/(a+b).  (Halving is exact in binary arithmetic, so this
// equals 0.5 * phi bit for bit.)
template <typename T, int LIM>
__device__ __forceinline__ T limiter_half(T a, T b, T beta) {
  T ab = a * b;
  if (LIM == LIM_VANLEER) {
    return ab > T(0) ? Ar<T>::div(ab, a + b) : T(0);
  } else {
    T aa = fabs(a), bb = fabs(b);
    T m;
    if (LIM == LIM_MINMOD) m = fmin(aa, bb);
    else m = fmax(fmin(aa, beta * bb), fmin(beta * aa, bb));
    return ab > T(0) ? copysign(T(0.5) * m, a) : T(0);
  }
}

// Eqs. (13)-(14): star pressure and normal velocity at a face from the
// reconstructed left/right (rho, u_n, p); then eq. (12) with the upwind state
// chosen by the sign of u*.  DIR = 0: x-face (normal velocity u), 1: y-face.
// qL, qR are primitive (rho, u, v, p, y_k).  F receives the flux along +x /
// +y; a species row is (rho_A y_k,A) u*, the mass flux's upwind side.
template <typename T, int DIR, int NF = 4>
__device__ __forceinline__ void lagrange_flux(const Phys<T>& P, const T qL[NF], const T qR[NF], T F[NF]) {
  const T rL = qL[0], pL = qL[3], rR = qR[0], pR = qR[3];
  const T unL = qL[1 + DIR], unR = qR[1 + DIR];
  T pstar, ustar;
  if (P.riemann == RIEMANN_MAXC) {
    // a = max(c_L, c_R) with c_k^2 = gamma p_k / rho_k; the larger c is the
    // larger c^2, so only one square root is needed.  With the weight
    // w = rho_L / (rho_L + rho_R), eqs. (13)-(14) read
    //   p* = p_L + w (p_R - p_L) - rho_R w a (u_R - u_L)
    //   u* = u_R - w (u_R - u_L) - (p_R - p_L) / ((rho_L + rho_R) a).
    T a2 = P.gamma * fmax(Ar<T>::div(pL, rL), Ar<T>::div(pR, rR));
    T a, ia;
    Ar<T>::sqrt_and_rsqrt(a2, a, ia);
    const T irs = Ar<T>::rcp(rL + rR);
    const T w = rL * irs, dp = pR - pL, du = unR - unL;
    pstar = fma_(-(rR * w * a), du, fma_(w, dp, pL));
    ustar = fma_(-dp, irs * ia, fma_(-w, du, unR));
  } else {
    // acoustic solver with Z_k = rho_k c_k
    T ZL = rL * Ar<T>::sqrt_(P.gamma * Ar<T>::div(pL, rL));
    T ZR = rR * Ar<T>::sqrt_(P.gamma * Ar<T>::div(pR, rR));
    T iZ = Ar<T>::rcp(ZL + ZR);
    pstar = fma_(-(ZL * ZR * iZ), unR - unL, fma_(ZR, pL, ZL * pR) * iZ);
    ustar = fma_(-(pR - pL), iZ, fma_(ZL, unL, ZR * unR) * iZ);
  }
  const bool left = ustar > T(0);
  const T r = left ? rL : rR;
  const T u = left ? qL[1] : qR[1];
  const T v = left ? qL[2] : qR[2];
  const T p = left ? pL : pR;
  const T rE = fma_(p, P.inv_gm1, T(0.5) * r * fma_(u, u, v * v));
  const T m = r * ustar;
  F[0] = m;
  F[1] = m * u;
  F[2] = m * v;
  F[3] = (rE + pstar) * ustar;
  F[1 + DIR] += pstar;
#pragma unroll
  for (int k = 4; k < NF; ++k) F[k] = (r * (left ? qL[k] : qR[k])) * ustar;
}

// Local CFL speed (|u|+c)/dx + (|v|+c)/dy (1D: (|u|+c)/dx) of a cell, and its
// positivity (rho > 0 and p > 0; false for NaN).
template <typename T, int DIM>
__device__ __forceinline__ T cell_speed(const Phys<T>& P, const T U[4], bool& ok) {
  const T ir = Ar<T>::rcp(U[0]);
  const T u = U[1] * ir, v = U[2] * ir;
  T q[4] = {U[0], u, v, P.gm1 * fma_(T(-0.5), fma_(U[1], u, U[2] * v), U[3])};
  ok = (q[0] > T(0)) && (q[3] > T(0));
  T c = Ar<T>::sqrt_(P.gamma * q[3] * ir);
  T s = (fabs(q[1]) + c) * P.rdx;
  if (DIM == 2) s = fma_(fabs(q[2]) + c, P.rdy, s);
  return s;
}

__device__ __forceinline__ int map_index(int c, int n, int bc) {
  if (bc == BC_PERIODIC) {
    c %= n;
    return c < 0 ? c + n : c;
  }
  return c < 0 ? 0 : (c >= n ? n - 1 : c);
}

// Max of positive doubles through their IEEE bit patterns (which order like
// the values); a NaN speed wins and is caught when dt is formed.
__device__ __forceinline__ void atomic_max_speed(unsigned long long* dst, double s) {
  atomicMax(dst, (unsigned long long)__double_as_longlong(s));
}

}  // namespace lf
