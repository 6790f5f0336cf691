// Device arithmetic of the Lagrange-flux scheme (arXiv:1607.08710):
// equation of state (eq. 1), slope limiter (eq. "sweby"), Lagrangian HLL /
// acoustic interface solver (eqs. 13-14) and upwind Lagrange flux (eq. 12),
// with NF = 4 + nspecies fields per cell: the transported mass fractions of
// Sec. 5 ride on the same upwind flux as (rho, rho u, rho v, rho E).
//
// FP64 uses IEEE division and square root throughout.  FP32 uses the
// hardware approximate reciprocal and reciprocal square root (the PTX
// instructions rcp.approx.ftz.f32 and rsqrt.approx.ftz.f32, one
// special-function instruction each): each is within a few ulp, far inside
// the FP32 error budget of the scheme; a quotient a / b is a * (1 / b).
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

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

template <> struct Ar<float> {
  static __device__ __forceinline__ float rcp(float x) { return rcp_approx(x); }
  static __device__ __forceinline__ float div(float a, float b) { return a * rcp_approx(b); }
  static __device__ __forceinline__ void sqrt_and_rsqrt(float x, float& a, float& ia) {
    ia = rsqrt_approx(x);
    a = x * ia;
  }
  static __device__ __forceinline__ float sqrt_(float x) { return x * rsqrt_approx(x); }
};

// Rounding is pinned: the kernels are compiled with -fmad=false, so a
// product and a sum are fused only where fma_ is written.  Every inlined copy
// of an expression (e.g. the first face of a row tile in its prologue and the
// same face inside the previous tile's march) then rounds identically, which
// makes results independent of the tile height and of the launch shape.
__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }

// ---------------------------------------------------------------------------
// Lane values.  The scheme's arithmetic is written once for a lane value V:
// one cell (float or double), or the two FP32 cells a lane owns held as one
// packed pair F2 and computed with Blackwell's paired FP32 add / multiply /
// fma instructions, one instruction for both cells.  Comparisons, selects,
// min/max and the special functions act per component.  Every packed
// operation rounds each component exactly like the scalar operation, so the
// pair computes, bit for bit, what two scalar passes would.
// ---------------------------------------------------------------------------
struct F2 {
  float2 v;
  F2() = default;
  __device__ __forceinline__ explicit F2(float s) { v.x = s; v.y = s; }
  __device__ __forceinline__ F2(float a, float b) { v.x = a; v.y = b; }
};
struct B2 {
  bool x, y;
};

__device__ __forceinline__ F2 f2_of(float2 t) {
  F2 r;
  r.v = t;
  return r;
}
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return f2_of(__fadd2_rn(a.v, b.v)); }
// a - b as b * (-1) + a: the product is exact, so this rounds like a
// subtraction.  (Measured on GB300 slightly faster than the paired
// subtraction instruction.)
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return f2_of(__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v)); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return f2_of(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 fma_(F2 a, F2 b, F2 c) { return f2_of(__ffma2_rn(a.v, b.v, c.v)); }

// Scalar type, mask type and cells per lane value.
template <typename V> struct LaneT;
template <> struct LaneT<float> { using S = float; using M = bool; static constexpr int N = 1; };
template <> struct LaneT<double> { using S = double; using M = bool; static constexpr int N = 1; };
template <> struct LaneT<F2> { using S = float; using M = B2; static constexpr int N = 2; };

template <typename V> __device__ __forceinline__ V splat(double s) { return V(typename LaneT<V>::S(s)); }

__device__ __forceinline__ float get(float v, int) { return v; }
__device__ __forceinline__ double get(double v, int) { return v; }
__device__ __forceinline__ float get(F2 v, int j) { return j ? v.v.y : v.v.x; }
__device__ __forceinline__ bool get(bool m, int) { return m; }
__device__ __forceinline__ bool get(B2 m, int j) { return j ? m.y : m.x; }

template <typename T> __device__ __forceinline__ T vmax(T a, T b) { return fmax(a, b); }
template <typename T> __device__ __forceinline__ T vmin(T a, T b) { return fmin(a, b); }
template <typename T> __device__ __forceinline__ T vabs(T a) { return fabs(a); }
template <typename T> __device__ __forceinline__ T vcopysign(T m, T a) { return copysign(m, a); }
template <typename T> __device__ __forceinline__ bool gt0(T a) { return a > T(0); }
template <typename T> __device__ __forceinline__ T vsel(bool c, T a, T b) { return c ? a : b; }
__device__ __forceinline__ bool land(bool a, bool b) { return a && b; }

template <> __device__ __forceinline__ F2 vmax(F2 a, F2 b) { return F2(fmaxf(a.v.x, b.v.x), fmaxf(a.v.y, b.v.y)); }
template <> __device__ __forceinline__ F2 vmin(F2 a, F2 b) { return F2(fminf(a.v.x, b.v.x), fminf(a.v.y, b.v.y)); }
template <> __device__ __forceinline__ F2 vabs(F2 a) { return F2(fabsf(a.v.x), fabsf(a.v.y)); }
template <> __device__ __forceinline__ F2 vcopysign(F2 m, F2 a) {
  return F2(copysignf(m.v.x, a.v.x), copysignf(m.v.y, a.v.y));
}
__device__ __forceinline__ B2 gt0(F2 a) { return B2{a.v.x > 0.0f, a.v.y > 0.0f}; }
__device__ __forceinline__ F2 vsel(B2 c, F2 a, F2 b) { return F2(c.x ? a.v.x : b.v.x, c.y ? a.v.y : b.v.y); }
__device__ __forceinline__ B2 land(B2 a, B2 b) { return B2{a.x && b.x, a.y && b.y}; }

template <> struct Ar<F2> {
  static __device__ __forceinline__ F2 rcp(F2 x) { return F2(rcp_approx(x.v.x), rcp_approx(x.v.y)); }
  static __device__ __forceinline__ F2 div(F2 a, F2 b) { return a * rcp(b); }
  static __device__ __forceinline__ void sqrt_and_rsqrt(F2 x, F2& a, F2& ia) {
    ia = F2(rsqrt_approx(x.v.x), rsqrt_approx(x.v.y));
    a = x * ia;
  }
  static __device__ __forceinline__ F2 sqrt_(F2 x) { return x * F2(rsqrt_approx(x.v.x), rsqrt_approx(x.v.y)); }
};

// Physics constants of one launch, as lane values.
template <typename V>
struct Phys {
  using S = typename LaneT<V>::S;
  V gamma, gm1, inv_gm1, beta, rdx, rdy;
  int riemann;
  __device__ __forceinline__ explicit Phys(const MeshDesc& m)
      : gamma(V(S(m.gamma))), gm1(V(S(m.gamma - 1.0))), inv_gm1(V(S(1) / S(m.gamma - 1.0))), beta(V(S(m.beta))),
        rdx(V(S(m.rdx))), rdy(V(S(m.rdy))), riemann(m.riemann) {}
};

// Conservative (rho, rho u, rho v, rho E, rho y_k) -> primitive
// (rho, u, v, p, y_k), eq. (1); y_k = (rho y_k) / rho.
template <typename V, int NF = 4>
__device__ __forceinline__ void to_prim(const Phys<V>& P, const V U[NF], V q[NF]) {
  const V ir = Ar<V>::rcp(U[0]);
  const V u = U[1] * ir, v = U[2] * ir;
  q[0] = U[0];
  q[1] = u;
  q[2] = v;
  q[3] = P.gm1 * fma_(splat<V>(-0.5), fma_(U[1], u, U[2] * v), U[3]);
#pragma unroll
  for (int k = 4; k < NF; ++k) q[k] = U[k] * ir;
}

// Half of the limited slope, phi(a,b)/2, so that the face states are
// q +/- limiter_half: eq. (sweby) for LIM_MINMOD / LIM_SWEBY, and van Leer's
// limiter (ab>0) 2ab/(a+b).  (Halving is exact in binary arithmetic, so this
// equals 0.5 * phi bit for bit.)
template <typename V, int LIM>
__device__ __forceinline__ V limiter_half(V a, V b, V beta) {
  const V ab = a * b;
  const auto pos = gt0(ab);
  if (LIM == LIM_VANLEER) {
    // one cell: the quotient is formed only where it is used (an IEEE FP64
    // division is a long instruction sequence); a pair computes both lanes
    if constexpr (LaneT<V>::N == 1) return pos ? Ar<V>::div(ab, a + b) : V(0);
    else return vsel(pos, Ar<V>::div(ab, a + b), splat<V>(0.0));
  } else {
    const V aa = vabs(a), bb = vabs(b);
    V m;
    if (LIM == LIM_MINMOD) m = vmin(aa, bb);
    else m = vmax(vmin(aa, beta * bb), vmin(beta * aa, bb));
    return vsel(pos, vcopysign(splat<V>(0.5) * m, a), splat<V>(0.0));
  }
}

// max(pL / rL, pR / rR) for rL, rR > 0.  A packed pair forms both quotients
// (two special-function instructions per component, cheap); one cell
// compares the cross products and forms only the larger quotient, which in
// FP64 saves an IEEE division (a long instruction sequence).  Equal cross
// products take the left quotient.
template <typename V>
__device__ __forceinline__ V max_quotient(V pL, V rL, V pR, V rR) {
  if constexpr (LaneT<V>::N == 1) return pL * rR >= pR * rL ? Ar<V>::div(pL, rL) : Ar<V>::div(pR, rR);
  else return vmax(Ar<V>::div(pL, rL), Ar<V>::div(pR, rR));
}

// Eqs. (13)-(14): star pressure and normal velocity at a face from the
// reconstructed left/right (rho, u_n, p); then eq. (12) with the upwind state
// chosen by the sign of u*.  DIR = 0: x-face (normal velocity u), 1: y-face.
// qL, qR are primitive (rho, u, v, p, y_k).  F receives the flux along +x /
// +y; a species row is (rho_A y_k,A) u*, the mass flux's upwind side.
template <typename V, int DIR, int NF = 4>
__device__ __forceinline__ void lagrange_flux(const Phys<V>& P, const V qL[NF], const V qR[NF], V F[NF]) {
  const V rL = qL[0], pL = qL[3], rR = qR[0], pR = qR[3];
  const V unL = qL[1 + DIR], unR = qR[1 + DIR];
  // jumps in both orientations: a product with a negated jump is exact, so
  // fma(x, -d, y) below rounds like y - x d
  const V ndu = unL - unR, ndp = pL - pR;
  V pstar, ustar;
  if (P.riemann == RIEMANN_MAXC) {
    // a = max(c_L, c_R) with c_k^2 = gamma p_k / rho_k; the larger c is the
    // larger c^2, so only one square root is needed.  With the weight
    // w = rho_L / (rho_L + rho_R), eqs. (13)-(14) read
    //   p* = p_L + w (p_R - p_L) - rho_R w a (u_R - u_L)
    //   u* = u_R - w (u_R - u_L) - (p_R - p_L) / ((rho_L + rho_R) a).
    const V a2 = P.gamma * max_quotient(pL, rL, pR, rR);
    V a, irs, irs_ia;  // a, 1/(rho_L + rho_R), 1/((rho_L + rho_R) a)
    if constexpr (LaneT<V>::N == 1 && sizeof(typename LaneT<V>::S) == 8) {
      // FP64: both reciprocals from one IEEE division (a division is a long
      // instruction sequence on the FP64 pipe)
      a = Ar<V>::sqrt_(a2);
      irs_ia = Ar<V>::rcp(a * (rL + rR));
      irs = a * irs_ia;
    } else {
      V ia;
      Ar<V>::sqrt_and_rsqrt(a2, a, ia);
      irs = Ar<V>::rcp(rL + rR);
      irs_ia = irs * ia;
    }
    const V w = rL * irs, dp = pR - pL;
    pstar = fma_(rR * w * a, ndu, fma_(w, dp, pL));
    ustar = fma_(ndp, irs_ia, fma_(w, ndu, unR));
  } else {
    // acoustic solver with Z_k = rho_k c_k
    const V ZL = rL * Ar<V>::sqrt_(P.gamma * Ar<V>::div(pL, rL));
    const V ZR = rR * Ar<V>::sqrt_(P.gamma * Ar<V>::div(pR, rR));
    const V iZ = Ar<V>::rcp(ZL + ZR);
    pstar = fma_(ZL * ZR * iZ, ndu, fma_(ZR, pL, ZL * pR) * iZ);
    ustar = fma_(ndp, iZ, fma_(ZL, unL, ZR * unR) * iZ);
  }
  const auto left = gt0(ustar);
  const V r = vsel(left, rL, rR);
  const V u = vsel(left, qL[1], qR[1]);
  const V v = vsel(left, qL[2], qR[2]);
  const V p = vsel(left, pL, pR);
  const V rE = fma_(p, P.inv_gm1, splat<V>(0.5) * r * fma_(u, u, v * v));
  const V m = r * ustar;
  F[0] = m;
  F[1] = m * u;
  F[2] = m * v;
  F[3] = (rE + pstar) * ustar;
  F[1 + DIR] = F[1 + DIR] + pstar;
#pragma unroll
  for (int k = 4; k < NF; ++k) F[k] = (r * vsel(left, qL[k], qR[k])) * ustar;
}

// Local CFL speed (|u|+c)/dx + (|v|+c)/dy (1D: (|u|+c)/dx) of a cell, and its
// positivity (rho > 0 and p > 0; false for NaN).
template <typename V, int DIM>
__device__ __forceinline__ V cell_speed(const Phys<V>& P, const V U[4], typename LaneT<V>::M& ok) {
  const V ir = Ar<V>::rcp(U[0]);
  const V u = U[1] * ir, v = U[2] * ir;
  const V p = P.gm1 * fma_(splat<V>(-0.5), fma_(U[1], u, U[2] * v), U[3]);
  ok = land(gt0(U[0]), gt0(p));
  const V c = Ar<V>::sqrt_(P.gamma * p * ir);
  V s = (vabs(u) + c) * P.rdx;
  if (DIM == 2) s = fma_(vabs(v) + c, P.rdy, s);
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
