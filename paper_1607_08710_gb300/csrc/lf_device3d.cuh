// Device arithmetic of the three-dimensional Lagrange-flux step
// (arXiv:1607.08710: eq. 1 with a third velocity component, eqs. 12-14 on
// faces normal to x, y or z).  A 3D cell carries NF = 5 + nspecies fields,
// (rho, rho u, rho v, rho w, rho E, rho y_k); its primitive state is
// (rho, u, v, w, p, y_k).  Lane values, rounding and the limiter are those of
// lf_device.cuh.
#pragma once

#include "lf_device.cuh"

namespace lf {

// Conservative -> primitive, eq. (1): p = (gamma-1) (rho E - |rho u|^2 / (2 rho)).
template <typename V, int NF>
__device__ __forceinline__ void to_prim3(const Phys<V>& P, const V U[NF], V q[NF]) {
  const V ir = Ar<V>::rcp(U[0]);
  const V u = U[1] * ir, v = U[2] * ir, w = U[3] * ir;
  q[0] = U[0];
  q[1] = u;
  q[2] = v;
  q[3] = w;
  q[4] = P.gm1 * fma_(splat<V>(-0.5), fma_(U[1], u, fma_(U[2], v, U[3] * w)), U[4]);
#pragma unroll
  for (int k = 5; k < NF; ++k) q[k] = U[k] * ir;
}

// Eqs. (13)-(14) and (12) on a face normal to axis DIR (0 = x, 1 = y, 2 = z),
// from the reconstructed primitive states qL, qR; F is the flux along +DIR.
// The same arithmetic as lagrange_flux, with w and the 3D field order.
template <typename V, int DIR, int NF>
__device__ __forceinline__ void lagrange_flux3(const Phys<V>& P, const V qL[NF], const V qR[NF], V F[NF]) {
  const V rL = qL[0], pL = qL[4], rR = qR[0], pR = qR[4];
  const V unL = qL[1 + DIR], unR = qR[1 + DIR];
  const V ndu = unL - unR, ndp = pL - pR;
  V pstar, ustar;
  if (P.riemann == RIEMANN_MAXC) {
    const V a2 = P.gamma * max_quotient(pL, rL, pR, rR);
    V a, irs, irs_ia;  // as lagrange_flux
    if constexpr (LaneT<V>::N == 1 && sizeof(typename LaneT<V>::S) == 8) {
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
  const V wv = vsel(left, qL[3], qR[3]);
  const V p = vsel(left, pL, pR);
  const V rE = fma_(p, P.inv_gm1, splat<V>(0.5) * r * fma_(u, u, fma_(v, v, wv * wv)));
  const V m = r * ustar;
  F[0] = m;
  F[1] = m * u;
  F[2] = m * v;
  F[3] = m * wv;
  F[4] = (rE + pstar) * ustar;
  F[1 + DIR] = F[1 + DIR] + pstar;
#pragma unroll
  for (int k = 5; k < NF; ++k) F[k] = (r * vsel(left, qL[k], qR[k])) * ustar;
}

// Local CFL speed (|u|+c)/dx + (|v|+c)/dy + (|w|+c)/dz and positivity.
template <typename V>
__device__ __forceinline__ V cell_speed3(const Phys<V>& P, V rdz, const V U[5], typename LaneT<V>::M& ok) {
  const V ir = Ar<V>::rcp(U[0]);
  const V u = U[1] * ir, v = U[2] * ir, w = U[3] * ir;
  const V p = P.gm1 * fma_(splat<V>(-0.5), fma_(U[1], u, fma_(U[2], v, U[3] * w)), U[4]);
  ok = land(gt0(U[0]), gt0(p));
  const V c = Ar<V>::sqrt_(P.gamma * p * ir);
  V s = (vabs(u) + c) * P.rdx;
  s = fma_(vabs(v) + c, P.rdy, s);
  return fma_(vabs(w) + c, rdz, s);
}

}  // namespace lf
