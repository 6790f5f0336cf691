"""Exact solution of the 1D Riemann problem for the ideal-gas Euler equations.

TEST INFRASTRUCTURE ONLY.  The paper compares its shock-tube results with the
exact solution (Sec. 4.2, all four tubes); this module supplies that
solution so the oracle can be pinned against it.  It follows the classical
construction in Toro's book (cited by the paper as [Toro], ch. 4):

* the star pressure p* is the root of f(p) = f_L(p) + f_R(p) + (u_R - u_L),
  where f_K is the shock (Rankine-Hugoniot) branch for p > p_K and the
  rarefaction (isentropic) branch for p <= p_K; f is increasing in p, so the
  root is bracketed and found by bisection-type root finding;
* u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2;
* the solution is self-similar in xi = (x - x0)/t and is sampled wave by wave.

It is pinned independently in tests/test_exact_riemann.py by the jump
conditions it must satisfy (Rankine-Hugoniot across shocks, constant entropy
and Riemann invariant through rarefactions, continuous p and u across the
contact), by symmetric problems, and by the small-amplitude acoustic limit.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.optimize import brentq


@dataclass(frozen=True)
class State:
    rho: float
    u: float
    p: float

    def c(self, gamma: float) -> float:
        return math.sqrt(gamma * self.p / self.rho)


def _f_side(p: float, s: State, g: float) -> float:
    """Velocity change across the wave that joins state s to pressure p."""
    if p > s.p:  # shock branch (Rankine-Hugoniot)
        A = 2.0 / ((g + 1.0) * s.rho)
        B = (g - 1.0) / (g + 1.0) * s.p
        return (p - s.p) * math.sqrt(A / (p + B))
    # rarefaction branch (isentropic)
    return 2.0 * s.c(g) / (g - 1.0) * ((p / s.p) ** ((g - 1.0) / (2.0 * g)) - 1.0)


@dataclass(frozen=True)
class StarRegion:
    p: float
    u: float
    rho_L: float
    rho_R: float


def star_region(L: State, R: State, gamma: float = 1.4) -> StarRegion:
    g = gamma
    if 2.0 / (g - 1.0) * (L.c(g) + R.c(g)) <= R.u - L.u:
        raise ValueError("initial data generate vacuum")

    def f(p):
        return _f_side(p, L, g) + _f_side(p, R, g) + (R.u - L.u)

    lo, hi = 1e-14 * min(L.p, R.p), max(L.p, R.p)
    while f(hi) < 0.0:
        hi *= 2.0
    pstar = brentq(f, lo, hi, xtol=1e-300, rtol=4 * np.finfo(float).eps, maxiter=500)
    ustar = 0.5 * (L.u + R.u) + 0.5 * (_f_side(pstar, R, g) - _f_side(pstar, L, g))

    def rho_star(s: State) -> float:
        if pstar > s.p:
            r = (g - 1.0) / (g + 1.0)
            return s.rho * (pstar / s.p + r) / (r * pstar / s.p + 1.0)
        return s.rho * (pstar / s.p) ** (1.0 / g)

    return StarRegion(pstar, ustar, rho_star(L), rho_star(R))


def wave_speeds(L: State, R: State, gamma: float = 1.4) -> dict:
    """Speeds of the wave fronts (shock speed, or head and tail of a fan)."""
    g = gamma
    st = star_region(L, R, g)
    out = {"contact": st.u}
    if st.p > L.p:
        out["left_shock"] = L.u - L.c(g) * math.sqrt((g + 1) / (2 * g) * st.p / L.p + (g - 1) / (2 * g))
    else:
        out["left_head"] = L.u - L.c(g)
        out["left_tail"] = st.u - L.c(g) * (st.p / L.p) ** ((g - 1) / (2 * g))
    if st.p > R.p:
        out["right_shock"] = R.u + R.c(g) * math.sqrt((g + 1) / (2 * g) * st.p / R.p + (g - 1) / (2 * g))
    else:
        out["right_head"] = R.u + R.c(g)
        out["right_tail"] = st.u + R.c(g) * (st.p / R.p) ** ((g - 1) / (2 * g))
    return out


def sample(L: State, R: State, xi, gamma: float = 1.4):
    """Primitive solution (rho, u, p) at similarity coordinates xi = (x-x0)/t."""
    g = gamma
    st = star_region(L, R, g)
    ws = wave_speeds(L, R, g)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    cL, cR = L.c(g), R.c(g)
    for k, s in np.ndenumerate(xi):
        if s <= st.u:  # left of the contact
            if st.p > L.p:
                val = (L.rho, L.u, L.p) if s <= ws["left_shock"] else (st.rho_L, st.u, st.p)
            elif s <= ws["left_head"]:
                val = (L.rho, L.u, L.p)
            elif s >= ws["left_tail"]:
                val = (st.rho_L, st.u, st.p)
            else:  # inside the left fan
                uf = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * L.u + s)
                cf = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * (L.u - s))
                val = (L.rho * (cf / cL) ** (2.0 / (g - 1.0)), uf, L.p * (cf / cL) ** (2.0 * g / (g - 1.0)))
        else:  # right of the contact
            if st.p > R.p:
                val = (R.rho, R.u, R.p) if s >= ws["right_shock"] else (st.rho_R, st.u, st.p)
            elif s >= ws["right_head"]:
                val = (R.rho, R.u, R.p)
            elif s <= ws["right_tail"]:
                val = (st.rho_R, st.u, st.p)
            else:  # inside the right fan
                uf = 2.0 / (g + 1.0) * (-cR + 0.5 * (g - 1.0) * R.u + s)
                cf = 2.0 / (g + 1.0) * (cR - 0.5 * (g - 1.0) * (R.u - s))
                val = (R.rho * (cf / cR) ** (2.0 / (g - 1.0)), uf, R.p * (cf / cR) ** (2.0 * g / (g - 1.0)))
        rho[k], u[k], p[k] = val
    return rho, u, p


def solution_on_cells(L: State, R: State, nx: int, t: float, x0: float = 0.5, gamma: float = 1.4,
                      xmin: float = 0.0, xmax: float = 1.0, sub: int = 8):
    """Cell averages (by `sub`-point midpoint sampling) of the exact solution."""
    dx = (xmax - xmin) / nx
    offs = (np.arange(sub) + 0.5) / sub
    x = xmin + (np.arange(nx)[:, None] + offs[None, :]) * dx
    rho, u, p = sample(L, R, (x - x0) / t, gamma)
    return rho.mean(axis=1), u.mean(axis=1), p.mean(axis=1)
