"""Seeded synthetic initial conditions.

This module only draws and lays out primitive fields (rho, u, v, p, and
optionally mass fractions y_k) on cell centres; it holds none of the scheme's
arithmetic (no equation of state, no flux), so that the CUDA path and the CPU
oracle can both start from exactly the same input.  Every array is float64
with shape (ny, nx), x fastest; 1D problems have ny == 1.

Workloads:
  * shock tubes of Sec. 4.2 (Sod, two-rarefaction, sonic rarefaction,
    shock-shock) on [0, 1] with the interface at x = 0.5;
  * seeded four-quadrant 2D Riemann problems on [0, 1]^2;
  * a smooth density wave rho = 1 + 0.2 sin(2 pi (x + y)), u = v = 0.5, p = 1,
    whose exact solution is a translation;
  * a seeded Kelvin-Helmholtz shear layer;
  * seeded mesh sizes for batches of independent problems;
  * transported mass fractions (Sec. 5): a smooth scalar carried by a uniform
    flow (exact solution: a translation), a seeded three-region, two-material
    problem on the (0, 7) x (0, 3) vessel of the paper's triple-point case,
    and material indicators of the shear layer;
  * 3D: seeded eight-octant Riemann problems, a smooth density wave carried
    along the main diagonal, and a three-dimensional shear layer.
3D fields have shape (nz, ny, nx).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# (rho, u, p) left and right states of the shock tubes of Sec. 4.2.
SHOCK_TUBES = {
    "sod": ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1)),
    "two_rarefaction": ((1.0, -2.0, 0.4), (1.0, 2.0, 0.4)),
    "sonic_rarefaction": ((5.0, 0.0, 5.0), (0.125, 0.0, 0.1)),
    "shock_shock": ((1.0, 5.0, 1.0), (1.0, -5.0, 0.01)),
}


@dataclass
class Primitive:
    """Primitive fields on cell centres, each of shape (ny, nx)."""

    rho: np.ndarray
    u: np.ndarray
    v: np.ndarray
    p: np.ndarray
    y: np.ndarray | None = None  # mass fractions, shape (nspecies,) + field shape
    w: np.ndarray | None = None  # third velocity component (3D fields only)

    @property
    def nspecies(self) -> int:
        return 0 if self.y is None else int(self.y.shape[0])

    def stack(self) -> np.ndarray:
        """(4 + nspecies, ny, nx): rho, u, v, p, then y_1 .. y_nspecies;
        3D: (5 + nspecies, nz, ny, nx) with w after v."""
        planes = [self.rho, self.u, self.v] + ([self.w] if self.w is not None else []) + [self.p]
        if self.y is not None:
            planes += list(self.y)
        return np.stack(planes).astype(np.float64)

    @property
    def shape(self):
        return self.rho.shape


def cell_centres(n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    return lo + (np.arange(n, dtype=np.float64) + 0.5) * ((hi - lo) / n)


def shock_tube(nx: int, left, right, x0: float = 0.5) -> Primitive:
    """1D Riemann problem on [0, 1]: left state for x < x0, right state otherwise."""
    x = cell_centres(nx)
    is_left = x < x0
    rho = np.where(is_left, left[0], right[0])[None, :]
    u = np.where(is_left, left[1], right[1])[None, :]
    p = np.where(is_left, left[2], right[2])[None, :]
    return Primitive(rho.copy(), u.copy(), np.zeros_like(rho), p.copy())


def named_shock_tube(name: str, nx: int) -> Primitive:
    left, right = SHOCK_TUBES[name]
    return shock_tube(nx, left, right)


def quadrant_states(seed: int) -> np.ndarray:
    """Four constant states, rows in the order NE, NW, SW, SE, columns (rho, u, v, p).

    rho ~ U[0.5, 1.5], u, v ~ U[-0.75, 0.75], p ~ U[0.1, 1.0], drawn quadrant by
    quadrant in the order rho, u, v, p from numpy's default generator.
    """
    rng = np.random.default_rng(seed)
    out = np.empty((4, 4))
    for q in range(4):
        out[q, 0] = rng.uniform(0.5, 1.5)
        out[q, 1] = rng.uniform(-0.75, 0.75)
        out[q, 2] = rng.uniform(-0.75, 0.75)
        out[q, 3] = rng.uniform(0.1, 1.0)
    return out


def quadrant(nx: int, ny: int | None = None, seed: int = 0) -> Primitive:
    """Four-quadrant 2D Riemann problem on [0, 1]^2, split at x = y = 0.5."""
    ny = nx if ny is None else ny
    st = quadrant_states(seed)
    x = cell_centres(nx)[None, :]
    y = cell_centres(ny)[:, None]
    east, north = x >= 0.5, y >= 0.5
    idx = np.where(north & east, 0, np.where(north, 1, np.where(east, 3, 2)))
    return Primitive(st[idx, 0], st[idx, 1], st[idx, 2], st[idx, 3])


def smooth_wave(nx: int, ny: int | None = None, t: float = 0.0) -> Primitive:
    """rho = 1 + 0.2 sin(2 pi (x + y - t)), u = v = 0.5, p = 1 (periodic square).

    With u = v = 0.5 the exact solution at time t is the initial profile moved
    by (t/2, t/2), i.e. the phase x + y - t.
    """
    ny = nx if ny is None else ny
    x = cell_centres(nx)[None, :]
    y = cell_centres(ny)[:, None]
    rho = 1.0 + 0.2 * np.sin(2.0 * math.pi * (x + y - t))
    one = np.ones((ny, nx))
    return Primitive(rho, 0.5 * one, 0.5 * one, one.copy())


def smooth_wave_1d(nx: int, t: float = 0.0) -> Primitive:
    """rho = 1 + 0.2 sin(2 pi (x - t)), u = 1, p = 1 on the periodic unit interval."""
    x = cell_centres(nx)[None, :]
    rho = 1.0 + 0.2 * np.sin(2.0 * math.pi * (x - t))
    one = np.ones((1, nx))
    return Primitive(rho, one.copy(), np.zeros((1, nx)), one.copy())


def kelvin_helmholtz_profiles(nx: int, ny: int | None = None, seed: int = 0, amplitude: float = 0.01,
                              modes: int = 8):
    """The shear layer of kelvin_helmholtz as its 1D profiles: (rho_y, u_y,
    v_x, p) with rho_y, u_y of shape (ny,) (functions of y), v_x of shape
    (nx,) (a function of x) and the constant p; rho(j, i) = rho_y[j],
    u(j, i) = u_y[j], v(j, i) = v_x[i].  For meshes too large to lay out on
    the host."""
    ny = nx if ny is None else ny
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.0, 1.0, modes)
    phi = rng.uniform(0.0, 2.0 * math.pi, modes)
    x = cell_centres(nx)
    y = cell_centres(ny)
    k = np.arange(1, modes + 1)[:, None]
    S = (a[:, None] * np.sin(2.0 * math.pi * k * x[None, :] + phi[:, None])).sum(axis=0)
    vrow = amplitude * S / np.max(np.abs(S))
    inside = np.abs(y - 0.5) < 0.25
    return np.where(inside, 2.0, 1.0), np.where(inside, 0.5, -0.5), vrow, 2.5


def kelvin_helmholtz(nx: int, ny: int | None = None, seed: int = 0, amplitude: float = 0.01,
                     modes: int = 8) -> Primitive:
    """Shear layer: rho = 2, u = +0.5 inside |y - 0.5| < 0.25; rho = 1, u = -0.5 outside; p = 2.5.

    v = amplitude * S(x) / max|S| with S(x) = sum_{k=1..modes} a_k sin(2 pi k x + phi_k),
    a_k ~ U[0, 1], phi_k ~ U[0, 2 pi) drawn (all a_k, then all phi_k) from
    numpy's default generator.
    """
    ny = nx if ny is None else ny
    rho_y, u_y, v_x, p = kelvin_helmholtz_profiles(nx, ny, seed, amplitude, modes)
    rho = np.broadcast_to(rho_y[:, None], (ny, nx)).copy()
    u = np.broadcast_to(u_y[:, None], (ny, nx)).copy()
    v = np.broadcast_to(v_x[None, :], (ny, nx)).copy()
    return Primitive(rho, u, v, np.full((ny, nx), p))


def smooth_perturbation(nx: int, ny: int | None = None, seed: int = 0, modes: int = 4) -> np.ndarray:
    """Seeded smooth periodic field of unit max amplitude (a sum of low Fourier modes)."""
    ny = nx if ny is None else ny
    rng = np.random.default_rng(seed)
    x = cell_centres(nx)[None, :]
    y = cell_centres(ny)[:, None]
    f = np.zeros((ny, nx))
    for _ in range(modes):
        kx, ky = rng.integers(1, 4, size=2)
        ph = rng.uniform(0.0, 2.0 * math.pi)
        amp = rng.uniform(0.5, 1.0)
        f += amp * np.sin(2.0 * math.pi * (kx * x + ky * y) + ph)
    return f / np.max(np.abs(f))


def batched_sizes(nprob: int, seed: int = 0, lo: int = 64, hi: int = 1024) -> np.ndarray:
    """(nprob, 2) array of (nx, ny), each side round(exp(U[ln lo, ln hi])), drawn nx then ny."""
    rng = np.random.default_rng(seed)
    out = np.empty((nprob, 2), dtype=np.int64)
    for k in range(nprob):
        out[k, 0] = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        out[k, 1] = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
    return out


def with_species(prim: Primitive, y) -> Primitive:
    """The same flow carrying the mass fractions y (shape (nspecies,) + field shape)."""
    y = np.asarray(y, dtype=np.float64)
    if y.ndim == prim.rho.ndim:
        y = y[None]
    assert y.shape[1:] == prim.shape
    return Primitive(prim.rho, prim.u, prim.v, prim.p, y.copy(), prim.w)


def advected_scalar_1d(nx: int, t: float = 0.0) -> Primitive:
    """rho = 1, u = 1, p = 1 on the periodic unit interval carrying
    y = 0.5 + 0.4 sin(2 pi (x - t)): the exact solution at time t."""
    x = cell_centres(nx)[None, :]
    one = np.ones((1, nx))
    y = 0.5 + 0.4 * np.sin(2.0 * math.pi * (x - t))
    return Primitive(one.copy(), one.copy(), np.zeros((1, nx)), one.copy(), y[None])


def advected_scalar(nx: int, ny: int | None = None, t: float = 0.0) -> Primitive:
    """rho = 1, u = v = 0.5, p = 1 on the periodic unit square carrying
    y = 0.5 + 0.4 sin(2 pi (x + y - t)): the exact solution at time t."""
    ny = nx if ny is None else ny
    x = cell_centres(nx)[None, :]
    yc = cell_centres(ny)[:, None]
    one = np.ones((ny, nx))
    y = 0.5 + 0.4 * np.sin(2.0 * math.pi * (x + yc - t))
    return Primitive(one.copy(), 0.5 * one, 0.5 * one, one.copy(), y[None])


def advected_indicator(nx: int, ny: int | None = None) -> Primitive:
    """rho = 1, u = 0.6, v = -0.3, p = 1 (periodic unit square) carrying the
    indicator of the disc |(x, y) - (0.4, 0.6)| < 0.2."""
    ny = nx if ny is None else ny
    x = cell_centres(nx)[None, :]
    yc = cell_centres(ny)[:, None]
    one = np.ones((ny, nx))
    y = ((x - 0.4) ** 2 + (yc - 0.6) ** 2 < 0.04).astype(np.float64)
    return Primitive(one.copy(), 0.6 * one, -0.3 * one, one.copy(), y[None])


TRIPLE_DOMAIN = (7.0, 3.0)  # the vessel (0, 7) x (0, 3) of the triple-point case


def three_region_states(seed: int) -> np.ndarray:
    """Three resting states, rows for regions 1, 2, 3, columns (rho, p):
    rho ~ U[0.1, 1.0], p ~ U[0.1, 1.0], drawn region by region (rho, then p)."""
    rng = np.random.default_rng(seed)
    out = np.empty((3, 2))
    for r in range(3):
        out[r, 0] = rng.uniform(0.1, 1.0)
        out[r, 1] = rng.uniform(0.1, 1.0)
    return out


def three_region(nx: int, ny: int, seed: int = 0) -> Primitive:
    """Three-state, two-material problem on (0, 7) x (0, 3) at rest.

    Region 1 is x < 1, region 2 is x > 1, y < 1.5 and region 3 is x > 1,
    y > 1.5 (the layout of the triple-point case of Sec. 5; its geometry
    figure is not part of the text, so the split lines are this module's
    choice).  States are seeded.  Material A fills regions 1 and 3 and
    material B region 2; y_1 and y_2 are their indicators (y_1 + y_2 = 1).
    """
    lx, ly = TRIPLE_DOMAIN
    st = three_region_states(seed)
    x = cell_centres(nx, 0.0, lx)[None, :] * np.ones((ny, 1))
    yc = cell_centres(ny, 0.0, ly)[:, None] * np.ones((1, nx))
    region = np.where(x < 1.0, 0, np.where(yc < 1.5, 1, 2))
    zero = np.zeros((ny, nx))
    yA = (region != 1).astype(np.float64)
    return Primitive(st[region, 0], zero.copy(), zero.copy(), st[region, 1], np.stack([yA, 1.0 - yA]))


def shear_layer_tracers(nx: int, ny: int | None = None, seed: int = 0, nspecies: int = 2) -> Primitive:
    """The Kelvin-Helmholtz shear layer carrying nspecies mass fractions: y_1 is
    the indicator of the layer |y - 0.5| < 0.25, y_2 = 1 - y_1, and further
    species (if any) are smooth seeded fields in [0.1, 0.9]."""
    ny = nx if ny is None else ny
    kh = kelvin_helmholtz(nx, ny, seed=seed)
    yc = cell_centres(ny)[:, None] * np.ones((1, nx))
    inside = (np.abs(yc - 0.5) < 0.25).astype(np.float64)
    ys = [inside, 1.0 - inside]
    for k in range(2, nspecies):
        ys.append(0.5 + 0.4 * smooth_perturbation(nx, ny, seed=seed * 31 + k))
    return with_species(kh, np.stack(ys[:nspecies]))


# ---------------------------------------------------------------------------
# 3D fields, shape (nz, ny, nx) on the unit cube unless stated
# ---------------------------------------------------------------------------
def _grid3(nx: int, ny: int, nz: int):
    x = cell_centres(nx)[None, None, :]
    y = cell_centres(ny)[None, :, None]
    z = cell_centres(nz)[:, None, None]
    return x, y, z


def octant_states(seed: int) -> np.ndarray:
    """Eight constant states, rows for octants o = 4 [z >= 1/2] + 2 [y >= 1/2] + [x >= 1/2],
    columns (rho, u, v, w, p): rho ~ U[0.5, 1.5], u, v, w ~ U[-0.75, 0.75],
    p ~ U[0.1, 1.0], drawn octant by octant in that order."""
    rng = np.random.default_rng(seed)
    out = np.empty((8, 5))
    for o in range(8):
        out[o, 0] = rng.uniform(0.5, 1.5)
        out[o, 1:4] = [rng.uniform(-0.75, 0.75) for _ in range(3)]
        out[o, 4] = rng.uniform(0.1, 1.0)
    return out


def octant(nx: int, ny: int | None = None, nz: int | None = None, seed: int = 0) -> Primitive:
    """Eight-octant 3D Riemann problem on [0, 1]^3, split at x = y = z = 0.5."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    st = octant_states(seed)
    x, y, z = _grid3(nx, ny, nz)
    o = 4 * (z >= 0.5) + 2 * (y >= 0.5) + (x >= 0.5)
    o = np.broadcast_to(o, (nz, ny, nx))
    return Primitive(st[o, 0], st[o, 1], st[o, 2], st[o, 4], None, st[o, 3])


def smooth_wave_3d(nx: int, ny: int | None = None, nz: int | None = None, t: float = 0.0) -> Primitive:
    """rho = 1 + 0.2 sin(2 pi (x + y + z - t)), u = v = w = 1/3, p = 1 (periodic
    cube): the exact solution at time t is the initial profile moved by t/3
    along each axis."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    x, y, z = _grid3(nx, ny, nz)
    rho = 1.0 + 0.2 * np.sin(2.0 * math.pi * (x + y + z - t))
    one = np.ones((nz, ny, nx))
    return Primitive(rho * one, one / 3.0, one / 3.0, one.copy(), None, one / 3.0)


def shear_layer_3d(nx: int, ny: int | None = None, nz: int | None = None, seed: int = 0,
                   amplitude: float = 0.01, modes: int = 8) -> Primitive:
    """The Kelvin-Helmholtz layer of kelvin_helmholtz (rho 2 / u +0.5 inside
    |y - 0.5| < 0.25, rho 1 / u -0.5 outside, p 2.5) with the seeded
    perturbation v = amplitude S(x) / max|S| of that function times
    cos(2 pi z), and w = 0."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    kh = kelvin_helmholtz(nx, ny, seed=seed, amplitude=amplitude, modes=modes)
    z = cell_centres(nz)[:, None, None]
    one = np.ones((nz, ny, nx))
    v = kh.v[None] * np.cos(2.0 * math.pi * z)
    return Primitive(kh.rho[None] * one, kh.u[None] * one, v * one, kh.p[None] * one, None, np.zeros((nz, ny, nx)))
