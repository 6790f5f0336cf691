// CPU oracle for the second-order Lagrange-flux scheme of De Vuyst, Gasc,
// Motte, Peybernes and Poncet, "Lagrange-flux schemes: reformulating
// second-order accurate Lagrange-remap schemes for better node-based HPC
// performance" (arXiv:1607.08710).
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
// reference that the CUDA path is checked against.  Only the test suite, the
// smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
// no code, header, table or constant with the CUDA library, and it includes
// nothing from it.
//
// Everything is FP64 (or a forward-mode dual number built on FP64), single
// threaded, with one loop per step of the paper's Heun algorithm (Sec. 4) and
// every face flux stored before any cell is updated.  Compiled with
// -ffp-contract=off so that no fused multiply-add changes the rounding.
//
// The `#pragma omp` lines act only in a second build of this same file with
// -fopenmp, used to time the oracle on all host cores beside the GPU.  Every
// loop they split writes each element from one iteration, and the only
// reductions are a logical AND and an exact maximum, so that build returns
// the same bits as the plain single-threaded one.
//
// Readings of points where the paper is silent (the CUDA library takes the
// same readings):
//   * CFL condition (Sec. 4, Heun step 1 requires a CFL condition without
//     writing it out): dt = CFL / max_K sum_d (|u_d,K| + c_K) / dx_d over the
//     mesh's axes (1D: x; 2D: x, y; 3D: x, y, z), from U^n, the same dt for
//     all stages; clipped to t_end - t when a final time is given.
//   * Three dimensions (the finite-volume form of Sec. 4 is written for any
//     polygonal/polyhedral cell): the same face formulas with a third flux
//     direction; the state gains rho w, the primitive state w.
//   * MUSCL (Sec. 4, eq. "sweby" and Heun step 2): limited undivided slopes of
//     the primitive variables (rho, u, v, [w,] p), direction by direction,
//     with face values q_i +/- sigma_i / 2.
//   * Upwind edge value (eq. 12 and Heun step 4): the conservative vector
//     rebuilt from the primitive state reconstructed on the upwind side,
//     L if u* > 0, else R.
//   * Ghost cells: two layers; transmissive = copy of the boundary cell,
//     periodic = wrap-around.
//   * Species (Sec. 5, conservative form of the mass-fraction transport):
//     each mass fraction y_k = (rho y_k)/rho is one more primitive variable,
//     reconstructed with the same limiter as (rho, u, v, p); the edge value of
//     rho y_k is rebuilt from the upwind primitive state like the other
//     conservative variables, so its flux is (rho_A y_k,A) u*.  The species do
//     not enter the pressure, the sound speed or the CFL condition (one gamma
//     for the mixture).
//   * Derivative conventions for the dual number at non-smooth points:
//     max/min pick the first argument on ties, the limiter is 0 (with zero
//     derivative) when ab <= 0, and the upwind branch follows the value of u*.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------------------
// Scalar types: plain double, and a forward-mode dual number (value and one
// tangent) used to compute exact directional derivatives of the scheme.
// ---------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual sqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}

inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
inline double sq_root(double x) { return std::sqrt(x); }
inline Dual sq_root(const Dual& x) { return sqrt(x); }

// Op-counting scalar: a double that tallies each arithmetic operation it
// takes part in (add or subtract, multiply, divide, square root), used only to
// count the method's flops per cell (oracle_count_ops), never to step.
// Negation, absolute values, comparisons and sign tests are not counted.
struct OpTally {
  double add = 0, mul = 0, div = 0, sqrt = 0;
};
OpTally g_tally;
struct Counted {
  double v;
  Counted() : v(0) {}
  Counted(double x) : v(x) {}
};
inline Counted operator+(Counted a, Counted b) { g_tally.add += 1; return Counted(a.v + b.v); }
inline Counted operator-(Counted a, Counted b) { g_tally.add += 1; return Counted(a.v - b.v); }
inline Counted operator-(Counted a) { return Counted(-a.v); }
inline Counted operator*(Counted a, Counted b) { g_tally.mul += 1; return Counted(a.v * b.v); }
inline Counted operator/(Counted a, Counted b) { g_tally.div += 1; return Counted(a.v / b.v); }
inline double val(const Counted& x) { return x.v; }
inline Counted sq_root(const Counted& x) { g_tally.sqrt += 1; return Counted(std::sqrt(x.v)); }

template <class S> inline S abs_s(const S& a) { return val(a) < 0.0 ? S(-a) : a; }
// First argument on ties.
template <class S> inline S max_first(const S& a, const S& b) { return val(a) >= val(b) ? a : b; }
template <class S> inline S min_first(const S& a, const S& b) { return val(a) <= val(b) ? a : b; }

// ---------------------------------------------------------------------------
// Configuration, mirrored field by field by the ctypes structure in oracle.py.
// ---------------------------------------------------------------------------
enum { LIM_MINMOD = 0, LIM_SWEBY = 1, LIM_VANLEER = 2 };
enum { BC_TRANSMISSIVE = 0, BC_PERIODIC = 1 };
enum { RIEMANN_MAXC = 0, RIEMANN_PER_SIDE = 1 };
enum { ORC_OK = 0, ORC_NONPHYSICAL = 1, ORC_ARG = 2 };

constexpr int MAX_SPECIES = 8;
constexpr int MAXF = 5 + MAX_SPECIES;  // largest number of transported fields

struct OracleConfig {
  int32_t dim;      // 1, 2 or 3
  int32_t nx, ny;   // cells (ny == 1 when dim == 1)
  int32_t limiter;  // LIM_*
  int32_t bc;       // BC_*
  int32_t riemann;  // RIEMANN_*
  double dx, dy;    // cell sizes (dy unused in 1D)
  double gamma;     // perfect-gas ratio of specific heats, in (1, 3]
  double cfl;       // CFL number
  double beta;      // Sweby coefficient, in [1, 2]
  int32_t time_order;  // 2: Heun (Sec. 4); 3: third-order SSP Runge-Kutta
  int32_t nspecies;    // transported mass fractions (Sec. 5), 0 .. MAX_SPECIES
  int32_t nz;          // cells in z (1 unless dim == 3)
  int32_t pad;
  double dz;           // cell size in z (dim == 3)
};

// Velocity components carried: (u, v) in 1D and 2D (v = 0 in 1D), (u, v, w) in 3D.
inline int nvel(const OracleConfig& c) { return c.dim == 3 ? 3 : 2; }
// Index of rho E in the conservative vector and of p in the primitive one.
inline int ien(const OracleConfig& c) { return 1 + nvel(c); }
// Fields per cell: (rho, rho u, rho v, [rho w,] rho E, rho y_1 .. rho y_nspecies).
inline int nfields(const OracleConfig& c) { return 2 + nvel(c) + c.nspecies; }

bool config_ok(const OracleConfig* c) {
  if (!c) return false;
  if (c->dim < 1 || c->dim > 3) return false;
  if (c->nx < 1 || c->ny < 1 || c->nz < 1) return false;
  if (c->dim == 1 && c->ny != 1) return false;
  if (c->dim < 3 && c->nz != 1) return false;
  if (c->dim == 3 && !(c->dz > 0)) return false;
  if (c->limiter < 0 || c->limiter > 2) return false;
  if (c->bc < 0 || c->bc > 1) return false;
  if (c->riemann < 0 || c->riemann > 1) return false;
  if (!(c->dx > 0) || (c->dim >= 2 && !(c->dy > 0))) return false;
  if (!(c->gamma > 1.0)) return false;
  if (c->time_order != 2 && c->time_order != 3) return false;
  if (c->nspecies < 0 || c->nspecies > MAX_SPECIES) return false;
  return true;
}

// ---------------------------------------------------------------------------
// Eq. (1): perfect-gas EOS p = (gamma-1) rho (E - |u|^2/2), c = sqrt(gamma p / rho).
// Primitive vector q = (rho, u, v, [w,] p, y_1 ..); conservative
// U = (rho, rho u, rho v, [rho w,] rho E, rho y_1 ..), nfields(c) entries each.
// ---------------------------------------------------------------------------
template <class S>
void prim_from_cons(const OracleConfig& c, const S U[], S q[]) {
  const int nv = nvel(c), e = ien(c);
  S rho = U[0];
  S kin = S(0.0);  // |u|^2
  for (int d = 0; d < nv; ++d) {
    q[1 + d] = U[1 + d] / rho;
    kin = kin + q[1 + d] * q[1 + d];
  }
  S E = U[e] / rho;
  q[0] = rho;
  q[e] = (c.gamma - 1.0) * rho * (E - 0.5 * kin);
  for (int k = 0; k < c.nspecies; ++k) q[e + 1 + k] = U[e + 1 + k] / rho;
}

template <class S>
void cons_from_prim(const OracleConfig& c, const S q[], S U[]) {
  const int nv = nvel(c), e = ien(c);
  S rho = q[0], p = q[e];
  S kin = S(0.0);
  U[0] = rho;
  for (int d = 1; d <= nv; ++d) {
    U[d] = rho * q[d];
    kin = kin + q[d] * q[d];
  }
  U[e] = p / (c.gamma - 1.0) + 0.5 * rho * kin;
  for (int k = 0; k < c.nspecies; ++k) U[e + 1 + k] = rho * q[e + 1 + k];
}

template <class S>
S sound_speed(const OracleConfig& c, const S& rho, const S& p) {
  return sq_root(c.gamma * p / rho);
}

// ---------------------------------------------------------------------------
// Eq. (sweby): phi(a,b) = (ab>0) sign(a) max(min(|a|, beta|b|), min(beta|a|, |b|)),
// beta in [1,2]; beta = 1 is minmod (Sec. 4.2, last shock tube).  The van Leer
// limiter (ab>0) 2ab/(a+b) is the one other classical limiter offered.
// ---------------------------------------------------------------------------
template <class S>
S limiter(const OracleConfig& c, const S& a, const S& b) {
  if (!(val(a) * val(b) > 0.0)) return S(0.0);
  if (c.limiter == LIM_VANLEER) return 2.0 * a * b / (a + b);
  double beta = (c.limiter == LIM_MINMOD) ? 1.0 : c.beta;
  S aa = abs_s(a), bb = abs_s(b);
  S m = max_first(min_first(aa, S(beta * bb)), min_first(S(beta * aa), bb));
  return val(a) > 0.0 ? m : S(-m);
}

// ---------------------------------------------------------------------------
// Sec. 4.1, eqs. (13)-(14): Lagrangian HLL / acoustic interface solver.
//   p* = (rho_R p_L + rho_L p_R)/(rho_L+rho_R)
//        - rho_L rho_R/(rho_L+rho_R) max(c_L,c_R) (u_R - u_L)
//   u* = (rho_L u_L + rho_R u_R)/(rho_L+rho_R)
//        - (p_R - p_L) / ((rho_L+rho_R) max(c_L,c_R))
// u_L, u_R are the velocities normal to the face.  The per-side variant uses
// the impedances Z_k = rho_k c_k in the same acoustic formulas.
// ---------------------------------------------------------------------------
template <class S>
void interface_solve(const OracleConfig& c, const S& rL, const S& uL, const S& pL,
                     const S& rR, const S& uR, const S& pR, S& pstar, S& ustar) {
  S cL = sound_speed(c, rL, pL);
  S cR = sound_speed(c, rR, pR);
  if (c.riemann == RIEMANN_MAXC) {
    S a = max_first(cL, cR);
    S rs = rL + rR;
    pstar = (rR * pL + rL * pR) / rs - (rL * rR / rs) * a * (uR - uL);
    ustar = (rL * uL + rR * uR) / rs - (pR - pL) / (rs * a);
  } else {
    S ZL = rL * cL, ZR = rR * cR;
    S Zs = ZL + ZR;
    pstar = (ZR * pL + ZL * pR) / Zs - (ZL * ZR / Zs) * (uR - uL);
    ustar = (ZL * uL + ZR * uR) / Zs - (pR - pL) / Zs;
  }
}

// ---------------------------------------------------------------------------
// Eq. (12) with the upwinding of Sec. 4 (Heun steps 3-5): for a face with unit
// normal nu along axis `dir` (0 = x, 1 = y, 2 = z), pointing from L to R,
//   Phi = U_A (u* ) + (0, p* nu, p* u*),
// U_A = U(q_L) if u* > 0 else U(q_R).  The species rows of Phi are
// (rho y_k)_A u*, with no pressure term.
// ---------------------------------------------------------------------------
template <class S>
void face_flux(const OracleConfig& c, int dir, const S qL[], const S qR[], S F[]) {
  const int e = ien(c);
  S pstar, ustar;
  interface_solve(c, qL[0], qL[1 + dir], qL[e], qR[0], qR[1 + dir], qR[e], pstar, ustar);
  const S* qup = (val(ustar) > 0.0) ? qL : qR;
  S Uup[MAXF];
  cons_from_prim(c, qup, Uup);
  for (int l = 0; l < nfields(c); ++l) F[l] = Uup[l] * ustar;
  F[1 + dir] = F[1 + dir] + pstar;
  F[e] = F[e] + pstar * ustar;
}

// ---------------------------------------------------------------------------
// Mesh bookkeeping: planes of nx*ny*nz values, x fastest (index
// (k*ny + j)*nx + i).  Ghost-extended primitive arrays carry G = 2 layers on
// each active axis (x; x, y; or x, y, z).  Inactive axes have one cell, no
// ghosts and size 1.
// ---------------------------------------------------------------------------
const int G = 2;

inline int wrap_index(int i, int n, int bc) {
  if (bc == BC_PERIODIC) {
    int r = i % n;
    return r < 0 ? r + n : r;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

template <class S>
struct Mesh {
  const OracleConfig& c;
  int n[3];      // cells per axis
  int g[3];      // ghost layers per axis
  int ext[3];    // ghost-extended extents
  double h[3];   // cell sizes
  explicit Mesh(const OracleConfig& cfg) : c(cfg) {
    n[0] = cfg.nx;
    n[1] = cfg.ny;
    n[2] = cfg.nz;
    h[0] = cfg.dx;
    h[1] = cfg.dim >= 2 ? cfg.dy : 1.0;
    h[2] = cfg.dim == 3 ? cfg.dz : 1.0;
    for (int d = 0; d < 3; ++d) {
      g[d] = d < cfg.dim ? G : 0;
      ext[d] = n[d] + 2 * g[d];
    }
  }
  size_t ncell() const { return (size_t)n[0] * n[1] * n[2]; }
  size_t cell(int i, int j, int k) const { return ((size_t)k * n[1] + j) * n[0] + i; }
  // ghost-extended index of interior-relative cell (i, j, k)
  size_t gidx(int i, int j, int k) const {
    return ((size_t)(k + g[2]) * ext[1] + (j + g[1])) * ext[0] + (i + g[0]);
  }
  // Faces normal to axis d: n[d] + 1 of them along d; face (i, j, k) lies
  // between the cell one step back along d and cell (i, j, k).
  size_t nfaces(int d) const { return (size_t)(n[0] + (d == 0)) * (n[1] + (d == 1)) * (n[2] + (d == 2)); }
  size_t fidx(int d, int i, int j, int k) const {
    return ((size_t)k * (n[1] + (d == 1)) + j) * (n[0] + (d == 0)) + i;
  }
};

// Builds the ghost-extended primitive field from the conservative planes.
template <class S>
bool build_primitives(const Mesh<S>& m, const std::vector<S> U[], std::vector<S> qg[]) {
  const OracleConfig& c = m.c;
  const int nf = nfields(c);
  for (int l = 0; l < nf; ++l) qg[l].assign((size_t)m.ext[0] * m.ext[1] * m.ext[2], S(0.0));
  bool physical = true;
#pragma omp parallel for collapse(2) reduction(&& : physical)
  for (int k = -m.g[2]; k < m.n[2] + m.g[2]; ++k)
    for (int j = -m.g[1]; j < m.n[1] + m.g[1]; ++j)
      for (int i = -m.g[0]; i < m.n[0] + m.g[0]; ++i) {
        // A ghost cell takes the primitive state of the interior cell it maps to.
        size_t s = m.cell(wrap_index(i, m.n[0], c.bc), wrap_index(j, m.n[1], c.bc), wrap_index(k, m.n[2], c.bc));
        S Uc[MAXF], q[MAXF];
        for (int l = 0; l < nf; ++l) Uc[l] = U[l][s];
        prim_from_cons(c, Uc, q);
        if (!(val(q[0]) > 0.0) || !(val(q[ien(c)]) > 0.0)) physical = false;
        size_t gi = m.gidx(i, j, k);
        for (int l = 0; l < nf; ++l) qg[l][gi] = q[l];
      }
  return physical;
}

// All face fluxes of a state (Heun steps 2-5, or 7-10): F[d][l] holds field
// l's flux through every face normal to axis d (indexed by Mesh::fidx).
template <class S>
bool all_face_fluxes(const Mesh<S>& m, const std::vector<S> U[], std::vector<S> F[3][MAXF]) {
  const OracleConfig& c = m.c;
  const int nf = nfields(c);
  std::vector<S> qg[MAXF];
  bool physical = build_primitives(m, U, qg);
  // primitive l of the cell s steps along axis d from cell (i, j, k)
  auto q_at = [&](int l, int d, int s, int i, int j, int k) -> S {
    int o[3] = {i, j, k};
    o[d] += s;
    return qg[l][m.gidx(o[0], o[1], o[2])];
  };
  for (int d = 0; d < c.dim; ++d) {
    for (int l = 0; l < nf; ++l) F[d][l].assign(m.nfaces(d), S(0.0));
    int e[3] = {m.n[0], m.n[1], m.n[2]};
    e[d] += 1;
#pragma omp parallel for collapse(2)
    for (int k = 0; k < e[2]; ++k)
      for (int j = 0; j < e[1]; ++j)
        for (int i = 0; i < e[0]; ++i) {
          // left cell: one step back along d; right cell: (i, j, k)
          S qL[MAXF], qR[MAXF];
          for (int l = 0; l < nf; ++l) {
            S sL = limiter(c, q_at(l, d, -1, i, j, k) - q_at(l, d, -2, i, j, k),
                           q_at(l, d, 0, i, j, k) - q_at(l, d, -1, i, j, k));
            S sR = limiter(c, q_at(l, d, 0, i, j, k) - q_at(l, d, -1, i, j, k),
                           q_at(l, d, 1, i, j, k) - q_at(l, d, 0, i, j, k));
            qL[l] = q_at(l, d, -1, i, j, k) + 0.5 * sL;
            qR[l] = q_at(l, d, 0, i, j, k) - 0.5 * sR;
          }
          S Fv[MAXF];
          face_flux(c, d, qL, qR, Fv);
          for (int l = 0; l < nf; ++l) F[d][l][m.fidx(d, i, j, k)] = Fv[l];
        }
  }
  return physical;
}

// Sum over the faces of cell K of |A| Phi_A . nu_A (outward), divided by |K|
// (Sec. 4, semi-discrete scheme after eq. 11).  Fluxes are stored with the
// normal pointing along +d; the face behind the cell enters with a minus sign.
template <class S>
S flux_balance(const Mesh<S>& m, const std::vector<S> F[3][MAXF], int l, int i, int j, int k) {
  const double K = m.h[0] * m.h[1] * m.h[2];
  S acc = S(0.0);
  for (int d = 0; d < m.c.dim; ++d) {
    const double A = m.h[(d + 1) % 3] * m.h[(d + 2) % 3];
    int hi[3] = {i, j, k};
    hi[d] += 1;
    S ahead = F[d][l][m.fidx(d, hi[0], hi[1], hi[2])], behind = F[d][l][m.fidx(d, i, j, k)];
    acc = acc + A * ahead - A * behind;
  }
  return acc / K;
}

// The CFL reading stated at the top of this file: sum over the mesh's axes
// of (|u_d| + c) / dx_d for one cell's primitive state q.
template <class S>
S wave_speed_sum(const OracleConfig& c, const double h[3], const S q[]) {
  S a = sound_speed(c, q[0], q[ien(c)]);
  S s = S(0.0);
  for (int d = 0; d < c.dim; ++d) s = s + (abs_s(q[1 + d]) + a) / h[d];
  return s;
}

// Heun step 1 under the CFL reading stated at the top of this file.
double cfl_dt(const OracleConfig& c, const std::vector<double> U[]) {
  Mesh<double> m(c);
  double smax = 0.0;
#pragma omp parallel for reduction(max : smax)
  for (size_t k = 0; k < m.ncell(); ++k) {
    double Uc[MAXF], q[MAXF];
    for (int l = 0; l < nfields(c); ++l) Uc[l] = U[l][k];
    prim_from_cons(c, Uc, q);
    double s = wave_speed_sum(c, m.h, q);
    if (s > smax) smax = s;
  }
  return c.cfl / smax;
}

// Positivity of a state (rho > 0 and p > 0 in every cell).
template <class S>
bool state_physical(const Mesh<S>& m, const std::vector<S> U[]) {
  const OracleConfig& c = m.c;
  bool ok = true;
#pragma omp parallel for reduction(&& : ok)
  for (size_t k = 0; k < m.ncell(); ++k) {
    S Uc[MAXF], q[MAXF];
    for (int l = 0; l < nfields(c); ++l) Uc[l] = U[l][k];
    prim_from_cons(c, Uc, q);
    if (!(val(q[0]) > 0.0) || !(val(q[ien(c)]) > 0.0)) ok = false;
  }
  return ok;
}

// One Heun step (Sec. 4, steps 2-11) with a given dt.
template <class S>
bool heun_step(const OracleConfig& c, std::vector<S> U[], double dt) {
  Mesh<S> m(c);
  const int nf = nfields(c);
  std::vector<S> Fn[3][MAXF], Fs[3][MAXF], Us[MAXF];
  bool ok = all_face_fluxes(m, U, Fn);  // steps 2-5
  for (int l = 0; l < nf; ++l) Us[l].resize(m.ncell());
#pragma omp parallel for collapse(2)
  for (int k = 0; k < m.n[2]; ++k)  // step 6: predicted states
    for (int j = 0; j < m.n[1]; ++j)
      for (int i = 0; i < m.n[0]; ++i) {
        size_t x = m.cell(i, j, k);
        for (int l = 0; l < nf; ++l) Us[l][x] = U[l][x] - dt * flux_balance(m, Fn, l, i, j, k);
      }
  ok = all_face_fluxes(m, Us, Fs) && ok;  // steps 7-10
#pragma omp parallel for collapse(2)
  for (int k = 0; k < m.n[2]; ++k)  // step 11: averaged fluxes
    for (int j = 0; j < m.n[1]; ++j)
      for (int i = 0; i < m.n[0]; ++i) {
        size_t x = m.cell(i, j, k);
        for (int l = 0; l < nf; ++l) {
          S bn = flux_balance(m, Fn, l, i, j, k);
          S bs = flux_balance(m, Fs, l, i, j, k);
          U[l][x] = U[l][x] - dt * ((bn + bs) / 2.0);
        }
      }
  return state_physical(m, U) && ok;
}

// Third-order strong-stability-preserving Runge-Kutta step of Shu and Osher
// (J. Comput. Phys. 77, 1988) for the semi-discrete scheme dU/dt = L(U),
// L(U) = -(1/|K|) sum_A |A| Phi_A (Sec. 4 leaves the Runge-Kutta family open as time advance
// schemes):
//   U1 = U^n + dt L(U^n)
//   U2 = 3/4 U^n + 1/4 (U1 + dt L(U1))
//   U^{n+1} = 1/3 U^n + 2/3 (U2 + dt L(U2))
template <class S>
bool ssprk3_step(const OracleConfig& c, std::vector<S> U[], double dt) {
  Mesh<S> m(c);
  const int nf = nfields(c);
  std::vector<S> F[3][MAXF], U1[MAXF], U2[MAXF];
  bool ok = all_face_fluxes(m, U, F);
  for (int l = 0; l < nf; ++l) U1[l].resize(m.ncell());
  for (int k = 0; k < m.n[2]; ++k)
    for (int j = 0; j < m.n[1]; ++j)
      for (int i = 0; i < m.n[0]; ++i) {
        size_t x = m.cell(i, j, k);
        for (int l = 0; l < nf; ++l) U1[l][x] = U[l][x] - dt * flux_balance(m, F, l, i, j, k);
      }
  ok = all_face_fluxes(m, U1, F) && ok;
  for (int l = 0; l < nf; ++l) U2[l].resize(m.ncell());
  for (int k = 0; k < m.n[2]; ++k)
    for (int j = 0; j < m.n[1]; ++j)
      for (int i = 0; i < m.n[0]; ++i) {
        size_t x = m.cell(i, j, k);
        for (int l = 0; l < nf; ++l)
          U2[l][x] = 0.75 * U[l][x] + 0.25 * (U1[l][x] - dt * flux_balance(m, F, l, i, j, k));
      }
  ok = all_face_fluxes(m, U2, F) && ok;
  for (int k = 0; k < m.n[2]; ++k)
    for (int j = 0; j < m.n[1]; ++j)
      for (int i = 0; i < m.n[0]; ++i) {
        size_t x = m.cell(i, j, k);
        for (int l = 0; l < nf; ++l)
          U[l][x] = U[l][x] / 3.0 + (2.0 / 3.0) * (U2[l][x] - dt * flux_balance(m, F, l, i, j, k));
      }
  return state_physical(m, U) && ok;
}

template <class S>
bool time_step(const OracleConfig& c, std::vector<S> U[], double dt) {
  return c.time_order == 3 ? ssprk3_step(c, U, dt) : heun_step(c, U, dt);
}

void load_planes(const OracleConfig& c, const double* src, std::vector<double> U[]) {
  size_t n = (size_t)c.nx * c.ny * c.nz;
  for (int l = 0; l < nfields(c); ++l) U[l].assign(src + l * n, src + (l + 1) * n);
}
void store_planes(const OracleConfig& c, const std::vector<double> U[], double* dst) {
  size_t n = (size_t)c.nx * c.ny * c.nz;
  for (int l = 0; l < nfields(c); ++l) std::memcpy(dst + l * n, U[l].data(), n * sizeof(double));
}

// Flops of one stage of the method on state U, in the minimal schedule: each
// cell's primitive state, each cell's limited slope per axis and field, each
// face's states and Lagrange flux, and each cell's flux balance formed once
// (the step above stores both face states' slopes and re-forms the flux
// balance of U^n in step 11; those repeats are the oracle's literal form, not
// work the method needs).  Faces wrap around on every axis, so a row of n
// cells has n faces.  tally[s] receives the operations of part s, summed over
// all cells: 0 primitives, 1 slopes, 2 face states and fluxes, 3 flux
// balances, 4 the predictor update U - dt b, 5 the corrector update
// U - dt (b_n + b_*)/2 (whose b_n the predictor already formed), 6 the
// wave-speed sum of the CFL condition.
constexpr int kCountParts = 7;
void count_stage_ops(const OracleConfig& c, const std::vector<double> U[], OpTally tally[kCountParts]) {
  Mesh<Counted> m(c);
  const int nf = nfields(c);
  const size_t n = m.ncell();
  auto wrapped = [&](int i, int j, int k, int d, int s) {  // cell s steps along axis d, periodic
    int o[3] = {i, j, k};
    o[d] = wrap_index(o[d] + s, m.n[d], BC_PERIODIC);
    return m.cell(o[0], o[1], o[2]);
  };
  std::vector<Counted> q[MAXF], sig[3][MAXF], F[3][MAXF];
  for (int l = 0; l < nf; ++l) q[l].resize(n);
  g_tally = OpTally();
  for (size_t x = 0; x < n; ++x) {  // 0: primitives
    Counted Uc[MAXF], qc[MAXF];
    for (int l = 0; l < nf; ++l) Uc[l] = Counted(U[l][x]);
    prim_from_cons(c, Uc, qc);
    for (int l = 0; l < nf; ++l) q[l][x] = qc[l];
  }
  tally[0] = g_tally;
  g_tally = OpTally();
  for (int d = 0; d < c.dim; ++d)  // 1: limited slopes
    for (int l = 0; l < nf; ++l) {
      sig[d][l].resize(n);
      for (int k = 0; k < m.n[2]; ++k)
        for (int j = 0; j < m.n[1]; ++j)
          for (int i = 0; i < m.n[0]; ++i) {
            size_t x = m.cell(i, j, k);
            sig[d][l][x] = limiter(c, q[l][x] - q[l][wrapped(i, j, k, d, -1)], q[l][wrapped(i, j, k, d, 1)] - q[l][x]);
          }
    }
  tally[1] = g_tally;
  g_tally = OpTally();
  for (int d = 0; d < c.dim; ++d) {  // 2: face states and fluxes (face behind each cell)
    for (int l = 0; l < nf; ++l) F[d][l].resize(m.nfaces(d));
    for (int k = 0; k < m.n[2]; ++k)
      for (int j = 0; j < m.n[1]; ++j)
        for (int i = 0; i < m.n[0]; ++i) {
          size_t xr = m.cell(i, j, k), xl = wrapped(i, j, k, d, -1);
          Counted qL[MAXF], qR[MAXF], Fv[MAXF];
          for (int l = 0; l < nf; ++l) {
            qL[l] = q[l][xl] + 0.5 * sig[d][l][xl];
            qR[l] = q[l][xr] - 0.5 * sig[d][l][xr];
          }
          face_flux(c, d, qL, qR, Fv);
          int hi[3] = {i, j, k};
          for (int l = 0; l < nf; ++l) F[d][l][m.fidx(d, i, j, k)] = Fv[l];
          if (hi[d] == 0) {  // the same face closes the far end of the row
            hi[d] = m.n[d];
            for (int l = 0; l < nf; ++l) F[d][l][m.fidx(d, hi[0], hi[1], hi[2])] = Fv[l];
          }
        }
  }
  tally[2] = g_tally;
  std::vector<Counted> b[MAXF];
  g_tally = OpTally();
  for (int l = 0; l < nf; ++l) {  // 3: flux balances
    b[l].resize(n);
    for (int k = 0; k < m.n[2]; ++k)
      for (int j = 0; j < m.n[1]; ++j)
        for (int i = 0; i < m.n[0]; ++i) b[l][m.cell(i, j, k)] = flux_balance(m, F, l, i, j, k);
  }
  tally[3] = g_tally;
  const Counted dt(1e-3);
  g_tally = OpTally();
  for (int l = 0; l < nf; ++l)  // 4: predictor update
    for (size_t x = 0; x < n; ++x) (void)(Counted(U[l][x]) - dt * b[l][x]);
  tally[4] = g_tally;
  g_tally = OpTally();
  for (int l = 0; l < nf; ++l)  // 5: corrector update (b stands for both b_n and b_*)
    for (size_t x = 0; x < n; ++x) (void)(Counted(U[l][x]) - dt * ((b[l][x] + b[l][x]) / 2.0));
  tally[5] = g_tally;
  g_tally = OpTally();
  for (size_t x = 0; x < n; ++x) {  // 6: wave-speed sum
    Counted qc[MAXF];
    for (int l = 0; l < nf; ++l) qc[l] = q[l][x];
    (void)wave_speed_sum(c, m.h, qc);
  }
  tally[6] = g_tally;
}

}  // namespace

// ===========================================================================
// C entry points used through ctypes.  A state is nfields = 4 + nspecies
// planes stored plane after plane (rho, rho u, rho v, rho E, rho y_1 ..), each
// plane nx*ny values, x fastest.
// Return ORC_OK, ORC_NONPHYSICAL (a non-positive density or pressure met) or
// ORC_ARG (invalid configuration or argument).
// ===========================================================================
extern "C" {

int oracle_limiter(const OracleConfig* c, int64_t n, const double* a, const double* b, double* out) {
  if (!c || n < 0) return ORC_ARG;
  for (int64_t k = 0; k < n; ++k) out[k] = limiter(*c, a[k], b[k]);
  return ORC_OK;
}

// L and R are n x 3 arrays of (rho, u_normal, p).
int oracle_interface_solve(const OracleConfig* c, int64_t n, const double* L, const double* R,
                           double* pstar, double* ustar) {
  if (!c || n < 0) return ORC_ARG;
  for (int64_t k = 0; k < n; ++k)
    interface_solve(*c, L[3 * k], L[3 * k + 1], L[3 * k + 2], R[3 * k], R[3 * k + 1], R[3 * k + 2],
                    pstar[k], ustar[k]);
  return ORC_OK;
}

// qL, qR, F are n x nfields arrays; q = (rho, u, v, p, y_1 ..).
int oracle_face_flux(const OracleConfig* c, int dir, int64_t n, const double* qL, const double* qR,
                     double* F) {
  if (!c || n < 0 || (dir != 0 && dir != 1) || c->nspecies < 0 || c->nspecies > MAX_SPECIES) return ORC_ARG;
  const int nf = nfields(*c);
  for (int64_t k = 0; k < n; ++k) face_flux(*c, dir, qL + nf * k, qR + nf * k, F + nf * k);
  return ORC_OK;
}

int oracle_prim_to_cons(const OracleConfig* c, const double* q, double* U) {
  if (!config_ok(c)) return ORC_ARG;
  size_t n = (size_t)c->nx * c->ny * c->nz;
  const int nf = nfields(*c);
  for (size_t k = 0; k < n; ++k) {
    double qc[MAXF] = {}, Uc[MAXF];
    for (int l = 0; l < nf; ++l) qc[l] = q[l * n + k];
    cons_from_prim(*c, qc, Uc);
    for (int l = 0; l < nf; ++l) U[l * n + k] = Uc[l];
  }
  return ORC_OK;
}

int oracle_cons_to_prim(const OracleConfig* c, const double* U, double* q) {
  if (!config_ok(c)) return ORC_ARG;
  size_t n = (size_t)c->nx * c->ny * c->nz;
  const int nf = nfields(*c);
  for (size_t k = 0; k < n; ++k) {
    double Uc[MAXF] = {}, qc[MAXF];
    for (int l = 0; l < nf; ++l) Uc[l] = U[l * n + k];
    prim_from_cons(*c, Uc, qc);
    for (int l = 0; l < nf; ++l) q[l * n + k] = qc[l];
  }
  return ORC_OK;
}

int oracle_dt(const OracleConfig* c, const double* Uin, double* dt) {
  if (!config_ok(c) || !Uin || !dt) return ORC_ARG;
  std::vector<double> U[MAXF];
  load_planes(*c, Uin, U);
  *dt = cfl_dt(*c, U);
  return ORC_OK;
}

// L(U) = -(1/|K|) sum_A |A| Phi_A, the right-hand side of the semi-discrete
// scheme after eq. (11).
int oracle_residual(const OracleConfig* c, const double* Uin, double* LU) {
  if (!config_ok(c) || !Uin || !LU) return ORC_ARG;
  std::vector<double> U[MAXF], F[3][MAXF];
  load_planes(*c, Uin, U);
  Mesh<double> m(*c);
  bool ok = all_face_fluxes(m, U, F);
  size_t n = m.ncell();
  for (int k = 0; k < m.n[2]; ++k)
    for (int j = 0; j < m.n[1]; ++j)
      for (int i = 0; i < m.n[0]; ++i)
        for (int l = 0; l < nfields(*c); ++l) LU[l * n + m.cell(i, j, k)] = -flux_balance(m, F, l, i, j, k);
  return ok ? ORC_OK : ORC_NONPHYSICAL;
}

// Runs up to max_steps time steps (Heun, or SSP-RK3 when time_order == 3).  If dts_in is given, step n uses dts_in[n]
// (a frozen dt sequence); otherwise dt comes from the CFL condition and is
// clipped so that t never passes t_end (t_end <= 0: no final time).  The run
// stops early once t reaches t_end.  dts_out (nullable) receives the dt used
// by each step.
int oracle_run(const OracleConfig* c, double* Uio, int32_t max_steps, double t0, double t_end,
               const double* dts_in, double* dts_out, int32_t* steps_done, double* t_out) {
  if (!config_ok(c) || !Uio || max_steps < 0) return ORC_ARG;
  std::vector<double> U[MAXF];
  load_planes(*c, Uio, U);
  double t = t0;
  int n = 0;
  int status = ORC_OK;
  for (; n < max_steps; ++n) {
    if (t_end > 0.0 && !dts_in && t >= t_end) break;
    double dt = dts_in ? dts_in[n] : cfl_dt(*c, U);
    if (!dts_in && t_end > 0.0 && t + dt > t_end) dt = t_end - t;
    if (dts_out) dts_out[n] = dt;
    if (!time_step(*c, U, dt)) {
      status = ORC_NONPHYSICAL;
      ++n;
      t += dt;
      break;
    }
    t += dt;
  }
  store_planes(*c, U, Uio);
  if (steps_done) *steps_done = n;
  if (t_out) *t_out = t;
  return status;
}

// Forward-mode directional derivative of nsteps Heun steps with the frozen
// dt sequence dts.  q0 and dq0 are the initial primitive planes (rho, u, v, p,
// y_1 ..) and their tangent; U_out and dU_out receive the final conservative
// planes and their tangent.
int oracle_run_tangent(const OracleConfig* c, const double* q0, const double* dq0, int32_t nsteps,
                       const double* dts, double* U_out, double* dU_out) {
  if (!config_ok(c) || !q0 || !dq0 || !dts || nsteps < 0) return ORC_ARG;
  size_t n = (size_t)c->nx * c->ny * c->nz;
  const int nf = nfields(*c);
  std::vector<Dual> U[MAXF];
  for (int l = 0; l < nf; ++l) U[l].resize(n);
  for (size_t k = 0; k < n; ++k) {
    Dual qc[MAXF], Uc[MAXF];
    for (int l = 0; l < nf; ++l) qc[l] = Dual(q0[l * n + k], dq0[l * n + k]);
    cons_from_prim(*c, qc, Uc);
    for (int l = 0; l < nf; ++l) U[l][k] = Uc[l];
  }
  int status = ORC_OK;
  for (int s = 0; s < nsteps; ++s)
    if (!time_step(*c, U, dts[s])) status = ORC_NONPHYSICAL;
  for (int l = 0; l < nf; ++l)
    for (size_t k = 0; k < n; ++k) {
      U_out[l * n + k] = U[l][k].v;
      dU_out[l * n + k] = U[l][k].d;
    }
  return status;
}

// Flops per cell of the method on the state U (count_stage_ops): out[4 s + k]
// for part s = 0 .. 6 and k = add, multiply, divide, square root, each summed
// over the mesh and divided by the number of cells.  Counting is serial: the
// OpenMP build refuses it (ORC_ARG).
int oracle_count_ops(const OracleConfig* c, const double* U_in, double* out) {
#ifdef _OPENMP
  (void)c;
  (void)U_in;
  (void)out;
  return ORC_ARG;
#else
  if (!config_ok(c) || !U_in || !out) return ORC_ARG;
  std::vector<double> U[MAXF];
  load_planes(*c, U_in, U);
  OpTally t[kCountParts];
  count_stage_ops(*c, U, t);
  const double n = (double)c->nx * c->ny * c->nz;
  for (int s = 0; s < kCountParts; ++s) {
    out[4 * s + 0] = t[s].add / n;
    out[4 * s + 1] = t[s].mul / n;
    out[4 * s + 2] = t[s].div / n;
    out[4 * s + 3] = t[s].sqrt / n;
  }
  return ORC_OK;
#endif
}

// Threads of the OpenMP timing build: sets the count when n > 0 and returns
// the count the next parallel loop will use (always 1 in the plain build).
int oracle_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

}  // extern "C"
