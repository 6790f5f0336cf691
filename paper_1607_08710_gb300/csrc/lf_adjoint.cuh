// Discrete adjoint of the Lagrange-flux step (arXiv:1607.08710, Sec. 4).
//
// With the flux divergence D_K(U) = (F_{i+1/2} - F_{i-1/2})/dx +
// (G_{j+1/2} - G_{j-1/2})/dy, the Heun step is U* = U - dt D(U),
// U' = (U + U*)/2 - dt/2 D(U*).  With dt frozen, its transpose maps a
// cotangent lambda of U' to
//     lambda* = lambda/2 - dt/2 (dD/dU)(U*)^T lambda
//     lambda_U = lambda/2 + lambda* - dt (dD/dU)(U)^T lambda*.
// The product w = (dD/dU)^T mu is formed in gather form, without atomics:
//   0. prep kernels: the primitives of every cell (eq. 1), and for every
//      position p = -1 .. n of every row (x) and column (y), i.e. every cell
//      and the first ghost cell on each side, the limiter value and its two
//      partial derivatives for each field (eq. "sweby" / van Leer) -- the
//      forward quantities the two passes below read, computed once;
//   1. face kernel: for every face f (between positions f-1 and f), the face
//      states from those tables, the face cotangent nu_f = (mu_{f-1} -
//      mu_f) / h (mu = 0 outside the mesh), and the reverse of the interface
//      solve and upwind flux into the cotangents of the two face states (8
//      values per face);
//   2. cell kernel: for every cell, sum the face-state cotangents that reach
//      it directly and through the limited slopes of itself and its two
//      neighbours (the tabulated partial derivatives), over every image of the
//      cell under the boundary map (ghost copies, periodic images), then
//      reverse the primitive conversion (eq. 1) and apply the RK combination.
// Derivative conventions at non-smooth points are those of the oracle's dual
// numbers: ties of max/min take the first argument, the limiter is constant 0
// where ab <= 0, and the upwind side follows the value of u*.
#pragma once

#include "lf_device.cuh"

namespace lf {

// Limiter value and partial derivatives (phi, dphi/da, dphi/db).
template <typename T, int LIM>
__device__ __forceinline__ void limiter_d(T a, T b, T beta, T& phi, T& da, T& db) {
  if (!(a * b > T(0))) {
    phi = da = db = T(0);
    return;
  }
  if (LIM == LIM_VANLEER) {
    const T s = a + b, is = T(1) / s;
    phi = T(2) * a * b * is;
    da = T(2) * b * b * is * is;
    db = T(2) * a * a * is * is;
    return;
  }
  const T be = LIM == LIM_MINMOD ? T(1) : beta;
  const T aa = fabs(a), bb = fabs(b);
  const bool m1a = aa <= be * bb;  // min(|a|, beta|b|) takes |a|
  const T m1 = m1a ? aa : be * bb;
  const bool m2a = be * aa <= bb;  // min(beta|a|, |b|) takes beta|a|
  const T m2 = m2a ? be * aa : bb;
  const bool first = m1 >= m2;
  // phi = sign(a) * (selected term); with ab > 0, c|a| -> c a and c|b| -> c b
  if (first) {
    da = m1a ? T(1) : T(0);
    db = m1a ? T(0) : be;
  } else {
    da = m2a ? be : T(0);
    db = m2a ? T(0) : T(1);
  }
  phi = copysign(first ? m1 : m2, a);
}

// Reverse of lagrange_flux (eqs. 13-14 with a = max(c_L, c_R), eq. 12) at
// the face states qL, qR for the flux cotangent Fb: adds the cotangents of
// qL and qR to qLb, qRb.
template <typename T, int DIR>
__device__ __forceinline__ void lagrange_flux_vjp(const Phys<T>& P, const T qL[4], const T qR[4], const T Fb[4],
                                                  T qLb[4], T qRb[4]) {
  const T g = P.gamma;
  const T rL = qL[0], pL = qL[3], rR = qR[0], pR = qR[3];
  const T unL = qL[1 + DIR], unR = qR[1 + DIR];
  const T c2L = g * pL / rL, c2R = g * pR / rR;
  const bool useL = c2L >= c2R;  // max(c_L, c_R) takes c_L on ties
  const T a = sqrt(useL ? c2L : c2R);
  const T rs = rL + rR, irs = T(1) / rs, irs2 = irs * irs;
  const T du = unR - unL, dp = pR - pL;
  const T pstar = (rR * pL + rL * pR) * irs - rL * rR * irs * a * du;
  const T ustar = (rL * unL + rR * unR) * irs - dp * irs / a;
  const bool left = ustar > T(0);
  const T* qs = left ? qL : qR;
  T* qsb = left ? qLb : qRb;
  const T r = qs[0], u = qs[1], v = qs[2], p = qs[3];
  const T E = p * P.inv_gm1 + T(0.5) * r * (u * u + v * v);
  // flux: F0 = r u*, F1 = r u u* (+p* for x), F2 = r v u* (+p* for y), F3 = (E + p*) u*
  const T ustar_b = Fb[0] * r + Fb[1] * r * u + Fb[2] * r * v + Fb[3] * (E + pstar);
  const T pstar_b = (DIR == 0 ? Fb[1] : Fb[2]) + Fb[3] * ustar;
  const T E_b = Fb[3] * ustar;
  qsb[0] += Fb[0] * ustar + Fb[1] * u * ustar + Fb[2] * v * ustar + E_b * T(0.5) * (u * u + v * v);
  qsb[1] += Fb[1] * r * ustar + E_b * r * u;
  qsb[2] += Fb[2] * r * ustar + E_b * r * v;
  qsb[3] += E_b * P.inv_gm1;
  // p* and u* as functions of (rL, unL, pL, rR, unR, pR, a)
  const T a_b = pstar_b * (-rL * rR * du * irs) + ustar_b * (dp * irs / (a * a));
  qLb[3] += pstar_b * rR * irs + ustar_b * irs / a;
  qRb[3] += pstar_b * rL * irs - ustar_b * irs / a;
  qLb[1 + DIR] += pstar_b * rL * rR * a * irs + ustar_b * rL * irs;
  qRb[1 + DIR] += -pstar_b * rL * rR * a * irs + ustar_b * rR * irs;
  qLb[0] += pstar_b * (rR * dp - a * du * rR * rR) * irs2 + ustar_b * (rR * (unL - unR) * irs2 + dp * irs2 / a);
  qRb[0] += pstar_b * (-rL * dp - a * du * rL * rL) * irs2 + ustar_b * (rL * (unR - unL) * irs2 + dp * irs2 / a);
  // a = sqrt(gamma p_k / r_k) of the side k with the larger sound speed
  T* kb = useL ? qLb : qRb;
  const T rk = useL ? rL : rR;
  kb[3] += a_b * g / (T(2) * a * rk);
  kb[0] += -a_b * a / (T(2) * rk);
}

template <typename T>
__device__ __forceinline__ void load_prim(const Phys<T>& P, const T* U, long long plane, long long idx, T q[4]) {
  T Uc[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) Uc[k] = U[k * plane + idx];
  // plain division here: the adjoint recomputes the forward in the precision of the run
  const T r = Uc[0], u = Uc[1] / r, v = Uc[2] / r;
  q[0] = r;
  q[1] = u;
  q[2] = v;
  q[3] = P.gm1 * (Uc[3] - T(0.5) * (Uc[1] * u + Uc[2] * v));
}

// Slot of face f (0 .. n) of line `line` in the face-cotangent arrays: x-faces
// row by row ([row][face]), y-faces face row by face row ([face][column]), so
// that neighbouring threads, which take neighbouring x positions, touch
// neighbouring slots and neighbouring cells in both directions.
template <int DIR>
__device__ __forceinline__ long long face_slot(const MeshDesc& m, int line, int f) {
  return DIR == 0 ? (long long)line * (m.nx + 1) + f : (long long)f * m.nx + line;
}

// Slot of position p (-1 .. n) of line `line` in the slope tables, laid out
// like the faces.  A slot holds 12 values: phi, dphi/da, dphi/db per field.
template <int DIR>
__device__ __forceinline__ long long pos_slot(const MeshDesc& m, int line, int p) {
  return DIR == 0 ? (long long)line * (m.nx + 2) + (p + 1) : (long long)(p + 1) * m.nx + line;
}

// Dense index of the mapped cell at position c of line `line`.
template <int DIR>
__device__ __forceinline__ long long line_cell(const MeshDesc& m, int line, int c) {
  const int n = DIR == 0 ? m.nx : m.ny;
  const int cm = map_index(c, n, m.bc);
  return DIR == 0 ? (long long)line * m.nx + cm : (long long)cm * m.nx + line;
}

// Primitives of every cell, 4 dense planes of nx*ny.
template <typename T>
__global__ void prim_planes_kernel(const MeshDesc m, const T* __restrict__ U, T* Q) {
  const Phys<T> P(m);
  const long long total = (long long)m.nx * m.ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(t / m.nx), i = (int)(t - (long long)j * m.nx);
    T q[4];
    load_prim(P, U, m.plane, (long long)j * m.pitch + i, q);
#pragma unroll
    for (int k = 0; k < 4; ++k) Q[k * total + t] = q[k];
  }
}

// Limiter value and partial derivatives at every position p = -1 .. n of
// every line, from the primitives of positions p-1, p, p+1 (boundary-mapped).
template <typename T, int LIM, int DIR>
__global__ void slope_table_kernel(const MeshDesc m, const T* __restrict__ Q, T* tab) {
  const int n = DIR == 0 ? m.nx : m.ny;
  const int lines = DIR == 0 ? m.ny : m.nx;
  const long long cells = (long long)m.nx * m.ny;
  const long long total = (long long)(n + 2) * lines;
  const T beta = T(m.beta);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int line = DIR == 0 ? (int)(t / (n + 2)) : (int)(t % lines);
    const int p = (DIR == 0 ? (int)(t - (long long)line * (n + 2)) : (int)(t / lines)) - 1;
    const long long cm = line_cell<DIR>(m, line, p - 1), c0 = line_cell<DIR>(m, line, p),
                    cp = line_cell<DIR>(m, line, p + 1);
    T* o = tab + pos_slot<DIR>(m, line, p) * 12;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const T qm = Q[k * cells + cm], q0 = Q[k * cells + c0], qp = Q[k * cells + cp];
      T phi, da, db;
      limiter_d<T, LIM>(q0 - qm, qp - q0, beta, phi, da, db);
      o[k] = phi;
      o[4 + k] = da;
      o[8 + k] = db;
    }
  }
}

// Face kernel.  DIR 0: x-faces, nx + 1 per row, ny rows; DIR 1: y-faces,
// ny + 1 per column, nx columns.  Output Fq[face_slot * 8 + ...]: cotangents
// of (qL[0..3], qR[0..3]).
template <typename T, int DIR>
__global__ void face_vjp_kernel(const MeshDesc m, const T* __restrict__ Q, const T* __restrict__ tab,
                                const T* __restrict__ mu, T* Fq) {
  const Phys<T> P(m);
  const int n = DIR == 0 ? m.nx : m.ny;        // cells along the direction
  const int lines = DIR == 0 ? m.ny : m.nx;    // rows (x) or columns (y)
  const long long cells = (long long)m.nx * m.ny;
  const long long total = (long long)(n + 1) * lines;
  const T h = DIR == 0 ? T(m.rdx) : T(m.rdy);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    // consecutive threads: consecutive faces of a row (x) or columns (y)
    const int line = DIR == 0 ? (int)(t / (n + 1)) : (int)(t % lines);
    const int f = DIR == 0 ? (int)(t - (long long)line * (n + 1)) : (int)(t / lines);
    const long long cl = line_cell<DIR>(m, line, f - 1), cr = line_cell<DIR>(m, line, f);
    const T* sl = tab + pos_slot<DIR>(m, line, f - 1) * 12;
    const T* sr = tab + pos_slot<DIR>(m, line, f) * 12;
    T qL[4], qR[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      qL[k] = Q[k * cells + cl] + T(0.5) * sl[k];
      qR[k] = Q[k * cells + cr] - T(0.5) * sr[k];
    }
    T nu[4];
    const bool hasL = f - 1 >= 0, hasR = f < n;  // cells of the mesh on each side
    const long long il = DIR == 0 ? (long long)line * m.pitch + (f - 1) : (long long)(f - 1) * m.pitch + line;
    const long long ir = DIR == 0 ? (long long)line * m.pitch + f : (long long)f * m.pitch + line;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const T muL = hasL ? mu[k * m.plane + il] : T(0);
      const T muR = hasR ? mu[k * m.plane + ir] : T(0);
      nu[k] = (muL - muR) * h;
    }
    T qLb[4] = {T(0), T(0), T(0), T(0)}, qRb[4] = {T(0), T(0), T(0), T(0)};
    lagrange_flux_vjp<T, DIR>(P, qL, qR, nu, qLb, qRb);
    T* o = Fq + face_slot<DIR>(m, line, f) * 8;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      o[k] = qLb[k];
      o[4 + k] = qRb[k];
    }
  }
}

// Cotangents of the primitives of one cell along one direction, gathered
// from the face-state cotangents Fq (see face_vjp_kernel) and the reversed
// limited slopes (the tabulated partial derivatives).  `pos` is the cell's
// index along the direction, `line` the transverse index.
template <typename T, int DIR>
__device__ __forceinline__ void gather_dir(const MeshDesc& m, const T* Fq, const T* tab, int pos, int line, T qb[4]) {
  const int n = DIR == 0 ? m.nx : m.ny;
  auto face = [&](int f, int part, int k) -> T {  // part 0: qL cotangent, 1: qR cotangent
    if (f < 0 || f > n) return T(0);
    return Fq[face_slot<DIR>(m, line, f) * 8 + part * 4 + k];
  };
  // every image v of this cell in [-2, n+1] (itself, ghost copies, periodic images)
  int cand[9] = {pos, -2, -1, n, n + 1, pos - n, pos + n, pos - 2 * n, pos + 2 * n};
  for (int ci = 0; ci < 9; ++ci) {
    const int v = cand[ci];
    if (v < -2 || v > n + 1 || map_index(v, n, m.bc) != pos) continue;
    bool dup = false;
    for (int cj = 0; cj < ci; ++cj) dup |= cand[cj] == v;
    if (dup) continue;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      T acc = face(v + 1, 0, k) + face(v, 1, k);  // v as the left cell of face v+1/2, right cell of v-1/2
      for (int w = v - 1; w <= v + 1; ++w) {       // slopes of cells v-1, v, v+1
        if (w < -1 || w > n) continue;             // only these slopes enter a face
        const T sb = T(0.5) * (face(w + 1, 0, k) - face(w, 1, k));
        // sigma_w = phi(q_w - q_{w-1}, q_{w+1} - q_w)
        const T* d = tab + pos_slot<DIR>(m, line, w) * 12;
        const T da = d[4 + k], db = d[8 + k];
        if (w == v) acc += (da - db) * sb;
        else if (w == v - 1) acc += db * sb;
        else acc -= da * sb;
      }
      qb[k] += acc;
    }
  }
}

// out = alpha X + beta Y + c (dD/dU)^T mu, cell by cell (X, Y nullable).
template <typename T>
__global__ void cell_vjp_kernel(const MeshDesc m, const T* __restrict__ Q, const T* __restrict__ Fx,
                                const T* __restrict__ Fy, const T* __restrict__ tabx, const T* __restrict__ taby,
                                const T* X, T alpha, const T* Y, T beta, T c, T* out) {
  const Phys<T> P(m);
  const long long total = (long long)m.nx * m.ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(t / m.nx), i = (int)(t - (long long)j * m.nx);
    const long long idx = (long long)j * m.pitch + i;
    T qb[4] = {T(0), T(0), T(0), T(0)};
    gather_dir<T, 0>(m, Fx, tabx, i, j, qb);
    gather_dir<T, 1>(m, Fy, taby, j, i, qb);
    // reverse of the primitive conversion at this cell
    const T r = Q[t], u = Q[total + t], v = Q[2 * total + t];
    T w[4];
    w[0] = qb[0] - qb[1] * u / r - qb[2] * v / r + qb[3] * P.gm1 * T(0.5) * (u * u + v * v);
    w[1] = qb[1] / r - qb[3] * P.gm1 * u;
    w[2] = qb[2] / r - qb[3] * P.gm1 * v;
    w[3] = qb[3] * P.gm1;
    T res[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      res[k] = c * w[k];
      if (X) res[k] += alpha * X[k * m.plane + idx];
      if (Y) res[k] += beta * Y[k * m.plane + idx];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) out[k * m.plane + idx] = res[k];
  }
}

// Direct variants of the face and cell passes: every face and every cell
// recomputes the primitives and limited slopes it needs from U (no prep
// tables).  Used in FP32, where the recomputation is cheaper than the three
// extra passes and the table traffic; FP64 pays for its divisions and uses
// the tables.
template <typename T, int LIM, int DIR>
__global__ void face_vjp_direct_kernel(const MeshDesc m, const T* __restrict__ U, const T* __restrict__ mu, T* Fq) {
  const Phys<T> P(m);
  const int n = DIR == 0 ? m.nx : m.ny;        // cells along the direction
  const int lines = DIR == 0 ? m.ny : m.nx;    // rows (x) or columns (y)
  const long long total = (long long)(n + 1) * lines;
  const T h = DIR == 0 ? T(m.rdx) : T(m.rdy);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    // consecutive threads: consecutive faces of a row (x) or columns (y)
    const int line = DIR == 0 ? (int)(t / (n + 1)) : (int)(t % lines);
    const int f = DIR == 0 ? (int)(t - (long long)line * (n + 1)) : (int)(t / lines);
    auto cell_idx = [&](int c) -> long long {
      const int cm = map_index(c, n, m.bc);
      return DIR == 0 ? (long long)line * m.pitch + cm : (long long)cm * m.pitch + line;
    };
    T q[4][4];  // cells f-2, f-1, f, f+1
#pragma unroll
    for (int s = 0; s < 4; ++s) load_prim(P, U, m.plane, cell_idx(f - 2 + s), q[s]);
    T qL[4], qR[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      T phi, da, db;
      limiter_d<T, LIM>(q[1][k] - q[0][k], q[2][k] - q[1][k], P.beta, phi, da, db);
      qL[k] = q[1][k] + T(0.5) * phi;
      limiter_d<T, LIM>(q[2][k] - q[1][k], q[3][k] - q[2][k], P.beta, phi, da, db);
      qR[k] = q[2][k] - T(0.5) * phi;
    }
    T nu[4];
    const bool hasL = f - 1 >= 0, hasR = f < n;  // cells of the mesh on each side
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const T muL = hasL ? mu[k * m.plane + cell_idx(f - 1)] : T(0);
      const T muR = hasR ? mu[k * m.plane + cell_idx(f)] : T(0);
      nu[k] = (muL - muR) * h;
    }
    T qLb[4] = {T(0), T(0), T(0), T(0)}, qRb[4] = {T(0), T(0), T(0), T(0)};
    lagrange_flux_vjp<T, DIR>(P, qL, qR, nu, qLb, qRb);
    T* o = Fq + face_slot<DIR>(m, line, f) * 8;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      o[k] = qLb[k];
      o[4 + k] = qRb[k];
    }
  }
}

// Cotangents of the primitives of one cell along one direction, gathered
// from the face-state cotangents Fq (see face_vjp_kernel) and the reversed
// limited slopes.  `pos` is the cell's index along the direction, `line` the
// transverse index.
template <typename T, int LIM, int DIR>
__device__ __forceinline__ void gather_dir_direct(const Phys<T>& P, const MeshDesc& m, const T* U, const T* Fq, int pos,
                                           int line, T qb[4]) {
  const int n = DIR == 0 ? m.nx : m.ny;
  auto cell_idx = [&](int c) -> long long {
    const int cm = map_index(c, n, m.bc);
    return DIR == 0 ? (long long)line * m.pitch + cm : (long long)cm * m.pitch + line;
  };
  auto face = [&](int f, int part, int k) -> T {  // part 0: qL cotangent, 1: qR cotangent
    if (f < 0 || f > n) return T(0);
    return Fq[face_slot<DIR>(m, line, f) * 8 + part * 4 + k];
  };
  // every image v of this cell in [-2, n+1] (itself, ghost copies, periodic images)
  int cand[9] = {pos, -2, -1, n, n + 1, pos - n, pos + n, pos - 2 * n, pos + 2 * n};
  for (int ci = 0; ci < 9; ++ci) {
    const int v = cand[ci];
    if (v < -2 || v > n + 1 || map_index(v, n, m.bc) != pos) continue;
    bool dup = false;
    for (int cj = 0; cj < ci; ++cj) dup |= cand[cj] == v;
    if (dup) continue;
    T qw[5][4];  // primitives of cells v-2 .. v+2
    for (int s = 0; s < 5; ++s) load_prim(P, U, m.plane, cell_idx(v - 2 + s), qw[s]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      T acc = face(v + 1, 0, k) + face(v, 1, k);  // v as the left cell of face v+1/2, right cell of v-1/2
      for (int w = v - 1; w <= v + 1; ++w) {       // slopes of cells v-1, v, v+1
        if (w < -1 || w > n) continue;             // only these slopes enter a face
        const T sb = T(0.5) * (face(w + 1, 0, k) - face(w, 1, k));
        const int s = w - v + 2;                   // qw index of cell w
        T phi, da, db;
        limiter_d<T, LIM>(qw[s][k] - qw[s - 1][k], qw[s + 1][k] - qw[s][k], P.beta, phi, da, db);
        // sigma_w = phi(q_w - q_{w-1}, q_{w+1} - q_w)
        if (w == v) acc += (da - db) * sb;
        else if (w == v - 1) acc += db * sb;
        else acc -= da * sb;
      }
      qb[k] += acc;
    }
  }
}

// out = alpha X + beta Y + c (dD/dU)^T mu, cell by cell (X, Y nullable).
template <typename T, int LIM>
__global__ void cell_vjp_direct_kernel(const MeshDesc m, const T* __restrict__ U, const T* __restrict__ Fx,
                                const T* __restrict__ Fy, const T* X, T alpha, const T* Y, T beta, T c, T* out) {
  const Phys<T> P(m);
  const long long total = (long long)m.nx * m.ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(t / m.nx), i = (int)(t - (long long)j * m.nx);
    const long long idx = (long long)j * m.pitch + i;
    T qb[4] = {T(0), T(0), T(0), T(0)};
    gather_dir_direct<T, LIM, 0>(P, m, U, Fx, i, j, qb);
    gather_dir_direct<T, LIM, 1>(P, m, U, Fy, j, i, qb);
    // reverse of the primitive conversion at this cell
    T q[4];
    load_prim(P, U, m.plane, idx, q);
    const T r = q[0], u = q[1], v = q[2];
    T w[4];
    w[0] = qb[0] - qb[1] * u / r - qb[2] * v / r + qb[3] * P.gm1 * T(0.5) * (u * u + v * v);
    w[1] = qb[1] / r - qb[3] * P.gm1 * u;
    w[2] = qb[2] / r - qb[3] * P.gm1 * v;
    w[3] = qb[3] * P.gm1;
    T res[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      res[k] = c * w[k];
      if (X) res[k] += alpha * X[k * m.plane + idx];
      if (Y) res[k] += beta * Y[k * m.plane + idx];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) out[k * m.plane + idx] = res[k];
  }
}

// Cotangent of the conservative initial state -> gradient with respect to
// the primitive initial fields (rho, u, v, p), written densely (nx*ny planes).
template <typename T>
__global__ void grad_prim_kernel(const MeshDesc m, const T* __restrict__ U0, const T* __restrict__ lam, T* gq) {
  const Phys<T> P(m);
  const long long total = (long long)m.nx * m.ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(t / m.nx), i = (int)(t - (long long)j * m.nx);
    const long long idx = (long long)j * m.pitch + i;
    T q[4];
    load_prim(P, U0, m.plane, idx, q);
    T L[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) L[k] = lam[k * m.plane + idx];
    const T r = q[0], u = q[1], v = q[2];
    // U = (r, r u, r v, p/(gamma-1) + r (u^2+v^2)/2)
    gq[t] = L[0] + L[1] * u + L[2] * v + L[3] * T(0.5) * (u * u + v * v);
    gq[total + t] = (L[1] + L[3] * u) * r;
    gq[2 * total + t] = (L[2] + L[3] * v) * r;
    gq[3 * total + t] = L[3] * P.inv_gm1;
  }
}

}  // namespace lf
