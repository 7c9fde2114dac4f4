// Masked uniform grids: inflow-outflow domains made of active squares of a
// bounding box (Sec. 3, Test problem 3, the flow over a step).
//
// Layout.  The unknowns live on the full lattice of the bounding box (nx x ny
// square elements of side h): Q2 velocity nodes (2nx+1) x (2ny+1), Q1 nodes
// (nx+1) x (ny+1), P0 elements nx*ny, ordered as on the square grid.  Unknowns
// of inactive nodes and elements are kept with identity rows (value 0 in every
// solution).  Velocity rows are identity at the Dirichlet nodes: the active
// nodes on the boundary of the active region, except those strictly inside the
// outflow edge (the right edge of the box), where the weak form leaves the
// natural (do-nothing) condition.  The frame vector k (1 on the active Q1
// nodes, -1 on the active elements) spans the pressure null space (Sec. 2): an
// outflow boundary removes the constant pressure mode.
//
// Operators.  One element pass computes, per active element, the 23 element
// outputs of K (18 velocity rows, 4 Q1 rows, 1 P0 row) with the closed-form /
// Gauss element arithmetic of the square grid (q2_elem), with the velocity of
// the Dirichlet and inactive nodes masked to zero; one node pass gathers them
// (fixed order, no atomics) and applies the identity rows.
//
// Solver.  The two-stage PCD method of Sec. 3.1 (Step I on the reduced Q1
// system with the PCD Schur approximation M_S^{-1} = Ap^{-1} F1 Q1^{-1}, F1
// carrying the inflow Robin term; Step II on the full system with M_1) by
// restarted flexible GMRES, velocity blocks by one FP32 V-cycle of a masked
// geometric multigrid hierarchy (halving nx and ny while the mask stays
// 2 x 2-nested), dense exact solve on the coarsest level; the pressure solves
// (Ap^{-1}, the Schur complement of M_Q) by a few CG steps preconditioned by
// masked Q1 V-cycles; Picard iteration around it.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>
#include "common.cuh"
#include "q1ops.cuh"
#include "q2tile.cuh"

namespace eth {
namespace msk {

constexpr int NE = 23;   // element outputs: 9 + 9 velocity rows, 4 Q1 rows, 1 P0 row

inline unsigned nblk(size_t m, int t = 256) {
  size_t b = (m + t - 1) / t;
  if (b < 1) b = 1;
  if (b > 4096) b = 4096;
  return (unsigned)b;
}

// ---------------------------------------------------------------------------
// element pass: E[k * n0 + e] = output k of active element e
// ---------------------------------------------------------------------------
template <class TI, class CT, int F>
__global__ void __launch_bounds__(128) k_elem(int nx, int ny, CT h, CT nu, CT sdc, const unsigned char* __restrict__ act,
                                              const unsigned char* __restrict__ fix, int mask_in, const TI* __restrict__ x,
                                              const TI* __restrict__ p, const TI* __restrict__ w, CT* __restrict__ E) {
  constexpr bool XIN = F & QF_XIN, PIN = F & QF_PIN, HP0 = F & QF_P0, UOUT = F & QF_UOUT, POUT = F & QF_POUT,
                 WIND = (F & QF_CONV) || (F & QF_SD);
  const int Nx = 2 * nx + 1;
  const size_t nv = (size_t)Nx * (2 * ny + 1), n0 = (size_t)nx * ny, n1 = (size_t)(nx + 1) * (ny + 1);
  const CT ih = CT(1) / h, area = h * h;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n0; e += (size_t)gridDim.x * blockDim.x) {
    if (!act[e]) continue;
    const int ex = (int)(e % nx), ey = (int)(e / nx);
    CT U[2][9], Wn[2][9], P1[4] = {0, 0, 0, 0}, P0 = 0, Y[2][9], YP1[4], YP0 = 0;
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const size_t g = (size_t)(2 * ey + b) * Nx + 2 * ex + a;
        if (XIN) {
          // mask_in 1: Dirichlet/inactive velocity zeroed (D_I x); 2: only those kept (D_B x)
          const bool m = mask_in == 1 ? fix[g] != 0 : (mask_in == 2 ? fix[g] == 0 : false);
          U[0][b * 3 + a] = m ? CT(0) : (CT)x[g];
          U[1][b * 3 + a] = m ? CT(0) : (CT)x[g + nv];
        } else {
          U[0][b * 3 + a] = 0;
          U[1][b * 3 + a] = 0;
        }
        if (WIND) {
          Wn[0][b * 3 + a] = (CT)w[g];
          Wn[1][b * 3 + a] = (CT)w[g + nv];
        } else {
          Wn[0][b * 3 + a] = 0;
          Wn[1][b * 3 + a] = 0;
        }
      }
    if (PIN) {
#pragma unroll
      for (int k = 0; k < 4; ++k) P1[k] = (CT)p[(size_t)(ey + (k >> 1)) * (nx + 1) + ex + (k & 1)];
      if (HP0) P0 = (CT)p[n1 + e];
    }
    q2_elem<CT, F>(U, Wn, P1, P0, nu, ih, ih, area, sdc, Y, YP1, YP0);
    if (UOUT) {
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int i = 0; i < 9; ++i) E[(size_t)(c * 9 + i) * n0 + e] = Y[c][i];
    }
    if (POUT) {
#pragma unroll
      for (int k = 0; k < 4; ++k) E[(size_t)(18 + k) * n0 + e] = YP1[k];
      E[(size_t)22 * n0 + e] = YP0;
    }
  }
}

// Element diagonal of the velocity operator (both components share it):
// E[i * n0 + e] = (F_e)_{ii}, from the element action on unit vectors.
template <class CT, int F>
__global__ void __launch_bounds__(128) k_elem_diag(int nx, int ny, CT h, CT nu, CT sdc, const unsigned char* __restrict__ act,
                                                   const CT* __restrict__ w, CT* __restrict__ E) {
  constexpr bool WIND = (F & QF_CONV) || (F & QF_SD);
  const int Nx = 2 * nx + 1;
  const size_t nv = (size_t)Nx * (2 * ny + 1), n0 = (size_t)nx * ny;
  const CT ih = CT(1) / h, area = h * h;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n0; e += (size_t)gridDim.x * blockDim.x) {
    if (!act[e]) continue;
    const int ex = (int)(e % nx), ey = (int)(e / nx);
    CT Wn[2][9];
    for (int q = 0; q < 9; ++q) {
      const size_t g = (size_t)(2 * ey + q / 3) * Nx + 2 * ex + q % 3;
      Wn[0][q] = WIND ? w[g] : CT(0);
      Wn[1][q] = WIND ? w[g + nv] : CT(0);
    }
    const CT P1[4] = {0, 0, 0, 0};
#pragma unroll 1
    for (int i = 0; i < 9; ++i) {
      CT U[2][9], Y[2][9], YP1[4], YP0;
      for (int j = 0; j < 9; ++j) { U[0][j] = (j == i) ? CT(1) : CT(0); U[1][j] = 0; }
      q2_elem<CT, F>(U, Wn, P1, CT(0), nu, ih, ih, area, sdc, Y, YP1, YP0);
      E[(size_t)i * n0 + e] = Y[0][i];
    }
  }
}

// Full 9 x 9 scalar element matrix (set-up of the coarsest level, FP64):
// M[e * 81 + i * 9 + j] = (F_e)_{ij}.
template <int F>
__global__ void k_elem_mat(int nx, int ny, double h, double nu, double sdc, const unsigned char* __restrict__ act,
                           const double* __restrict__ w, double* __restrict__ M) {
  constexpr bool WIND = (F & QF_CONV) || (F & QF_SD);
  const int Nx = 2 * nx + 1;
  const size_t nv = (size_t)Nx * (2 * ny + 1), n0 = (size_t)nx * ny;
  using CT = double;
  const CT ih = 1.0 / h, area = h * h;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n0; e += (size_t)gridDim.x * blockDim.x) {
    if (!act[e]) continue;
    const int ex = (int)(e % nx), ey = (int)(e / nx);
    CT Wn[2][9];
    for (int q = 0; q < 9; ++q) {
      const size_t g = (size_t)(2 * ey + q / 3) * Nx + 2 * ex + q % 3;
      Wn[0][q] = WIND ? w[g] : 0.0;
      Wn[1][q] = WIND ? w[g + nv] : 0.0;
    }
    const CT P1[4] = {0, 0, 0, 0};
#pragma unroll 1
    for (int j = 0; j < 9; ++j) {
      CT U[2][9], Y[2][9], YP1[4], YP0;
      for (int k = 0; k < 9; ++k) { U[0][k] = (k == j) ? 1.0 : 0.0; U[1][k] = 0; }
      q2_elem<CT, F>(U, Wn, P1, 0.0, nu, ih, ih, area, sdc, Y, YP1, YP0);
      for (int i = 0; i < 9; ++i) M[e * 81 + i * 9 + j] = Y[0][i];
    }
  }
}

// ---------------------------------------------------------------------------
// node passes
// ---------------------------------------------------------------------------
// Sum of the element rows of Q2 node (i, j), component c, over its active
// elements in a fixed order (low element first in y, then in x).
template <class CT>
__device__ __forceinline__ CT vsum(int nx, int ny, int i, int j, int c, size_t n0, const unsigned char* __restrict__ act,
                                   const CT* __restrict__ E) {
  CT s = 0;
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    int ey, bb;
    if (j & 1) { if (u) break; ey = j >> 1; bb = 1; }
    else { ey = (j >> 1) - 1 + u; bb = u ? 0 : 2; }
    if (ey < 0 || ey >= ny) continue;
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      int ex, aa;
      if (i & 1) { if (v) break; ex = i >> 1; aa = 1; }
      else { ex = (i >> 1) - 1 + v; aa = v ? 0 : 2; }
      if (ex < 0 || ex >= nx) continue;
      const size_t e = (size_t)ey * nx + ex;
      if (!act[e]) continue;
      s += E[(size_t)(c * 9 + bb * 3 + aa) * n0 + e];
    }
  }
  return s;
}

enum : int {
  V_ID = 0,      // y = fixed ? a : S            (K, F: identity rows)
  V_ZERO = 1,    // y = fixed ? 0 : S            (B^T)
  V_RHS = 2,     // y = fixed ? a : -S           (lifted right-hand side)
  V_RESID = 3,   // y = fixed ? 0 : a - S        (a: level right-hand side)
  V_SMOOTH = 4,  // y = fixed ? 0 : x + omega d (a - S)
  V_SCALE = 5,   // y = fixed ? 0 : d S
  V_BSUB = 6,    // y = fixed ? a : a - S
  V_DINV = 7     // y = fixed ? 0 : 1 / S        (component 0 only)
};

template <class CT, class TA, class TO>
__global__ void k_vgather(int nx, int ny, int mode, const unsigned char* __restrict__ act, const unsigned char* __restrict__ fix,
                          const CT* __restrict__ E, const TA* __restrict__ a, const CT* __restrict__ x,
                          const CT* __restrict__ d, CT omega, TO* __restrict__ y, int ncomp) {
  const int Nx = 2 * nx + 1;
  const size_t nv = (size_t)Nx * (2 * ny + 1), n0 = (size_t)nx * ny;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < ncomp * nv; k += (size_t)gridDim.x * blockDim.x) {
    const int c = k >= nv ? 1 : 0;
    const size_t g = k - c * nv;
    const int j = (int)(g / Nx), i = (int)(g - (size_t)j * Nx);
    if (fix[g]) {
      TO v = TO(0);
      if (mode == V_ID || mode == V_RHS || mode == V_BSUB) v = (TO)a[k];
      y[k] = v;
      continue;
    }
    const CT s = vsum<CT>(nx, ny, i, j, c, n0, act, E);
    CT out;
    switch (mode) {
      case V_ID: case V_ZERO: out = s; break;
      case V_RHS: out = -s; break;
      case V_RESID: out = (CT)a[k] - s; break;
      case V_SMOOTH: out = x[k] + omega * d[g] * ((CT)a[k] - s); break;
      case V_SCALE: out = d[g] * s; break;
      case V_BSUB: out = (CT)a[k] - s; break;
      default: out = s != CT(0) ? CT(1) / s : CT(0); break;
    }
    y[k] = (TO)out;
  }
}

enum : int {
  P_PIN = 0,     // y = active ? S : a           (K, K1: identity rows of the inactive unknowns)
  P_PLAIN = 1,   // y = active ? S : 0           (B)
  P_NEG = 2      // y = active ? -S : 0          (lifted right-hand side)
};

// Pressure rows: Q1 node (I, J) sums the Q1 outputs of its (up to four) active
// elements; an active element's P0 row is its own output.  count = n1 (Q1 rows
// only, the reduced system) or n1 + n0.
template <class CT, class TA, class TO>
__global__ void k_pgather(int nx, int ny, int mode, size_t count, const unsigned char* __restrict__ act,
                          const unsigned char* __restrict__ q1a, const CT* __restrict__ E, const TA* __restrict__ a,
                          TO* __restrict__ y) {
  const size_t n0 = (size_t)nx * ny, n1 = (size_t)(nx + 1) * (ny + 1);
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < count; k += (size_t)gridDim.x * blockDim.x) {
    bool on;
    CT s = 0;
    if (k < n1) {
      on = q1a[k] != 0;
      if (on) {
        const int J = (int)(k / (nx + 1)), I = (int)(k - (size_t)J * (nx + 1));
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
          for (int dx = 0; dx < 2; ++dx) {
            const int ex = I - 1 + dx, ey = J - 1 + dy;
            if (ex < 0 || ex >= nx || ey < 0 || ey >= ny) continue;
            const size_t e = (size_t)ey * nx + ex;
            if (!act[e]) continue;
            const int c = 1 - dx, dd = 1 - dy;
            s += E[(size_t)(18 + dd * 2 + c) * n0 + e];
          }
      }
    } else {
      const size_t e = k - n1;
      on = act[e] != 0;
      if (on) s = E[(size_t)22 * n0 + e];
    }
    TO v;
    if (on) v = (TO)(mode == P_NEG ? -s : s);
    else v = (mode == P_PIN) ? (TO)a[k] : TO(0);
    y[k] = v;
  }
}

// ---------------------------------------------------------------------------
// multigrid transfers and smoothing helpers (levels nested 2:1)
// ---------------------------------------------------------------------------
// 1D Q2 restriction weight of the fine lattice node at offset o in [-3, 3]
// from 2I (coarse node I odd: element midpoint; I even: element vertex).
__device__ __forceinline__ float rw1(int odd, int o) {
  if (o == 0) return 1.f;
  if (odd) return (o == -1 || o == 1) ? 0.75f : 0.f;
  return (o == -1 || o == 1) ? 0.375f : ((o == -3 || o == 3) ? -0.125f : 0.f);
}
// 1D Q2 interpolation to fine lattice index i: base coarse index and weights
// (even i: injection; i = 4E+1: 3/8, 3/4, -1/8; i = 4E+3: -1/8, 3/4, 3/8).
__device__ __forceinline__ int pw1(int i, float& w0, float& w1, float& w2) {
  if (!(i & 1)) { w0 = 1.f; w1 = 0.f; w2 = 0.f; return i >> 1; }
  const int E = i >> 2;
  if ((i & 3) == 1) { w0 = 0.375f; w1 = 0.75f; w2 = -0.125f; }
  else { w0 = -0.125f; w1 = 0.75f; w2 = 0.375f; }
  return 2 * E;
}

// b_c = P^T r_f on the free coarse nodes (0 on the fixed ones); r_f vanishes
// on the fixed fine nodes.  Fine offsets outside the lattice are skipped (the
// free outflow nodes sit on the box edge).
template <class T>
__global__ void k_restrict(int nxc, int nyc, const unsigned char* __restrict__ fixc, const T* __restrict__ rf, T* __restrict__ bc) {
  const int Nxc = 2 * nxc + 1, Nyc = 2 * nyc + 1, Nxf = 4 * nxc + 1, Nyf = 4 * nyc + 1;
  const size_t nvc = (size_t)Nxc * Nyc, nvf = (size_t)Nxf * Nyf;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < nvc; g += (size_t)gridDim.x * blockDim.x) {
    if (fixc[g]) { bc[g] = 0; bc[g + nvc] = 0; continue; }
    const int J = (int)(g / Nxc), I = (int)(g - (size_t)J * Nxc);
    const int ox = I & 1, oy = J & 1;
    T s0 = 0, s1 = 0;
#pragma unroll
    for (int u = -3; u <= 3; ++u) {
      const float wy = rw1(oy, u);
      const int fj = 2 * J + u;
      if (wy == 0.f || fj < 0 || fj >= Nyf) continue;
      T t0 = 0, t1 = 0;
#pragma unroll
      for (int v = -3; v <= 3; ++v) {
        const float wx = rw1(ox, v);
        const int fi = 2 * I + v;
        if (wx == 0.f || fi < 0 || fi >= Nxf) continue;
        const size_t f = (size_t)fj * Nxf + fi;
        t0 += (T)wx * rf[f];
        t1 += (T)wx * rf[f + nvf];
      }
      s0 += (T)wy * t0;
      s1 += (T)wy * t1;
    }
    bc[g] = s0;
    bc[g + nvc] = s1;
  }
}

// x_f += P x_c on the free fine nodes
template <class T>
__global__ void k_prolong_add(int nxc, int nyc, const unsigned char* __restrict__ fixf, const T* __restrict__ xc, T* __restrict__ xf) {
  const int Nxc = 2 * nxc + 1, Nyc = 2 * nyc + 1, Nxf = 4 * nxc + 1, Nyf = 4 * nyc + 1;
  const size_t nvc = (size_t)Nxc * Nyc, nvf = (size_t)Nxf * Nyf;
  for (size_t f = blockIdx.x * (size_t)blockDim.x + threadIdx.x; f < nvf; f += (size_t)gridDim.x * blockDim.x) {
    if (fixf[f]) continue;
    const int j = (int)(f / Nxf), i = (int)(f - (size_t)j * Nxf);
    float wx[3], wy[3];
    const int cx = pw1(i, wx[0], wx[1], wx[2]), cy = pw1(j, wy[0], wy[1], wy[2]);
    T s0 = 0, s1 = 0;
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        if (wx[v] == 0.f || wy[u] == 0.f) continue;
        const size_t c = (size_t)(cy + u) * Nxc + cx + v;
        const T fw = (T)(wx[v] * wy[u]);
        s0 += fw * xc[c];
        s1 += fw * xc[c + nvc];
      }
    xf[f] += s0;
    xf[f + nvf] += s1;
  }
}

// coarse wind = fine wind at the coarse nodes (coarse Q2 nodes are fine Q2 nodes)
template <class TI, class T>
__global__ void k_inject(int nxc, int nyc, const TI* __restrict__ wf, T* __restrict__ wc) {
  const int Nxc = 2 * nxc + 1, Nyc = 2 * nyc + 1, Nxf = 4 * nxc + 1, Nyf = 4 * nyc + 1;
  const size_t nvc = (size_t)Nxc * Nyc, nvf = (size_t)Nxf * Nyf;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < nvc; g += (size_t)gridDim.x * blockDim.x) {
    const int J = (int)(g / Nxc), I = (int)(g - (size_t)J * Nxc);
    const size_t f = (size_t)(2 * J) * Nxf + 2 * I;
    wc[g] = (T)wf[f];
    wc[g + nvc] = (T)wf[f + nvf];
  }
}

template <class TI, class T>
__global__ void k_cast(size_t m, const TI* __restrict__ a, T* __restrict__ b) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) b[k] = (T)a[k];
}

// level right-hand side from an FP64 vector (0 on fixed nodes) and the first
// Jacobi sweep from a zero guess: b = v, x = omega D^{-1} b
template <class TI, class T>
__global__ void k_jac0(size_t nv, const unsigned char* __restrict__ fix, const T* __restrict__ dinv, T omega,
                       const TI* __restrict__ v, T* __restrict__ b, T* __restrict__ x) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < 2 * nv; k += (size_t)gridDim.x * blockDim.x) {
    const size_t g = k >= nv ? k - nv : k;
    const T bv = fix[g] ? T(0) : (T)v[k];
    if ((const void*)v != (const void*)b) b[k] = bv;
    x[k] = omega * dinv[g] * bv;
  }
}

// coarsest level: x = A_c^{-1} b on the free nodes (column-major inverse over
// the free-node list idx), both components (blockIdx.y); fixed nodes stay 0.
template <class T>
__global__ void k_cdense(int m, size_t nv, const int* __restrict__ idx, const T* __restrict__ Ainv, const T* __restrict__ b,
                         T* __restrict__ x) {
  const size_t off = (size_t)blockIdx.y * nv;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
    T s = 0;
    for (int k = 0; k < m; ++k) s += Ainv[(size_t)k * m + r] * b[off + idx[k]];
    x[off + idx[r]] = s;
  }
}

// z_u = x (free nodes), v (fixed nodes: the identity rows of F)
template <class T>
__global__ void k_vout(size_t nv, const unsigned char* __restrict__ fix, const T* __restrict__ x, const double* __restrict__ v,
                       double* __restrict__ z) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < 2 * nv; k += (size_t)gridDim.x * blockDim.x) {
    const size_t g = k >= nv ? k - nv : k;
    z[k] = fix[g] ? v[k] : (double)x[k];
  }
}

// ---------------------------------------------------------------------------
// pressure-space operators on the masked grid (FP64)
// ---------------------------------------------------------------------------
// Q1 matrix F1_e = nu K1_e + C_e(w) + R_e(w) of every active element (row =
// test node, local index d*2 + c), Sec. 3.1 Eq. discrete-commutator1x: K1 the Q1
// stiffness, C the Q1 convection int psi_i (w_h . grad psi_j) (3x3 Gauss, Q2
// wind), R the inflow Robin term -int_{Gamma_in} (w.n) psi_i psi_j ds on the
// element's boundary edges (edges of the active region) where the wind enters
// (w.n < 0 at the edge midpoint), 3-point Gauss on the edge with the Q2 trace of
// w.  w == nullptr: the Stokes case (F1 = nu K1).
__global__ void k_f1_elem(int nx, int ny, double h, double nu, const unsigned char* __restrict__ act,
                          const double* __restrict__ w, double* __restrict__ F1e) {
  const int Nx = 2 * nx + 1;
  const size_t nv = (size_t)Nx * (2 * ny + 1), n0 = (size_t)nx * ny;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n0; e += (size_t)gridDim.x * blockDim.x) {
    if (!act[e]) continue;
    const int ex = (int)(e % nx), ey = (int)(e / nx);
    double c[4][4];
    for (int li = 0; li < 4; ++li)
      for (int lj = 0; lj < 4; ++lj) {
        const int ci = li & 1, di = li >> 1, cj = lj & 1, dj = lj >> 1;
        c[li][lj] = nu * (q1k(ci, cj) * q1m(di, dj) + q1m(ci, cj) * q1k(di, dj));
      }
    if (w != nullptr) {
      for (int qy = 0; qy < 3; ++qy)
        for (int qx = 0; qx < 3; ++qx) {
          double wx = 0, wy = 0;
          for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a) {
              const double f = q2v(a, gq(qx)) * q2v(b, gq(qy));
              const size_t g = (size_t)(2 * ey + b) * Nx + 2 * ex + a;
              wx += f * w[g];
              wy += f * w[g + nv];
            }
          const double W = gw(qx) * gw(qy) * h * h;
          for (int li = 0; li < 4; ++li) {
            const double psi = q1v(li & 1, gq(qx)) * q1v(li >> 1, gq(qy));
            for (int lj = 0; lj < 4; ++lj) {
              const int cj = lj & 1, dj = lj >> 1;
              const double dx = q1d(cj) * q1v(dj, gq(qy)) / h, dy = q1v(cj, gq(qx)) * q1d(dj) / h;
              c[li][lj] += W * psi * (wx * dx + wy * dy);
            }
          }
        }
      // inflow Robin term on the boundary edges
      for (int s = 0; s < 4; ++s) {
        const int fx = ex + (s == 0 ? -1 : (s == 1 ? 1 : 0)), fy = ey + (s == 2 ? -1 : (s == 3 ? 1 : 0));
        if (fx >= 0 && fx < nx && fy >= 0 && fy < ny && act[(size_t)fy * nx + fx]) continue;   // interior edge
        const double onx = s == 0 ? -1.0 : (s == 1 ? 1.0 : 0.0), ony = s == 2 ? -1.0 : (s == 3 ? 1.0 : 0.0);
        double wn[3];
        for (int k = 0; k < 3; ++k) {
          const int gi = s == 0 ? 2 * ex : (s == 1 ? 2 * ex + 2 : 2 * ex + k);
          const int gj = s == 2 ? 2 * ey : (s == 3 ? 2 * ey + 2 : 2 * ey + k);
          const size_t g = (size_t)gj * Nx + gi;
          wn[k] = w[g] * onx + w[g + nv] * ony;
        }
        if (wn[1] >= 0.0) continue;   // not an inflow edge
        // local Q1 indices of the edge's two end nodes, in the direction of t
        const int l0 = s == 0 ? 0 : (s == 1 ? 1 : (s == 2 ? 0 : 2));
        const int l1 = s == 0 ? 2 : (s == 1 ? 3 : (s == 2 ? 1 : 3));
        const int lid[2] = {l0, l1};
        for (int q = 0; q < 3; ++q) {
          const double t = gq(q);
          const double wng = q2v(0, t) * wn[0] + q2v(1, t) * wn[1] + q2v(2, t) * wn[2];
          const double lin[2] = {1.0 - t, t};
          for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) c[lid[a]][lid[b]] -= gw(q) * wng * h * lin[a] * lin[b];
        }
      }
    }
    for (int li = 0; li < 4; ++li)
      for (int lj = 0; lj < 4; ++lj) F1e[e * 16 + li * 4 + lj] = c[li][lj];
  }
}

// Q1 node operator with identity rows on the inactive nodes:
// y_I = sum over active elements T around I of (M_T x)_I, M_T = F1e[T]
// (F1e != nullptr) or h^2 (m (x) m + c1) (c1 = 0: the Q1 mass; c1 = -1/16: the
// Schur complement S = Qk - R^T Q0^{-1} R of M_Q, element by element).
__global__ void k_q1apply(int nx, int ny, double h, const unsigned char* __restrict__ act, const unsigned char* __restrict__ q1a,
                          const double* __restrict__ F1e, double c1, const double* __restrict__ x, double* __restrict__ y) {
  const int M = nx + 1;
  const size_t n1 = (size_t)M * (ny + 1);
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n1; k += (size_t)gridDim.x * blockDim.x) {
    if (!q1a[k]) { y[k] = x[k]; continue; }
    const int J = (int)(k / M), I = (int)(k - (size_t)J * M);
    double s = 0;
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        const int ex = I - 1 + dx, ey = J - 1 + dy;
        if (ex < 0 || ex >= nx || ey < 0 || ey >= ny) continue;
        const size_t e = (size_t)ey * nx + ex;
        if (!act[e]) continue;
        const int c = 1 - dx, d = 1 - dy, li = d * 2 + c;
        for (int lj = 0; lj < 4; ++lj) {
          const int cj = lj & 1, dj = lj >> 1;
          const double m = F1e != nullptr ? F1e[e * 16 + li * 4 + lj] : h * h * (q1m(c, cj) * q1m(d, dj) + c1);
          s += m * x[(size_t)(ey + dj) * M + ex + cj];
        }
      }
    y[k] = s;
  }
}

// Two-field pressure mass M_Q = [Qk R^T; R Q0] (Sec. 2.3; R = |T|/4, Q0 = |T|)
// over the active elements; rows of the inactive unknowns: identity (pin) or zero.
__global__ void k_mq_apply(int nx, int ny, double h, const unsigned char* __restrict__ act, const unsigned char* __restrict__ q1a,
                           int pin, const double* __restrict__ x, double* __restrict__ y) {
  const int M = nx + 1;
  const size_t n1 = (size_t)M * (ny + 1), n0 = (size_t)nx * ny;
  const double area = h * h;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n1 + n0; k += (size_t)gridDim.x * blockDim.x) {
    if (k < n1) {
      if (!q1a[k]) { y[k] = pin ? x[k] : 0.0; continue; }
      const int J = (int)(k / M), I = (int)(k - (size_t)J * M);
      double s = 0;
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const int ex = I - 1 + dx, ey = J - 1 + dy;
          if (ex < 0 || ex >= nx || ey < 0 || ey >= ny) continue;
          const size_t e = (size_t)ey * nx + ex;
          if (!act[e]) continue;
          const int c = 1 - dx, d = 1 - dy;
          for (int lj = 0; lj < 4; ++lj) {
            const int cj = lj & 1, dj = lj >> 1;
            s += area * q1m(c, cj) * q1m(d, dj) * x[(size_t)(ey + dj) * M + ex + cj];
          }
          s += 0.25 * area * x[n1 + e];
        }
      y[k] = s;
    } else {
      const size_t e = k - n1;
      if (!act[e]) { y[k] = pin ? x[k] : 0.0; continue; }
      const int ex = (int)(e % nx), ey = (int)(e / nx);
      const double s1 = x[(size_t)ey * M + ex] + x[(size_t)ey * M + ex + 1] + x[(size_t)(ey + 1) * M + ex] +
                        x[(size_t)(ey + 1) * M + ex + 1];
      y[k] = 0.25 * area * s1 + area * x[k];
    }
  }
}

// Diagonal data of the PCD and M_Q solves:
//  mdinv (N_v): inverse diagonal of the velocity mass matrix on the free nodes, 0 on fixed ones
//  (the Md of Ap = B1 Md^{-1} B1^T);
//  q1dinv (N_1): inverse diagonal of the Q1 mass (1 on inactive nodes);
//  kv (N_1 + N_0): the frame vector k (1 on active Q1 nodes, -1 on active elements).
__global__ void k_diag_setup(int nx, int ny, double h, const unsigned char* __restrict__ act, const unsigned char* __restrict__ fix,
                             const unsigned char* __restrict__ q1a, double* __restrict__ mdinv, double* __restrict__ q1dinv,
                             double* __restrict__ kv) {
  const int Nx = 2 * nx + 1, M = nx + 1;
  const size_t nv = (size_t)Nx * (2 * ny + 1), n1 = (size_t)M * (ny + 1), n0 = (size_t)nx * ny;
  const double area = h * h;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < nv + n1 + n0; k += (size_t)gridDim.x * blockDim.x) {
    if (k < nv) {
      if (fix[k]) { mdinv[k] = 0; continue; }
      const int j = (int)(k / Nx), i = (int)(k - (size_t)j * Nx);
      double s = 0;
      for (int u = 0; u < 2; ++u) {
        int ey, bb;
        if (j & 1) { if (u) break; ey = j >> 1; bb = 1; } else { ey = (j >> 1) - 1 + u; bb = u ? 0 : 2; }
        if (ey < 0 || ey >= ny) continue;
        for (int v = 0; v < 2; ++v) {
          int ex, aa;
          if (i & 1) { if (v) break; ex = i >> 1; aa = 1; } else { ex = (i >> 1) - 1 + v; aa = v ? 0 : 2; }
          if (ex < 0 || ex >= nx || !act[(size_t)ey * nx + ex]) continue;
          s += area * m1d(aa, aa) * m1d(bb, bb);
        }
      }
      mdinv[k] = 1.0 / s;
    } else if (k < nv + n1) {
      const size_t q = k - nv;
      double cnt = 0;
      if (q1a[q]) {
        const int J = (int)(q / M), I = (int)(q - (size_t)J * M);
        for (int dy = 0; dy < 2; ++dy)
          for (int dx = 0; dx < 2; ++dx) {
            const int ex = I - 1 + dx, ey = J - 1 + dy;
            if (ex >= 0 && ex < nx && ey >= 0 && ey < ny && act[(size_t)ey * nx + ex]) cnt += 1.0;
          }
      }
      const double d = cnt * area / 9.0;
      q1dinv[q] = q1a[q] ? 1.0 / d : 1.0;
      kv[q] = q1a[q] ? 1.0 : 0.0;
    } else {
      const size_t e = k - nv - n1;
      kv[n1 + e] = act[e] ? -1.0 : 0.0;
    }
  }
}

// ---------------------------------------------------------------------------
// vector kernels and deterministic reductions (FP64)
// ---------------------------------------------------------------------------
constexpr int RB = 256;     // threads per reduction block
inline int rblocks(size_t m) {
  size_t b = (m + 4 * RB - 1) / (4 * RB);
  if (b < 1) b = 1;
  if (b > 1024) b = 1024;
  return (int)b;
}

// out[0] = <a, b> (and out[1] = <c, d> when c != nullptr); scale: out *= s
__global__ void __launch_bounds__(RB) k_dot(size_t m, const double* __restrict__ a, const double* __restrict__ b,
                                            const double* __restrict__ c, const double* __restrict__ d, Slot sl, double* out) {
  double v[2] = {0.0, 0.0};
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) {
    v[0] += a[k] * b[k];
    if (c != nullptr) v[1] += c[k] * d[k];
  }
  if (slot_arrive<2>(sl, blockIdx.x, v)) { out[0] = v[0]; out[1] = v[1]; }
}

// y = a x + b y
__global__ void k_axpby(size_t m, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) y[k] = a * x[k] + b * y[k];
}
// y = x - (s[0] / kk) k   (removes the component of x along k; s[0] = <k, x>)
__global__ void k_proj(size_t m, const double* __restrict__ x, const double* __restrict__ kv, const double* __restrict__ s,
                       double kk, double* __restrict__ y) {
  const double f = s[0] / kk;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) y[k] = x[k] - f * kv[k];
}
__global__ void k_scale(size_t m, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) y[k] = a * x[k];
}

// ---- preconditioned CG with device-resident scalars (Jacobi preconditioner)
struct PcgS {
  double rz, rr0, alpha, beta, tol2;
  int done, its, pad;
};

// alpha = rz / <p, q>
__global__ void __launch_bounds__(RB) k_pcg_alpha(size_t m, const double* __restrict__ p, const double* __restrict__ q, PcgS* st, Slot sl) {
  if (st->done) return;
  double v[1] = {0.0};
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) v[0] += p[k] * q[k];
  if (slot_arrive<1>(sl, blockIdx.x, v)) {
    if (v[0] > 0.0) st->alpha = st->rz / v[0];
    else st->done = 1;
  }
}
// p = z + beta p
__global__ void k_pcg_p(size_t m, const double* __restrict__ z, double* __restrict__ p, const PcgS* st) {
  if (st->done) return;
  const double be = st->beta;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) p[k] = z[k] + be * p[k];
}

// ---- GMRES basis kernels (basis vectors V_i at V + i * ld)
// part[i * nb + b] = <V_i, w> over block b's share (grid nb x nvec)
__global__ void __launch_bounds__(RB) k_mdot(size_t n, const double* __restrict__ V, size_t ld, const double* __restrict__ w,
                                             double* __restrict__ part) {
  const int i = blockIdx.y, nb = gridDim.x;
  const double* v = V + (size_t)i * ld;
  double acc = 0.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)nb * blockDim.x) acc += v[k] * w[k];
  double a[1] = {acc};
  block_sum<1>(a);
  if (threadIdx.x == 0) part[(size_t)i * nb + blockIdx.x] = a[0];
}
// h[i] (+)= sum_b part[i * nb + b] in block order (one warp per i)
__global__ void k_msum(int nvec, int nb, const double* __restrict__ part, double* __restrict__ h, int accumulate) {
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= nvec) return;
  double a = 0.0;
  for (int b = lane; b < nb; b += 32) a += part[(size_t)i * nb + b];
  a = warp_sum(a);
  if (lane == 0) h[i] = accumulate ? h[i] + a : a;
}
// w -= sum_i h[i] V_i
__global__ void k_mupd(size_t n, const double* __restrict__ V, size_t ld, int nvec, const double* __restrict__ h,
                       double* __restrict__ w) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    double s = w[k];
    for (int i = 0; i < nvec; ++i) s -= h[i] * V[(size_t)i * ld + k];
    w[k] = s;
  }
}
// v = w / sqrt(h[j1]) (h[j1] = <w, w>; v = 0 if it vanishes).  h[j1] itself is
// replaced by the norm in a separate launch (k_hsqrt), after every block has read it.
__global__ void k_vnext(size_t n, const double* __restrict__ w, double* __restrict__ v, const double* h, int j1) {
  const double nn = sqrt(fmax(h[j1], 0.0));
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
    v[k] = nn > 0.0 ? w[k] / nn : 0.0;
}
__global__ void k_hsqrt(double* h, int j1) { h[j1] = sqrt(fmax(h[j1], 0.0)); }
// x += sum_i y[i] Z_i
__global__ void k_zupd(size_t n, const double* __restrict__ Z, size_t ld, int k, const double* __restrict__ y, double* __restrict__ x) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    double s = x[t];
    for (int i = 0; i < k; ++i) s += y[i] * Z[(size_t)i * ld + t];
    x[t] = s;
  }
}
// r = b - r (r holds K x on entry)
__global__ void k_bminus(size_t n, const double* __restrict__ b, double* __restrict__ r) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) r[k] = b[k] - r[k];
}

}  // namespace msk
}  // namespace eth

// ===========================================================================
// host side
// ===========================================================================
namespace eth {
namespace msk {

// one level of the masked velocity hierarchy (FP32)
struct MLev {
  int nx = 0, ny = 0;
  double h = 0;
  size_t nv = 0, n0 = 0;
  unsigned char *act = nullptr, *fix = nullptr;   // device masks
  std::vector<unsigned char> hact;                // host element mask
  bool own = false;                               // masks owned (coarse levels)
  float *dinv = nullptr, *w = nullptr, *x = nullptr, *b = nullptr, *r = nullptr, *t = nullptr;
};

// one level of a masked Q1 hierarchy (FP64)
struct QLev {
  int nx = 0, ny = 0;
  size_t n1 = 0;
  const unsigned char* act = nullptr;    // the velocity level's element mask
  unsigned char* q1a = nullptr;          // active Q1 nodes (device)
  std::vector<unsigned char> hq1a;
  double *d = nullptr, *x = nullptr, *b = nullptr, *r = nullptr;
};
struct QHier {
  std::vector<QLev> lv;
  double shift = 0.0;
  double* cinv = nullptr;
  int* cidx = nullptr;
  int ncf = 0;
};

// Node roles of a masked grid (the definitions of the header comment).
static void node_roles(int nx, int ny, int outflow, const std::vector<unsigned char>& act, std::vector<unsigned char>& fix,
                       std::vector<unsigned char>& dir, std::vector<unsigned char>& q1a) {
  const int Nx = 2 * nx + 1, Ny = 2 * ny + 1;
  const size_t nv = (size_t)Nx * Ny;
  fix.assign(nv, 0);
  dir.assign(nv, 0);
  q1a.assign((size_t)(nx + 1) * (ny + 1), 0);
  std::vector<unsigned char> q2a(nv, 0), bnd(nv, 0);
  auto on = [&](int ex, int ey) { return ex >= 0 && ex < nx && ey >= 0 && ey < ny && act[(size_t)ey * nx + ex]; };
  for (int j = 0; j < Ny; ++j)
    for (int i = 0; i < Nx; ++i) {
      int exs[2], eys[2], nex = 0, ney = 0;
      if (i & 1) exs[nex++] = i >> 1; else { exs[nex++] = (i >> 1) - 1; exs[nex++] = i >> 1; }
      if (j & 1) eys[ney++] = j >> 1; else { eys[ney++] = (j >> 1) - 1; eys[ney++] = j >> 1; }
      bool any = false, all = true;
      for (int a = 0; a < ney; ++a)
        for (int b = 0; b < nex; ++b) {
          const bool o = on(exs[b], eys[a]);
          any = any || o;
          all = all && o;
        }
      const size_t g = (size_t)j * Nx + i;
      q2a[g] = any;
      bnd[g] = any && !all;
    }
  std::vector<unsigned char> outf(nv, 0);
  if (outflow) {
    int jmin = Ny, jmax = -1;
    for (int j = 0; j < Ny; ++j)
      if (bnd[(size_t)j * Nx + Nx - 1]) { jmin = std::min(jmin, j); jmax = std::max(jmax, j); }
    for (int j = jmin + 1; j < jmax; ++j)
      if (bnd[(size_t)j * Nx + Nx - 1]) outf[(size_t)j * Nx + Nx - 1] = 1;
  }
  for (size_t g = 0; g < nv; ++g) {
    dir[g] = bnd[g] && !outf[g];
    fix[g] = dir[g] || !q2a[g];
  }
  for (int J = 0; J <= ny; ++J)
    for (int I = 0; I <= nx; ++I)
      q1a[(size_t)J * (nx + 1) + I] = on(I - 1, J - 1) || on(I, J - 1) || on(I - 1, J) || on(I, J);
}

// In-place Gauss-Jordan inverse with partial pivoting (row-major m x m)
static bool invert_dense(std::vector<double>& A, int m) {
  std::vector<double> I((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) I[(size_t)i * m + i] = 1.0;
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int r = c + 1; r < m; ++r)
      if (std::fabs(A[(size_t)r * m + c]) > std::fabs(A[(size_t)piv * m + c])) piv = r;
    if (!(std::fabs(A[(size_t)piv * m + c]) > 0.0)) return false;
    if (piv != c)
      for (int k = 0; k < m; ++k) {
        std::swap(A[(size_t)piv * m + k], A[(size_t)c * m + k]);
        std::swap(I[(size_t)piv * m + k], I[(size_t)c * m + k]);
      }
    const double d = 1.0 / A[(size_t)c * m + c];
    for (int k = 0; k < m; ++k) { A[(size_t)c * m + k] *= d; I[(size_t)c * m + k] *= d; }
    for (int r = 0; r < m; ++r) {
      if (r == c) continue;
      const double f = A[(size_t)r * m + c];
      if (f == 0.0) continue;
      for (int k = 0; k < m; ++k) { A[(size_t)r * m + k] -= f * A[(size_t)c * m + k]; I[(size_t)r * m + k] -= f * I[(size_t)c * m + k]; }
    }
  }
  A.swap(I);
  return true;
}

}  // namespace msk
}  // namespace eth

using eth::msk::MLev;
using eth::msk::QHier;
using eth::msk::QLev;
using eth::msk::PcgS;

struct eth_mgrid {
  int dev = 0;
  cudaStream_t s = nullptr;
  int nx = 0, ny = 0, outflow = 0;
  double h = 0, x0 = 0, y0 = 0;
  size_t nv = 0, n1 = 0, n0 = 0, nu2 = 0, np = 0, nt = 0;
  double nu = 1.0;
  bool has_coef = false, conv = false, prec_ok = false;
  std::vector<unsigned char> h_act, h_fix, h_dir, h_q1a;
  unsigned char *act = nullptr, *fix = nullptr, *q1a = nullptr;
  double* wind = nullptr;       // 2 N_v
  double* E = nullptr;          // element outputs (23 N_0)
  double* part = nullptr;       // reduction partials
  unsigned* ticket = nullptr;
  double* red = nullptr;        // reduction results (device, 64)
  double* redh = nullptr;       // pinned mirror (64)
  double *mdinv = nullptr, *q1dinv = nullptr, *kv = nullptr, *f1e = nullptr;
  double kk = 0.0;
  double *t0 = nullptr, *t1 = nullptr, *t2 = nullptr, *xs = nullptr;          // N_t scratch
  double *pr = nullptr, *pz = nullptr, *pp = nullptr, *pq = nullptr, *px = nullptr, *pa = nullptr, *pb = nullptr;  // N_1 + N_0
  PcgS* pcg = nullptr;           // inner CG scalars (device)
  std::vector<MLev> lv;
  eth::msk::QHier qh[2];        // Q1 hierarchies: [0] Ap preconditioner, [1] Schur complement of M_Q
  float* E32 = nullptr;         // level element outputs (18 N_0 of level 0)
  float* cinv = nullptr;
  int* cidx = nullptr;
  int ncf = 0;
  double *V = nullptr, *Z = nullptr, *hd = nullptr, *hd2 = nullptr, *yd = nullptr, *hh = nullptr, *mpart = nullptr;
  int gm_m = 0;                 // restart length the GMRES workspace holds
  double* bv = nullptr;         // right-hand side buffer of the Picard iteration (N_t)
  double* zo = nullptr;         // preconditioned vector of the captured Arnoldi step (N_t)
  cudaStream_t si = nullptr;    // internal stream of the solver (capturable)
  cudaEvent_t ev[2] = {nullptr, nullptr};
  // captured "z = P^{-1} v, w = K z" of each stage (v in xs, z in zo, w in t2) and the
  // launch parameters they were captured with
  cudaGraphExec_t gx[2] = {nullptr, nullptr};
  double gsig[2][5] = {{0}};
  long gnodes[2] = {0, 0};       // nodes of each captured graph
  long launches = 0;
};

namespace eth {
namespace msk {

using G = eth_mgrid;
constexpr double SDC = 0.5;     // streamline-diffusion coefficient of the preconditioner's levels
constexpr int DOT_NB = 1024;    // partial slots of k_dot

static Slot slot(G* g, int nb) {
  Slot s{};
  s.part = g->part;
  s.ticket = g->ticket;
  s.out = nullptr;
  s.total = nb;
  return s;
}

// red[o], red[o+1] = <a, b>, <c, d> (asynchronous)
static eth_status dot2(G* g, size_t m, const double* a, const double* b, const double* c, const double* d, int o) {
  const int nb = rblocks(m);
  k_dot<<<nb, RB, 0, g->s>>>(m, a, b, c, d, slot(g, nb), g->red + o);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  return ETH_OK;
}
static eth_status fetch(G* g, int count) {
  ETH_CUDA(cudaMemcpyAsync(g->redh, g->red, count * sizeof(double), cudaMemcpyDeviceToHost, g->s));
  ETH_CUDA(cudaStreamSynchronize(g->s));
  return ETH_OK;
}

// ---- FP64 operator applies on level 0
template <int F>
static eth_status elem64(G* g, int mask_in, const double* x, const double* p, const double* w) {
  k_elem<double, double, F><<<nblk(g->n0, 128), 128, 0, g->s>>>(g->nx, g->ny, g->h, g->nu, 0.0, g->act, g->fix, mask_in, x, p, w, g->E);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  return ETH_OK;
}
static eth_status vgat64(G* g, int mode, const double* a, const double* d, double* y) {
  k_vgather<double, double, double><<<nblk(2 * g->nv), 256, 0, g->s>>>(g->nx, g->ny, mode, g->act, g->fix, g->E, a, nullptr, d,
                                                                         0.0, y, 2);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  return ETH_OK;
}
static eth_status pgat64(G* g, int mode, size_t count, const double* a, double* y) {
  k_pgather<double, double, double><<<nblk(count), 256, 0, g->s>>>(g->nx, g->ny, mode, count, g->act, g->q1a, g->E, a, y);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  return ETH_OK;
}

// y = K x (full) or K1 x (reduced: velocity and Q1 pressure)
static eth_status apply_K(G* g, bool reduced, const double* x, double* y) {
  const double* p = x + g->nu2;
  constexpr int FK = QF_DIFF | QF_XIN | QF_PIN | QF_UOUT | QF_POUT;
  if (reduced) {
    if (g->conv) ETH_TRY((elem64<FK | QF_CONV>(g, 1, x, p, g->wind)));
    else ETH_TRY((elem64<FK>(g, 1, x, p, nullptr)));
    ETH_TRY(vgat64(g, V_ID, x, nullptr, y));
    return pgat64(g, P_PIN, g->n1, p, y + g->nu2);
  }
  if (g->conv) ETH_TRY((elem64<FK | QF_P0 | QF_CONV>(g, 1, x, p, g->wind)));
  else ETH_TRY((elem64<FK | QF_P0>(g, 1, x, p, nullptr)));
  ETH_TRY(vgat64(g, V_ID, x, nullptr, y));
  return pgat64(g, P_PIN, g->np, p, y + g->nu2);
}

// y_u = r_u - D_I B^T zp (B1^T only when !p0); fixed rows keep r_u
static eth_status bsub(G* g, bool p0, const double* ru, const double* zp, double* y) {
  if (p0) ETH_TRY((elem64<QF_PIN | QF_P0 | QF_UOUT>(g, 0, nullptr, zp, nullptr)));
  else ETH_TRY((elem64<QF_PIN | QF_UOUT>(g, 0, nullptr, zp, nullptr)));
  return vgat64(g, V_BSUB, ru, nullptr, y);
}

}  // namespace msk
}  // namespace eth

// ---------------------------------------------------------------------------
// masked multigrid for the velocity blocks (FP32 levels)
// ---------------------------------------------------------------------------
namespace eth {
namespace msk {

constexpr int FV = QF_DIFF | QF_XIN | QF_UOUT;              // level operator nu A
constexpr int FVC = FV | QF_CONV | QF_SD;                    // + N(w) + streamline diffusion
constexpr int MAX_COARSE_FREE = 2048;                        // dense coarsest-level solve

static void mg_free(G* g) {
  for (MLev& L : g->lv) {
    if (L.own) { cudaFree(L.act); cudaFree(L.fix); }
    cudaFree(L.dinv); cudaFree(L.w); cudaFree(L.x); cudaFree(L.b); cudaFree(L.r); cudaFree(L.t);
  }
  g->lv.clear();
  for (QHier& Q : g->qh) {
    for (QLev& L : Q.lv) { cudaFree(L.q1a); cudaFree(L.d); cudaFree(L.x); cudaFree(L.b); cudaFree(L.r); }
    Q.lv.clear();
    cudaFree(Q.cinv); cudaFree(Q.cidx);
    Q.cinv = nullptr; Q.cidx = nullptr; Q.ncf = 0;
  }
  cudaFree(g->E32); g->E32 = nullptr;
  cudaFree(g->cinv); g->cinv = nullptr;
  cudaFree(g->cidx); g->cidx = nullptr;
  g->ncf = 0;
}

// Level geometry: halve nx and ny while both are even and every 2 x 2 block of
// elements is wholly active or wholly inactive.
static eth_status mg_build_geometry(G* g) {
  std::vector<unsigned char> act = g->h_act;
  int nx = g->nx, ny = g->ny;
  double h = g->h;
  for (int l = 0;; ++l) {
    MLev L;
    L.nx = nx; L.ny = ny; L.h = h;
    L.hact = act;
    L.nv = (size_t)(2 * nx + 1) * (2 * ny + 1);
    L.n0 = (size_t)nx * ny;
    if (l == 0) {
      L.act = g->act; L.fix = g->fix; L.own = false;
    } else {
      std::vector<unsigned char> fix, dir, q1a;
      node_roles(nx, ny, g->outflow, act, fix, dir, q1a);
      L.own = true;
      ETH_CUDA(cudaMalloc((void**)&L.act, L.n0));
      ETH_CUDA(cudaMalloc((void**)&L.fix, L.nv));
      ETH_CUDA(cudaMemcpy(L.act, act.data(), L.n0, cudaMemcpyHostToDevice));
      ETH_CUDA(cudaMemcpy(L.fix, fix.data(), L.nv, cudaMemcpyHostToDevice));
    }
    ETH_CUDA(cudaMalloc((void**)&L.dinv, L.nv * sizeof(float)));
    ETH_CUDA(cudaMalloc((void**)&L.w, 2 * L.nv * sizeof(float)));
    ETH_CUDA(cudaMalloc((void**)&L.x, 2 * L.nv * sizeof(float)));
    ETH_CUDA(cudaMalloc((void**)&L.b, 2 * L.nv * sizeof(float)));
    ETH_CUDA(cudaMalloc((void**)&L.r, 2 * L.nv * sizeof(float)));
    ETH_CUDA(cudaMalloc((void**)&L.t, 2 * L.nv * sizeof(float)));
    ETH_CUDA(cudaMemset(L.w, 0, 2 * L.nv * sizeof(float)));
    ETH_CUDA(cudaMemset(L.x, 0, 2 * L.nv * sizeof(float)));
    ETH_CUDA(cudaMemset(L.t, 0, 2 * L.nv * sizeof(float)));
    g->lv.push_back(L);
    bool nest = nx % 2 == 0 && ny % 2 == 0 && nx >= 2 && ny >= 2;
    std::vector<unsigned char> ca;
    if (nest) {
      const int cx = nx / 2, cy = ny / 2;
      ca.assign((size_t)cx * cy, 0);
      for (int ey = 0; ey < cy && nest; ++ey)
        for (int ex = 0; ex < cx && nest; ++ex) {
          const unsigned char a0 = act[(size_t)(2 * ey) * nx + 2 * ex], a1 = act[(size_t)(2 * ey) * nx + 2 * ex + 1],
                              a2 = act[(size_t)(2 * ey + 1) * nx + 2 * ex], a3 = act[(size_t)(2 * ey + 1) * nx + 2 * ex + 1];
          if (a0 != a1 || a0 != a2 || a0 != a3) nest = false;
          ca[(size_t)ey * cx + ex] = a0;
        }
    }
    if (!nest) break;
    act.swap(ca);
    nx /= 2; ny /= 2; h *= 2.0;
  }
  ETH_CUDA(cudaMalloc((void**)&g->E32, (size_t)18 * g->n0 * sizeof(float)));
  // coarsest level: free-node list
  const MLev& C = g->lv.back();
  std::vector<unsigned char> fix(C.nv);
  ETH_CUDA(cudaMemcpy(fix.data(), C.fix, C.nv, cudaMemcpyDeviceToHost));
  std::vector<int> idx;
  for (size_t k = 0; k < C.nv; ++k)
    if (!fix[k]) idx.push_back((int)k);
  if ((int)idx.size() > MAX_COARSE_FREE) {
    set_error("masked grid: the coarsest multigrid level keeps %d free nodes (> %d): the mask must coarsen further "
              "(nx, ny divisible by powers of 2 with 2 x 2-nested active blocks)", (int)idx.size(), MAX_COARSE_FREE);
    return ETH_EINVAL;
  }
  g->ncf = (int)idx.size();
  ETH_CUDA(cudaMalloc((void**)&g->cidx, std::max<size_t>(1, idx.size()) * sizeof(int)));
  if (!idx.empty()) ETH_CUDA(cudaMemcpy(g->cidx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice));
  ETH_CUDA(cudaMalloc((void**)&g->cinv, std::max<size_t>(1, idx.size() * idx.size()) * sizeof(float)));
  return ETH_OK;
}

// Coefficient-dependent data: level winds, Jacobi diagonals, coarsest inverse.
static eth_status mg_prepare(G* g) {
  const float nu = (float)g->nu;
  const size_t nl = g->lv.size();
  for (size_t l = 0; l < nl; ++l) {
    MLev& L = g->lv[l];
    if (g->conv) {
      if (l == 0) k_cast<double, float><<<nblk(2 * L.nv), 256, 0, g->s>>>(2 * L.nv, g->wind, L.w);
      else k_inject<float, float><<<nblk(L.nv), 256, 0, g->s>>>(L.nx, L.ny, g->lv[l - 1].w, L.w);
      ETH_CUDA(cudaGetLastError());
      k_elem_diag<float, FVC><<<nblk(L.n0, 128), 128, 0, g->s>>>(L.nx, L.ny, (float)L.h, nu, (float)SDC, L.act, L.w, g->E32);
    } else {
      k_elem_diag<float, FV><<<nblk(L.n0, 128), 128, 0, g->s>>>(L.nx, L.ny, (float)L.h, nu, 0.f, L.act, L.w, g->E32);
    }
    ETH_CUDA(cudaGetLastError());
    k_vgather<float, float, float><<<nblk(L.nv), 256, 0, g->s>>>(L.nx, L.ny, V_DINV, L.act, L.fix, g->E32, (const float*)nullptr,
                                                               nullptr, nullptr, 0.f, L.dinv, 1);
    ETH_CUDA(cudaGetLastError());
    g->launches += 2;
  }
  // coarsest operator: element matrices (FP64) assembled over the free nodes and inverted on the host
  const MLev& C = g->lv.back();
  const int m = g->ncf;
  if (m > 0) {
    double *M = nullptr, *wd = nullptr;
    ETH_CUDA(cudaMalloc((void**)&M, C.n0 * 81 * sizeof(double)));
    ETH_CUDA(cudaMemsetAsync(M, 0, C.n0 * 81 * sizeof(double), g->s));
    if (g->conv) {
      ETH_CUDA(cudaMalloc((void**)&wd, 2 * C.nv * sizeof(double)));
      k_cast<float, double><<<nblk(2 * C.nv), 256, 0, g->s>>>(2 * C.nv, C.w, wd);
      k_elem_mat<FVC><<<nblk(C.n0, 64), 64, 0, g->s>>>(C.nx, C.ny, C.h, g->nu, SDC, C.act, wd, M);
    } else {
      k_elem_mat<FV><<<nblk(C.n0, 64), 64, 0, g->s>>>(C.nx, C.ny, C.h, g->nu, 0.0, C.act, nullptr, M);
    }
    ETH_CUDA(cudaGetLastError());
    std::vector<double> Mh(C.n0 * 81);
    std::vector<unsigned char> act(C.n0), fix(C.nv);
    std::vector<int> idx(m);
    ETH_CUDA(cudaMemcpyAsync(Mh.data(), M, Mh.size() * sizeof(double), cudaMemcpyDeviceToHost, g->s));
    ETH_CUDA(cudaMemcpyAsync(act.data(), C.act, C.n0, cudaMemcpyDeviceToHost, g->s));
    ETH_CUDA(cudaMemcpyAsync(fix.data(), C.fix, C.nv, cudaMemcpyDeviceToHost, g->s));
    ETH_CUDA(cudaMemcpyAsync(idx.data(), g->cidx, m * sizeof(int), cudaMemcpyDeviceToHost, g->s));
    ETH_CUDA(cudaStreamSynchronize(g->s));
    cudaFree(M);
    cudaFree(wd);
    std::vector<int> pos(C.nv, -1);
    for (int k = 0; k < m; ++k) pos[idx[k]] = k;
    std::vector<double> A((size_t)m * m, 0.0);
    const int Nx = 2 * C.nx + 1;
    for (size_t e = 0; e < C.n0; ++e) {
      if (!act[e]) continue;
      const int ex = (int)(e % C.nx), ey = (int)(e / C.nx);
      for (int i = 0; i < 9; ++i) {
        const int ri = pos[(size_t)(2 * ey + i / 3) * Nx + 2 * ex + i % 3];
        if (ri < 0) continue;
        for (int j = 0; j < 9; ++j) {
          const int cj = pos[(size_t)(2 * ey + j / 3) * Nx + 2 * ex + j % 3];
          if (cj < 0) continue;
          A[(size_t)ri * m + cj] += Mh[e * 81 + i * 9 + j];
        }
      }
    }
    if (!invert_dense(A, m)) { set_error("masked grid: singular coarsest-level operator"); return ETH_EINVAL; }
    std::vector<float> Af((size_t)m * m);
    for (int r = 0; r < m; ++r)
      for (int k = 0; k < m; ++k) Af[(size_t)k * m + r] = (float)A[(size_t)r * m + k];   // column-major
    ETH_CUDA(cudaMemcpyAsync(g->cinv, Af.data(), Af.size() * sizeof(float), cudaMemcpyHostToDevice, g->s));
    ETH_CUDA(cudaStreamSynchronize(g->s));
  }
  return ETH_OK;
}

// level operator pass: E32 = element rows of F_l x
static eth_status mg_elem(G* g, const MLev& L, const float* x) {
  if (g->conv)
    k_elem<float, float, FVC><<<nblk(L.n0, 128), 128, 0, g->s>>>(L.nx, L.ny, (float)L.h, (float)g->nu, (float)SDC, L.act, L.fix, 1,
                                                                 x, (const float*)nullptr, L.w, g->E32);
  else
    k_elem<float, float, FV><<<nblk(L.n0, 128), 128, 0, g->s>>>(L.nx, L.ny, (float)L.h, (float)g->nu, 0.f, L.act, L.fix, 1, x,
                                                                (const float*)nullptr, (const float*)nullptr, g->E32);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  return ETH_OK;
}
static eth_status mg_gather(G* g, const MLev& L, int mode, const float* a, const float* x, float* y, float omega) {
  k_vgather<float, float, float><<<nblk(2 * L.nv), 256, 0, g->s>>>(L.nx, L.ny, mode, L.act, L.fix, g->E32, a, x, L.dinv, omega, y, 2);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  return ETH_OK;
}

// z_u = V(v_u): one V-cycle (pre / post damped-Jacobi sweeps) on both velocity
// components; z equals v on the fixed nodes (identity rows of F).
static eth_status vcycle(G* g, const double* v, double* z, int pre, int post, float omega) {
  const int nl = (int)g->lv.size();
  {
    MLev& L = g->lv[0];
    k_jac0<double, float><<<nblk(2 * L.nv), 256, 0, g->s>>>(L.nv, L.fix, L.dinv, omega, v, L.b, L.x);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
  }
  for (int l = 0; l < nl - 1; ++l) {
    MLev& L = g->lv[l];
    for (int s = 1; s < pre; ++s) {
      ETH_TRY(mg_elem(g, L, L.x));
      ETH_TRY(mg_gather(g, L, V_SMOOTH, L.b, L.x, L.t, omega));
      std::swap(L.x, L.t);
    }
    ETH_TRY(mg_elem(g, L, L.x));
    ETH_TRY(mg_gather(g, L, V_RESID, L.b, nullptr, L.r, omega));
    MLev& C = g->lv[l + 1];
    k_restrict<float><<<nblk(C.nv), 256, 0, g->s>>>(C.nx, C.ny, C.fix, L.r, C.b);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
    if (l + 1 < nl - 1) {
      k_jac0<float, float><<<nblk(2 * C.nv), 256, 0, g->s>>>(C.nv, C.fix, C.dinv, omega, C.b, C.b, C.x);
      ETH_CUDA(cudaGetLastError());
      g->launches++;
    }
  }
  {
    MLev& C = g->lv[nl - 1];   // (nl == 1: the exact solve alone)
    ETH_CUDA(cudaMemsetAsync(C.x, 0, 2 * C.nv * sizeof(float), g->s));
    if (g->ncf > 0) {
      k_cdense<float><<<dim3(cdiv(g->ncf, 128), 2), 128, 0, g->s>>>(g->ncf, C.nv, g->cidx, g->cinv, C.b, C.x);
      ETH_CUDA(cudaGetLastError());
      g->launches++;
    }
  }
  for (int l = nl - 2; l >= 0; --l) {
    MLev& L = g->lv[l];
    const MLev& C = g->lv[l + 1];
    k_prolong_add<float><<<nblk(L.nv), 256, 0, g->s>>>(C.nx, C.ny, L.fix, C.x, L.x);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
    for (int s = 0; s < post; ++s) {
      ETH_TRY(mg_elem(g, L, L.x));
      ETH_TRY(mg_gather(g, L, V_SMOOTH, L.b, L.x, L.t, omega));
      std::swap(L.x, L.t);
    }
  }
  MLev& L0 = g->lv[0];
  k_vout<float><<<nblk(2 * L0.nv), 256, 0, g->s>>>(L0.nv, L0.fix, L0.x, v, z);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  return ETH_OK;
}

}  // namespace msk
}  // namespace eth

// ---------------------------------------------------------------------------
// masked Q1 multigrid: the preconditioner of the PCD matrix Ap (Q1 Laplacian
// plus a unit shift on the outflow nodes, where Ap = B1 Md^{-1} B1^T does not
// annihilate the constants) and of the Schur complement S = Qk - R^T Q0^{-1} R
// of M_Q (pure Q1 Laplacian with natural boundary conditions, singular on the
// constants, pseudo-inverse on the coarsest level)
// ---------------------------------------------------------------------------
namespace eth {
namespace msk {

constexpr double Q1_SHIFT = 1.0;   // outflow shift of the Ap preconditioner's operator
constexpr double Q1_OMEGA = 0.8;   // damped Jacobi of the Q1 levels

// K1 node operator over the active elements (+ shift on the outflow nodes when
// shift > 0): mode 0 y = K1 x (identity rows on inactive nodes), mode 1
// y = b - K1 x, mode 2 y = x + omega d (b - K1 x) (0 on inactive nodes)
__global__ void k_k1node(int nx, int ny, int mode, double shift, const unsigned char* __restrict__ act,
                         const unsigned char* __restrict__ q1a, const double* __restrict__ x, const double* __restrict__ b,
                         const double* __restrict__ d, double omega, double* __restrict__ y) {
  const int M = nx + 1;
  const size_t n1 = (size_t)M * (ny + 1);
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n1; k += (size_t)gridDim.x * blockDim.x) {
    if (!q1a[k]) { y[k] = mode == 0 ? x[k] : 0.0; continue; }
    const int J = (int)(k / M), I = (int)(k - (size_t)J * M);
    double s = (shift > 0.0 && I == nx) ? shift * x[k] : 0.0;
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        const int ex = I - 1 + dx, ey = J - 1 + dy;
        if (ex < 0 || ex >= nx || ey < 0 || ey >= ny || !act[(size_t)ey * nx + ex]) continue;
        const int c = 1 - dx, dd = 1 - dy;
        for (int lj = 0; lj < 4; ++lj) {
          const int cj = lj & 1, dj = lj >> 1;
          s += (q1k(c, cj) * q1m(dd, dj) + q1m(c, cj) * q1k(dd, dj)) * x[(size_t)(ey + dj) * M + ex + cj];
        }
      }
    y[k] = mode == 0 ? s : (mode == 1 ? b[k] - s : x[k] + omega * d[k] * (b[k] - s));
  }
}
// inverse diagonal of the level operator: 2/3 per active element around the node (+ shift), 0 on inactive nodes
__global__ void k_k1dinv(int nx, int ny, double shift, const unsigned char* __restrict__ act, const unsigned char* __restrict__ q1a,
                         double* __restrict__ d) {
  const int M = nx + 1;
  const size_t n1 = (size_t)M * (ny + 1);
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n1; k += (size_t)gridDim.x * blockDim.x) {
    if (!q1a[k]) { d[k] = 0.0; continue; }
    const int J = (int)(k / M), I = (int)(k - (size_t)J * M);
    double s = (shift > 0.0 && I == nx) ? shift : 0.0;
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        const int ex = I - 1 + dx, ey = J - 1 + dy;
        if (ex >= 0 && ex < nx && ey >= 0 && ey < ny && act[(size_t)ey * nx + ex]) s += 2.0 / 3.0;
      }
    d[k] = 1.0 / s;
  }
}
// b_c = P^T r_f (bilinear interpolation transposed), 0 on inactive coarse nodes
__global__ void k_q1r(int nxc, int nyc, const unsigned char* __restrict__ q1ac, const double* __restrict__ rf, double* __restrict__ bc) {
  const int Mc = nxc + 1, Mf = 2 * nxc + 1, Nyf = 2 * nyc + 1;
  const size_t n1c = (size_t)Mc * (nyc + 1);
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n1c; k += (size_t)gridDim.x * blockDim.x) {
    if (!q1ac[k]) { bc[k] = 0.0; continue; }
    const int J = (int)(k / Mc), I = (int)(k - (size_t)J * Mc);
    double s = 0.0;
    for (int u = -1; u <= 1; ++u) {
      const int fj = 2 * J + u;
      if (fj < 0 || fj >= Nyf) continue;
      for (int v = -1; v <= 1; ++v) {
        const int fi = 2 * I + v;
        if (fi < 0 || fi >= Mf) continue;
        s += (u ? 0.5 : 1.0) * (v ? 0.5 : 1.0) * rf[(size_t)fj * Mf + fi];
      }
    }
    bc[k] = s;
  }
}
// x_f += P x_c on the active fine nodes
__global__ void k_q1p(int nxc, int nyc, const unsigned char* __restrict__ q1af, const double* __restrict__ xc, double* __restrict__ xf) {
  const int Mc = nxc + 1, Mf = 2 * nxc + 1;
  const size_t n1f = (size_t)Mf * (2 * nyc + 1);
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n1f; k += (size_t)gridDim.x * blockDim.x) {
    if (!q1af[k]) continue;
    const int j = (int)(k / Mf), i = (int)(k - (size_t)j * Mf);
    const int I0 = i >> 1, J0 = j >> 1, I1 = (i & 1) ? I0 + 1 : I0, J1 = (j & 1) ? J0 + 1 : J0;
    const double wx = (i & 1) ? 0.5 : 1.0, wy = (j & 1) ? 0.5 : 1.0;
    double s = wx * wy * xc[(size_t)J0 * Mc + I0];
    if (i & 1) s += wx * wy * xc[(size_t)J0 * Mc + I1];
    if (j & 1) s += wx * wy * xc[(size_t)J1 * Mc + I0];
    if ((i & 1) && (j & 1)) s += wx * wy * xc[(size_t)J1 * Mc + I1];
    xf[k] += s;
  }
}
// level right-hand side b = v (0 on inactive nodes) and x = omega D^{-1} b
__global__ void k_q1j0(size_t m, const unsigned char* __restrict__ q1a, const double* __restrict__ d, double omega,
                       const double* __restrict__ v, double* __restrict__ b, double* __restrict__ x) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) {
    const double bv = q1a[k] ? v[k] : 0.0;
    b[k] = bv;
    x[k] = omega * d[k] * bv;
  }
}
// coarsest level: x = A_c^+ b over the active nodes (column-major)
__global__ void k_q1dense(int m, const int* __restrict__ idx, const double* __restrict__ Ainv, const double* __restrict__ b,
                          double* __restrict__ x) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < m; ++k) s += Ainv[(size_t)k * m + r] * b[idx[k]];
    x[idx[r]] = s;
  }
}
// Q0 elimination of M_Q [x1; x0] = [r1; r0]: t_I = r1_I - (1/4) sum_{active T around I} r0_T
// on active Q1 nodes (R = |T|/4, Q0 = |T|), 0 elsewhere
__global__ void k_mq_elim(int nx, int ny, const unsigned char* __restrict__ act, const unsigned char* __restrict__ q1a,
                          const double* __restrict__ r, double* __restrict__ t) {
  const int M = nx + 1;
  const size_t n1 = (size_t)M * (ny + 1);
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n1; k += (size_t)gridDim.x * blockDim.x) {
    if (!q1a[k]) { t[k] = 0.0; continue; }
    const int J = (int)(k / M), I = (int)(k - (size_t)J * M);
    double s = 0.0;
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        const int ex = I - 1 + dx, ey = J - 1 + dy;
        if (ex >= 0 && ex < nx && ey >= 0 && ey < ny && act[(size_t)ey * nx + ex]) s += r[n1 + (size_t)ey * nx + ex];
      }
    t[k] = r[k] - 0.25 * s;
  }
}
// back substitution: z1 = x1, z0_T = r0_T / |T| - (1/4) sum_{I in T} x1_I (active);
// inactive unknowns keep r (identity rows)
__global__ void k_mq_back(int nx, int ny, double h, const unsigned char* __restrict__ act, const unsigned char* __restrict__ q1a,
                          const double* __restrict__ x1, const double* __restrict__ r, double* __restrict__ z) {
  const int M = nx + 1;
  const size_t n1 = (size_t)M * (ny + 1), n0 = (size_t)nx * ny;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n1 + n0; k += (size_t)gridDim.x * blockDim.x) {
    if (k < n1) { z[k] = q1a[k] ? x1[k] : r[k]; continue; }
    const size_t e = k - n1;
    if (!act[e]) { z[k] = r[k]; continue; }
    const int ex = (int)(e % nx), ey = (int)(e / nx);
    const double s = x1[(size_t)ey * M + ex] + x1[(size_t)ey * M + ex + 1] + x1[(size_t)(ey + 1) * M + ex] +
                     x1[(size_t)(ey + 1) * M + ex + 1];
    z[k] = r[k] / (h * h) - 0.25 * s;
  }
}
// CG with a given preconditioned residual z: p = z, rz = <r, z>
__global__ void __launch_bounds__(RB) k_pcg2_start(size_t m, const double* __restrict__ r, const double* __restrict__ z,
                                                   double* __restrict__ p, PcgS* st, Slot sl) {
  double v[1] = {0.0};
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) {
    p[k] = z[k];
    v[0] += r[k] * z[k];
  }
  if (slot_arrive<1>(sl, blockIdx.x, v)) {
    st->rz = v[0]; st->its = 0; st->alpha = 0; st->beta = 0;
    st->done = v[0] > 0.0 ? 0 : 1;
  }
}
// x += alpha p, r -= alpha q
__global__ void k_pcg2_xr(size_t m, const double* __restrict__ p, const double* __restrict__ q, double* __restrict__ x,
                          double* __restrict__ r, PcgS* st) {
  if (st->done) return;
  const double al = st->alpha;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) {
    x[k] += al * p[k];
    r[k] -= al * q[k];
  }
}
// beta = <r, z>_new / <r, z>
__global__ void __launch_bounds__(RB) k_pcg2_beta(size_t m, const double* __restrict__ r, const double* __restrict__ z, PcgS* st,
                                                  Slot sl) {
  if (st->done) return;
  double v[1] = {0.0};
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) v[0] += r[k] * z[k];
  if (slot_arrive<1>(sl, blockIdx.x, v)) {
    if (v[0] > 0.0) { st->beta = v[0] / st->rz; st->rz = v[0]; st->its += 1; }
    else st->done = 1;
  }
}

// host: build the two Q1 hierarchies on the velocity levels' element masks
static eth_status q_build(G* g) {
  for (int w = 0; w < 2; ++w) {
    QHier& Q = g->qh[w];
    const double shift = (w == 0 && g->outflow) ? Q1_SHIFT : 0.0;
    Q.shift = shift;
    for (const MLev& V : g->lv) {
      QLev L;
      L.nx = V.nx; L.ny = V.ny;
      L.n1 = (size_t)(V.nx + 1) * (V.ny + 1);
      L.act = V.act;
      std::vector<unsigned char> fix, dir, q1a;
      node_roles(V.nx, V.ny, g->outflow, V.hact, fix, dir, q1a);
      L.hq1a = q1a;
      ETH_CUDA(cudaMalloc((void**)&L.q1a, L.n1));
      ETH_CUDA(cudaMemcpy(L.q1a, q1a.data(), L.n1, cudaMemcpyHostToDevice));
      for (double** p : {&L.d, &L.x, &L.b, &L.r}) {
        ETH_CUDA(cudaMalloc((void**)p, L.n1 * sizeof(double)));
        ETH_CUDA(cudaMemset(*p, 0, L.n1 * sizeof(double)));
      }
      k_k1dinv<<<nblk(L.n1), 256, 0, g->s>>>(L.nx, L.ny, shift, L.act, L.q1a, L.d);
      ETH_CUDA(cudaGetLastError());
      Q.lv.push_back(L);
    }
    // coarsest: dense (pseudo-)inverse over the active nodes
    const QLev& C = Q.lv.back();
    const MLev& CV = g->lv.back();
    std::vector<int> idx, pos(C.n1, -1);
    for (size_t k = 0; k < C.n1; ++k)
      if (C.hq1a[k]) { pos[k] = (int)idx.size(); idx.push_back((int)k); }
    const int m = (int)idx.size();
    std::vector<double> A((size_t)m * m, 0.0);
    const int M = C.nx + 1;
    for (int ey = 0; ey < C.ny; ++ey)
      for (int ex = 0; ex < C.nx; ++ex) {
        if (!CV.hact[(size_t)ey * C.nx + ex]) continue;
        for (int li = 0; li < 4; ++li)
          for (int lj = 0; lj < 4; ++lj) {
            const int ri = pos[(size_t)(ey + (li >> 1)) * M + ex + (li & 1)], cj = pos[(size_t)(ey + (lj >> 1)) * M + ex + (lj & 1)];
            A[(size_t)ri * m + cj] += q1k(li & 1, lj & 1) * q1m(li >> 1, lj >> 1) + q1m(li & 1, lj & 1) * q1k(li >> 1, lj >> 1);
          }
      }
    if (shift > 0.0)
      for (int k = 0; k < m; ++k)
        if (idx[k] % M == C.nx) A[(size_t)k * m + k] += shift;
    if (shift == 0.0)   // singular on the constants: (A + e e^T)^{-1} - e e^T, e = 1/sqrt(m)
      for (size_t k = 0; k < A.size(); ++k) A[k] += 1.0 / m;
    if (!invert_dense(A, m)) { set_error("masked grid: singular coarsest Q1 operator"); return ETH_EINVAL; }
    if (shift == 0.0)
      for (size_t k = 0; k < A.size(); ++k) A[k] -= 1.0 / m;
    std::vector<double> Ac((size_t)m * m);
    for (int r = 0; r < m; ++r)
      for (int k = 0; k < m; ++k) Ac[(size_t)k * m + r] = A[(size_t)r * m + k];
    Q.ncf = m;
    ETH_CUDA(cudaMalloc((void**)&Q.cidx, std::max(1, m) * sizeof(int)));
    ETH_CUDA(cudaMalloc((void**)&Q.cinv, std::max<size_t>(1, Ac.size()) * sizeof(double)));
    ETH_CUDA(cudaMemcpy(Q.cidx, idx.data(), m * sizeof(int), cudaMemcpyHostToDevice));
    ETH_CUDA(cudaMemcpy(Q.cinv, Ac.data(), Ac.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  return ETH_OK;
}

// z = V(r): one V-cycle of hierarchy w (V(1,1), damped Jacobi); z may alias nothing of the hierarchy
static eth_status qvcycle(G* g, int w, const double* r, double* z) {
  QHier& Q = g->qh[w];
  const int nl = (int)Q.lv.size();
  const double sh = Q.shift, om = Q1_OMEGA;
  {
    QLev& L = Q.lv[0];
    k_q1j0<<<nblk(L.n1), 256, 0, g->s>>>(L.n1, L.q1a, L.d, om, r, L.b, L.x);
    g->launches++;
  }
  for (int l = 0; l < nl - 1; ++l) {
    QLev& L = Q.lv[l];
    QLev& C = Q.lv[l + 1];
    k_k1node<<<nblk(L.n1), 256, 0, g->s>>>(L.nx, L.ny, 1, sh, L.act, L.q1a, L.x, L.b, L.d, om, L.r);
    k_q1r<<<nblk(C.n1), 256, 0, g->s>>>(C.nx, C.ny, C.q1a, L.r, C.b);
    if (l + 1 < nl - 1) k_q1j0<<<nblk(C.n1), 256, 0, g->s>>>(C.n1, C.q1a, C.d, om, C.b, C.b, C.x);
    g->launches += 3;
  }
  {
    QLev& C = Q.lv[nl - 1];
    ETH_CUDA(cudaMemsetAsync(C.x, 0, C.n1 * sizeof(double), g->s));
    k_q1dense<<<cdiv(Q.ncf, 128), 128, 0, g->s>>>(Q.ncf, Q.cidx, Q.cinv, C.b, C.x);
    g->launches++;
  }
  for (int l = nl - 2; l >= 0; --l) {
    QLev& L = Q.lv[l];
    const QLev& C = Q.lv[l + 1];
    k_q1p<<<nblk(L.n1), 256, 0, g->s>>>(C.nx, C.ny, L.q1a, C.x, L.x);
    k_k1node<<<nblk(L.n1), 256, 0, g->s>>>(L.nx, L.ny, 2, sh, L.act, L.q1a, L.x, L.b, L.d, om, l == 0 ? z : L.r);
    if (l > 0) std::swap(L.x, L.r);
    g->launches += 2;
  }
  if (nl == 1) ETH_CUDA(cudaMemcpyAsync(z, Q.lv[0].x, Q.lv[0].n1 * sizeof(double), cudaMemcpyDeviceToDevice, g->s));
  ETH_CUDA(cudaGetLastError());
  return ETH_OK;
}

}  // namespace msk
}  // namespace eth

// ---------------------------------------------------------------------------
// pressure solves and the block-triangular preconditioners
// ---------------------------------------------------------------------------
namespace eth {
namespace msk {

constexpr int AP_ITS = 3;           // CG steps on Ap (Q1 V-cycle preconditioner)
constexpr int MQ_ITS = 3;           // CG steps on the Schur complement of M_Q (Q1 V-cycle preconditioner)
constexpr int Q1_CHEB = 10;         // Chebyshev steps of the Q1 mass solve

// Chebyshev semi-iteration on D^{-1} Q (spectrum in [1/4, 9/4] for the Q1 mass
// matrix on squares, element-wise bound, identity rows included)
__global__ void k_cheb_init(size_t m, double theta, const double* __restrict__ b, const double* __restrict__ dinv,
                            double* __restrict__ r, double* __restrict__ x, double* __restrict__ d) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) {
    r[k] = b[k]; x[k] = 0.0; d[k] = dinv[k] * b[k] / theta;
  }
}
__global__ void k_cheb_upd(size_t m, double c1, double c2, const double* __restrict__ d, const double* __restrict__ q,
                           const double* __restrict__ dinv, double* __restrict__ x, double* __restrict__ r, double* __restrict__ dn) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) {
    x[k] += d[k];
    const double rv = r[k] - q[k];
    r[k] = rv;
    dn[k] = c1 * d[k] + c2 * dinv[k] * rv;
  }
}
__global__ void k_hadd(int n, const double* __restrict__ a, double* __restrict__ h) {
  const int i = threadIdx.x;
  if (i < n) h[i] += a[i];
}
// x = [D_B b_u; 0]: the lifted boundary data, zero elsewhere
__global__ void k_x0(size_t nv, size_t np, const unsigned char* __restrict__ fix, const double* __restrict__ b, double* __restrict__ x) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < 2 * nv + np; k += (size_t)gridDim.x * blockDim.x) {
    if (k < 2 * nv) {
      const size_t g = k >= nv ? k - nv : k;
      x[k] = fix[g] ? b[k] : 0.0;
    } else {
      x[k] = 0.0;
    }
  }
}

// x ~= Q1^{-1} b (Q1 mass with identity rows), Q1_CHEB Chebyshev steps
static eth_status q1_mass_inv(G* g, const double* b, double* x) {
  const size_t m = g->n1;
  const double lmin = 0.25, lmax = 2.25, theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
  double *r = g->pr, *d = g->pz, *dn = g->pp, *q = g->pq;
  k_cheb_init<<<nblk(m), 256, 0, g->s>>>(m, theta, b, g->q1dinv, r, x, d);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  double rho = 1.0 / sigma;
  for (int k = 0; k < Q1_CHEB; ++k) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    k_q1apply<<<nblk(m), 256, 0, g->s>>>(g->nx, g->ny, g->h, g->act, g->q1a, nullptr, 0.0, d, q);
    k_cheb_upd<<<nblk(m), 256, 0, g->s>>>(m, rn * rho, 2.0 * rn / delta, d, q, g->q1dinv, x, r, dn);
    ETH_CUDA(cudaGetLastError());
    g->launches += 2;
    std::swap(d, dn);
    rho = rn;
  }
  return ETH_OK;
}

// q = (Ap + pin) p, Ap = B1 Md^{-1} B1^T over the free velocity columns
static eth_status ap_apply(G* g, const double* p, double* q) {
  ETH_TRY((elem64<QF_PIN | QF_UOUT>(g, 0, nullptr, p, nullptr)));
  ETH_TRY(vgat64(g, V_SCALE, (const double*)nullptr, g->mdinv, g->t1));
  ETH_TRY((elem64<QF_XIN | QF_POUT>(g, 1, g->t1, nullptr, nullptr)));
  return pgat64(g, P_PIN, g->n1, p, q);
}

// x ~= A^{-1} b by `its` CG steps preconditioned with one Q1 V-cycle: op 0 A = Ap
// + pin (V-cycle of the Q1 Laplacian with the outflow shift), op 1 A = S + pin,
// S = Qk - R^T Q0^{-1} R (V-cycle of the natural-boundary Q1 Laplacian; b and
// the result are defined up to constants).  A fixed step count, scalars on the
// device: no host synchronisation.
static eth_status pcg_mg(G* g, int op, const double* b, double* x, int its) {
  const size_t m = g->n1;
  const int nb = rblocks(m);
  double *r = g->pr, *z = g->pz, *p = g->pp, *q = g->pq;
  ETH_CUDA(cudaMemcpyAsync(r, b, m * sizeof(double), cudaMemcpyDeviceToDevice, g->s));
  ETH_CUDA(cudaMemsetAsync(x, 0, m * sizeof(double), g->s));
  ETH_TRY(qvcycle(g, op, r, z));
  k_pcg2_start<<<nb, RB, 0, g->s>>>(m, r, z, p, g->pcg, slot(g, nb));
  g->launches++;
  for (int it = 0; it < its; ++it) {
    if (op == 0) ETH_TRY(ap_apply(g, p, q));
    else {
      k_q1apply<<<nblk(m), 256, 0, g->s>>>(g->nx, g->ny, g->h, g->act, g->q1a, nullptr, -1.0 / 16.0, p, q);
      g->launches++;
    }
    k_pcg_alpha<<<nb, RB, 0, g->s>>>(m, p, q, g->pcg, slot(g, nb));
    k_pcg2_xr<<<nblk(m), 256, 0, g->s>>>(m, p, q, x, r, g->pcg);
    g->launches += 2;
    if (it + 1 == its) break;
    ETH_TRY(qvcycle(g, op, r, z));
    k_pcg2_beta<<<nb, RB, 0, g->s>>>(m, r, z, g->pcg, slot(g, nb));
    k_pcg_p<<<nblk(m), 256, 0, g->s>>>(m, z, p, g->pcg);
    g->launches += 2;
  }
  ETH_CUDA(cudaGetLastError());
  return ETH_OK;
}

// Step I (reduced system [u; p1]): z_p = -M_S^{-1} r_p = -Ap^{-1} F1 Q1^{-1} r_p,
// z_u = V(r_u - B1^T z_p)  (Sec. 3.1, Eq. discrete-commutator1x)
// Without a wind (the Stokes step) F1 = nu K1 annihilates the constants while the
// outflow Schur complement does not: there the Stokes limit of the commutator,
// F1 = nu Ap, gives M_S^{-1} = nu Q1^{-1}.
static eth_status prec_pcd(G* g, const eth_opts* o, const double* r, double* z) {
  const double* rp = r + g->nu2;
  double* zp = z + g->nu2;
  ETH_TRY(q1_mass_inv(g, rp, g->pa));
  if (g->conv) {
    k_q1apply<<<nblk(g->n1), 256, 0, g->s>>>(g->nx, g->ny, g->h, g->act, g->q1a, g->f1e, 0.0, g->pa, g->pb);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
    ETH_TRY(pcg_mg(g, 0, g->pb, g->px, AP_ITS));
    k_scale<<<nblk(g->n1), 256, 0, g->s>>>(g->n1, -1.0, g->px, zp);
  } else {
    k_scale<<<nblk(g->n1), 256, 0, g->s>>>(g->n1, -g->nu, g->pa, zp);
  }
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  ETH_TRY(bsub(g, false, r, zp, g->t0));
  return vcycle(g, g->t0, z, std::max(1, o->mg_pre), std::max(1, o->mg_post), (float)(o->mg_omega > 0 ? o->mg_omega : 0.85));
}

// Step II (full system): z_p = -nu M_Q^+ r_p (k projected out), z_u = V(r_u - B^T z_p)
// (Sec. 3.1, the preconditioner M_1 of Eq. nse-precon-ref)
// M_Q^+ r_p: k projected out of r_p, Q0 eliminated, CG on the Schur complement,
// back substitution, k projected out of the result.
static eth_status prec_m1(G* g, const eth_opts* o, const double* r, double* z) {
  double* zp = z + g->nu2;
  const double* rp = r + g->nu2;
  ETH_TRY(dot2(g, g->np, g->kv, rp, nullptr, nullptr, 4));
  k_proj<<<nblk(g->np), 256, 0, g->s>>>(g->np, rp, g->kv, g->red + 4, g->kk, g->pa);
  k_mq_elim<<<nblk(g->n1), 256, 0, g->s>>>(g->nx, g->ny, g->act, g->q1a, g->pa, g->pb);
  ETH_CUDA(cudaGetLastError());
  g->launches += 2;
  ETH_TRY(pcg_mg(g, 1, g->pb, g->px, MQ_ITS));
  k_mq_back<<<nblk(g->np), 256, 0, g->s>>>(g->nx, g->ny, g->h, g->act, g->q1a, g->px, g->pa, g->pb);
  ETH_CUDA(cudaGetLastError());
  ETH_TRY(dot2(g, g->np, g->kv, g->pb, nullptr, nullptr, 4));
  k_proj<<<nblk(g->np), 256, 0, g->s>>>(g->np, g->pb, g->kv, g->red + 4, g->kk, g->pb);
  k_scale<<<nblk(g->np), 256, 0, g->s>>>(g->np, -g->nu, g->pb, zp);
  ETH_CUDA(cudaGetLastError());
  g->launches += 3;
  ETH_TRY(bsub(g, true, r, zp, g->t0));
  return vcycle(g, g->t0, z, std::max(1, o->mg_pre), std::max(1, o->mg_post), (float)(o->mg_omega > 0 ? o->mg_omega : 0.85));
}

static eth_status prepare(G* g) {
  if (g->prec_ok) return ETH_OK;
  ETH_TRY(mg_prepare(g));
  k_f1_elem<<<nblk(g->n0, 128), 128, 0, g->s>>>(g->nx, g->ny, g->h, g->nu, g->act, g->conv ? g->wind : nullptr, g->f1e);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  g->prec_ok = true;
  return ETH_OK;
}

}  // namespace msk
}  // namespace eth

// ---------------------------------------------------------------------------
// flexible restarted GMRES, the two-stage method, Picard
// ---------------------------------------------------------------------------
namespace eth {
namespace msk {

constexpr int MD_NB = 128;   // blocks per basis vector in k_mdot

static eth_status gm_alloc(G* g, int m) {
  if (g->gm_m >= m) return ETH_OK;
  cudaFree(g->V); cudaFree(g->Z); cudaFree(g->hd); cudaFree(g->hd2); cudaFree(g->yd); cudaFree(g->mpart);
  if (g->hh) cudaFreeHost(g->hh);
  g->V = g->Z = g->hd = g->hd2 = g->yd = g->mpart = g->hh = nullptr;
  g->gm_m = 0;
  ETH_CUDA(cudaMalloc((void**)&g->V, (size_t)(m + 1) * g->nt * sizeof(double)));
  ETH_CUDA(cudaMalloc((void**)&g->Z, (size_t)m * g->nt * sizeof(double)));
  ETH_CUDA(cudaMalloc((void**)&g->hd, (size_t)(m + 2) * sizeof(double)));
  ETH_CUDA(cudaMalloc((void**)&g->hd2, (size_t)(m + 2) * sizeof(double)));
  ETH_CUDA(cudaMalloc((void**)&g->yd, (size_t)(m + 1) * sizeof(double)));
  ETH_CUDA(cudaMalloc((void**)&g->mpart, (size_t)(m + 1) * MD_NB * sizeof(double)));
  ETH_CUDA(cudaMallocHost((void**)&g->hh, (size_t)(m + 2) * sizeof(double)));
  g->gm_m = m;
  return ETH_OK;
}

static eth_status sys_apply(G* g, int stage, const double* x, double* y) { return apply_K(g, stage == 1, x, y); }
static eth_status sys_prec(G* g, const eth_opts* o, int stage, const double* r, double* z) {
  return stage == 1 ? prec_pcd(g, o, r, z) : prec_m1(g, o, r, z);
}

// h[0..nvec) = V^T w (pass 0) or hd2 = V^T w then w -= V hd2, h += hd2 (pass 1)
static eth_status cgs_pass(G* g, size_t n, int nvec, double* w, bool second) {
  double* h = second ? g->hd2 : g->hd;
  k_mdot<<<dim3(MD_NB, nvec), RB, 0, g->s>>>(n, g->V, g->nt, w, g->mpart);
  k_msum<<<cdiv(nvec, 8), 256, 0, g->s>>>(nvec, MD_NB, g->mpart, h, 0);
  k_mupd<<<nblk(n), 256, 0, g->s>>>(n, g->V, g->nt, nvec, h, w);
  g->launches += 3;
  if (second) {
    k_hadd<<<1, 1024, 0, g->s>>>(nvec, g->hd2, g->hd);
    g->launches++;
  }
  ETH_CUDA(cudaGetLastError());
  return ETH_OK;
}

// The preconditioner and operator of one Arnoldi step (xs -> zo -> t2) as a CUDA
// graph, captured at first use and again whenever a launch parameter baked into
// it (wind on/off, nu, smoother damping and sweeps) changes; every buffer it
// touches keeps its address for the life of the handle.
static eth_status step_graph(G* g, const eth_opts* o, int stage) {
  const int k = stage - 1;
  const double sig[5] = {g->conv ? 1.0 : 0.0, g->nu, o->mg_omega, (double)o->mg_pre, (double)o->mg_post};
  if (g->gx[k] && std::memcmp(sig, g->gsig[k], sizeof(sig)) != 0) {
    cudaGraphExecDestroy(g->gx[k]);
    g->gx[k] = nullptr;
  }
  if (!g->gx[k]) {
    cudaGraph_t graph = nullptr;
    ETH_CUDA(cudaStreamBeginCapture(g->s, cudaStreamCaptureModeThreadLocal));
    const long l0 = g->launches;
    eth_status st = sys_prec(g, o, stage, g->xs, g->zo);
    if (st == ETH_OK) st = sys_apply(g, stage, g->zo, g->t2);
    const cudaError_t ce = cudaStreamEndCapture(g->s, &graph);
    g->launches = l0;
    if (st != ETH_OK) { if (graph) cudaGraphDestroy(graph); return st; }
    if (ce != cudaSuccess) return cuda_status(ce, "masked grid: graph capture");
    const cudaError_t ie = cudaGraphInstantiate(&g->gx[k], graph, 0);
    size_t nodes = 0;
    cudaGraphGetNodes(graph, nullptr, &nodes);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return cuda_status(ie, "masked grid: graph instantiation");
    g->gnodes[k] = (long)nodes;
    std::memcpy(g->gsig[k], sig, sizeof(sig));
  }
  ETH_CUDA(cudaGraphLaunch(g->gx[k], g->s));
  g->launches += g->gnodes[k];
  return ETH_OK;
}

// Restarted right-preconditioned flexible GMRES on the stage's system (n
// unknowns) from x; stops when the residual norm is <= tol_abs (the true
// residual, recomputed at every restart) or after maxit iterations.
static eth_status gmres(G* g, const eth_opts* o, int stage, size_t n, const double* b, double* x, double tol_abs, int restart,
                        int maxit, int* its, double* res) {
  const size_t ld = g->nt;
  double* r = g->t2;
  *its = 0;
  ETH_TRY(sys_apply(g, stage, x, r));
  k_bminus<<<nblk(n), 256, 0, g->s>>>(n, b, r);
  ETH_CUDA(cudaGetLastError());
  ETH_TRY(dot2(g, n, r, r, nullptr, nullptr, 0));
  ETH_TRY(fetch(g, 1));
  double beta = std::sqrt(g->redh[0]);
  const int m = restart;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
  while (beta > tol_abs && *its < maxit) {
    if (!std::isfinite(beta)) { set_error("masked grid GMRES: non-finite residual"); return ETH_ENAN; }
    k_scale<<<nblk(n), 256, 0, g->s>>>(n, 1.0 / beta, r, g->V);
    ETH_CUDA(cudaGetLastError());
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int k = 0;
    for (int j = 0; j < m; ++j) {
      double* vj = g->V + (size_t)j * ld;
      double* zj = g->Z + (size_t)j * ld;
      if (o->graph) {   // z_j = P^{-1} v_j and w = K z_j by one graph launch (staged through xs / zo)
        ETH_CUDA(cudaMemcpyAsync(g->xs, vj, n * sizeof(double), cudaMemcpyDeviceToDevice, g->s));
        ETH_TRY(step_graph(g, o, stage));
        ETH_CUDA(cudaMemcpyAsync(zj, g->zo, n * sizeof(double), cudaMemcpyDeviceToDevice, g->s));
      } else {
        ETH_TRY(sys_prec(g, o, stage, vj, zj));
        ETH_TRY(sys_apply(g, stage, zj, r));   // r: the new direction w
      }
      ETH_TRY(cgs_pass(g, n, j + 1, r, false));
      ETH_TRY(cgs_pass(g, n, j + 1, r, true));
      k_mdot<<<dim3(MD_NB, 1), RB, 0, g->s>>>(n, r, ld, r, g->mpart);
      k_msum<<<1, 32, 0, g->s>>>(1, MD_NB, g->mpart, g->hd + j + 1, 0);
      k_vnext<<<nblk(n), 256, 0, g->s>>>(n, r, g->V + (size_t)(j + 1) * ld, g->hd, j + 1);
      k_hsqrt<<<1, 1, 0, g->s>>>(g->hd, j + 1);
      ETH_CUDA(cudaGetLastError());
      g->launches += 4;
      ETH_CUDA(cudaMemcpyAsync(g->hh, g->hd, (size_t)(j + 2) * sizeof(double), cudaMemcpyDeviceToHost, g->s));
      ETH_CUDA(cudaStreamSynchronize(g->s));
      for (int i = 0; i <= j + 1; ++i) H[(size_t)i * m + j] = g->hh[i];
      for (int i = 0; i < j; ++i) {
        const double a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * bb;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      const double a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
      const double d = std::hypot(a, bb);
      cs[j] = d > 0.0 ? a / d : 1.0;
      sn[j] = d > 0.0 ? bb / d : 0.0;
      H[(size_t)j * m + j] = d;
      H[(size_t)(j + 1) * m + j] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      ++*its;
      k = j + 1;
      if (d == 0.0) { k = j; break; }
      if (std::fabs(gv[j + 1]) <= tol_abs || *its >= maxit || g->hh[j + 1] == 0.0) break;
    }
    for (int i = k - 1; i >= 0; --i) {
      double s = gv[i];
      for (int l = i + 1; l < k; ++l) s -= H[(size_t)i * m + l] * y[l];
      y[i] = s / H[(size_t)i * m + i];
    }
    if (k > 0) {
      ETH_CUDA(cudaMemcpyAsync(g->yd, y.data(), k * sizeof(double), cudaMemcpyHostToDevice, g->s));
      k_zupd<<<nblk(n), 256, 0, g->s>>>(n, g->Z, ld, k, g->yd, x);
      ETH_CUDA(cudaGetLastError());
      g->launches++;
    }
    ETH_TRY(sys_apply(g, stage, x, r));
    k_bminus<<<nblk(n), 256, 0, g->s>>>(n, b, r);
    ETH_CUDA(cudaGetLastError());
    ETH_TRY(dot2(g, n, r, r, nullptr, nullptr, 0));
    ETH_TRY(fetch(g, 1));
    beta = std::sqrt(g->redh[0]);
    if (k == 0) break;   // breakdown before any progress
  }
  *res = beta;
  return ETH_OK;
}

// The two-stage PCD method (Sec. 3.1) from the lifted boundary data.
static eth_status two_stage(G* g, const eth_opts* o, const double* b, double* x, eth_stats* st) {
  const double eta = o->tol, c = o->c_stage > 0 ? o->c_stage : 10.0;
  const int restart = o->restart > 0 ? o->restart : 50;
  const int maxit = o->maxit > 0 ? o->maxit : 2000;
  ETH_TRY(gm_alloc(g, restart));
  ETH_TRY(prepare(g));
  const size_t nred = g->nu2 + g->n1;
  k_x0<<<nblk(g->nt), 256, 0, g->s>>>(g->nv, g->np, g->fix, b, x);
  ETH_CUDA(cudaGetLastError());
  ETH_TRY(dot2(g, nred, b, b, nullptr, nullptr, 0));     // ||b_red||^2, and ||b||^2 below
  ETH_TRY(dot2(g, g->nt, b, b, nullptr, nullptr, 2));
  ETH_TRY(fetch(g, 3));
  const double nbred = std::sqrt(g->redh[0]), nb = std::sqrt(g->redh[2]);
  if (!(nb > 0.0)) {
    ETH_CUDA(cudaMemsetAsync(x, 0, g->nt * sizeof(double), g->s));
    if (st) { std::memset(st, 0, sizeof(*st)); }
    return ETH_OK;
  }
  int its1 = 0, its2 = 0;
  double res1 = 0, res2 = 0;
  ETH_TRY(gmres(g, o, 1, nred, b, x, c * eta * nbred, restart, maxit, &its1, &res1));
  // Prop. 2: z* = b - K [u1*; p1*; 0], and the bound c^2 eta^2 ||b_red||^2 + ||r0*||^2
  ETH_TRY(apply_K(g, false, x, g->t2));
  k_bminus<<<nblk(g->nt), 256, 0, g->s>>>(g->nt, b, g->t2);
  ETH_CUDA(cudaGetLastError());
  ETH_TRY(dot2(g, g->nt, g->t2, g->t2, nullptr, nullptr, 0));
  ETH_TRY(dot2(g, g->n0, g->t2 + nred, g->t2 + nred, nullptr, nullptr, 2));
  ETH_TRY(fetch(g, 3));
  const double z2 = g->redh[0], r02 = g->redh[2];
  ETH_TRY(gmres(g, o, 2, g->nt, b, x, eta * nb, restart, std::max(0, maxit - its1), &its2, &res2));
  // canonical pressure: k^T p = 0
  ETH_TRY(dot2(g, g->np, g->kv, x + g->nu2, nullptr, nullptr, 0));
  k_proj<<<nblk(g->np), 256, 0, g->s>>>(g->np, x + g->nu2, g->kv, g->red, g->kk, x + g->nu2);
  ETH_CUDA(cudaGetLastError());
  ETH_TRY(apply_K(g, false, x, g->t2));
  k_bminus<<<nblk(g->nt), 256, 0, g->s>>>(g->nt, b, g->t2);
  ETH_CUDA(cudaGetLastError());
  ETH_TRY(dot2(g, g->nt, g->t2, g->t2, nullptr, nullptr, 0));
  ETH_TRY(fetch(g, 1));
  const double rel = std::sqrt(g->redh[0]) / nb;
  if (st) {
    st->iters_stage1 = its1;
    st->iters_stage2 = its2;
    st->iters_total = its1 + its2;
    st->refine_passes = 0;
    st->relres_true = rel;
    st->prop2_lhs = z2;
    st->prop2_bound = (c * eta * nbred) * (c * eta * nbred) + r02;
    st->status = rel <= eta * (1.0 + 1e-9) ? ETH_OK : ETH_ENOTCONV;
  }
  return ETH_OK;
}

}  // namespace msk
}  // namespace eth

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
using namespace eth;
using namespace eth::msk;

static void mgrid_free(eth_mgrid* g) {
  if (!g) return;
  mg_free(g);
  cudaFree(g->act); cudaFree(g->fix); cudaFree(g->q1a); cudaFree(g->wind); cudaFree(g->E);
  cudaFree(g->part); cudaFree(g->ticket); cudaFree(g->red);
  if (g->redh) cudaFreeHost(g->redh);
  if (g->hh) cudaFreeHost(g->hh);
  cudaFree(g->pcg);
  cudaFree(g->mdinv); cudaFree(g->q1dinv); cudaFree(g->kv); cudaFree(g->f1e);
  cudaFree(g->t0); cudaFree(g->t1); cudaFree(g->t2); cudaFree(g->xs); cudaFree(g->bv);
  cudaFree(g->pr); cudaFree(g->pz); cudaFree(g->pp); cudaFree(g->pq); cudaFree(g->px); cudaFree(g->pa); cudaFree(g->pb);
  cudaFree(g->V); cudaFree(g->Z); cudaFree(g->hd); cudaFree(g->hd2); cudaFree(g->yd); cudaFree(g->mpart); cudaFree(g->zo);
  for (cudaGraphExec_t& e : g->gx)
    if (e) cudaGraphExecDestroy(e);
  for (cudaEvent_t& e : g->ev)
    if (e) cudaEventDestroy(e);
  if (g->si) cudaStreamDestroy(g->si);
  delete g;
}

static eth_status mgrid_init(eth_mgrid* g, const unsigned char* active) {
  const size_t n0 = (size_t)g->nx * g->ny;
  g->h_act.resize(n0);
  for (size_t e = 0; e < n0; ++e) g->h_act[e] = active[e] ? 1 : 0;
  node_roles(g->nx, g->ny, g->outflow, g->h_act, g->h_fix, g->h_dir, g->h_q1a);
  g->nv = (size_t)(2 * g->nx + 1) * (2 * g->ny + 1);
  g->n1 = (size_t)(g->nx + 1) * (g->ny + 1);
  g->n0 = n0;
  g->nu2 = 2 * g->nv;
  g->np = g->n1 + g->n0;
  g->nt = g->nu2 + g->np;
  auto A = [&](void** p, size_t bytes) { return cudaMalloc(p, bytes < 8 ? 8 : bytes); };
  ETH_CUDA(A((void**)&g->act, n0));
  ETH_CUDA(A((void**)&g->fix, g->nv));
  ETH_CUDA(A((void**)&g->q1a, g->n1));
  ETH_CUDA(cudaMemcpy(g->act, g->h_act.data(), n0, cudaMemcpyHostToDevice));
  ETH_CUDA(cudaMemcpy(g->fix, g->h_fix.data(), g->nv, cudaMemcpyHostToDevice));
  ETH_CUDA(cudaMemcpy(g->q1a, g->h_q1a.data(), g->n1, cudaMemcpyHostToDevice));
  ETH_CUDA(A((void**)&g->wind, g->nu2 * 8));
  ETH_CUDA(A((void**)&g->E, (size_t)NE * n0 * 8));
  ETH_CUDA(A((void**)&g->part, (size_t)2 * DOT_NB * 8));
  ETH_CUDA(A((void**)&g->ticket, 16 * sizeof(unsigned)));
  ETH_CUDA(cudaMemset(g->ticket, 0, 16 * sizeof(unsigned)));
  ETH_CUDA(A((void**)&g->red, 64 * 8));
  ETH_CUDA(cudaMallocHost((void**)&g->redh, 64 * 8));
  ETH_CUDA(A((void**)&g->pcg, sizeof(PcgS)));
  ETH_CUDA(A((void**)&g->mdinv, g->nv * 8));
  ETH_CUDA(A((void**)&g->q1dinv, g->n1 * 8));
  ETH_CUDA(A((void**)&g->kv, g->np * 8));
  ETH_CUDA(A((void**)&g->f1e, n0 * 16 * 8));
  for (double** p : {&g->t0, &g->t1, &g->t2, &g->xs, &g->bv, &g->zo}) ETH_CUDA(A((void**)p, g->nt * 8));
  ETH_CUDA(cudaStreamCreateWithFlags(&g->si, cudaStreamNonBlocking));
  for (cudaEvent_t& e : g->ev) ETH_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  for (double** p : {&g->pr, &g->pz, &g->pp, &g->pq, &g->px, &g->pa, &g->pb}) ETH_CUDA(A((void**)p, g->np * 8));
  k_diag_setup<<<nblk(g->nv + g->np), 256, 0, g->s>>>(g->nx, g->ny, g->h, g->act, g->fix, g->q1a, g->mdinv, g->q1dinv, g->kv);
  ETH_CUDA(cudaGetLastError());
  size_t cnt = 0;
  for (unsigned char v : g->h_q1a) cnt += v;
  for (unsigned char v : g->h_act) cnt += v;
  g->kk = (double)cnt;
  ETH_CUDA(cudaStreamSynchronize(g->s));
  ETH_TRY(mg_build_geometry(g));
  ETH_TRY(q_build(g));
  ETH_CUDA(cudaStreamSynchronize(g->s));
  return ETH_OK;
}

extern "C" {

eth_status eth_mgrid_create(int nx, int ny, double h, double x0, double y0, const unsigned char* active_host, int outflow,
                            void* cuda_stream, eth_mgrid** out) {
  if (!out || !active_host) { set_error("eth_mgrid_create: NULL argument"); return ETH_EINVAL; }
  *out = nullptr;
  if (nx < 1 || ny < 1 || !(h > 0.0) || (outflow != 0 && outflow != 1)) {
    set_error("eth_mgrid_create: need nx, ny >= 1, h > 0, outflow in {0, 1}");
    return ETH_EINVAL;
  }
  const double nt = 2.0 * (2.0 * nx + 1) * (2.0 * ny + 1) + (nx + 1.0) * (ny + 1.0) + (double)nx * ny;
  if (nt > 2.0e9) { set_error("eth_mgrid_create: grid too large"); return ETH_EINVAL; }
  size_t nact = 0;
  for (size_t e = 0; e < (size_t)nx * ny; ++e) nact += active_host[e] ? 1 : 0;
  if (nact == 0) { set_error("eth_mgrid_create: no active element"); return ETH_EINVAL; }
  eth_mgrid* g = new eth_mgrid();
  cudaGetDevice(&g->dev);
  g->s = (cudaStream_t)cuda_stream;
  g->nx = nx; g->ny = ny; g->h = h; g->x0 = x0; g->y0 = y0; g->outflow = outflow;
  const eth_status s = mgrid_init(g, active_host);
  if (s != ETH_OK) { mgrid_free(g); return s; }
  *out = g;
  return ETH_OK;
}

void eth_mgrid_destroy(eth_mgrid* g) {
  if (!g) return;
  DeviceGuard dg(g->dev);
  cudaStreamSynchronize(g->s);
  mgrid_free(g);
}

eth_status eth_mask_roles(int nx, int ny, const unsigned char* active_host, int outflow, unsigned char* fixed_host,
                          unsigned char* dirichlet_host, unsigned char* q1_active_host) {
  if (!active_host || nx < 1 || ny < 1 || (outflow != 0 && outflow != 1)) {
    set_error("eth_mask_roles: need nx, ny >= 1, an element mask and outflow in {0, 1}");
    return ETH_EINVAL;
  }
  std::vector<unsigned char> act((size_t)nx * ny), fix, dir, q1a;
  for (size_t e = 0; e < act.size(); ++e) act[e] = active_host[e] ? 1 : 0;
  node_roles(nx, ny, outflow, act, fix, dir, q1a);
  if (fixed_host) std::memcpy(fixed_host, fix.data(), fix.size());
  if (dirichlet_host) std::memcpy(dirichlet_host, dir.data(), dir.size());
  if (q1_active_host) std::memcpy(q1_active_host, q1a.data(), q1a.size());
  return ETH_OK;
}

eth_status eth_mgrid_sizes(const eth_mgrid* g, long long* nv, long long* n1, long long* n0, long long* nt) {
  if (!g) { set_error("eth_mgrid_sizes: NULL grid"); return ETH_EINVAL; }
  if (nv) *nv = (long long)g->nv;
  if (n1) *n1 = (long long)g->n1;
  if (n0) *n0 = (long long)g->n0;
  if (nt) *nt = (long long)g->nt;
  return ETH_OK;
}

eth_status eth_mgrid_roles(const eth_mgrid* g, unsigned char* fixed_host, unsigned char* dirichlet_host,
                           unsigned char* q1_active_host, int* levels, int* coarse_free) {
  if (!g) { set_error("eth_mgrid_roles: NULL grid"); return ETH_EINVAL; }
  if (fixed_host) std::memcpy(fixed_host, g->h_fix.data(), g->nv);
  if (dirichlet_host) std::memcpy(dirichlet_host, g->h_dir.data(), g->nv);
  if (q1_active_host) std::memcpy(q1_active_host, g->h_q1a.data(), g->n1);
  if (levels) *levels = (int)g->lv.size();
  if (coarse_free) *coarse_free = g->ncf;
  return ETH_OK;
}

eth_status eth_mgrid_set_coefficients(eth_mgrid* g, double nu, const double* wind_dev) {
  if (!g) { set_error("eth_mgrid_set_coefficients: NULL grid"); return ETH_EINVAL; }
  if (!(nu > 0.0)) { set_error("eth_mgrid_set_coefficients: nu must be > 0"); return ETH_EINVAL; }
  ETH_ON_DEVICE(g);
  g->nu = nu;
  g->conv = wind_dev != nullptr;
  if (wind_dev) ETH_CUDA(cudaMemcpyAsync(g->wind, wind_dev, g->nu2 * 8, cudaMemcpyDeviceToDevice, g->s));
  g->has_coef = true;
  g->prec_ok = false;
  return ETH_OK;
}

eth_status eth_mgrid_apply(eth_mgrid* g, eth_op op, const double* x, double* y) {
  if (!g || !x || !y) { set_error("eth_mgrid_apply: NULL argument"); return ETH_EINVAL; }
  if (!g->has_coef) { set_error("eth_mgrid_apply: call eth_mgrid_set_coefficients first"); return ETH_EINVAL; }
  ETH_ON_DEVICE(g);
  constexpr int FF = QF_DIFF | QF_XIN | QF_UOUT;
  switch (op) {
    case ETH_OP_K: return apply_K(g, false, x, y);
    case ETH_OP_K1: return apply_K(g, true, x, y);
    case ETH_OP_A:
      ETH_TRY((elem64<FF>(g, 1, x, nullptr, nullptr)));
      return vgat64(g, V_ID, x, nullptr, y);
    case ETH_OP_F:
      if (g->conv) ETH_TRY((elem64<FF | QF_CONV>(g, 1, x, nullptr, g->wind)));
      else ETH_TRY((elem64<FF>(g, 1, x, nullptr, nullptr)));
      return vgat64(g, V_ID, x, nullptr, y);
    case ETH_OP_B:
      ETH_TRY((elem64<QF_XIN | QF_POUT>(g, 1, x, nullptr, nullptr)));
      return pgat64(g, P_PLAIN, g->np, (const double*)nullptr, y);
    case ETH_OP_BT:
      ETH_TRY((elem64<QF_PIN | QF_P0 | QF_UOUT>(g, 0, nullptr, x, nullptr)));
      return vgat64(g, V_ZERO, (const double*)nullptr, nullptr, y);
    case ETH_OP_MQ:
      k_mq_apply<<<nblk(g->np), 256, 0, g->s>>>(g->nx, g->ny, g->h, g->act, g->q1a, 0, x, y);
      ETH_CUDA(cudaGetLastError());
      g->launches++;
      return ETH_OK;
    default:
      set_error("eth_mgrid_apply: operator %d not available on masked grids", (int)op);
      return ETH_EINVAL;
  }
}

eth_status eth_mgrid_rhs(eth_mgrid* g, const double* ubc, double* b) {
  if (!g || !ubc || !b) { set_error("eth_mgrid_rhs: NULL argument"); return ETH_EINVAL; }
  if (!g->has_coef) { set_error("eth_mgrid_rhs: call eth_mgrid_set_coefficients first"); return ETH_EINVAL; }
  ETH_ON_DEVICE(g);
  constexpr int FR = QF_DIFF | QF_XIN | QF_UOUT | QF_POUT;
  if (g->conv) ETH_TRY((elem64<FR | QF_CONV>(g, 2, ubc, nullptr, g->wind)));
  else ETH_TRY((elem64<FR>(g, 2, ubc, nullptr, nullptr)));
  ETH_TRY(vgat64(g, V_RHS, ubc, nullptr, b));
  return pgat64(g, P_NEG, g->np, (const double*)nullptr, b + g->nu2);
}

// The solve runs on the handle's internal stream (capturable), after the work
// already queued on the user stream, and is joined back to it.
static eth_status mgrid_solve(eth_mgrid* g, const eth_opts* o, const double* b, double* x, eth_stats* st) {
  eth_stats tmp{};
  const long l0 = g->launches;
  const auto t0 = std::chrono::steady_clock::now();
  const cudaStream_t user = g->s;
  ETH_CUDA(cudaEventRecord(g->ev[0], user));
  ETH_CUDA(cudaStreamWaitEvent(g->si, g->ev[0], 0));
  g->s = g->si;
  const eth_status s2 = two_stage(g, o, b, x, &tmp);
  g->s = user;
  ETH_CUDA(cudaEventRecord(g->ev[1], g->si));
  ETH_CUDA(cudaStreamWaitEvent(user, g->ev[1], 0));
  if (s2 != ETH_OK) { cudaStreamSynchronize(g->si); return s2; }
  ETH_CUDA(cudaStreamSynchronize(g->s));
  tmp.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  tmp.kernel_launches = (int)(g->launches - l0);
  if (st) *st = tmp;
  return ETH_OK;
}

static bool opts_ok(const eth_opts* o) {
  return o && o->tol > 0.0 && o->tol < 1.0 && o->maxit >= 1 && o->restart >= 1 && o->restart <= 1000 && o->mg_pre <= 64 &&
         o->mg_post <= 64 && o->c_stage >= 0.0;
}

eth_status eth_mgrid_solve(eth_mgrid* g, const eth_opts* opts, const double* b, double* x, eth_stats* stats) {
  if (!g || !b || !x) { set_error("eth_mgrid_solve: NULL argument"); return ETH_EINVAL; }
  if (!g->has_coef) { set_error("eth_mgrid_solve: call eth_mgrid_set_coefficients first"); return ETH_EINVAL; }
  if (!g->outflow) { set_error("eth_mgrid_solve: the masked-grid solver needs an outflow boundary (outflow = 1)"); return ETH_EINVAL; }
  eth_opts def;
  eth_default_opts(&def);
  const eth_opts* o = opts ? opts : &def;
  if (!opts_ok(o)) { set_error("eth_mgrid_solve: bad options"); return ETH_EINVAL; }
  ETH_ON_DEVICE(g);
  return mgrid_solve(g, o, b, x, stats);
}

eth_status eth_mgrid_picard(eth_mgrid* g, const eth_opts* opts, const double* ubc, int steps, double* x, double* xs,
                            double* nlres_host, eth_stats* stats_host) {
  if (!g || !ubc || !x) { set_error("eth_mgrid_picard: NULL argument"); return ETH_EINVAL; }
  if (!g->has_coef) { set_error("eth_mgrid_picard: set the viscosity with eth_mgrid_set_coefficients first"); return ETH_EINVAL; }
  if (!g->outflow) { set_error("eth_mgrid_picard: the masked-grid solver needs an outflow boundary (outflow = 1)"); return ETH_EINVAL; }
  if (steps < 1 || steps > 1000) { set_error("eth_mgrid_picard: steps must be in 1..1000"); return ETH_EINVAL; }
  eth_opts def;
  eth_default_opts(&def);
  const eth_opts* o = opts ? opts : &def;
  if (!opts_ok(o)) { set_error("eth_mgrid_picard: bad options"); return ETH_EINVAL; }
  ETH_ON_DEVICE(g);
  g->conv = false;       // step 1: the Stokes problem
  g->prec_ok = false;
  for (int k = 0; k < steps; ++k) {
    ETH_TRY(eth_mgrid_rhs(g, ubc, g->bv));
    eth_stats st{};
    ETH_TRY(mgrid_solve(g, o, g->bv, x, &st));
    if (stats_host) stats_host[k] = st;   // ETH_ENOTCONV of a step is reported there and does not stop the iteration
    if (xs) ETH_CUDA(cudaMemcpyAsync(xs + (size_t)k * g->nt, x, g->nt * 8, cudaMemcpyDeviceToDevice, g->s));
    // linearise at the new iterate: w = u_k, and the nonlinear residual there
    ETH_CUDA(cudaMemcpyAsync(g->wind, x, g->nu2 * 8, cudaMemcpyDeviceToDevice, g->s));
    g->conv = true;
    g->prec_ok = false;
    ETH_TRY(eth_mgrid_rhs(g, ubc, g->bv));
    ETH_TRY(apply_K(g, false, x, g->t2));
    k_bminus<<<nblk(g->nt), 256, 0, g->s>>>(g->nt, g->bv, g->t2);
    ETH_CUDA(cudaGetLastError());
    ETH_TRY(dot2(g, g->nt, g->t2, g->t2, g->bv, g->bv, 0));
    ETH_TRY(fetch(g, 2));
    if (nlres_host) nlres_host[k] = g->redh[1] > 0.0 ? std::sqrt(g->redh[0] / g->redh[1]) : 0.0;
  }
  ETH_CUDA(cudaStreamSynchronize(g->s));
  return ETH_OK;
}

}  // extern "C"
