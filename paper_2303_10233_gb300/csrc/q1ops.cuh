// Pressure-space operators on the Q1 lattice and the P0 elements.
//
// Closed-form element matrices of a rectangle hx x hy with bilinear shape
// functions (local node (c,d), c,d in {0,1}):
//   mass       M1_e = hx*hy * m(c,c') m(d,d'),          m = [[1/3,1/6],[1/6,1/3]]
//   stiffness  K1_e = hy/hx * k(c,c') m(d,d') + hx/hy * m(c,c') k(d,d'),  k = [[1,-1],[-1,1]]
//   ones       O_e  = 1 (all 16 entries)
// A Q1 node operator is y_I = sum_{T ni I} sum_{J in T} (cm*M1_e + ck*K1_e +
// c1*O_e + C_T)[I,J] x_J, where C_T is an optional per-element 4x4 matrix
// (the Q1 convection of Sec. 3.1, precomputed at set-up).  With cm = 1,
// c1 = -|T|/16 this is the Schur complement S = Qk - R^T Q0^{-1} R of the
// two-field pressure mass matrix M_Q = [Qk R^T; R Q0] (Sec. 2.3): R has the
// entries |T|/4 and Q0 = diag|T|.
#pragma once
#include "common.cuh"

namespace eth {

enum : int { Q1E_APPLY = 0, Q1E_SMOOTH = 1, Q1E_RESID = 2 };

template <class TI, class TO, class CT>
struct Q1Params {
  int n;
  CT hx, hy;
  CT cm, ck, c1;         // element-matrix coefficients
  const CT* conv;        // per-element 4x4 (row = test node), or null
  int conv_trans;        // use C_T^T
  const TI* x;           // Q1 input ((n+1)^2)
  const TI* x0;          // optional P0 input (n^2): y_I += r0 * sum_{T ni I} |T|/4 x0_T
  CT r0;
  TO* y;                 // Q1 output
  const CT* b;           // smoother rhs
  const CT* dinv;        // smoother inverse diagonal
  CT omega;
  Slot slot;             // optional fused dot <y, x>
  int slot_off;
  int dot;
  const int* done;
};

__host__ __device__ constexpr double q1m(int a, int b) { return a == b ? 1.0 / 3.0 : 1.0 / 6.0; }
__host__ __device__ constexpr double q1k(int a, int b) { return a == b ? 1.0 : -1.0; }

// Visits the (up to) four elements around Q1 node (I, J) with compile-time local
// indices: f(ex, ey, c, d) gets the element and the node's local position (c, d)
// in it (c, d are constants after unrolling, so coefficient products fold).
#define Q1_FOR_ELEMENTS(n, I, J, ...)                                   \
  _Pragma("unroll") for (int dy_ = 0; dy_ < 2; ++dy_)                    \
  _Pragma("unroll") for (int dx_ = 0; dx_ < 2; ++dx_) {                  \
    const int ex = (I) - 1 + dx_, ey = (J) - 1 + dy_;                    \
    if (ex < 0 || ex >= (n) || ey < 0 || ey >= (n)) continue;            \
    const int c = 1 - dx_, d = 1 - dy_;                                  \
    __VA_ARGS__                                                          \
  }

template <class TI, class TO, class CT, int EPI>
__global__ void __launch_bounds__(256) k_q1node(Q1Params<TI, TO, CT> P) {
  ETH_GRID_DEP_WAIT();
  if (P.done != nullptr && *P.done) return;
  const int n = P.n, M = n + 1;
  const int tot = M * M;
  double dacc = 0.0;
  const CT area = P.hx * P.hy, rxy = P.hy / P.hx, ryx = P.hx / P.hy;
  for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < tot; node += gridDim.x * blockDim.x) {
    const int J = node / M, I = node - J * M;
    CT acc = 0;
    Q1_FOR_ELEMENTS(n, I, J, {
      const int e = ey * n + ex;
#pragma unroll
      for (int dd = 0; dd < 2; ++dd)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          CT coef = P.cm * area * (CT)(q1m(c, cc) * q1m(d, dd)) +
                    P.ck * (rxy * (CT)(q1k(c, cc) * q1m(d, dd)) + ryx * (CT)(q1m(c, cc) * q1k(d, dd))) + P.c1;
          if (P.conv != nullptr) {
            const int li = d * 2 + c, lj = dd * 2 + cc;
            coef += P.conv_trans ? P.conv[(size_t)e * 16 + lj * 4 + li] : P.conv[(size_t)e * 16 + li * 4 + lj];
          }
          acc += coef * (CT)P.x[(size_t)(ey + dd) * M + ex + cc];
        }
      if (P.x0 != nullptr) acc += P.r0 * area * CT(0.25) * (CT)P.x0[e];
    })
    TO out;
    if (EPI == Q1E_APPLY) out = (TO)acc;
    else if (EPI == Q1E_SMOOTH) out = (TO)((CT)P.x[node] + P.omega * P.dinv[node] * (P.b[node] - acc));
    else out = (TO)(P.b[node] - acc);
    P.y[node] = out;
    if (P.dot) dacc += (double)out * (double)P.x[node];
  }
  if (P.dot) {
    double v[1] = {dacc};
    if (slot_arrive<1>(P.slot, P.slot_off + blockIdx.x, v)) finish_slot(P.slot, v[0]);
  }
}

// P0 rows of M_Q: y0_T = cr * |T|/4 * sum_{I in T} x1_I + cq * |T| * x0_T
template <class TI, class TO, class CT>
__global__ void k_p0rows(int n, CT area, CT cr, CT cq, const TI* __restrict__ x1, const TI* __restrict__ x0,
                         TO* __restrict__ y0, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done != nullptr && *done) return;
  const int tot = n * n, M = n + 1;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
    const int ey = e / n, ex = e - ey * n;
    CT s = (CT)x1[(size_t)ey * M + ex] + (CT)x1[(size_t)ey * M + ex + 1] + (CT)x1[(size_t)(ey + 1) * M + ex] +
           (CT)x1[(size_t)(ey + 1) * M + ex + 1];
    CT v = cr * area * CT(0.25) * s;
    if (x0 != nullptr) v += cq * area * (CT)x0[e];
    y0[e] = (TO)v;
  }
}

inline unsigned q1_blocks(int n) {
  long tot = (long)(n + 1) * (n + 1);
  long b = (tot + 255) / 256;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace eth
