// Warp-strip form of the fused K apply (FP64 input and output, Dirichlet rows
// identity): the operator kernel of the Krylov loops and of eth_apply.
//
// One warp walks up a strip of element columns: lane L holds element column
// ex = ex0 - 1 + L.  Lanes 1..30 own the nodes at the lower-left of their
// element (vertex (2ex, 2ey), the two edge midpoints (2ex+1, 2ey) and
// (2ex, 2ey+1), the centre (2ex+1, 2ey+1), the Q1 vertex (ex, ey) and the P0
// element (ex, ey)); lane 0 computes the element to the left of the strip (its
// right-hand contributions) and lane 31 only loads the column of nodes to the
// right of the strip (the third node column of lane 30's element).  Phantom
// element columns and rows up to index n own the nodes on the right and top
// boundary lines.  The warp walks element rows ey0-1 .. ey0+rows-1; the first
// row only seeds the carried sums.
//
// Per element row a lane loads the two new node rows of its element (the
// bottom row is the previous element's top row, kept in registers), converts
// them to the element arithmetic type, takes the third node column from its
// right neighbour by a warp shuffle, forms the element contributions with the
// closed-form element matrices (q2_elem), takes its left neighbour's right-hand
// contributions by a shuffle, adds the sums carried from the element row below
// and writes the owned outputs.  No shared memory, no atomics: every node sums
// its (at most four) element contributions in one fixed order.  The next row's
// loads are issued before the current row is computed.
#pragma once
#include "q2tile.cuh"

namespace eth {

constexpr int QS_OWN = 30;     // owned element columns per warp (lanes 1 .. 30)
constexpr int QS_WARPS = 4;    // warps per CTA
constexpr int TILE_STRIP = 200;   // tile codes TILE_STRIP + rows select this kernel
#ifndef ETH_STRIP_MINB
#define ETH_STRIP_MINB 5       // resident CTAs per SM the FP32 Stokes form is compiled for
#endif
#ifndef ETH_STRIP_STCS
#define ETH_STRIP_STCS 1       // 1: outputs stored with the streaming (evict-first) hint
#endif
// output store: the outputs are not read again by the kernel
__device__ __forceinline__ void strip_st(double* p, double v) {
#if ETH_STRIP_STCS
  __stcs(p, v);
#else
  *p = v;
#endif
}

// ---------------------------------------------------------------------------
// Element arithmetic in the even/odd basis, one velocity component at a time.
//
// The 1D quadratic stiffness and mass matrices are centrosymmetric, and the
// linear-quadratic couplings of B are centrosymmetric or antisymmetric under
// the reflection of the element.  In the basis (v0 + v2, v1, v0 - v2) of a
// node triple ("e", "m", "o") and (q0 + q1, q0 - q1) of a Q1 pair ("e", "o"),
// with outputs taken as ((y0 + y2)/2, y1, (y0 - y2)/2), the element matrices
// split by parity: per component A needs 25 multiply-adds instead of 77, the
// B^T p coupling 9 + 2 and the B u coupling 9 + 2, at the price of 12 additions
// for the input transform and 12 for the output.  Transformed 1D matrices:
//   K^ = [4/3 -8/3 0; -8/3 16/3 0; 0 0 1]   (stiffness (1/3)[7 -8 1; ...])
//   M^ = [1/20 1/15 0; 1/15 8/15 0; 0 0 1/12]   (mass (1/30)[4 2 -1; ...])
// c12 (int N_c L_a') maps the odd Q1 part to (e, m) with -1/3, 2/3 and the
// even part to o with -1/2; g12 (int N_d L_b) maps e to (e, m) with 1/12, 1/3
// and o to o with 1/12 (outputs in the halved basis); for B u the transposed
// maps with unhalved inputs: c12: o -> e with -1, (e, m) -> o with -2/3, 4/3;
// g12: (e, m) -> e with 1/6, 2/3, o -> o with 1/6.  g0 = int L_b gives
// (1/6, 2/3, 0), c0 = L_a(1) - L_a(0) gives -o.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr double eoK(int i, int j) {
  return (i == 2 || j == 2) ? (i == j ? 1.0 : 0.0) : (i == 0 ? (j == 0 ? 4.0 / 3.0 : -8.0 / 3.0) : (j == 0 ? -8.0 / 3.0 : 16.0 / 3.0));
}
__host__ __device__ constexpr double eoM(int i, int j) {
  return (i == 2 || j == 2) ? (i == j ? 1.0 / 12.0 : 0.0) : (i == 0 ? (j == 0 ? 1.0 / 20.0 : 1.0 / 15.0) : (j == 0 ? 1.0 / 15.0 : 8.0 / 15.0));
}
// B^T maps (output class i in {e, m, o} from Q1 class k in {e, o}), halved outputs
__host__ __device__ constexpr double eoC(int i, int k) {   // c12
  return k == 1 ? (i == 0 ? -1.0 / 3.0 : (i == 1 ? 2.0 / 3.0 : 0.0)) : (i == 2 ? -0.5 : 0.0);
}
__host__ __device__ constexpr double eoG(int i, int k) {   // g12
  return k == 0 ? (i == 0 ? 1.0 / 12.0 : (i == 1 ? 1.0 / 3.0 : 0.0)) : (i == 2 ? 1.0 / 12.0 : 0.0);
}
// B maps (Q1 class k from input class i), unhalved inputs
__host__ __device__ constexpr double eoCt(int k, int i) {   // c12
  return k == 0 ? (i == 2 ? -1.0 : 0.0) : (i == 0 ? -2.0 / 3.0 : (i == 1 ? 4.0 / 3.0 : 0.0));
}
__host__ __device__ constexpr double eoGt(int k, int i) {   // g12
  return k == 0 ? (i == 0 ? 1.0 / 6.0 : (i == 1 ? 2.0 / 3.0 : 0.0)) : (i == 2 ? 1.0 / 6.0 : 0.0);
}
__host__ __device__ constexpr double eoG0(int i) { return i == 0 ? 1.0 / 6.0 : (i == 1 ? 2.0 / 3.0 : 0.0); }

// (v0, v1, v2) -> (v0 + v2, v1, v0 - v2) along x (a) then y (b): Uh[beta][alpha]
template <class CT>
__device__ __forceinline__ void eo_fwd(const CT (&U)[9], CT (&Uh)[3][3]) {
  CT X[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    X[b][0] = U[b * 3] + U[b * 3 + 2];
    X[b][1] = U[b * 3 + 1];
    X[b][2] = U[b * 3] - U[b * 3 + 2];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Uh[0][a] = X[0][a] + X[2][a];
    Uh[1][a] = X[1][a];
    Uh[2][a] = X[0][a] - X[2][a];
  }
}
// halved-basis outputs Yh[beta][alpha] -> nodal Y[b*3 + a]
template <class CT>
__device__ __forceinline__ void eo_inv(const CT (&Yh)[3][3], CT (&Y)[9]) {
  CT R[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    R[0][a] = Yh[0][a] + Yh[2][a];
    R[1][a] = Yh[1][a];
    R[2][a] = Yh[0][a] - Yh[2][a];
  }
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    Y[b * 3] = R[b][0] + R[b][2];
    Y[b * 3 + 1] = R[b][1];
    Y[b * 3 + 2] = R[b][0] - R[b][2];
  }
}

// Velocity component C of one element: Y = nu A u_C + (B^T p)_C (nodal), and this
// component's part of B u added to Zh[delta][gamma] (Q1, transformed, 4x the
// nodal values) and Z0 (P0).  Ph[delta][gamma]: the transformed Q1 pressure.
template <class CT, int F, int C>
__device__ __forceinline__ void eo_comp(const CT (&U)[9], const CT (&Ph)[2][2], CT P0, CT skm, CT smk, CT hx, CT hy,
                                        CT (&Y)[9], CT (&Zh)[2][2], CT& Z0) {
  constexpr bool DIFF = F & QF_DIFF, PIN = F & QF_PIN, HP0 = F & QF_P0, POUT = F & QF_POUT;
  CT Uh[3][3], Yh[3][3];
  eo_fwd<CT>(U, Uh);
#pragma unroll
  for (int bb = 0; bb < 3; ++bb)
#pragma unroll
    for (int aa = 0; aa < 3; ++aa) Yh[bb][aa] = 0;
  if (DIFF) {
    if (skm == smk) {
#pragma unroll
      for (int bb = 0; bb < 3; ++bb)
#pragma unroll
        for (int aa = 0; aa < 3; ++aa) {
          CT acc = 0;
#pragma unroll
          for (int b2 = 0; b2 < 3; ++b2)
#pragma unroll
            for (int a2 = 0; a2 < 3; ++a2) {
              const double cf = eoM(bb, b2) * eoK(aa, a2) + eoK(bb, b2) * eoM(aa, a2);
              if (cf != 0.0) acc += (CT)cf * Uh[b2][a2];
            }
          Yh[bb][aa] = skm * acc;
        }
    } else {
#pragma unroll
      for (int bb = 0; bb < 3; ++bb)
#pragma unroll
        for (int aa = 0; aa < 3; ++aa) {
          CT a1 = 0, a2s = 0;
#pragma unroll
          for (int b2 = 0; b2 < 3; ++b2)
#pragma unroll
            for (int a2 = 0; a2 < 3; ++a2) {
              const double c1 = eoM(bb, b2) * eoK(aa, a2), c2 = eoK(bb, b2) * eoM(aa, a2);
              if (c1 != 0.0) a1 += (CT)c1 * Uh[b2][a2];
              if (c2 != 0.0) a2s += (CT)c2 * Uh[b2][a2];
            }
          Yh[bb][aa] = skm * a1 + smk * a2s;
        }
    }
  }
  if (PIN) {   // + B^T p: x component c12 along x, g12 along y (scaled -hy); y component swapped (-hx)
    const CT s = C == 0 ? -hy : -hx;
#pragma unroll
    for (int bb = 0; bb < 3; ++bb)
#pragma unroll
      for (int aa = 0; aa < 3; ++aa) {
        CT acc = 0;
#pragma unroll
        for (int dl = 0; dl < 2; ++dl)
#pragma unroll
          for (int gm = 0; gm < 2; ++gm) {
            const double cf = C == 0 ? eoG(bb, dl) * eoC(aa, gm) : eoC(bb, dl) * eoG(aa, gm);
            if (cf != 0.0) acc += (CT)cf * Ph[dl][gm];
          }
        if (HP0) {   // B0^T: -c0 (odd) in the derivative direction, g0 in the other
          const double c0 = C == 0 ? (aa == 2 ? -eoG0(bb) : 0.0) : (bb == 2 ? -eoG0(aa) : 0.0);
          if (c0 != 0.0) acc += (CT)c0 * P0;
        }
        Yh[bb][aa] += s * acc;
      }
  }
  if (POUT) {   // B u: Zh[delta][gamma] += s * sum (maps) Uh
    const CT s = C == 0 ? -hy : -hx;
#pragma unroll
    for (int dl = 0; dl < 2; ++dl)
#pragma unroll
      for (int gm = 0; gm < 2; ++gm) {
        CT acc = 0;
#pragma unroll
        for (int bb = 0; bb < 3; ++bb)
#pragma unroll
          for (int aa = 0; aa < 3; ++aa) {
            const double cf = C == 0 ? eoGt(dl, bb) * eoCt(gm, aa) : eoCt(dl, bb) * eoGt(gm, aa);
            if (cf != 0.0) acc += (CT)cf * Uh[bb][aa];
          }
        Zh[dl][gm] += s * acc;
      }
    if (HP0) {
      CT acc = 0;
#pragma unroll
      for (int i = 0; i < 2; ++i) acc += (CT)eoG0(i) * (C == 0 ? Uh[i][2] : Uh[2][i]);
      Z0 += (C == 0 ? hy : hx) * acc;
    }
  }
  eo_inv<CT>(Yh, Y);
}

// Wind at the 3x3 Gauss points of an element (both components).
template <class CT>
__device__ __forceinline__ void wind_gauss(const CT (&Wn)[2][9], CT (&WQ)[2][9]) {
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    CT T2[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int q = 0; q < 3; ++q)
        T2[b][q] = LV(q, 0) * Wn[c][b * 3] + LV(q, 1) * Wn[c][b * 3 + 1] + LV(q, 2) * Wn[c][b * 3 + 2];
#pragma unroll
    for (int qy = 0; qy < 3; ++qy)
#pragma unroll
      for (int qx = 0; qx < 3; ++qx)
        WQ[c][qy * 3 + qx] = LV(qy, 0) * T2[0][qx] + LV(qy, 1) * T2[1][qx] + LV(qy, 2) * T2[2][qx];
  }
}

// Convection (or its element transpose) of one velocity component, added to Y:
// the same 3x3 Gauss sum factorisation as q2_elem.
template <class CT, int F>
__device__ __forceinline__ void conv_comp(const CT (&U)[9], const CT (&WQ)[2][9], CT ihx, CT ihy, CT area, CT (&Y)[9]) {
  constexpr bool TRANS = F & QF_TRANS;
  CT T1[3][3], T2[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (!TRANS) T1[b][q] = LD(q, 0) * U[b * 3] + LD(q, 1) * U[b * 3 + 1] + LD(q, 2) * U[b * 3 + 2];
      T2[b][q] = LV(q, 0) * U[b * 3] + LV(q, 1) * U[b * 3 + 1] + LV(q, 2) * U[b * 3 + 2];
    }
  CT GX[9], GY[9], CV[9];
#pragma unroll
  for (int qy = 0; qy < 3; ++qy)
#pragma unroll
    for (int qx = 0; qx < 3; ++qx) {
      const int q = qy * 3 + qx;
      const CT wq = GW(qx) * GW(qy) * area;
      if (!TRANS) {
        const CT dx = ihx * (LV(qy, 0) * T1[0][qx] + LV(qy, 1) * T1[1][qx] + LV(qy, 2) * T1[2][qx]);
        const CT dy = ihy * (LD(qy, 0) * T2[0][qx] + LD(qy, 1) * T2[1][qx] + LD(qy, 2) * T2[2][qx]);
        CV[q] = wq * (WQ[0][q] * dx + WQ[1][q] * dy);
        GX[q] = 0; GY[q] = 0;
      } else {
        const CT vl = LV(qy, 0) * T2[0][qx] + LV(qy, 1) * T2[1][qx] + LV(qy, 2) * T2[2][qx];
        GX[q] = wq * ihx * WQ[0][q] * vl;
        GY[q] = wq * ihy * WQ[1][q] * vl;
        CV[q] = 0;
      }
    }
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    CT H1[3], H2[3];
#pragma unroll
    for (int qx = 0; qx < 3; ++qx) {
      if (TRANS) {
        H1[qx] = LV(0, b) * GX[qx] + LV(1, b) * GX[3 + qx] + LV(2, b) * GX[6 + qx];
        H2[qx] = LD(0, b) * GY[qx] + LD(1, b) * GY[3 + qx] + LD(2, b) * GY[6 + qx];
      } else {
        H1[qx] = 0;
        H2[qx] = LV(0, b) * CV[qx] + LV(1, b) * CV[3 + qx] + LV(2, b) * CV[6 + qx];
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
      Y[b * 3 + a] += LD(0, a) * H1[0] + LD(1, a) * H1[1] + LD(2, a) * H1[2] +
                      LV(0, a) * H2[0] + LV(1, a) * H2[1] + LV(2, a) * H2[2];
  }
}

// FP64 -> element type for K values at once: the short integer conversion on
// every lane, and the full one only when some lane of the warp holds a value
// outside the normal binary32 range (one vote for the whole batch).  Every lane
// of the warp must call it.
template <class CT, int K>
__device__ __forceinline__ void cvt_batch(const double (&v)[K], const bool (&ok)[K], CT (&out)[K]) {
  if constexpr (sizeof(CT) == 8) {
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = ok[k] ? (CT)v[k] : CT(0);
  } else {
    bool bad = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const unsigned long long u = (unsigned long long)__double_as_longlong(v[k]);
      const unsigned hi = (unsigned)(u >> 32);
      const unsigned t = (unsigned)((u + (1ull << 28)) >> 29) + 0x40000000u;
      out[k] = ok[k] ? __uint_as_float((t & 0x7fffffffu) | (hi & 0x80000000u)) : 0.0f;
      bad |= ok[k] && ((hi & 0x7ff00000u) - (897u << 20) >= (254u << 20));
    }
    if (__any_sync(0xffffffffu, bad)) {
#pragma unroll
      for (int k = 0; k < K; ++k) out[k] = ok[k] ? f64_to_f32_bits(v[k]) : 0.0f;
    }
  }
}

// The rows [ey0, ey1) of one warp's strip.  INT: the warp touches no boundary
// node and no phantom element (every load, element and output exists and is an
// interior one), so every bounds test below folds away.
template <class CT, int F, bool INT>
__device__ __forceinline__ void strip_warp(const Q2Params<double, double, CT>& P, int lane, int ex, int ey0, int ey1,
                                           double& dacc) {
  constexpr bool CONV = F & QF_CONV, PIN = F & QF_PIN, HP0 = F & QF_P0, POUT = F & QF_POUT, DOT = F & QF_DOT;
  // outputs: the conversion instruction (FP64 pipe) for everything in the plain apply;
  // with the fused dot (FP64 products on the same pipe) the second velocity component
  // goes through the integer bit path instead
  constexpr bool HW1 = false;
  const unsigned FULL = 0xffffffffu;
  const int n = P.n, N = 2 * n + 1, nv = N * N, M = n + 1, n1 = M * M;
  const bool comp = lane <= QS_OWN;                    // lanes that compute an element
  const bool owner = lane >= 1 && lane <= QS_OWN && (INT || ex <= n);
  const int i0 = 2 * ex, i1 = 2 * ex + 1;
  const bool c0in = INT || (i0 > 0 && i0 < 2 * n);     // interior node columns
  const bool c1in = comp && (INT || (i1 > 0 && i1 < 2 * n));
  const bool c0ex = INT || (i0 >= 0 && i0 <= 2 * n);   // existing node columns (wind)
  const bool c1ex = comp && (INT || (i1 >= 0 && i1 <= 2 * n));
  const bool cP = INT || (ex >= 0 && ex <= n);         // existing Q1 column
  const bool colB = !INT && (i0 == 0 || i0 == 2 * n);  // node column 2ex on the boundary
  const CT ihx = CT(1) / P.hx, ihy = CT(1) / P.hy, area = P.hx * P.hy;
  const CT skm = P.nu * P.hy * ihx, smk = P.nu * P.hx * ihy;
  const double* __restrict__ X = P.x;

  // raw FP64 inputs of the next element row: node rows 2ey+1, 2ey+2 at columns 2ex
  // and 2ex+1 for both components, the Q1 vertex (ex, ey+1), P0 (ex, ey)
  double raw[10];
  bool rok[10];
  auto load = [&](int ey) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int j = 2 * ey + 1 + r;
      const bool rin = INT || (j > 0 && j < 2 * n);
      const bool la = rin && c0in, lb = rin && c1in;
      const int ga = j * N + i0, gb = ga + 1;
      rok[r * 4 + 0] = rok[r * 4 + 1] = la;
      rok[r * 4 + 2] = rok[r * 4 + 3] = lb;
      raw[r * 4 + 0] = la ? X[ga] : 0.0;
      raw[r * 4 + 1] = la ? X[ga + nv] : 0.0;
      raw[r * 4 + 2] = lb ? X[gb] : 0.0;
      raw[r * 4 + 3] = lb ? X[gb + nv] : 0.0;
    }
    rok[8] = PIN && cP && (INT || (ey + 1 >= 0 && ey + 1 <= n));
    raw[8] = rok[8] ? P.p[(ey + 1) * M + ex] : 0.0;
    rok[9] = PIN && HP0 && comp && (INT || (ex >= 0 && ex < n && ey >= 0 && ey < n));
    raw[9] = rok[9] ? P.p[n1 + ey * n + ex] : 0.0;
  };
  auto wld = [&](int j, int i, bool colok, int c) -> CT {
    return (colok && (INT || (j >= 0 && j <= 2 * n))) ? P.w[j * N + i + c * nv] : CT(0);
  };

  // bottom node row of the seed element row ey0-1 (node row 2ey0-2, Q1 row ey0-1)
  CT uB[2][3], pB[2], wB[2][3];
  {
    const int j = 2 * ey0 - 2;
    const bool rin = INT || (j > 0 && j < 2 * n);
    double v[5];
    bool ok[5];
    ok[0] = ok[1] = rin && c0in;
    ok[2] = ok[3] = rin && c1in;
    ok[4] = PIN && cP && (INT || ey0 - 1 >= 0);
    v[0] = ok[0] ? X[j * N + i0] : 0.0;
    v[1] = ok[1] ? X[j * N + i0 + nv] : 0.0;
    v[2] = ok[2] ? X[j * N + i1] : 0.0;
    v[3] = ok[3] ? X[j * N + i1 + nv] : 0.0;
    v[4] = ok[4] ? P.p[(ey0 - 1) * M + ex] : 0.0;
    CT c[5];
    cvt_batch<CT, 5>(v, ok, c);
    uB[0][0] = c[0]; uB[1][0] = c[1]; uB[0][1] = c[2]; uB[1][1] = c[3];
    uB[0][2] = __shfl_down_sync(FULL, uB[0][0], 1);
    uB[1][2] = __shfl_down_sync(FULL, uB[1][0], 1);
    pB[0] = PIN ? c[4] : CT(0);
    pB[1] = __shfl_down_sync(FULL, pB[0], 1);
    if (CONV) {
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        wB[cc][0] = wld(j, i0, c0ex, cc);
        wB[cc][1] = wld(j, i1, c1ex, cc);
        wB[cc][2] = __shfl_down_sync(FULL, wB[cc][0], 1);
      }
    }
  }
  CT carV[2] = {0, 0}, carE[2] = {0, 0}, carP = 0;
  load(ey0 - 1);
  for (int ey = ey0 - 1; ey < ey1; ++ey) {
    // this row's new inputs (converted), then the next row's loads in flight
    CT cvv[10];
    cvt_batch<CT, 10>(raw, rok, cvv);
    CT u1[2][3], u2[2][3], pT[2], p0v;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      u1[c][0] = cvv[c]; u1[c][1] = cvv[2 + c];
      u2[c][0] = cvv[4 + c]; u2[c][1] = cvv[6 + c];
      u1[c][2] = __shfl_down_sync(FULL, u1[c][0], 1);
      u2[c][2] = __shfl_down_sync(FULL, u2[c][0], 1);
    }
    pT[0] = PIN ? cvv[8] : CT(0);
    pT[1] = __shfl_down_sync(FULL, pT[0], 1);
    p0v = (PIN && HP0) ? cvv[9] : CT(0);
    CT w1[2][3], w2[2][3];
    if (CONV) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        w1[c][0] = wld(2 * ey + 1, i0, c0ex, c); w1[c][1] = wld(2 * ey + 1, i1, c1ex, c);
        w2[c][0] = wld(2 * ey + 2, i0, c0ex, c); w2[c][1] = wld(2 * ey + 2, i1, c1ex, c);
        w1[c][2] = __shfl_down_sync(FULL, w1[c][0], 1);
        w2[c][2] = __shfl_down_sync(FULL, w2[c][0], 1);
      }
    }
    if (ey + 1 < ey1) load(ey + 1);

    const bool valid = comp && (INT || (ex >= 0 && ex < n && ey >= 0 && ey < n));
    const bool emitrow = owner && ey >= ey0;
    const int j0 = 2 * ey;
    const bool rowB = !INT && (ey == 0 || ey == n);     // node row 2ey on the boundary
    const bool xin = INT || ex < n, yin = INT || ey < n;
    // transformed Q1 pressure of the element
    CT Ph[2][2] = {{0, 0}, {0, 0}};
    if (PIN) {
      const CT e0 = pB[0] + pB[1], o0 = pB[0] - pB[1], e1 = pT[0] + pT[1], o1 = pT[0] - pT[1];
      Ph[0][0] = e0 + e1; Ph[0][1] = o0 + o1; Ph[1][0] = e0 - e1; Ph[1][1] = o0 - o1;
    }
    CT WQ[2][9];
    if (CONV && valid) {
      CT Wn[2][9];
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int a = 0; a < 3; ++a) { Wn[c][a] = wB[c][a]; Wn[c][3 + a] = w1[c][a]; Wn[c][6 + a] = w2[c][a]; }
      wind_gauss<CT>(Wn, WQ);
    }
    CT Zh[2][2] = {{0, 0}, {0, 0}}, Z0 = 0;
    CT fdot = 0;   // FP32 element arithmetic: this row's dot partial (inputs are FP32 already)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      CT Y[9];
      if (valid) {
        CT U[9];
#pragma unroll
        for (int a = 0; a < 3; ++a) { U[a] = uB[c][a]; U[3 + a] = u1[c][a]; U[6 + a] = u2[c][a]; }
        if (c == 0) eo_comp<CT, F, 0>(U, Ph, p0v, skm, smk, P.hx, P.hy, Y, Zh, Z0);
        else eo_comp<CT, F, 1>(U, Ph, p0v, skm, smk, P.hx, P.hy, Y, Zh, Z0);
        if (CONV) conv_comp<CT, F>(U, WQ, ihx, ihy, area, Y);
      } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) Y[k] = 0;
      }
      // left neighbour's right-hand contributions
      const CT L2 = __shfl_up_sync(FULL, Y[2], 1);
      const CT L5 = __shfl_up_sync(FULL, Y[5], 1);
      const CT L8 = __shfl_up_sync(FULL, Y[8], 1);
      if (emitrow) {
        double* __restrict__ yc = P.y + (size_t)c * nv;
        const double* __restrict__ xc = X + (size_t)c * nv;
        // s: the node's sum; xf: the node's input in the element type (the dot partner)
        auto emit = [&](int i, int j, bool bnd, CT s, CT xf) {
          const int g = j * N + i;
          double o;
          if (bnd) {
            o = xc[g];
            if (DOT) dacc += o * o;
          } else {
            o = (c == 0 || HW1) ? cvt_out<double, CT>(s) : cvt<double, CT>(s);
            if (DOT) {
              if constexpr (sizeof(CT) == 4) fdot += s * xf;
              else dacc += o * xc[g];
            }
          }
          strip_st(yc + g, o);
        };
        emit(i0, j0, rowB || colB, Y[0] + L2 + carV[c], uB[c][0]);
        if (xin) emit(i1, j0, rowB, Y[1] + carE[c], uB[c][1]);
        if (yin) {
          emit(i0, j0 + 1, colB, Y[3] + L5, u1[c][0]);
          if (xin) emit(i1, j0 + 1, false, Y[4], u1[c][1]);
        }
      }
      carV[c] = Y[6] + L8;   // sums carried to the next element row
      carE[c] = Y[7];
    }
    if (POUT) {   // Q1 outputs: back from the transformed basis (factor 1/4), P0 output
      CT YP1[4];
      {
        const CT x0e = Zh[0][0] + Zh[0][1], x1e = Zh[0][0] - Zh[0][1];   // delta = e
        const CT x0o = Zh[1][0] + Zh[1][1], x1o = Zh[1][0] - Zh[1][1];   // delta = o
        YP1[0] = CT(0.25) * (x0e + x0o); YP1[1] = CT(0.25) * (x1e + x1o);
        YP1[2] = CT(0.25) * (x0e - x0o); YP1[3] = CT(0.25) * (x1e - x1o);
      }
      const CT LP1 = __shfl_up_sync(FULL, YP1[1], 1);
      const CT LP3 = __shfl_up_sync(FULL, YP1[3], 1);
      if (emitrow) {
        const int gp = ey * M + ex;
        const CT sp = YP1[0] + LP1 + carP;
        const double so = cvt_out<double, CT>(sp);
        strip_st(P.yp + gp, so);
        if (DOT) {
          if constexpr (sizeof(CT) == 4) fdot += sp * pB[0];
          else dacc += so * P.dvp[gp];
        }
        if (HP0 && xin && yin) {
          const int ge = n1 + ey * n + ex;
          const double s0 = cvt_out<double, CT>(Z0);
          strip_st(P.yp + ge, s0);
          if (DOT) {
            if constexpr (sizeof(CT) == 4) fdot += Z0 * p0v;
            else dacc += s0 * P.dvp[ge];
          }
        }
      }
      carP = YP1[2] + LP3;
    }
    if (DOT && sizeof(CT) == 4) dacc += (double)fdot;
    // the top node row becomes the bottom row of the next element row
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        uB[c][a] = u2[c][a];
        if (CONV) wB[c][a] = w2[c][a];
      }
    pB[0] = pT[0];
    pB[1] = pT[1];
  }
}

template <class CT, int F>
__global__ void __launch_bounds__(32 * QS_WARPS, (sizeof(CT) == 4 && !(F & QF_CONV)) ? ETH_STRIP_MINB : 1)
    k_q2s(Q2Params<double, double, CT> P, int rows, int nstrips, int nwork) {
  ETH_GRID_DEP_WAIT();
  constexpr bool DOT = F & QF_DOT;
  static_assert((F & QF_XIN) && (F & QF_UOUT) && !(F & (QF_NOBC | QF_MASS | QF_SD | QF_SRC_JB | QF_SRC_XPC)),
                "strip kernel: velocity in/out operator applies with Dirichlet rows");
  if (P.done != nullptr && *P.done) return;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * QS_WARPS + (threadIdx.x >> 5);
  double dacc = 0.0;
  if (gw < nwork) {   // warp-uniform
    const int n = P.n;
    const int strip = gw % nstrips, chunk = gw / nstrips;
    const int ex0 = strip * QS_OWN;
    const int ey0 = chunk * rows, ey1 = min(ey0 + rows, n + 1);
    // interior warp: every node it loads (columns 2ex0-2 .. 2ex0+60, rows 2ey0-2 .. 2ey1)
    // is an interior node and every element it computes exists
    const bool interior = ex0 >= 2 && ex0 + QS_OWN < n && ey0 >= 2 && ey1 < n;
    const int ex = ex0 - 1 + lane;
    if (interior) strip_warp<CT, F, true>(P, lane, ex, ey0, ey1, dacc);
    else strip_warp<CT, F, false>(P, lane, ex, ey0, ey1, dacc);
  }
  if (DOT) {
    double v[1] = {dacc};
    if (slot_arrive<1>(P.slot, P.slot_off + blockIdx.x, v)) finish_slot(P.slot, v[0]);
  }
}

inline int q2s_warps(int n, int rows) { return (int)(cdiv(n + 1, QS_OWN) * cdiv(n + 1, rows)); }
inline int q2s_blocks(int n, int rows) { return (int)cdiv(q2s_warps(n, rows), QS_WARPS); }
inline bool q2s_rows_ok(int rows) { return rows >= 2 && rows <= 32; }

template <class CT, int F>
static cudaError_t launch_q2s(const Q2Params<double, double, CT>& P, cudaStream_t s, int rows) {
  const int nstrips = (int)cdiv(P.n + 1, QS_OWN);
  const int nwork = q2s_warps(P.n, rows);
  k_q2s<CT, F><<<q2s_blocks(P.n, rows), 32 * QS_WARPS, 0, s>>>(P, rows, nstrips, nwork);
  return cudaGetLastError();
}

}  // namespace eth
