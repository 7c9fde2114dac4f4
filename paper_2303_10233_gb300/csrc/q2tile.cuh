// Matrix-free element-tile applies on the Q2 velocity lattice.
//
// One CTA owns the output nodes of a block of OX x OY elements and computes
// the element contributions of a (OX+1) x (OY+1) block (one halo element on
// the low side in each direction), so every owned node gathers all its
// element contributions from shared memory: no atomics, deterministic.
//
// Per element (3x3 Gauss, sum factorisation over the tensor-product basis):
//   velocity rows  y_i += int nu grad(phi_i) : grad(u)        (A, Sec. 2)
//                       + int (w_h . grad u) phi_i             (N(w), Sec. 3)
//                       - int p div(phi_i)                     (B^T p)
//   pressure rows  yp_k = -int psi_k div u   (Q1)   yp_0 = -int_T div u (P0)
// The transposed convection (for K^T) tests (w_h phi_i) against grad u's
// trial: y_i += int (w_h . grad phi_i) u.
#pragma once
#include "common.cuh"

namespace eth {

constexpr int TEX = 32, TEY = 8;                 // computed elements per CTA
constexpr int OEX = TEX - 1, OEY = TEY - 1;      // owned elements per CTA
constexpr int Q2T = TEX * TEY;                   // threads per CTA (1 element each)
constexpr int SQX = 2 * TEX + 1, SQY = 2 * TEY + 1;   // shared Q2 node tile
constexpr int SPX = TEX + 1, SPY = TEY + 1;           // shared Q1 node tile
constexpr int NEO = 23;                          // per-element outputs: 9+9 u, 4 p1, 1 p0

enum : int {
  QF_DIFF = 1,      // nu * A
  QF_CONV = 2,      // N(w)
  QF_TRANS = 4,     // transpose the convection (N^T)
  QF_XIN = 8,       // velocity input
  QF_PIN = 16,      // B^T p (Q1 part)
  QF_P0 = 32,       // include the P0 pressure in B^T p and B u
  QF_UOUT = 64,     // velocity output
  QF_POUT = 128,    // B u output
  QF_DOT = 256,     // fused dot <y, x> over all outputs (FP64)
  QF_MASS = 512,    // velocity mass term int u phi_i
  QF_NOBC = 1024,   // no Dirichlet masking / identity rows
  QF_SD = 2048,     // streamline diffusion sum_T d_T int (w.grad u)(w.grad v) (coarse levels)
};
enum : int { EPI_APPLY = 0, EPI_SMOOTH = 1, EPI_RESID = 2, EPI_SCALE = 3, EPI_BSUB = 4 };
// EPI_SCALE: y = dinv * (op x) on the interior, 0 on the boundary.
// EPI_BSUB:  y = bsrc - (op x) on the interior, bsrc on the boundary.

template <class TI, class TO, class CT>
struct Q2Params {
  int n;
  CT hx, hy, nu;
  const TI* x;      // velocity in (2 N_v)
  const TI* p;      // pressure in ([p1; p0])
  const CT* w;      // wind (2 N_v)
  TO* y;            // velocity out
  TO* yp;           // pressure out ([p1; p0])
  const CT* b;      // smoother / residual right-hand side (2 N_v)
  const CT* dinv;   // inverse diagonal (N_v), smoother
  CT omega;
  CT sd;            // QF_SD coefficient c: d_T = c h / (2|w|_T) (1 - 1/Pe_T) when Pe_T > 1
  Slot slot;        // QF_DOT
  int slot_off;
  const TO* dv;       // QF_DOT partner of the velocity output
  const TO* dvp;      // QF_DOT partner of the pressure output
  const TO* bsrc;     // EPI_SMOOTH: boundary rows copy bsrc (else 0); EPI_BSUB: minuend
  const int* done;    // optional early-exit flag
};

template <class CT, int F>
__device__ __forceinline__ void q2_elem(const CT (&U)[2][9], const CT (&Wn)[2][9], const CT (&P1)[4], CT P0,
                                        CT nu, CT ihx, CT ihy, CT area, CT sdc, CT (&Y)[2][9], CT (&YP1)[4], CT& YP0) {
  constexpr bool CONV = F & QF_CONV, TRANS = F & QF_TRANS, PIN = F & QF_PIN, HP0 = F & QF_P0,
                 DIFF = F & QF_DIFF, POUT = F & QF_POUT, MASS = F & QF_MASS, SD = F & QF_SD;
  constexpr bool NEEDVAL = (CONV && TRANS) || MASS;
  constexpr bool NEEDGRAD = DIFF || (CONV && !TRANS) || POUT;
  CT DX[2][9], DY[2][9], VL[2][9];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    CT T1[3][3], T2[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        T1[b][q] = LD(q, 0) * U[c][b * 3] + LD(q, 1) * U[c][b * 3 + 1] + LD(q, 2) * U[c][b * 3 + 2];
        T2[b][q] = LV(q, 0) * U[c][b * 3] + LV(q, 1) * U[c][b * 3 + 1] + LV(q, 2) * U[c][b * 3 + 2];
      }
#pragma unroll
    for (int qy = 0; qy < 3; ++qy)
#pragma unroll
      for (int qx = 0; qx < 3; ++qx) {
        if (NEEDGRAD) {
          DX[c][qy * 3 + qx] = ihx * (LV(qy, 0) * T1[0][qx] + LV(qy, 1) * T1[1][qx] + LV(qy, 2) * T1[2][qx]);
          DY[c][qy * 3 + qx] = ihy * (LD(qy, 0) * T2[0][qx] + LD(qy, 1) * T2[1][qx] + LD(qy, 2) * T2[2][qx]);
        }
        if (NEEDVAL) VL[c][qy * 3 + qx] = LV(qy, 0) * T2[0][qx] + LV(qy, 1) * T2[1][qx] + LV(qy, 2) * T2[2][qx];
      }
  }
  CT WQ[2][9];
  if (CONV) {
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
  CT delta = 0;
  if (SD) {   // element streamline-diffusion parameter from the mean wind speed
    CT wn = 0;
#pragma unroll
    for (int q = 0; q < 9; ++q) wn += sqrt(WQ[0][q] * WQ[0][q] + WQ[1][q] * WQ[1][q]);
    wn *= CT(1) / CT(9);
    const CT h = CT(1) / (ihx < ihy ? ihx : ihy);
    const CT pe = wn * h / (CT(2) * nu);
    if (pe > CT(1)) delta = sdc * h / (CT(2) * wn) * (CT(1) - CT(1) / pe);
  }
  CT PQ[9];
  if (PIN) {
#pragma unroll
    for (int qy = 0; qy < 3; ++qy)
#pragma unroll
      for (int qx = 0; qx < 3; ++qx) {
        CT v = NV(qy, 0) * (NV(qx, 0) * P1[0] + NV(qx, 1) * P1[1]) + NV(qy, 1) * (NV(qx, 0) * P1[2] + NV(qx, 1) * P1[3]);
        if (HP0) v += P0;
        PQ[qy * 3 + qx] = v;
      }
  }
  if (F & QF_UOUT) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      CT GX[9], GY[9], CV[9];
#pragma unroll
      for (int qy = 0; qy < 3; ++qy)
#pragma unroll
        for (int qx = 0; qx < 3; ++qx) {
          const int q = qy * 3 + qx;
          const CT wq = GW(qx) * GW(qy) * area;
          CT gx = 0, gy = 0, cv = 0;
          if (DIFF) { gx = nu * DX[c][q]; gy = nu * DY[c][q]; }
          if (PIN) { if (c == 0) gx -= PQ[q]; else gy -= PQ[q]; }
          if (CONV && !TRANS) cv = WQ[0][q] * DX[c][q] + WQ[1][q] * DY[c][q];
          if (SD) { gx += delta * WQ[0][q] * cv; gy += delta * WQ[1][q] * cv; }
          if (CONV && TRANS) { gx += WQ[0][q] * VL[c][q]; gy += WQ[1][q] * VL[c][q]; }
          if (MASS) cv += VL[c][q];
          GX[q] = wq * ihx * gx; GY[q] = wq * ihy * gy; CV[q] = wq * cv;
        }
      CT H1[3][3], H2[3][3];   // [qx][b]
#pragma unroll
      for (int qx = 0; qx < 3; ++qx)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          H1[qx][b] = LV(0, b) * GX[qx] + LV(1, b) * GX[3 + qx] + LV(2, b) * GX[6 + qx];
          H2[qx][b] = LD(0, b) * GY[qx] + LD(1, b) * GY[3 + qx] + LD(2, b) * GY[6 + qx] +
                      LV(0, b) * CV[qx] + LV(1, b) * CV[3 + qx] + LV(2, b) * CV[6 + qx];
        }
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a)
          Y[c][b * 3 + a] = LD(0, a) * H1[0][b] + LD(1, a) * H1[1][b] + LD(2, a) * H1[2][b] +
                            LV(0, a) * H2[0][b] + LV(1, a) * H2[1][b] + LV(2, a) * H2[2][b];
    }
  }
  if (POUT) {
    CT s[4] = {0, 0, 0, 0};
    CT s0 = 0;
#pragma unroll
    for (int qy = 0; qy < 3; ++qy)
#pragma unroll
      for (int qx = 0; qx < 3; ++qx) {
        const int q = qy * 3 + qx;
        const CT dv = -(GW(qx) * GW(qy) * area) * (DX[0][q] + DY[1][q]);
        s0 += dv;
#pragma unroll
        for (int d = 0; d < 2; ++d)
#pragma unroll
          for (int cc = 0; cc < 2; ++cc) s[d * 2 + cc] += NV(qy, d) * NV(qx, cc) * dv;
      }
#pragma unroll
    for (int k = 0; k < 4; ++k) YP1[k] = s[k];
    YP0 = s0;
  }
}

template <class TI, class TO, class CT, int F, int EPI>
__global__ void __launch_bounds__(Q2T) k_q2(Q2Params<TI, TO, CT> P) {
  constexpr bool CONV = F & QF_CONV, XIN = F & QF_XIN, PIN = F & QF_PIN, HP0 = F & QF_P0,
                 UOUT = F & QF_UOUT, POUT = F & QF_POUT, DOT = F & QF_DOT, NOBC = F & QF_NOBC;
  if (P.done != nullptr && *P.done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CT* sx = reinterpret_cast<CT*>(smem_raw);                 // [2][SQY][SQX]
  CT* sw = sx + 2 * SQY * SQX;                              // [2][SQY][SQX] (CONV)
  CT* sp1 = sw + (CONV ? 2 * SQY * SQX : 0);                // [SPY][SPX]
  CT* sp0 = sp1 + SPY * SPX;                                // [TEY][TEX]
  CT* eo = sp0 + TEY * TEX;                                 // [NEO][Q2T]

  const int n = P.n, N = 2 * n + 1;
  const size_t nv = (size_t)N * N;
  const int n1 = (n + 1) * (n + 1);
  const int ex0 = blockIdx.x * OEX, ey0 = blockIdx.y * OEY;
  const int gi0 = 2 * (ex0 - 1), gj0 = 2 * (ey0 - 1);
  const int tid = threadIdx.x;

  // ---- phase 0: stage inputs (masked velocity, wind, pressure) in shared memory
  if (XIN || CONV) {
    for (int k = tid; k < SQY * SQX; k += Q2T) {
      const int lj = k / SQX, li = k - lj * SQX;
      const int i = gi0 + li, j = gj0 + lj;
      CT v0 = 0, v1 = 0, w0 = 0, w1 = 0;
      if (i >= 0 && i < N && j >= 0 && j < N) {
        const size_t g = (size_t)j * N + i;
        const bool bnd = !NOBC && (i == 0 || j == 0 || i == N - 1 || j == N - 1);
        if (XIN && !bnd) { v0 = (CT)P.x[g]; v1 = (CT)P.x[g + nv]; }
        if (CONV) { w0 = P.w[g]; w1 = P.w[g + nv]; }
      }
      if (XIN) { sx[k] = v0; sx[SQY * SQX + k] = v1; }
      if (CONV) { sw[k] = w0; sw[SQY * SQX + k] = w1; }
    }
  }
  if (PIN) {
    for (int k = tid; k < SPY * SPX; k += Q2T) {
      const int lj = k / SPX, li = k - lj * SPX;
      const int I = ex0 - 1 + li, J = ey0 - 1 + lj;
      sp1[k] = (I >= 0 && I <= n && J >= 0 && J <= n) ? (CT)P.p[(size_t)J * (n + 1) + I] : CT(0);
    }
    if (HP0) {
      for (int k = tid; k < TEY * TEX; k += Q2T) {
        const int ly = k / TEX, lx = k - ly * TEX;
        const int ex = ex0 - 1 + lx, ey = ey0 - 1 + ly;
        sp0[k] = (ex >= 0 && ex < n && ey >= 0 && ey < n) ? (CT)P.p[n1 + (size_t)ey * n + ex] : CT(0);
      }
    }
  }
  __syncthreads();

  // ---- phase 1: one element per thread
  {
    const int lx = tid % TEX, ly = tid / TEX;
    const int ex = ex0 - 1 + lx, ey = ey0 - 1 + ly;
    CT Y[2][9], YP1[4], YP0 = 0;
    if (ex >= 0 && ex < n && ey >= 0 && ey < n) {
      CT U[2][9], Wn[2][9], P1[4], P0v = 0;
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const int s = (2 * ly + b) * SQX + 2 * lx + a;
          U[0][b * 3 + a] = XIN ? sx[s] : CT(0);
          U[1][b * 3 + a] = XIN ? sx[SQY * SQX + s] : CT(0);
          if (CONV) { Wn[0][b * 3 + a] = sw[s]; Wn[1][b * 3 + a] = sw[SQY * SQX + s]; }
        }
      if (PIN) {
#pragma unroll
        for (int d = 0; d < 2; ++d)
#pragma unroll
          for (int c = 0; c < 2; ++c) P1[d * 2 + c] = sp1[(ly + d) * SPX + lx + c];
        if (HP0) P0v = sp0[ly * TEX + lx];
      }
      const CT ihx = CT(1) / P.hx, ihy = CT(1) / P.hy, area = P.hx * P.hy;
      q2_elem<CT, F>(U, Wn, P1, P0v, P.nu, ihx, ihy, area, P.sd, Y, YP1, YP0);
    } else {
#pragma unroll
      for (int k = 0; k < 9; ++k) { Y[0][k] = 0; Y[1][k] = 0; }
#pragma unroll
      for (int k = 0; k < 4; ++k) YP1[k] = 0;
    }
    if (UOUT) {
#pragma unroll
      for (int k = 0; k < 9; ++k) { eo[k * Q2T + tid] = Y[0][k]; eo[(9 + k) * Q2T + tid] = Y[1][k]; }
    }
    if (POUT) {
#pragma unroll
      for (int k = 0; k < 4; ++k) eo[(18 + k) * Q2T + tid] = YP1[k];
      eo[22 * Q2T + tid] = YP0;
    }
  }
  __syncthreads();

  double dacc = 0.0;
  // ---- phase 2a: owned velocity nodes gather their element contributions
  if (UOUT) {
    const int iend = (ex0 + OEX >= n) ? N : 2 * (ex0 + OEX);
    const int jend = (ey0 + OEY >= n) ? N : 2 * (ey0 + OEY);
    const int nli = iend - gi0 - 2, nlj = jend - gj0 - 2;
    for (int k = tid; k < nli * nlj; k += Q2T) {
      const int lj = 2 + k / nli, li = 2 + k % nli;
      int xl[2], xa[2], nx, yl[2], yb[2], ny;
      if (li & 1) { xl[0] = (li - 1) >> 1; xa[0] = 1; nx = 1; }
      else { const int m = li >> 1; xl[0] = m - 1; xa[0] = 2; nx = 1; if (m < TEX) { xl[1] = m; xa[1] = 0; nx = 2; } }
      if (lj & 1) { yl[0] = (lj - 1) >> 1; yb[0] = 1; ny = 1; }
      else { const int m = lj >> 1; yl[0] = m - 1; yb[0] = 2; ny = 1; if (m < TEY) { yl[1] = m; yb[1] = 0; ny = 2; } }
      CT s0 = 0, s1 = 0;
      for (int u = 0; u < ny; ++u)
        for (int v = 0; v < nx; ++v) {
          const int t = yl[u] * TEX + xl[v];
          const int kk = yb[u] * 3 + xa[v];
          s0 += eo[kk * Q2T + t];
          s1 += eo[(9 + kk) * Q2T + t];
        }
      const int i = gi0 + li, j = gj0 + lj;
      const size_t g = (size_t)j * N + i;
      const bool bnd = !NOBC && (i == 0 || j == 0 || i == N - 1 || j == N - 1);
      TO o0, o1;
      if (EPI == EPI_APPLY) {
        if (bnd) {
          if (XIN) { o0 = (TO)P.x[g]; o1 = (TO)P.x[g + nv]; } else { o0 = 0; o1 = 0; }
        } else { o0 = (TO)s0; o1 = (TO)s1; }
      } else if (EPI == EPI_SMOOTH) {
        if (bnd) { if (P.bsrc) { o0 = (TO)P.bsrc[g]; o1 = (TO)P.bsrc[g + nv]; } else { o0 = 0; o1 = 0; } }
        else {
          const int s = lj * SQX + li;
          const CT di = P.omega * P.dinv[g];
          o0 = (TO)(sx[s] + di * (P.b[g] - s0));
          o1 = (TO)(sx[SQY * SQX + s] + di * (P.b[g + nv] - s1));
        }
      } else if (EPI == EPI_RESID) {
        if (bnd) { o0 = 0; o1 = 0; } else { o0 = (TO)(P.b[g] - s0); o1 = (TO)(P.b[g + nv] - s1); }
      } else if (EPI == EPI_SCALE) {
        if (bnd) { o0 = 0; o1 = 0; } else { o0 = (TO)(P.dinv[g] * s0); o1 = (TO)(P.dinv[g] * s1); }
      } else {  // EPI_BSUB
        if (bnd) { o0 = P.bsrc[g]; o1 = P.bsrc[g + nv]; } else { o0 = P.bsrc[g] - (TO)s0; o1 = P.bsrc[g + nv] - (TO)s1; }
      }
      P.y[g] = o0;
      P.y[g + nv] = o1;
      if (DOT) dacc += (double)o0 * P.dv[g] + (double)o1 * P.dv[g + nv];
    }
  }
  // ---- phase 2b: owned pressure rows (B u)
  if (POUT) {
    const int Iend = (ex0 + OEX >= n) ? n + 1 : ex0 + OEX;
    const int Jend = (ey0 + OEY >= n) ? n + 1 : ey0 + OEY;
    const int nI = Iend - ex0, nJ = Jend - ey0;
    for (int k = tid; k < nI * nJ; k += Q2T) {
      const int LJ = 1 + k / nI, LI = 1 + k % nI;
      CT s = 0;
#pragma unroll
      for (int dd = 0; dd < 2; ++dd) {
        const int ly = LJ - 1 + dd, d = 1 - dd;     // element below (d=1), above (d=0)
        if (ly >= TEY) continue;
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const int lx = LI - 1 + cc, c = 1 - cc;
          if (lx >= TEX) continue;
          s += eo[(18 + d * 2 + c) * Q2T + ly * TEX + lx];
        }
      }
      const size_t gp = (size_t)(ey0 - 1 + LJ) * (n + 1) + (ex0 - 1 + LI);
      P.yp[gp] = (TO)s;
      if (DOT) dacc += (double)(TO)s * P.dvp[gp];
    }
    if (HP0) {
      const int nEx = min(OEX, n - ex0), nEy = min(OEY, n - ey0);
      for (int k = tid; k < nEx * nEy; k += Q2T) {
        const int ly = 1 + k / nEx, lx = 1 + k % nEx;
        const size_t ge = (size_t)n1 + (size_t)(ey0 - 1 + ly) * n + (ex0 - 1 + lx);
        const CT s = eo[22 * Q2T + ly * TEX + lx];
        P.yp[ge] = (TO)s;
        if (DOT) dacc += (double)(TO)s * P.dvp[ge];
      }
    }
  }
  if (DOT) {
    double v[1] = {dacc};
    const int idx = P.slot_off + blockIdx.y * gridDim.x + blockIdx.x;
    if (slot_arrive<1>(P.slot, idx, v)) finish_slot(P.slot, v[0]);
  }
}

inline size_t q2_smem_bytes(int F, size_t ct_size) {
  const bool conv = F & QF_CONV;
  size_t nct = 2 * SQY * SQX + (conv ? 2 * SQY * SQX : 0) + SPY * SPX + TEY * TEX + NEO * Q2T;
  return nct * ct_size;
}

inline dim3 q2_grid(int n) { return dim3(cdiv(n, OEX), cdiv(n, OEY)); }
inline int q2_blocks(int n) { return (int)(cdiv(n, OEX) * cdiv(n, OEY)); }

template <class TI, class TO, class CT, int F, int EPI>
cudaError_t launch_q2(const Q2Params<TI, TO, CT>& P, cudaStream_t s) {
  static bool attr_set = false;
  const size_t smem = q2_smem_bytes(F, sizeof(CT));
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_q2<TI, TO, CT, F, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_q2<TI, TO, CT, F, EPI><<<q2_grid(P.n), Q2T, smem, s>>>(P);
  return cudaGetLastError();
}

}  // namespace eth
