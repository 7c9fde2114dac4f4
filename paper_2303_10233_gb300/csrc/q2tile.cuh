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

#ifndef ETH_TEY
#define ETH_TEY 8
#endif
#ifndef ETH_OUT_HWCVT
#define ETH_OUT_HWCVT 1
#endif
constexpr int TEX = 32, TEY = ETH_TEY;           // computed elements per CTA
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
  QF_SRC_JB = 4096, // x field = omega * dinv * b (first Jacobi sweep from zero), b read from bx
  QF_SRC_XPC = 8192,// x field = x + P xc (coarse-grid correction prolongated on the fly)
  QF_SRC_RJB = 16384,// with QF_SRC_JB: b = P^T r_f, the finer level's residual bx restricted on the fly
};
enum : int { EPI_APPLY = 0, EPI_SMOOTH = 1, EPI_RESID = 2, EPI_SCALE = 3, EPI_BSUB = 4, EPI_JR = 5 };
// EPI_JR (with QF_SRC_JB): y = b - F x and y2 = x = omega D^{-1} b; bcopy = b (optional).
// With QF_SRC_RJB, b is the restriction of the finer level's residual (bx, lattice
// 4n+1), gathered per staged node with the weights and in the order of the
// stand-alone restriction kernel, and bcopy receives it (required).
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
  const TI* bx;       // QF_SRC_JB: level right-hand side (masked on the boundary)
  CT* y2;             // EPI_JR: the iterate x
  CT* bcopy;          // EPI_JR: copy of b (CT), may be null
  const CT* xc;       // QF_SRC_XPC: coarse-level iterate (level n/2)
};

// Closed-form element integrals on the unit interval (shape functions as in
// common.cuh).  Quadratic stiffness / mass: k1d = (1/3)[7 -8 1; -8 16 -8; 1 -8 7],
// m1d = (1/30)[4 2 -1; 2 16 2; -1 2 4].  Linear-quadratic couplings:
// c12[c][a] = int N_c L_a', g12[d][b] = int N_d L_b, c0[a] = L_a(1) - L_a(0),
// g0[b] = int L_b.  On a rectangle hx x hy (local index b*3 + a):
//   A_e = (hy/hx) k1d (x) m1d + (hx/hy) m1d (x) k1d
//   B1x_e[(c,d),(a,b)] = -hy c12[c][a] g12[d][b],  B1y_e = -hx g12[c][a] c12[d][b]
//   B0x_e[(a,b)] = -hy c0[a] g0[b],                B0y_e = -hx g0[a] c0[b]
__host__ __device__ constexpr double k1d(int a, int b) {
  return a == b ? (a == 1 ? 16.0 / 3.0 : 7.0 / 3.0) : ((a == 1 || b == 1) ? -8.0 / 3.0 : 1.0 / 3.0);
}
__host__ __device__ constexpr double m1d(int a, int b) {
  return a == b ? (a == 1 ? 16.0 / 30.0 : 4.0 / 30.0) : ((a == 1 || b == 1) ? 2.0 / 30.0 : -1.0 / 30.0);
}
__host__ __device__ constexpr double c12(int c, int a) {
  return c == 0 ? (a == 0 ? -5.0 / 6.0 : (a == 1 ? 2.0 / 3.0 : 1.0 / 6.0)) : (a == 0 ? -1.0 / 6.0 : (a == 1 ? -2.0 / 3.0 : 5.0 / 6.0));
}
__host__ __device__ constexpr double g12(int d, int b) {
  return d == 0 ? (b == 0 ? 1.0 / 6.0 : (b == 1 ? 1.0 / 3.0 : 0.0)) : (b == 0 ? 0.0 : (b == 1 ? 1.0 / 3.0 : 1.0 / 6.0));
}
__host__ __device__ constexpr double c0v(int a) { return a == 0 ? -1.0 : (a == 1 ? 0.0 : 1.0); }
__host__ __device__ constexpr double g0v(int b) { return b == 1 ? 4.0 / 6.0 : 1.0 / 6.0; }

// FP64 -> FP32 of a staged input (warp-collective; masked lanes give 0).
template <class CT, class TI>
__device__ __forceinline__ CT cvt_stage(TI v, bool valid) {
  if constexpr (sizeof(TI) == 8 && sizeof(CT) == 4) {
#if ETH_IN_FASTCVT
    return f64_to_f32_warp(v, valid);
#else
    return valid ? f64_to_f32_bits(v) : 0.0f;
#endif
  } else {
    return valid ? (CT)v : CT(0);
  }
}

// FP32 -> FP64 of kernel outputs: the conversion instruction (FP64 pipe, idle in
// FP32 element kernels) or the integer bit path (ALU pipe).  The operator apply
// converts its first velocity component one way and the second the other,
// which balances the two pipes.
template <class TO, class CT>
__device__ __forceinline__ TO cvt_out(CT v) {
#if ETH_OUT_HWCVT
  return (TO)v;
#else
  return cvt<TO, CT>(v);
#endif
}

// 1D Q2 restriction weight of the fine node at offset o in [-3, 3] from 2I (coarse
// node I odd: an element midpoint; even: an element vertex).
__device__ __forceinline__ float rjb_w(int odd, int o) {
  if (o == 0) return 1.f;
  if (odd) return (o == -1 || o == 1) ? 0.75f : 0.f;
  return (o == -1 || o == 1) ? 0.375f : ((o == -3 || o == 3) ? -0.125f : 0.f);
}

// b at coarse node (i, j) (interior) = P^T r_f: fine lattice Nf = 2N - 1.
template <class CT, class TI>
__device__ __forceinline__ void rjb_gather(const TI* __restrict__ rf, int N, int i, int j, CT& b0, CT& b1) {
  const int Nf = 2 * N - 1;
  const int nvf = Nf * Nf;
  const int ox = i & 1, oy = j & 1;
  CT s0 = 0, s1 = 0;
#pragma unroll
  for (int u = -3; u <= 3; ++u) {
    const float wyv = rjb_w(oy, u);
    if (wyv == 0.f) continue;
    const int row = (2 * j + u) * Nf;
    CT t0 = 0, t1 = 0;
#pragma unroll
    for (int v = -3; v <= 3; ++v) {
      const float wxv = rjb_w(ox, v);
      if (wxv == 0.f) continue;
      const int f = row + 2 * i + v;
      t0 += (CT)wxv * (CT)rf[f];
      t1 += (CT)wxv * (CT)rf[f + nvf];
    }
    s0 += (CT)wyv * t0;
    s1 += (CT)wyv * t1;
  }
  b0 = s0;
  b1 = s1;
}

template <class CT, int F>
__device__ __forceinline__ void q2_elem(const CT (&U)[2][9], const CT (&Wn)[2][9], const CT (&P1)[4], CT P0,
                                        CT nu, CT ihx, CT ihy, CT area, CT sdc, CT (&Y)[2][9], CT (&YP1)[4], CT& YP0) {
  constexpr bool CONV = F & QF_CONV, TRANS = F & QF_TRANS, PIN = F & QF_PIN, HP0 = F & QF_P0,
                 DIFF = F & QF_DIFF, POUT = F & QF_POUT, MASS = F & QF_MASS, SD = F & QF_SD, UOUT = F & QF_UOUT;
  // ---- constant-coefficient parts with the closed-form element matrices (immediates)
  const CT hx = area * ihy, hy = area * ihx;
  if (UOUT) {
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int i = 0; i < 9; ++i) Y[c][i] = 0;
  }
  if (UOUT && DIFF) {
    const CT skm = nu * hy * ihx, smk = nu * hx * ihy;   // nu hy/hx, nu hx/hy
    if (skm == smk) {
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          CT acc = 0;
#pragma unroll
          for (int j = 0; j < 9; ++j)
            acc += (CT)(k1d(i % 3, j % 3) * m1d(i / 3, j / 3) + m1d(i % 3, j % 3) * k1d(i / 3, j / 3)) * U[c][j];
          Y[c][i] = skm * acc;
        }
    } else {
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          CT a1 = 0, a2 = 0;
#pragma unroll
          for (int j = 0; j < 9; ++j) {
            a1 += (CT)(k1d(i % 3, j % 3) * m1d(i / 3, j / 3)) * U[c][j];
            a2 += (CT)(m1d(i % 3, j % 3) * k1d(i / 3, j / 3)) * U[c][j];
          }
          Y[c][i] = skm * a1 + smk * a2;
        }
    }
  }
  if (UOUT && PIN) {   // B^T p: y_x -= hy (c12 (x) g12)^T p1 + hy c0 g0 p0, y_y with the roles swapped
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int a = i % 3, b = i / 3;
      CT sx_ = 0, sy_ = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int cc = k & 1, dd = k >> 1;
        sx_ += (CT)(c12(cc, a) * g12(dd, b)) * P1[k];
        sy_ += (CT)(g12(cc, a) * c12(dd, b)) * P1[k];
      }
      if (HP0) { sx_ += (CT)(c0v(a) * g0v(b)) * P0; sy_ += (CT)(g0v(a) * c0v(b)) * P0; }
      Y[0][i] -= hy * sx_;
      Y[1][i] -= hx * sy_;
    }
  }
  if (POUT) {          // B u: yp1 = -hy (c12 (x) g12) u_x - hx (g12 (x) c12) u_y ; yp0 likewise
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int cc = k & 1, dd = k >> 1;
      CT ax = 0, ay = 0;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const int a = i % 3, b = i / 3;
        ax += (CT)(c12(cc, a) * g12(dd, b)) * U[0][i];
        ay += (CT)(g12(cc, a) * c12(dd, b)) * U[1][i];
      }
      YP1[k] = -(hy * ax + hx * ay);
    }
    CT ax = 0, ay = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int a = i % 3, b = i / 3;
      if (c0v(a) * g0v(b) != 0.0) ax += (CT)(c0v(a) * g0v(b)) * U[0][i];
      if (g0v(a) * c0v(b) != 0.0) ay += (CT)(g0v(a) * c0v(b)) * U[1][i];
    }
    YP0 = -(hy * ax + hx * ay);
  }
  // ---- wind-dependent / mass terms by sum factorisation at the 3x3 Gauss points
  constexpr bool SUMF = UOUT && (CONV || MASS || SD);
  if (!SUMF) return;
  constexpr bool NEEDVAL = (CONV && TRANS) || MASS;
  constexpr bool NEEDGRAD = (CONV && !TRANS) || SD;
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
  if (CONV || SD) {
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
        if ((CONV && !TRANS) || SD) {
          const CT wgu = WQ[0][q] * DX[c][q] + WQ[1][q] * DY[c][q];
          if (CONV && !TRANS) cv = wgu;
          if (SD) { gx += delta * WQ[0][q] * wgu; gy += delta * WQ[1][q] * wgu; }
        }
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
        Y[c][b * 3 + a] += LD(0, a) * H1[0][b] + LD(1, a) * H1[1][b] + LD(2, a) * H1[2][b] +
                           LV(0, a) * H2[0][b] + LV(1, a) * H2[1][b] + LV(2, a) * H2[2][b];
  }
}

// Resident CTAs per SM the register allocation must allow.  The FP32 operator
// apply (32 x 8) is held to 5 CTAs without convection and 4 with it; the FP32
// Stokes smoothing sweep with FP64 output and the fused dot (the V-cycle exit) to
// 3: unbounded it takes 96 registers, 2 CTAs per SM, and the 333 tiles of a 256^2
// level need a second wave on 152 SMs.
template <class CT, int F, int EPI, int TY>
__host__ __device__ constexpr int q2_min_blocks() {
  return (TY == 8 && sizeof(CT) == 4 && EPI == EPI_APPLY) ? ((F & QF_CONV) ? 4 : 5)
       : (TY == 8 && sizeof(CT) == 4 && EPI == EPI_SMOOTH && !(F & QF_CONV)) ? 3 : 1;
}

// TY = element rows per CTA (tile 32 x TY computed, 31 x (TY-1) owned); the
// constants below shadow the default-shape ones of the namespace.
// The FP32 operator apply (32 x 8) is held to 5 resident CTAs per SM without
// convection (<= 51 registers, no spills) and to 4 with it (<= 64 registers,
// a few spills): the extra warps hide the staging loads (measured: Stokes
// 1024^2 57.9 -> 52.7 us; Oseen 1024^2 160 us at the 166 registers the
// compiler takes unbounded -> 82 us).
template <class TI, class TO, class CT, int F, int EPI, int TY = ETH_TEY>
__global__ void __launch_bounds__(TEX * TY, q2_min_blocks<CT, F, EPI, TY>())
    k_q2(Q2Params<TI, TO, CT> P) {
  ETH_GRID_DEP_WAIT();
  constexpr int TEY = TY, OEY = TY - 1, Q2T = TEX * TY, SQY = 2 * TY + 1, SPY = TY + 1;
  constexpr bool CONV = F & QF_CONV, XIN = F & QF_XIN, PIN = F & QF_PIN, HP0 = F & QF_P0,
                 UOUT = F & QF_UOUT, POUT = F & QF_POUT, DOT = F & QF_DOT, NOBC = F & QF_NOBC,
                 JB = F & QF_SRC_JB, XPC = F & QF_SRC_XPC, RJB = (F & QF_SRC_RJB) && (F & QF_SRC_JB);
  if (P.done != nullptr && *P.done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CT* sx = reinterpret_cast<CT*>(smem_raw);                 // [2][SQY][SQX]
  CT* sw = sx + 2 * SQY * SQX;                              // [2][SQY][SQX] (CONV)
  CT* sp1 = sw + (CONV ? 2 * SQY * SQX : 0);                // [SPY][SPX]
  CT* sp0 = sp1 + SPY * SPX;                                // [TEY][TEX]
  CT* eo = sp0 + TEY * TEX;                                 // [NEO][Q2T]
  CT* sb = eo + NEO * Q2T;                                  // [2][SQY][SQX] (RJB: the restricted b)

  const int n = P.n, N = 2 * n + 1;
  const int nv = N * N;   // 32-bit offsets: 2 N_v + N_1 + N_0 < 2^31 for n <= 8192
  const int n1 = (n + 1) * (n + 1);
  const int ex0 = blockIdx.x * OEX, ey0 = blockIdx.y * OEY;
  const int gi0 = 2 * (ex0 - 1), gj0 = 2 * (ey0 - 1);
  const int tid = threadIdx.x;

  // ---- phase 0: stage inputs (masked velocity, wind, pressure) in shared memory.
  // All global loads of a thread are issued before any is used (memory-level parallelism).
  if (XIN || CONV) {
    constexpr int NLD = (SQY * SQX + Q2T - 1) / Q2T;
    TI v0[NLD], v1[NLD];
    CT w0[NLD], w1[NLD];
    bool ok[NLD];
#pragma unroll
    for (int r = 0; r < NLD; ++r) {
      const int k = tid + r * Q2T;
      const int lj = k / SQX, li = k - lj * SQX;
      const int i = gi0 + li, j = gj0 + lj;
      v0[r] = 0; v1[r] = 0; w0[r] = 0; w1[r] = 0; ok[r] = false;
      if (k < SQY * SQX && i >= 0 && i < N && j >= 0 && j < N) {
        const int g = j * N + i;
        const bool bnd = !NOBC && (i == 0 || j == 0 || i == N - 1 || j == N - 1);
        if (XIN && !bnd) {
          ok[r] = true;
          if (RJB) { w0[r] = P.dinv[g]; }
          else if (JB) { v0[r] = P.bx[g]; v1[r] = P.bx[g + nv]; w0[r] = P.dinv[g]; }
          else { v0[r] = P.x[g]; v1[r] = P.x[g + nv]; }
        }
        if (CONV) { if (JB) w1[r] = P.w[g]; else { w0[r] = P.w[g]; w1[r] = P.w[g + nv]; } }
      }
    }
    if (RJB) {   // b = P^T r_f at the staged interior nodes, kept in sb for the epilogue
#pragma unroll 1
      for (int r = 0; r < NLD; ++r) {
        const int k = tid + r * Q2T;
        CT b0 = 0, b1 = 0;
        if (ok[r]) {
          const int lj = k / SQX, li = k - lj * SQX;
          rjb_gather<CT, TI>(P.bx, N, gi0 + li, gj0 + lj, b0, b1);
        }
        if (k < SQY * SQX) { sb[k] = b0; sb[SQY * SQX + k] = b1; }
        v0[r] = (TI)b0; v1[r] = (TI)b1;
      }
    }
#pragma unroll
    for (int r = 0; r < NLD; ++r) {
      const int k = tid + r * Q2T;
      // every lane converts (warp-collective); masked lanes give 0
      const CT c0 = XIN ? cvt_stage<CT, TI>(v0[r], ok[r]) : CT(0);
      const CT c1 = XIN ? cvt_stage<CT, TI>(v1[r], ok[r]) : CT(0);
      if (k < SQY * SQX) {
        if (JB) {
          const CT om = P.omega * w0[r];
          sx[k] = om * c0; sx[SQY * SQX + k] = om * c1;
        } else if (XIN) { sx[k] = c0; sx[SQY * SQX + k] = c1; }
        if (CONV && !JB) { sw[k] = w0[r]; sw[SQY * SQX + k] = w1[r]; }
      }
    }
    if (CONV && JB) {   // the wind's second component was not staged above
      for (int k = tid; k < SQY * SQX; k += Q2T) {
        const int lj = k / SQX, li = k - lj * SQX;
        const int i = gi0 + li, j = gj0 + lj;
        CT a = 0, b = 0;
        if (i >= 0 && i < N && j >= 0 && j < N) { const int g = j * N + i; a = P.w[g]; b = P.w[g + nv]; }
        sw[k] = a; sw[SQY * SQX + k] = b;
      }
    }
    if (XPC) {
      // coarse lattice (level n/2 has 2*(n/2)+1 = n+1 nodes per direction) covering the fine tile
      const int Nc = n + 1;
      const int nvc = Nc * Nc;
      const int cI0 = 2 * (gi0 >= 0 ? gi0 / 4 : -1), cJ0 = 2 * (gj0 >= 0 ? gj0 / 4 : -1);
      constexpr int CXW = (SQX + 3) / 2 + 4, CYW = (SQY + 3) / 2 + 4;
      CT* sc = eo;   // scratch: eo is unused until phase 1
      __syncthreads();
      for (int k = tid; k < CYW * CXW; k += Q2T) {
        const int lj = k / CXW, li = k - lj * CXW;
        const int I = cI0 + li, J = cJ0 + lj;
        CT a = 0, b = 0;
        if (I >= 0 && I < Nc && J >= 0 && J < Nc) { const int c = J * Nc + I; a = P.xc[c]; b = P.xc[c + nvc]; }
        sc[k] = a; sc[CYW * CXW + k] = b;
      }
      __syncthreads();
      for (int k = tid; k < SQY * SQX; k += Q2T) {
        const int lj = k / SQX, li = k - lj * SQX;
        const int i = gi0 + li, j = gj0 + lj;
        if (i <= 0 || j <= 0 || i >= N - 1 || j >= N - 1) continue;   // boundary / outside: no correction
        CT wx[3], wy[3];
        int cx, cy;
        if (!(i & 1)) { cx = i >> 1; wx[0] = 1; wx[1] = 0; wx[2] = 0; }
        else {
          cx = 2 * (i >> 2);
          if ((i & 3) == 1) { wx[0] = CT(0.375); wx[1] = CT(0.75); wx[2] = CT(-0.125); }
          else { wx[0] = CT(-0.125); wx[1] = CT(0.75); wx[2] = CT(0.375); }
        }
        if (!(j & 1)) { cy = j >> 1; wy[0] = 1; wy[1] = 0; wy[2] = 0; }
        else {
          cy = 2 * (j >> 2);
          if ((j & 3) == 1) { wy[0] = CT(0.375); wy[1] = CT(0.75); wy[2] = CT(-0.125); }
          else { wy[0] = CT(-0.125); wy[1] = CT(0.75); wy[2] = CT(0.375); }
        }
        CT a = 0, b = 0;
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
          for (int v = 0; v < 3; ++v) {
            if (wx[v] == CT(0) || wy[u] == CT(0)) continue;
            const int c = (cy + u - cJ0) * CXW + (cx + v - cI0);
            a += wx[v] * wy[u] * sc[c];
            b += wx[v] * wy[u] * sc[CYW * CXW + c];
          }
        sx[k] += a;
        sx[SQY * SQX + k] += b;
      }
    }
  }
  if (PIN) {
    constexpr int NLP = (SPY * SPX + Q2T - 1) / Q2T;
    TI pv[NLP], p0v = 0;
#pragma unroll
    for (int r = 0; r < NLP; ++r) {
      const int k = tid + r * Q2T;
      const int lj = k / SPX, li = k - lj * SPX;
      const int I = ex0 - 1 + li, J = ey0 - 1 + lj;
      pv[r] = (k < SPY * SPX && I >= 0 && I <= n && J >= 0 && J <= n) ? P.p[J * (n + 1) + I] : TI(0);
    }
    if (HP0) {
      const int ly = tid / TEX, lx = tid - ly * TEX;
      const int ex = ex0 - 1 + lx, ey = ey0 - 1 + ly;
      if (ex >= 0 && ex < n && ey >= 0 && ey < n) p0v = P.p[n1 + ey * n + ex];
      sp0[tid] = cvt<CT, TI>(p0v);
    }
#pragma unroll
    for (int r = 0; r < NLP; ++r) {
      const int k = tid + r * Q2T;
      if (k < SPY * SPX) sp1[k] = cvt<CT, TI>(pv[r]);
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
  // ---- phase 2: every owned element (tile-local lx, ly >= 1) gathers the four nodes it
  // owns (its lower-left vertex, the two adjacent edge midpoints, its centre) plus, on the
  // last element row / column of the domain, the nodes of the top / right boundary line.
  {
    const int lx = tid % TEX, ly = tid / TEX;
    const int ex = ex0 - 1 + lx, ey = ey0 - 1 + ly;
    const bool own = lx >= 1 && ly >= 1 && ex < n && ey < n;
    const int tL = tid - 1, tB = tid - TEX, tLB = tid - TEX - 1;
    auto E = [&](int a, int b, int t, int c) -> CT { return eo[(c * 9 + b * 3 + a) * Q2T + t]; };
    auto emit = [&](int i, int j, CT s0, CT s1) {
      const int g = j * N + i;
      const bool bnd = !NOBC && (i == 0 || j == 0 || i == N - 1 || j == N - 1);
      const int li = i - gi0, lj = j - gj0;
      TO o0, o1;
      if (EPI == EPI_APPLY) {
        if (bnd) {
          if (XIN) { o0 = (TO)P.x[g]; o1 = (TO)P.x[g + nv]; } else { o0 = 0; o1 = 0; }
        } else { o0 = cvt_out<TO, CT>(s0); o1 = cvt<TO, CT>(s1); }   // FP64 pipe / ALU pipe
      } else if (EPI == EPI_SMOOTH) {
        if (bnd) { if (P.bsrc) { o0 = (TO)P.bsrc[g]; o1 = (TO)P.bsrc[g + nv]; } else { o0 = 0; o1 = 0; } }
        else {
          const int sI = lj * SQX + li;
          const CT di = P.omega * P.dinv[g];
          o0 = cvt_out<TO, CT>(sx[sI] + di * (P.b[g] - s0));
          o1 = cvt_out<TO, CT>(sx[SQY * SQX + sI] + di * (P.b[g + nv] - s1));
        }
      } else if (EPI == EPI_RESID) {
        if (bnd) { o0 = 0; o1 = 0; } else { o0 = (TO)(P.b[g] - s0); o1 = (TO)(P.b[g + nv] - s1); }
      } else if (EPI == EPI_SCALE) {
        if (bnd) { o0 = 0; o1 = 0; } else { o0 = (TO)(P.dinv[g] * s0); o1 = (TO)(P.dinv[g] * s1); }
      } else if (EPI == EPI_BSUB) {
        if (bnd) { o0 = P.bsrc[g]; o1 = P.bsrc[g + nv]; } else { o0 = P.bsrc[g] - (TO)s0; o1 = P.bsrc[g + nv] - (TO)s1; }
      } else {  // EPI_JR
        const int sI = lj * SQX + li;
        if (bnd) {
          o0 = 0; o1 = 0;
          P.y2[g] = 0; P.y2[g + nv] = 0;
          if (P.bcopy) { P.bcopy[g] = 0; P.bcopy[g + nv] = 0; }
        } else {
          const CT b0 = RJB ? sb[sI] : cvt<CT, TI>(P.bx[g]), b1 = RJB ? sb[SQY * SQX + sI] : cvt<CT, TI>(P.bx[g + nv]);
          o0 = (TO)(b0 - s0); o1 = (TO)(b1 - s1);
          P.y2[g] = sx[sI]; P.y2[g + nv] = sx[SQY * SQX + sI];
          if (P.bcopy) { P.bcopy[g] = b0; P.bcopy[g + nv] = b1; }
        }
      }
      P.y[g] = o0;
      P.y[g + nv] = o1;
      if (DOT) dacc += (double)o0 * (double)P.dv[g] + (double)o1 * (double)P.dv[g + nv];
    };
    if (UOUT && own) {
      const int i0 = 2 * ex, j0 = 2 * ey;
      const bool lastx = ex == n - 1, lasty = ey == n - 1;
      // vertex (2ex, 2ey)
      emit(i0, j0, E(2, 2, tLB, 0) + E(0, 2, tB, 0) + E(2, 0, tL, 0) + E(0, 0, tid, 0),
                   E(2, 2, tLB, 1) + E(0, 2, tB, 1) + E(2, 0, tL, 1) + E(0, 0, tid, 1));
      emit(i0 + 1, j0, E(1, 2, tB, 0) + E(1, 0, tid, 0), E(1, 2, tB, 1) + E(1, 0, tid, 1));
      emit(i0, j0 + 1, E(2, 1, tL, 0) + E(0, 1, tid, 0), E(2, 1, tL, 1) + E(0, 1, tid, 1));
      emit(i0 + 1, j0 + 1, E(1, 1, tid, 0), E(1, 1, tid, 1));
      if (lastx) {
        emit(i0 + 2, j0, E(2, 2, tB, 0) + E(2, 0, tid, 0), E(2, 2, tB, 1) + E(2, 0, tid, 1));
        emit(i0 + 2, j0 + 1, E(2, 1, tid, 0), E(2, 1, tid, 1));
      }
      if (lasty) {
        emit(i0, j0 + 2, E(2, 2, tL, 0) + E(0, 2, tid, 0), E(2, 2, tL, 1) + E(0, 2, tid, 1));
        emit(i0 + 1, j0 + 2, E(1, 2, tid, 0), E(1, 2, tid, 1));
      }
      if (lastx && lasty) emit(i0 + 2, j0 + 2, E(2, 2, tid, 0), E(2, 2, tid, 1));
    }
    if (POUT && own) {
      auto Q = [&](int cc, int dd, int t) -> CT { return eo[(18 + dd * 2 + cc) * Q2T + t]; };
      auto pemit = [&](int I, int J, CT v) {
        const int gp = J * (n + 1) + I;
        const TO so = cvt_out<TO, CT>(v);
        P.yp[gp] = so;
        if (DOT) dacc += (double)so * (double)P.dvp[gp];
      };
      pemit(ex, ey, Q(1, 1, tLB) + Q(0, 1, tB) + Q(1, 0, tL) + Q(0, 0, tid));
      if (ex == n - 1) pemit(ex + 1, ey, Q(1, 1, tB) + Q(1, 0, tid));
      if (ey == n - 1) pemit(ex, ey + 1, Q(1, 1, tL) + Q(0, 1, tid));
      if (ex == n - 1 && ey == n - 1) pemit(ex + 1, ey + 1, Q(1, 1, tid));
      if (HP0) {
        const int ge = n1 + ey * n + ex;
        const TO so = cvt_out<TO, CT>(eo[22 * Q2T + tid]);
        P.yp[ge] = so;
        if (DOT) dacc += (double)so * (double)P.dvp[ge];
      }
    }
  }
  if (DOT) {
    double v[1] = {dacc};
    const int idx = P.slot_off + blockIdx.y * gridDim.x + blockIdx.x;
    if (slot_arrive<1>(P.slot, idx, v)) finish_slot(P.slot, v[0]);
  }
}

inline size_t q2_smem_bytes(int F, size_t ct_size, int ty = ETH_TEY) {
  const bool conv = F & QF_CONV;
  const size_t sqy = 2 * ty + 1, spy = ty + 1, q2t = (size_t)TEX * ty;
  size_t nct = 2 * sqy * SQX + (conv ? 2 * sqy * SQX : 0) + spy * SPX + q2t + NEO * q2t;
  if ((F & QF_SRC_RJB) && (F & QF_SRC_JB)) nct += 2 * sqy * SQX;
  return nct * ct_size;
}

inline dim3 q2_grid(int n, int ty = ETH_TEY) { return dim3(cdiv(n, OEX), cdiv(n, ty - 1)); }
inline int q2_blocks(int n, int ty = ETH_TEY) { return (int)(cdiv(n, OEX) * cdiv(n, ty - 1)); }

// Kernel stubs have internal linkage in every translation unit (each unit launches
// its own copy of a kernel), so the launcher and its record of the shared-memory
// attribute are per translation unit too (static).
template <class TI, class TO, class CT, int F, int EPI, int TY = ETH_TEY>
static cudaError_t launch_q2(const Q2Params<TI, TO, CT>& P, cudaStream_t s) {
  static SmemAttr attr;
  const size_t smem = q2_smem_bytes(F, sizeof(CT), TY);
  cudaError_t e = smem_attr(k_q2<TI, TO, CT, F, EPI, TY>, smem, attr);
  if (e != cudaSuccess) return e;
  k_q2<TI, TO, CT, F, EPI, TY><<<q2_grid(P.n, TY), TEX * TY, smem, s>>>(P);
  return cudaGetLastError();
}

// Tile heights a grid may select (the autotuned K apply); others use ETH_TEY.
constexpr int Q2_TILE_ROWS[3] = {4, 8, 16};
inline bool q2_tile_ok(int ty) { return ty == 4 || ty == 8 || ty == 16; }

template <class TI, class TO, class CT, int F, int EPI>
static cudaError_t launch_q2_ty(const Q2Params<TI, TO, CT>& P, cudaStream_t s, int ty) {
  switch (ty) {
    case 4: return launch_q2<TI, TO, CT, F, EPI, 4>(P, s);
    case 16: return launch_q2<TI, TO, CT, F, EPI, 16>(P, s);
    default: return launch_q2<TI, TO, CT, F, EPI, 8>(P, s);
  }
}

}  // namespace eth
