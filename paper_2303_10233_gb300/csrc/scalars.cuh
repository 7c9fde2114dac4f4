// Device-resident scalar state of the Krylov recurrences and the one-thread
// "finishers" that the last block of a grid-wide reduction runs.  Keeping the
// scalars on the device lets a whole iteration run without a host round trip
// (and be captured in a CUDA graph); the host polls `done` between chunks.
#pragma once
#include <cuda_runtime.h>

namespace eth {

struct Scalars {
  double v[96];          // solver scalars, indices S_* below
  double dots[16];       // plain finished reductions (FIN_STORE)
  int done;              // early-exit flag checked by every kernel of a chunk
  int status;            // eth_status raised on the device
  int iter;              // device iteration counter
  int inner_done;        // unused
  int idone[4];          // early-exit flags of inner (nested) PCG solves
  int loops, max_loops;  // bodies run by the device-side MINRES loop and their cap
  // Lanczos coefficients of the first MINRES run of a Stokes solve (EST-MINRES,
  // Sec. 2.4): lz_delta[j-1] = delta_j, lz_gamma[j-1] = gamma_{j+1}, j = 1 .. lz_n.
  double* lz_delta;
  double* lz_gamma;
  int lz_cap, lz_runs, lz_n;
};

// Inner PCG state blocks (exact preconditioner blocks): base index of each.
enum : int { PCG_VEL = 48, PCG_PRE = 64 };
enum : int { P_RZ = 0, P_ALPHA, P_BETA, P_TARGET, P_ITS, P_TOL };

// MINRES (Algorithm 1) state: gamma_{j-1}, gamma_j, c_{j-1}, c_j, s_{j-1}, s_j,
// eta, |eta_1|, delta_j and the coefficients of the fused vector updates.
enum : int {
  S_GPREV = 0, S_G, S_CPREV, S_C, S_SPREV, S_S, S_ETA, S_ETA1, S_DELTA, S_TOL,
  S_VA, S_VB, S_VC,            // v_{j+1} = VA*K z_j - VB*v_j - VC*v_{j-1}
  S_WZ, S_WO, S_WW, S_XC,      // w_{j+1} = WZ*z_j - WO*w_{j-1} - WW*w_j ; x += XC*w_{j+1}
  S_PEND,                      // convergence / breakdown seen (applied at iteration end)
  S_BETA,                      // k-projection coefficient k^T v / k^T k
  S_NP1, S_NP0,                // n_k and n_0
  S_MQC,                       // scale of the approximate Schur solve
  S_MQG,                       // constant gamma1 of the M_Q output (k^T z = 0)
  S_MQNU,                      // pressure block factor (nu)
  S_ITS,                       // iterations done (as double)
  S_INNER_TOL, S_RZ, S_RZ0, S_ALPHA, S_BETACG,   // inner PCG
  S_WXP,                       // 1 while the w/x update of the last Givens step is pending
  S_LAST
};

enum : int {
  FIN_STORE = 0,      // dots[...] = sums
  FIN_MINRES_INIT,    // gamma_1 from <z1, v1>
  FIN_MINRES_DELTA,   // delta_j from <K z_j, z_j>
  FIN_MINRES_GAMMA,   // gamma_{j+1}, Givens rotation, eta, convergence
  FIN_VSUMS,          // beta = (sum v_p1 - sum v_p0) / (n1 + n0)
  FIN_MQ,             // gamma1 of the M_Q output from (sum z~, sum adj*z~, sum v0)
  FIN_DONE,           // done = pending
  FIN_PCG_INIT,       // inner PCG: s = (<r, z>, <r, r>) -> rz, target = tol^2 <r, r>
  FIN_PCG_ALPHA,      // alpha = rz / <p, A p>
  FIN_PCG_RZ,         // beta = rz_new / rz; rz = rz_new
  FIN_PCG_RR,         // <r, r> <= target -> inner done
  FIN_V,              // beta from the v sums (the w/x update runs in its own kernel, k_minres_wx)
};

__device__ __forceinline__ void finish_minres_gamma(Scalars* sc, double g2) {
  double* v = sc->v;
  if (!(g2 > 0.0)) {             // breakdown: indefinite preconditioner or exhausted space
    if (g2 == 0.0) { v[S_PEND] = 1.0; }
    else { v[S_PEND] = 1.0; sc->status = 5; }
    g2 = 0.0;
  }
  const double gnew = sqrt(g2);
  if (sc->lz_runs == 1 && sc->lz_n < sc->lz_cap) {
    sc->lz_delta[sc->lz_n] = v[S_DELTA];
    sc->lz_gamma[sc->lz_n] = gnew;
    sc->lz_n += 1;
  }
  const double gj = v[S_G], delta = v[S_DELTA];
  const double a0 = v[S_C] * delta - v[S_CPREV] * v[S_S] * gj;
  const double a1 = sqrt(a0 * a0 + gnew * gnew);
  const double a2 = v[S_S] * delta + v[S_CPREV] * v[S_C] * gj;
  const double a3 = v[S_SPREV] * gj;
  const double cn = a0 / a1, sn = gnew / a1;
  v[S_WZ] = 1.0 / (gj * a1);
  v[S_WO] = a3 / a1;
  v[S_WW] = a2 / a1;
  v[S_XC] = cn * v[S_ETA];
  v[S_ETA] = -sn * v[S_ETA];
  v[S_GPREV] = gj; v[S_G] = gnew;
  v[S_CPREV] = v[S_C]; v[S_C] = cn;
  v[S_SPREV] = v[S_S]; v[S_S] = sn;
  v[S_ITS] += 1.0;
  v[S_WXP] = 1.0;
  if (fabs(v[S_ETA]) < v[S_TOL] * v[S_ETA1]) v[S_PEND] = 1.0;
  if (!isfinite(v[S_ETA])) { v[S_PEND] = 1.0; sc->status = 8; }
}

// Runs on one thread of the last block of a reduction; s[] holds the sums.
template <int NV_>
__device__ __forceinline__ void finish_slot_n(const Slot& sl, const double (&s)[NV_]) {
  Scalars* sc = sl.sc;
  double* v = sc ? sc->v : nullptr;
  switch (sl.op) {
    case FIN_STORE:
      for (int k = 0; k < NV_; ++k) sl.out[k] = s[k];
      break;
    case FIN_MINRES_INIT: {
      double g2 = s[0];
      if (!(g2 > 0.0)) { sc->status = g2 == 0.0 ? 0 : 5; v[S_PEND] = 1.0; g2 = 0.0; }
      const double g = sqrt(g2);
      v[S_G] = g; v[S_GPREV] = 0.0; v[S_ETA] = g; v[S_ETA1] = g;
      v[S_C] = v[S_CPREV] = 1.0; v[S_S] = v[S_SPREV] = 0.0; v[S_ITS] = 0.0;
      if (g == 0.0) v[S_PEND] = 1.0;
      sl.out[0] = s[0];
      break;
    }
    case FIN_MINRES_DELTA: {
      const double g = v[S_G];
      v[S_DELTA] = s[0] / (g * g);
      v[S_VA] = 1.0 / g;
      v[S_VB] = v[S_DELTA] / g;
      v[S_VC] = v[S_GPREV] > 0.0 ? g / v[S_GPREV] : 0.0;
      break;
    }
    case FIN_MINRES_GAMMA:
      finish_minres_gamma(sc, s[0]);
      break;
    case FIN_VSUMS:
      v[S_BETA] = (s[0] - s[1]) / (v[S_NP1] + v[S_NP0]);
      break;
    case FIN_V:
      v[S_BETA] = (s[0] - s[1]) / (v[S_NP1] + v[S_NP0]);
      sc->iter += 1;
      break;
    case FIN_MQ: {
      // z_k = c z~ + g1, z_0 = (v0+beta)/|T| - (c/4) sum_T z~ - g1 ; choose g1 so k^T z = 0
      // s[0] = sum z~, s[1] = sum_T sum_{I in T} z~_I, s[2] = sum_T (v0_T + beta)/|T|
      const double c = v[S_MQC];
      v[S_MQG] = -(c * s[0] - s[2] + 0.25 * c * s[1]) / (v[S_NP1] + v[S_NP0]);
      break;
    }
    case FIN_DONE:
      if (v[S_PEND] != 0.0) sc->done = 1;
      sc->iter += 1;
      break;
    case FIN_PCG_INIT: {
      double* q = v + sl.base;
      q[P_RZ] = s[0];
      q[P_TARGET] = q[P_TOL] * q[P_TOL] * s[NV_ > 1 ? 1 : 0];
      q[P_ITS] = 0.0;
      if (!(s[NV_ > 1 ? 1 : 0] > 0.0) || !(s[0] > 0.0)) sc->idone[sl.flag] = 1;
      break;
    }
    case FIN_PCG_ALPHA: {
      double* q = v + sl.base;
      q[P_ALPHA] = s[0] != 0.0 ? q[P_RZ] / s[0] : 0.0;
      q[P_ITS] += 1.0;
      break;
    }
    case FIN_PCG_RR: {
      double* q = v + sl.base;
      if (!(s[0] > q[P_TARGET])) sc->idone[sl.flag] = 1;
      break;
    }
    case FIN_PCG_RZ: {
      double* q = v + sl.base;
      q[P_BETA] = q[P_RZ] != 0.0 ? s[0] / q[P_RZ] : 0.0;
      q[P_RZ] = s[0];
      break;
    }
    default:
      break;
  }
}

__device__ __forceinline__ void finish_slot(const Slot& sl, double s0) {
  double s[1] = {s0};
  finish_slot_n<1>(sl, s);
}

}  // namespace eth
