// EST-MINRES estimate of the discrete inf-sup constant (Sec. 2.4).
//
// Preconditioned MINRES runs a Lanczos process on P^{-1} K; its coefficients
// delta_j (diagonal) and gamma_{j+1} (off the diagonal) form the tridiagonal
// T_j.  With P = blkdiag(A, M_Q) and k projected out of the M_Q solve, the
// eigenvalues of P^{-1} K are 1 and (1 +- sqrt(1 + 4 sigma)) / 2 for the
// eigenvalues sigma of B A^{-1} B^T v = sigma M_Q v (v orthogonal to k), so the
// negative eigenvalue closest to zero, theta_-, gives gamma^2 = theta_-^2 - theta_-.
// The estimate after j steps takes for theta_- the negative harmonic Ritz value
// closest to zero (the harmonic Ritz values are the zeros of the MINRES residual
// polynomial and never fall into the gap around zero, so the estimate comes
// from above).
//
// Harmonic Ritz values (target 0) of T_j are the theta with
// T_{j+1,j}^T T_{j+1,j} y = theta T_j y.  Expanding the determinant of that
// pencil shows they are the nonzero eigenvalues of the symmetric tridiagonal
// matrix of order j + 1
//
//     That = [ T_j                 gamma_{j+1} e_j ]
//            [ gamma_{j+1} e_j^T   gamma_{j+1}^2 e_j^T T_j^{-1} e_j ],
//
// which is singular by construction (its last pivot vanishes).  The corner
// entry is gamma_{j+1}^2 / d_j with d_j the last pivot of the LDL^T factorisation
// of T_j.  The eigenvalues of That below a shift are counted with the Sturm
// sequence of its pivots (Sylvester's law of inertia); the estimate is the largest
// eigenvalue below -1e-10 ||That|| (which leaves out the zero eigenvalue whatever
// rounding does to it), found by multisection.
#include <cmath>
#include "grid.cuh"
#include "scalars.cuh"

namespace eth {

// Number of eigenvalues of That (order m + 1) below s.
__device__ int that_count(const double* __restrict__ dl, const double* __restrict__ gm, int m, double corner, double s,
                          double pivmin) {
  int c = 0;
  double q = dl[0] - s;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0.0) ++c;
  for (int i = 1; i <= m; ++i) {
    const double a = i < m ? dl[i] : corner;
    const double b = gm[i - 1];             // coupling of rows i - 1 and i: gamma_{i+1}
    q = a - s - b * b / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) ++c;
  }
  return c;
}

// One warp per j.  The warp first finds the corner entry, the Gershgorin interval and
// the number `neg` of eigenvalues below the threshold (lane-parallel where the
// work is), then multisects: each round the 32 lanes count at 32 equally spaced
// interior points of [lo, hi), and the interval shrinks to the gap between the
// first point whose count reaches `neg` and the point before it (33x per round;
// count(lo) < neg <= count(hi) holds throughout, monotone counts or not).
__global__ void __launch_bounds__(128) k_est_infsup(const double* __restrict__ dl, const double* __restrict__ gm, int k,
                                                    double* __restrict__ est) {
  ETH_GRID_DEP_WAIT();
  const int lane = threadIdx.x & 31;
  const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (t >= k) return;   // whole warps leave together
  const int m = t + 1;  // Lanczos steps in T_m
  // last LDL^T pivot of T_m (every lane; IEEE arithmetic carries a zero pivot through as inf)
  double d = dl[0];
  for (int i = 1; i < m; ++i) d = dl[i] - gm[i - 1] * gm[i - 1] / d;
  const double gl = gm[m - 1];
  const double corner = gl * gl / d;
  if (!isfinite(corner) || !isfinite(d)) {
    if (lane == 0) est[t] = nan("");
    return;
  }
  // Gershgorin bounds and the norm of That, rows split over the lanes
  double lo = INFINITY, nrm = 0.0, b2max = 0.0;
  for (int i = lane; i <= m; i += 32) {
    const double a = i < m ? dl[i] : corner;
    const double r = (i > 0 ? fabs(gm[i - 1]) : 0.0) + (i < m ? fabs(gm[i]) : 0.0);
    lo = fmin(lo, a - r);
    nrm = fmax(nrm, fabs(a) + r);
    if (i < m) b2max = fmax(b2max, gm[i] * gm[i]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    nrm = fmax(nrm, __shfl_xor_sync(0xffffffffu, nrm, o));
    b2max = fmax(b2max, __shfl_xor_sync(0xffffffffu, b2max, o));
  }
  if (!(nrm > 0.0) || !isfinite(nrm)) {
    if (lane == 0) est[t] = nan("");
    return;
  }
  // smallest pivot magnitude kept (safe minimum times the largest squared coupling)
  const double pivmin = 2.3e-308 * fmax(1.0, b2max);
  double hi = -1e-10 * nrm;
  const int neg = that_count(dl, gm, m, corner, hi, pivmin);   // same value in every lane
  if (neg == 0) {
    if (lane == 0) est[t] = nan("");
    return;
  }
  lo -= 1e-12 * nrm;
  for (int round = 0; round < 40; ++round) {
    const double w = (hi - lo) / 33.0;
    const double x = lo + (double)(lane + 1) * w;
    const bool inside = x > lo && x < hi;
    const bool reach = inside && that_count(dl, gm, m, corner, x, pivmin) >= neg;
    const unsigned ge = __ballot_sync(0xffffffffu, reach);
    const unsigned in = __ballot_sync(0xffffffffu, inside);
    // ge and in are the same in every lane, so every branch below is taken warp-wide
    double nlo = lo, nhi = hi;
    unsigned before = in;                 // inside points whose count is below neg
    if (ge != 0u) {
      const int first = __ffs(ge) - 1;
      nhi = __shfl_sync(0xffffffffu, x, first);
      before = in & ((1u << first) - 1u);
    }
    if (before != 0u) nlo = __shfl_sync(0xffffffffu, x, 31 - __clz(before));
    const bool stuck = (nlo == lo && nhi == hi);
    lo = nlo;
    hi = nhi;
    if (stuck || hi - lo <= 2e-16 * fabs(hi)) break;
  }
  if (lane == 0) {
    const double th = 0.5 * (lo + hi);
    est[t] = th * th - th;
  }
}

}  // namespace eth

using namespace eth;

extern "C" {

eth_status eth_lanczos(eth_grid* g, int cap, double* delta_dev, double* gamma_dev, int* k_host) {
  if (!g || !k_host || cap < 0 || (cap > 0 && (!delta_dev || !gamma_dev))) {
    set_error("eth_lanczos: NULL argument or cap < 0");
    return ETH_EINVAL;
  }
  if (g->kind != ETH_STOKES) { set_error("eth_lanczos: Lanczos coefficients are kept by Stokes (MINRES) solves"); return ETH_EINVAL; }
  ETH_ON_DEVICE(g);
  ETH_CUDA(cudaMemcpyAsync(&g->sch->lz_n, &g->sc->lz_n, sizeof(int), cudaMemcpyDeviceToHost, g->s));
  ETH_CUDA(cudaMemcpyAsync(&g->sch->lz_runs, &g->sc->lz_runs, sizeof(int), cudaMemcpyDeviceToHost, g->s));
  ETH_CUDA(cudaStreamSynchronize(g->s));
  const int k = g->sch->lz_runs > 0 ? g->sch->lz_n : 0;
  *k_host = k;
  const int c = k < cap ? k : cap;
  if (c > 0) {
    ETH_CUDA(cudaMemcpyAsync(delta_dev, g->lz, (size_t)c * 8, cudaMemcpyDeviceToDevice, g->s));
    ETH_CUDA(cudaMemcpyAsync(gamma_dev, g->lz + ETH_LANCZOS_CAP, (size_t)c * 8, cudaMemcpyDeviceToDevice, g->s));
  }
  return ETH_OK;
}

eth_status eth_est_infsup(eth_grid* g, const double* delta_dev, const double* gamma_dev, int k, double* est_dev) {
  if (!g || k < 0 || (k > 0 && (!delta_dev || !gamma_dev || !est_dev))) {
    set_error("eth_est_infsup: NULL argument or k < 0");
    return ETH_EINVAL;
  }
  if (k == 0) return ETH_OK;
  ETH_ON_DEVICE(g);
  const int warps = 4;   // one warp per estimate, four per CTA
  k_est_infsup<<<(k + warps - 1) / warps, 32 * warps, 0, g->s>>>(delta_dev, gamma_dev, k, est_dev);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  return ETH_OK;
}

}  // extern "C"
