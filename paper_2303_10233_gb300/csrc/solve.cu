// Krylov drivers: preconditioned MINRES (Algorithm 1) for Stokes with the
// block-diagonal preconditioner blkdiag(V-cycle(nu A), nu M_Q^+) (Eq. stokes_pre,
// Sec. 2.2: the M_Q solve keeps z orthogonal to k), FP64 iterative refinement
// around mixed-precision inner solves, and the public solve entry points.
#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>
#include <chrono>
#include <cmath>
#include <cstring>
#include "solve.cuh"
#include "mg.cuh"

namespace eth {

static void work_free(void* p) {
  Work* w = (Work*)p;
  if (!w) return;
  gmres_free(w);
  lsc_free(w);
  mqcheb_free(w);
  mg_free(w->vf); mg_free(w->qf); mg_free(w->vd); mg_free(w->qd); mg_free(w->vft); mg_free(w->vdt);
  cudaFree(w->x); cudaFree(w->d); cudaFree(w->r); cudaFree(w->Kz); cudaFree(w->bp); cudaFree(w->pcg);
  for (int k = 0; k < 2; ++k) { cudaFree(w->V[k]); cudaFree(w->Z[k]); cudaFree(w->W[k]); }
  if (w->gexec) cudaGraphExecDestroy(w->gexec);
  if (w->s2) cudaStreamDestroy(w->s2);
  if (w->s3) cudaStreamDestroy(w->s3);
  if (w->evw) cudaEventDestroy(w->evw);
  if (w->evx) cudaEventDestroy(w->evx);
  if (w->sm) cudaStreamDestroy(w->sm);
  if (w->evu) cudaEventDestroy(w->evu);
  if (w->evf) cudaEventDestroy(w->evf);
  if (w->evj) cudaEventDestroy(w->evj);
  if (w->t0) cudaEventDestroy(w->t0);
  if (w->t1) cudaEventDestroy(w->t1);
  delete w;
}

void solver_free(eth_grid* g) {
  if (g->ws && g->ws_free) g->ws_free(g->ws);
  g->ws = nullptr;
}

eth_status solver_coefficients_changed(eth_grid* g) {
  Work* w = (Work*)g->ws;
  if (!w) return ETH_OK;
  mg_free(w->vf); mg_free(w->qf); mg_free(w->vd); mg_free(w->qd); mg_free(w->vft); mg_free(w->vdt);
  if (w->gexec) { cudaGraphExecDestroy(w->gexec); w->gexec = nullptr; w->gkey = -1; }
  gmres_free(w);
  return ETH_OK;
}

eth_status work_get(eth_grid* g, Work** out) {
  if (g->ws) { *out = (Work*)g->ws; return ETH_OK; }
  Work* w = new Work();
  g->ws = w;
  g->ws_free = work_free;
  const size_t nt = g->nt;
  double** bufs[] = {&w->x, &w->d, &w->r, &w->Kz, &w->bp, &w->V[0], &w->V[1], &w->Z[0], &w->Z[1], &w->W[0], &w->W[1]};
  for (double** b : bufs) ETH_CUDA(cudaMalloc((void**)b, nt * 8));
  ETH_CUDA(cudaStreamCreateWithFlags(&w->s2, cudaStreamNonBlocking));
  ETH_CUDA(cudaStreamCreateWithFlags(&w->s3, cudaStreamNonBlocking));
  ETH_CUDA(cudaEventCreateWithFlags(&w->evw, cudaEventDisableTiming));
  ETH_CUDA(cudaEventCreateWithFlags(&w->evx, cudaEventDisableTiming));
  ETH_CUDA(cudaStreamCreateWithFlags(&w->sm, cudaStreamNonBlocking));
  ETH_CUDA(cudaEventCreateWithFlags(&w->evu, cudaEventDisableTiming));
  ETH_CUDA(cudaEventCreateWithFlags(&w->evf, cudaEventDisableTiming));
  ETH_CUDA(cudaEventCreateWithFlags(&w->evj, cudaEventDisableTiming));
  ETH_CUDA(cudaEventCreate(&w->t0));
  ETH_CUDA(cudaEventCreate(&w->t1));
  *out = w;
  return ETH_OK;
}

int vblocks(size_t m) {
  size_t b = (m + 255) / 256;
  if (b > 152 * 4) b = 152 * 4;
  return (int)(b < 1 ? 1 : b);
}

Slot slot_of(eth_grid* g, int which, int total, int op) {
  Slot s = make_slot(g, which, total);
  s.op = op;
  return s;
}

// ---------------------------------------------------------------------------
// FP64 vector kernels (grid-stride, fused reductions through Slot)
// ---------------------------------------------------------------------------
__global__ void k_residual(size_t m, const double* __restrict__ b, const double* __restrict__ y, double* __restrict__ r, Slot sl) {
  ETH_GRID_DEP_WAIT();
  double acc = 0.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) {
    const double v = b[k] - y[k];
    r[k] = v;
    acc += v * v;
  }
  double v[1] = {acc};
  if (slot_arrive<1>(sl, blockIdx.x, v)) finish_slot(sl, v[0]);
}

// x_p1 -= sum_p1 / n1 ; x_p0 -= sum_p0 / n0  (sums in sums[0], sums[1])
__global__ void k_psub(size_t off, size_t n1, size_t n0, double* __restrict__ x, const double* __restrict__ sums) {
  ETH_GRID_DEP_WAIT();
  const double m1 = sums[0] / (double)n1, m0 = sums[1] / (double)n0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n1 + n0; k += (size_t)gridDim.x * blockDim.x)
    x[off + k] -= k < n1 ? m1 : m0;
}

__global__ void k_add(size_t m, double* __restrict__ x, const double* __restrict__ d) {
  ETH_GRID_DEP_WAIT();
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) x[k] += d[k];
}

__global__ void k_set_boundary(int n, double* __restrict__ u, const double* __restrict__ ub) {
  ETH_GRID_DEP_WAIT();
  const int N = 2 * n + 1;
  const size_t nv = (size_t)N * N;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < 2 * nv; k += (size_t)gridDim.x * blockDim.x) {
    const size_t gg = k < nv ? k : k - nv;
    const int j = (int)(gg / N), i = (int)(gg - (size_t)j * N);
    if (i == 0 || j == 0 || i == N - 1 || j == N - 1) u[k] = ub[k];
  }
}

// MINRES vector updates of iteration j, in two kernels so that the w/x part
// leaves the critical path: k_minres_v, after the K apply, forms
// v_{j+1} = VA K z_j - VB v_j - VC v_{j-1} (into vo) with the sums of its p1 / p0
// blocks (FIN_V); k_minres_wx, beside the K apply on a second stream, applies the
// update the previous Givens step left pending, w_j = WZ z_{j-1} - WO w_{j-2} -
// WW w_{j-1} (into wold), x += XC w_j; k_minres_flags, after both, retires the
// pending update and stops the loop once a converged step's update is applied.
// Neither of the two concurrent kernels changes a flag the other reads.
__global__ void k_minres_v(size_t nt, size_t nu2, size_t n1, const double* __restrict__ Kz, const double* __restrict__ vj,
                           double* __restrict__ vo, Scalars* __restrict__ sc, Slot sl) {
  ETH_GRID_DEP_WAIT();
  if (sc->done) return;
  const double a = sc->v[S_VA], b = sc->v[S_VB], c = sc->v[S_VC];
  double a1 = 0.0, a0 = 0.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < nt; k += (size_t)gridDim.x * blockDim.x) {
    const double v = a * Kz[k] - b * vj[k] - c * vo[k];
    vo[k] = v;
    if (k >= nu2) { if (k < nu2 + n1) a1 += v; else a0 += v; }
  }
  double v[2] = {a1, a0};
  if (slot_arrive<2>(sl, blockIdx.x, v)) finish_slot_n<2>(sl, v);
}

__global__ void k_minres_wx(size_t nt, const double* __restrict__ zprev, double* __restrict__ wold,
                            const double* __restrict__ wcur, double* __restrict__ x, const Scalars* __restrict__ sc) {
  ETH_GRID_DEP_WAIT();
  if (sc->done || sc->v[S_WXP] == 0.0) return;
  const double cz = sc->v[S_WZ], co = sc->v[S_WO], cw = sc->v[S_WW], cx = sc->v[S_XC];
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < nt; k += (size_t)gridDim.x * blockDim.x) {
    const double w = cz * zprev[k] - co * wold[k] - cw * wcur[k];
    wold[k] = w;
    x[k] += cx * w;
  }
}

__global__ void k_minres_flags(Scalars* sc) {
  ETH_GRID_DEP_WAIT();
  if (sc->done) return;
  if (sc->v[S_WXP] != 0.0) {
    sc->v[S_WXP] = 0.0;
    if (sc->v[S_PEND] != 0.0) sc->done = 1;
  }
}

// the w/x update left pending when the iteration loop stops (applied iff pending)
__global__ void k_minres_wx_tail(size_t nt, const double* __restrict__ zj, double* __restrict__ wo, const double* __restrict__ wj,
                                 double* __restrict__ x, Scalars* __restrict__ sc) {
  ETH_GRID_DEP_WAIT();
  if (sc->v[S_WXP] == 0.0) return;
  const double cz = sc->v[S_WZ], co = sc->v[S_WO], cw = sc->v[S_WW], cx = sc->v[S_XC];
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < nt; k += (size_t)gridDim.x * blockDim.x) {
    const double w = cz * zj[k] - co * wo[k] - cw * wj[k];
    wo[k] = w;
    x[k] += cx * w;
  }
}

__global__ void k_minres_wx_clear(Scalars* sc) {
  ETH_GRID_DEP_WAIT(); sc->v[S_WXP] = 0.0; }

// End of one body of the device-side MINRES loop (a conditional WHILE node of the
// solver graph): run the body again unless converged, broken down or out of
// iterations.  The body count is capped independently of the solver state, so
// the loop always ends.
__global__ void k_minres_loop(cudaGraphConditionalHandle h, Scalars* sc) {
  ETH_GRID_DEP_WAIT();
  const int l = ++sc->loops;
  const bool more = !sc->done && sc->status == 0 && l < sc->max_loops;
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

__global__ void k_init_scalars(Scalars* sc, double tol, double n1, double n0, double mqc, double nu, int maxit) {
  ETH_GRID_DEP_WAIT();
  sc->lz_runs += 1;             // Lanczos coefficients are kept for the first run only
  if (sc->lz_runs == 1) sc->lz_n = 0;
  sc->loops = 0;
  sc->max_loops = (maxit + 1) / 2;   // two MINRES iterations per loop body
  for (int k = 0; k < S_LAST; ++k) sc->v[k] = 0.0;
  sc->v[S_TOL] = tol;
  sc->v[S_NP1] = n1;
  sc->v[S_NP0] = n0;
  sc->v[S_MQC] = mqc;
  sc->v[S_MQNU] = nu;
  sc->done = 0;
  sc->status = 0;
  sc->iter = 0;
}

// ---------------------------------------------------------------------------
// pressure block: nu * M_Q^+ with k projected out (Sec. 2.2-2.3)
//   r = v - beta k  (beta = k^T v / k^T k)
//   t = r_k - R^T Q0^{-1} r_0            (t_I = r_k,I - 1/4 sum_{T ni I} r_0,T)
//   z_k = c V_K1(t) + g1                  (S ~ h^2/16 K1, c = 16/|T|)
//   z_0 = Q0^{-1}(r_0 - R z_k)
//   g1 chosen so that k^T z = 0; output nu * z.
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_mq_t(int n, const double* __restrict__ vp, const Scalars* __restrict__ sc, T* __restrict__ b,
                       T* __restrict__ x, const T* __restrict__ dinv, T omega, const int* done,
                       int sums, Slot sl, T inv_area) {
  ETH_GRID_DEP_WAIT();
  if (done != nullptr && *done) return;
  const int M = n + 1, n1 = M * M;
  const T beta = (T)sc->v[S_BETA];
  for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < n1; node += gridDim.x * blockDim.x) {
    const int J = node / M, I = node - J * M;
    T s = 0;
    Q1_FOR_ELEMENTS(n, I, J, { s += cvt<T, double>(vp[n1 + (size_t)ey * n + ex]) + beta; (void)c; (void)d; })
    const T t = cvt<T, double>(vp[node]) - beta - T(0.25) * s;
    b[node] = t;
    x[node] = omega * dinv[node] * t;
  }
  if (sums) {   // (0, 0, sum_T (v0_T + beta)/|T|) for the M_Q constant
    T s2 = 0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x)
      s2 += (cvt<T, double>(vp[n1 + e]) + beta) * inv_area;
    double v[3] = {0.0, 0.0, (double)s2};
    if (slot_arrive<3>(sl, blockIdx.x, v)) finish_slot_n<3>(sl, v);
  }
}

// sums for the k-orthogonality constant: (sum z~, sum_T sum_{I in T} z~_I, sum_T (v0_T + beta)/|T|)
template <class T>
__global__ void k_mq_sums(int n, const T* __restrict__ zt, const double* __restrict__ vp, T inv_area, Slot sl, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done != nullptr && *done) return;
  const int M = n + 1, n1 = M * M, n0 = n * n;
  const T beta = (T)sl.sc->v[S_BETA];
  T s0 = 0, s1 = 0, s2 = 0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n1 + n0; k += gridDim.x * blockDim.x) {
    if (k < n1) {
      const int J = k / M, I = k - J * M;
      const int ne = ((I > 0) + (I < n)) * ((J > 0) + (J < n));
      const T z = zt[k];
      s0 += z;
      s1 += (T)ne * z;
    } else {
      s2 += (cvt<T, double>(vp[k]) + beta) * inv_area;
    }
  }
  double v[3] = {(double)s0, (double)s1, (double)s2};
  if (slot_arrive<3>(sl, blockIdx.x, v)) finish_slot_n<3>(sl, v);
}

template <class T>
__global__ void k_mq_out(int n, const T* __restrict__ zt, const double* __restrict__ vp, double* __restrict__ zp, T inv_area,
                         const Scalars* __restrict__ sc, Slot gsl, int goff, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done != nullptr && *done) return;
  const int M = n + 1, n1 = M * M, n0 = n * n;
  const T beta = (T)sc->v[S_BETA], c = (T)sc->v[S_MQC], g1 = (T)sc->v[S_MQG], nu = (T)sc->v[S_MQNU];
  double acc = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n1 + n0; k += gridDim.x * blockDim.x) {
    T z;
    if (k < n1) {
      z = nu * (c * zt[k] + g1);
    } else {
      const int e = k - n1, ey = e / n, ex = e - ey * n;
      const T s = zt[(size_t)ey * M + ex] + zt[(size_t)ey * M + ex + 1] + zt[(size_t)(ey + 1) * M + ex] +
                  zt[(size_t)(ey + 1) * M + ex + 1];
      z = nu * ((cvt<T, double>(vp[k]) + beta) * inv_area - T(0.25) * c * s - g1);
    }
    const double zd = cvt<double, T>(z);
    zp[k] = zd;
    acc += zd * vp[k];
  }
  double v[1] = {acc};
  if (slot_arrive<1>(gsl, goff + blockIdx.x, v)) finish_slot(gsl, v[0]);
}

int mq_blocks(eth_grid* g) { return vblocks((size_t)g->n1 + g->n0); }

template <class T>
eth_status precond_pressure(eth_grid* g, Hier<T>& Q, const double* vp, double* zp, const Slot& gsl, int goff,
                            const int* done, cudaStream_t s) {
  Level<T>& L0 = Q.lv[0];
  const cudaStream_t keep = g->s;
  g->s = s;
  const int nbt = vblocks(g->n1), nbp = (int)q1_blocks(g->n);
  const T inv_area = (T)(1.0 / (g->hx * g->hy));
  const bool fold = q1_vcycle_fused<T>(Q, 1, 1);
  const int nb = mq_blocks(g);
  // the three sums of the M_Q constant come from k_mq_t (P0 part) and the last
  // Q1 smoothing sweep (Q1 part) when the fused V-cycle runs, else from k_mq_sums
  Slot sm = slot_of(g, SL_MQ, fold ? nbt + nbp : nb, FIN_MQ);
  k_mq_t<T><<<nbt, 256, 0, s>>>(g->n, vp, g->sc, L0.b, L0.x, L0.dinv, (T)Q.omega, done, fold ? 1 : 0, sm, inv_area);
  ETH_CUDA(cudaGetLastError());
  const T* zt = nullptr;
  eth_status st = vcycle_q1_from<T>(g, Q, 1, 1, done, &zt, fold ? &sm : nullptr, nbt);
  if (st != ETH_OK) { g->s = keep; return st; }
  if (!fold) {
    k_mq_sums<T><<<nb, 256, 0, s>>>(g->n, zt, vp, inv_area, sm, done);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
  }
  k_mq_out<T><<<nb, 256, 0, s>>>(g->n, zt, vp, zp, inv_area, g->sc, gsl, goff, done);
  ETH_CUDA(cudaGetLastError());
  g->launches += 2;
  g->s = keep;
  return ETH_OK;
}

template <>
Hier<float>& vel_hier<float>(Work* w) { return w->vf; }
template <>
Hier<double>& vel_hier<double>(Work* w) { return w->vd; }
template <>
Hier<float>& vel_hier_t<float>(Work* w) { return w->vft; }
template <>
Hier<double>& vel_hier_t<double>(Work* w) { return w->vdt; }
template <>
Hier<float>& q1_hier<float>(Work* w) { return w->qf; }
template <>
Hier<double>& q1_hier<double>(Work* w) { return w->qd; }
template eth_status precond_pressure<float>(eth_grid*, Hier<float>&, const double*, double*, const Slot&, int, const int*, cudaStream_t);
template eth_status precond_pressure<double>(eth_grid*, Hier<double>&, const double*, double*, const Slot&, int, const int*, cudaStream_t);

// ---------------------------------------------------------------------------
// exact preconditioner blocks (the P_1 form of Sec. 2.4): inner PCG solves of
// the velocity block (GMG V-cycle preconditioner) and of the Schur complement
// S = Qk - R^T Q0^{-1} R of M_Q (Q1 Laplacian V-cycle preconditioner), each to
// a relative residual opts.inner_tol, with device-side convergence flags so the
// whole outer iteration stays capturable in a CUDA graph.
// ---------------------------------------------------------------------------
__global__ void k_pcg_setup(Scalars* sc, int base, int flag, double tol) {
  ETH_GRID_DEP_WAIT();
  sc->v[base + P_TOL] = tol;
  sc->v[base + P_ITS] = 0.0;
  sc->idone[flag] = sc->done;
}

__global__ void k_pcg_start(size_t m, const double* __restrict__ b, double* __restrict__ r, double* __restrict__ x,
                            const int* done) {
  ETH_GRID_DEP_WAIT();
  if (*done) return;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) {
    r[k] = b[k];
    x[k] = 0.0;
  }
}

// (<a,b>, <a,a>) -> finisher
__global__ void k_dot2(size_t m, const double* __restrict__ a, const double* __restrict__ b, Slot sl, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (*done) return;
  double s0 = 0.0, s1 = 0.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) {
    s0 += a[k] * b[k];
    s1 += a[k] * a[k];
  }
  double v[2] = {s0, s1};
  if (slot_arrive<2>(sl, blockIdx.x, v)) finish_slot_n<2>(sl, v);
}

__global__ void k_pcg_copy(size_t m, const double* __restrict__ a, double* __restrict__ b, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (*done) return;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) b[k] = a[k];
}

// x += alpha p ; r -= alpha q ; <r, r> -> FIN_PCG_RR
__global__ void k_pcg_xr(size_t m, const double* __restrict__ p, const double* __restrict__ q, double* __restrict__ x,
                         double* __restrict__ r, Slot sl, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (*done) return;
  const double a = sl.sc->v[sl.base + P_ALPHA];
  double acc = 0.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) {
    x[k] += a * p[k];
    const double rv = r[k] - a * q[k];
    r[k] = rv;
    acc += rv * rv;
  }
  double v[1] = {acc};
  if (slot_arrive<1>(sl, blockIdx.x, v)) finish_slot(sl, v[0]);
}

// p = z + beta p
__global__ void k_pcg_pupd(size_t m, const double* __restrict__ z, double* __restrict__ p, const Scalars* sc, int base,
                           const int* done) {
  ETH_GRID_DEP_WAIT();
  if (*done) return;
  const double bt = sc->v[base + P_BETA];
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) p[k] = z[k] + bt * p[k];
}

// <a, b> -> finisher
__global__ void k_dot1(size_t m, const double* __restrict__ a, const double* __restrict__ b, Slot sl, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (*done) return;
  double s0 = 0.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) s0 += a[k] * b[k];
  double v[1] = {s0};
  if (slot_arrive<1>(sl, blockIdx.x, v)) finish_slot(sl, v[0]);
}

// Level-0 right-hand side b = a of the Q1 V-cycle and its first Jacobi step from
// zero, x = omega D^{-1} b, which vcycle_q1_from expects in place: without it
// level 0 would start from the previous call's iterate and the V-cycle would not
// be a linear (let alone symmetric) preconditioner.
template <class T>
__global__ void k_to_t(int m, const double* __restrict__ a, T omega, const T* __restrict__ dinv, T* __restrict__ b,
                       T* __restrict__ x, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (*done) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    const T v = cvt<T, double>(a[k]);
    b[k] = v;
    x[k] = omega * dinv[k] * v;
  }
}
template <class T>
__global__ void k_from_t(int m, const T* __restrict__ a, double* __restrict__ b, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (*done) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) b[k] = cvt<double, T>(a[k]);
}

// t = (r_k - beta) - 1/4 sum_{T ni I} (r_0,T + beta)  in FP64
__global__ void k_mq_t64(int n, const double* __restrict__ vp, const Scalars* __restrict__ sc, double* __restrict__ t,
                         const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done != nullptr && *done) return;
  const int M = n + 1, n1 = M * M;
  const double beta = sc->v[S_BETA];
  for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < n1; node += gridDim.x * blockDim.x) {
    const int J = node / M, I = node - J * M;
    double s = 0.0;
    for (int ey = J - 1; ey <= J; ++ey) {
      if (ey < 0 || ey >= n) continue;
      for (int ex = I - 1; ex <= I; ++ex) {
        if (ex < 0 || ex >= n) continue;
        s += vp[n1 + (size_t)ey * n + ex] + beta;
      }
    }
    t[node] = vp[node] - beta - 0.25 * s;
  }
}

static Slot pslot(eth_grid* g, int which, int total, int op, int base, int flag) {
  Slot s = slot_of(g, which, total, op);
  s.base = base;
  s.flag = flag;
  return s;
}

static eth_status ensure_pcg(eth_grid* g, Work* w) {
  if (w->pcg) return ETH_OK;
  const size_t nu2 = 2 * (size_t)g->nv;
  ETH_CUDA(cudaMalloc((void**)&w->pcg, (4 * nu2 + 6 * (size_t)g->n1) * 8));
  return ETH_OK;
}

// x = F^{-1} b (velocity block, identity boundary rows) by V-cycle-preconditioned CG.
template <class T>
static eth_status vel_pcg(eth_grid* g, Work* w, const eth_opts* o, const double* b, double* x, int maxit) {
  const size_t nu2 = 2 * (size_t)g->nv;
  double *r = w->pcg, *p = r + nu2, *q = p + nu2, *z = q + nu2;
  const int* idone = &g->sc->idone[0];
  const int nb = vblocks(nu2);
  k_pcg_setup<<<1, 1, 0, g->s>>>(g->sc, PCG_VEL, 0, o->inner_tol);
  k_pcg_start<<<nb, 256, 0, g->s>>>(nu2, b, r, x, idone);
  ETH_CUDA(cudaGetLastError());
  ETH_TRY(vcycle_vel<T>(g, vel_hier<T>(w), r, z, o->mg_pre, o->mg_post, idone, nullptr, 0));
  k_dot2<<<nb, 256, 0, g->s>>>(nu2, r, z, pslot(g, 9, nb, FIN_PCG_INIT, PCG_VEL, 0), idone);
  k_pcg_copy<<<nb, 256, 0, g->s>>>(nu2, z, p, idone);
  ETH_CUDA(cudaGetLastError());
  g->launches += 5;
  const bool fp32 = o->precision == ETH_MIXED;
  for (int it = 0; it < maxit; ++it) {
    {  // q = F p with the fused <q, p>
      Slot s = pslot(g, 10, q2_blocks(g->n), FIN_PCG_ALPHA, PCG_VEL, 0);
      if (fp32) {
        Q2Params<double, double, float> P{};
        P.n = g->n; P.hx = (float)g->hx; P.hy = (float)g->hy; P.nu = (float)g->nu;
        P.x = p; P.y = q; P.w = g->windf; P.done = idone; P.slot = s; P.dv = p;
        if (g->kind == ETH_OSEEN) ETH_CUDA((launch_q2<double, double, float, QF_DIFF | QF_CONV | QF_XIN | QF_UOUT | QF_DOT, EPI_APPLY>(P, g->s)));
        else ETH_CUDA((launch_q2<double, double, float, QF_DIFF | QF_XIN | QF_UOUT | QF_DOT, EPI_APPLY>(P, g->s)));
      } else {
        Q2Params<double, double, double> P{};
        P.n = g->n; P.hx = g->hx; P.hy = g->hy; P.nu = g->nu;
        P.x = p; P.y = q; P.w = g->wind; P.done = idone; P.slot = s; P.dv = p;
        if (g->kind == ETH_OSEEN) ETH_CUDA((launch_q2<double, double, double, QF_DIFF | QF_CONV | QF_XIN | QF_UOUT | QF_DOT, EPI_APPLY>(P, g->s)));
        else ETH_CUDA((launch_q2<double, double, double, QF_DIFF | QF_XIN | QF_UOUT | QF_DOT, EPI_APPLY>(P, g->s)));
      }
    }
    k_pcg_xr<<<nb, 256, 0, g->s>>>(nu2, p, q, x, r, pslot(g, 11, nb, FIN_PCG_RR, PCG_VEL, 0), idone);
    ETH_CUDA(cudaGetLastError());
    ETH_TRY(vcycle_vel<T>(g, vel_hier<T>(w), r, z, o->mg_pre, o->mg_post, idone, nullptr, 0));
    k_dot1<<<nb, 256, 0, g->s>>>(nu2, r, z, pslot(g, 9, nb, FIN_PCG_RZ, PCG_VEL, 0), idone);
    k_pcg_pupd<<<nb, 256, 0, g->s>>>(nu2, z, p, g->sc, PCG_VEL, idone);
    ETH_CUDA(cudaGetLastError());
    g->launches += 4;
  }
  return ETH_OK;
}

// x = S^+ t (Q1, FP64) by Q1-Laplacian-V-cycle-preconditioned CG.
template <class T>
static eth_status schur_pcg(eth_grid* g, Work* w, const eth_opts* o, const double* t, double* x, int maxit, cudaStream_t s) {
  const size_t nu2 = 2 * (size_t)g->nv;
  const int m = g->n1;
  double *r = w->pcg + 4 * nu2, *p = r + m, *q = p + m, *z = q + m;
  const int* idone = &g->sc->idone[1];
  const int nb = vblocks(m);
  Hier<T>& Q = q1_hier<T>(w);
  const cudaStream_t keep = g->s;
  g->s = s;
  auto precond = [&](const double* rr, double* zz) -> eth_status {
    k_to_t<T><<<nb, 256, 0, s>>>(m, rr, (T)Q.omega, Q.lv[0].dinv, Q.lv[0].b, Q.lv[0].x, idone);
    ETH_CUDA(cudaGetLastError());
    const T* res = nullptr;
    ETH_TRY(vcycle_q1_from<T>(g, Q, 1, 1, idone, &res));
    k_from_t<T><<<nb, 256, 0, s>>>(m, res, zz, idone);
    ETH_CUDA(cudaGetLastError());
    g->launches += 2;
    return ETH_OK;
  };
  k_pcg_setup<<<1, 1, 0, s>>>(g->sc, PCG_PRE, 1, o->inner_tol);
  k_pcg_start<<<nb, 256, 0, s>>>((size_t)m, t, r, x, idone);
  ETH_CUDA(cudaGetLastError());
  eth_status st = precond(r, z);
  if (st != ETH_OK) { g->s = keep; return st; }
  k_dot2<<<nb, 256, 0, s>>>((size_t)m, r, z, pslot(g, 12, nb, FIN_PCG_INIT, PCG_PRE, 1), idone);
  k_pcg_copy<<<nb, 256, 0, s>>>((size_t)m, z, p, idone);
  ETH_CUDA(cudaGetLastError());
  g->launches += 4;
  for (int it = 0; it < maxit; ++it) {
    Q1Params<double, double, double> P{};
    P.n = g->n; P.hx = g->hx; P.hy = g->hy; P.cm = 1.0; P.ck = 0.0; P.c1 = -g->hx * g->hy / 16.0;
    P.x = p; P.y = q; P.done = idone; P.dot = 1;
    const int nq = (int)q1_blocks(g->n);
    P.slot = pslot(g, 13, nq, FIN_PCG_ALPHA, PCG_PRE, 1);
    k_q1node<double, double, double, Q1E_APPLY><<<nq, 256, 0, s>>>(P);
    k_pcg_xr<<<nb, 256, 0, s>>>((size_t)m, p, q, x, r, pslot(g, 14, nb, FIN_PCG_RR, PCG_PRE, 1), idone);
    ETH_CUDA(cudaGetLastError());
    st = precond(r, z);
    if (st != ETH_OK) { g->s = keep; return st; }
    k_dot1<<<nb, 256, 0, s>>>((size_t)m, r, z, pslot(g, 12, nb, FIN_PCG_RZ, PCG_PRE, 1), idone);
    k_pcg_pupd<<<nb, 256, 0, s>>>((size_t)m, z, p, g->sc, PCG_PRE, idone);
    ETH_CUDA(cudaGetLastError());
    g->launches += 4;
  }
  g->s = keep;
  return ETH_OK;
}

// exact nu M_Q^+ r_p (k projected out): t = r_k - R^T Q0^{-1} r_0, z_k = S^+ t, z_0 = Q0^{-1}(r_0 - R z_k)
template <class T>
static eth_status precond_pressure_exact(eth_grid* g, Work* w, const eth_opts* o, const double* vp, double* zp,
                                         const Slot& gsl, int goff, const int* done, cudaStream_t s) {
  const size_t nu2 = 2 * (size_t)g->nv;
  const int m = g->n1;
  double* t = w->pcg + 4 * nu2 + 4 * (size_t)m;
  double* zt = t + m;
  k_mq_t64<<<vblocks(m), 256, 0, s>>>(g->n, vp, g->sc, t, done);
  ETH_CUDA(cudaGetLastError());
  ETH_TRY(schur_pcg<T>(g, w, o, t, zt, 60, s));
  const int nb = mq_blocks(g);
  Slot sm = slot_of(g, SL_MQ, nb, FIN_MQ);
  k_mq_sums<double><<<nb, 256, 0, s>>>(g->n, zt, vp, 1.0 / (g->hx * g->hy), sm, done);
  k_mq_out<double><<<nb, 256, 0, s>>>(g->n, zt, vp, zp, 1.0 / (g->hx * g->hy), g->sc, gsl, goff, done);
  ETH_CUDA(cudaGetLastError());
  g->launches += 3;
  return ETH_OK;
}

// exact velocity block with the fused <z_u, v_u> partials into the gamma slot
__global__ void k_vel_out(size_t m, const double* __restrict__ x, const double* __restrict__ v, double* __restrict__ z,
                          Slot gsl, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done != nullptr && *done) return;
  double acc = 0.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) {
    z[k] = x[k];
    acc += x[k] * v[k];
  }
  double a[1] = {acc};
  if (slot_arrive<1>(gsl, blockIdx.x, a)) finish_slot(gsl, a[0]);
}

// z = P^{-1} v with the fused <z, v> into the gamma slot (finisher fin).
// The velocity V-cycle and the pressure block run on two streams (fork/join).
template <class T>
static eth_status precond_stokes(eth_grid* g, Work* w, const eth_opts* o, const double* v, double* z, int fin, const int* done) {
  const size_t nu2 = 2 * (size_t)g->nv;
  const int nbv = o->a_exact ? vblocks(nu2) : vel_final_blocks(g->n), nbp = mq_blocks(g);
  Slot gs = slot_of(g, SL_GAMMA, nbv + nbp, fin);
  ETH_CUDA(cudaEventRecord(w->evf, g->s));
  ETH_CUDA(cudaStreamWaitEvent(w->s2, w->evf, 0));
  if (o->mq_mode == ETH_MQ_EXACT) ETH_TRY(precond_pressure_exact<T>(g, w, o, v + nu2, z + nu2, gs, nbv, done, w->s2));
  else if (o->mq_mode == ETH_MQ_CHEB) ETH_TRY(precond_pressure_cheb<T>(g, w, o, v + nu2, z + nu2, gs, nbv, done, w->s2));
  else ETH_TRY(precond_pressure<T>(g, q1_hier<T>(w), v + nu2, z + nu2, gs, nbv, done, w->s2));
  if (o->a_exact) {
    ETH_TRY(vel_pcg<T>(g, w, o, v, z, 60));
    // <z_u, v_u> partials (z_u already in place)
    k_vel_out<<<nbv, 256, 0, g->s>>>(nu2, z, v, z, gs, done);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
  } else {
    ETH_TRY(vcycle_vel<T>(g, vel_hier<T>(w), v, z, o->mg_pre, o->mg_post, done, &gs, 0));
  }
  ETH_CUDA(cudaEventRecord(w->evj, w->s2));
  ETH_CUDA(cudaStreamWaitEvent(g->s, w->evj, 0));
  return ETH_OK;
}

// one MINRES iteration j (buffers by parity)
template <class T>
static eth_status minres_iter(eth_grid* g, Work* w, const eth_opts* o, bool fp32, int j) {
  const size_t nt = g->nt, nu2 = 2 * (size_t)g->nv;
  const int* done = &g->sc->done;
  double* zj = w->Z[j & 1];
  double* zn = w->Z[(j + 1) & 1];
  double* vj = w->V[j & 1];
  double* vo = w->V[(j + 1) & 1];
  double* wj = w->W[j & 1];
  double* wo = w->W[(j + 1) & 1];   // w_{j-2}, overwritten by w_j
  const int nb = vblocks(nt);
  // the pending w/x update of iteration j-1 (z_{j-1} = zn's buffer, not yet overwritten)
  // on the side stream, beside the K apply and the v update
  ETH_CUDA(cudaEventRecord(w->evw, g->s));
  ETH_CUDA(cudaStreamWaitEvent(w->s3, w->evw, 0));
  k_minres_wx<<<nb, 256, 0, w->s3>>>(nt, zn, wj, wo, w->d, g->sc);
  ETH_CUDA(cudaGetLastError());
  ETH_TRY(op_apply_K_dot(g, fp32, false, zj, w->Kz, slot_of(g, SL_DELTA, 0, FIN_MINRES_DELTA), done));
  const int nbv = std::min(nb, 2 * 152);   // measured: 608 -> 304 blocks, 5.67 -> 5.58 ms at 256^2
  k_minres_v<<<nbv, 256, 0, g->s>>>(nt, nu2, (size_t)g->n1, w->Kz, vj, vo, g->sc, slot_of(g, SL_VSUM, nbv, FIN_V));
  ETH_CUDA(cudaGetLastError());
  ETH_CUDA(cudaEventRecord(w->evx, w->s3));
  ETH_CUDA(cudaStreamWaitEvent(g->s, w->evx, 0));
  k_minres_flags<<<1, 1, 0, g->s>>>(g->sc);
  ETH_CUDA(cudaGetLastError());
  ETH_TRY(precond_stokes<T>(g, w, o, vo, zn, FIN_MINRES_GAMMA, done));
  g->launches += 3;
  return ETH_OK;
}

// Programmatic dependent launch inside the captured graphs (ETH_PDL=1 in the
// environment): every kernel -> kernel edge becomes a programmatic edge from the
// upstream kernel's launch-completion port, so the downstream grid is scheduled
// while the upstream one runs and waits in griddepcontrol.wait (first statement
// of every kernel) for its completion.  Off by default: measured on GB300 it
// cost 3 % at n = 256 and gained 1 % at n = 512 (the waiting CTAs hold SM slots
// the producer's blocks could use).
bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("ETH_PDL");
    return e && e[0] == '1';
  }();
  return on;
}

eth_status make_programmatic(cudaGraph_t graph) {
  size_t ne = 0;
  ETH_CUDA(cudaGraphGetEdges(graph, nullptr, nullptr, nullptr, &ne));
  if (ne == 0) return ETH_OK;
  std::vector<cudaGraphNode_t> from(ne), to(ne);
  std::vector<cudaGraphEdgeData> ed(ne);
  ETH_CUDA(cudaGraphGetEdges(graph, from.data(), to.data(), ed.data(), &ne));
  for (size_t k = 0; k < ne; ++k) {
    cudaGraphNodeType ta, tb;
    ETH_CUDA(cudaGraphNodeGetType(from[k], &ta));
    ETH_CUDA(cudaGraphNodeGetType(to[k], &tb));
    if (ta != cudaGraphNodeTypeKernel || tb != cudaGraphNodeTypeKernel || ed[k].type != cudaGraphDependencyTypeDefault) continue;
    ETH_CUDA(cudaGraphRemoveDependencies(graph, &from[k], &to[k], &ed[k], 1));
    cudaGraphEdgeData p{};
    p.from_port = cudaGraphKernelNodePortLaunchCompletion;
    p.type = cudaGraphDependencyTypeProgrammatic;
    ETH_CUDA(cudaGraphAddDependencies(graph, &from[k], &to[k], &p, 1));
  }
  return ETH_OK;
}

eth_status read_scalars(eth_grid* g) {
  ETH_CUDA(cudaMemcpyAsync(g->sch, g->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, g->s));
  ETH_CUDA(cudaStreamSynchronize(g->s));
  return ETH_OK;
}

// Inner MINRES on K d = r (d from zero).  Returns iterations and device status.
template <class T>
static eth_status minres_solve(eth_grid* g, Work* w, const eth_opts* o, bool fp32, double tol, int maxit, int* its, int* dstat) {
  const size_t nt = g->nt;
  const double area = g->hx * g->hy;
  k_init_scalars<<<1, 1, 0, g->s>>>(g->sc, tol, (double)g->n1, (double)g->n0,
                                    o->mq_mode == ETH_MQ_EXACT ? 1.0 : 16.0 / area, g->nu, maxit);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  ETH_CUDA(cudaMemsetAsync(w->d, 0, nt * 8, g->s));
  ETH_CUDA(cudaMemsetAsync(w->W[0], 0, nt * 8, g->s));
  ETH_CUDA(cudaMemsetAsync(w->W[1], 0, nt * 8, g->s));
  ETH_CUDA(cudaMemsetAsync(w->V[0], 0, nt * 8, g->s));
  ETH_CUDA(cudaMemcpyAsync(w->V[1], w->r, nt * 8, cudaMemcpyDeviceToDevice, g->s));
  // beta of v_1 for the k-projection, then z_1 = P^{-1} v_1 and gamma_1
  {
    const int nb = vblocks((size_t)g->n1 + g->n0);
    Slot s = slot_of(g, SL_VSUM, nb, FIN_VSUMS);
    k_psums<0><<<nb, 256, 0, g->s>>>(2 * (size_t)g->nv, (size_t)g->n1, (size_t)g->n0, w->V[1], s);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
  }
  ETH_TRY(precond_stokes<T>(g, w, o, w->V[1], w->Z[1], FIN_MINRES_INIT, nullptr));
  ETH_TRY(read_scalars(g));
  if (g->sch->v[S_PEND] != 0.0) { *its = 0; *dstat = g->sch->status; return ETH_OK; }
  int j = 1;
  const bool use_graph = o->graph != 0;
  // 1: the whole loop on the device; 2 (or a driver without conditional graph nodes): host-checked replays
  bool device_loop = o->graph == 1 && !w->no_cond_nodes;
  // every option the captured graph depends on, in separate digit fields (mixed radix)
  const long long key =
      ((((((long long)o->graph * 4 + o->mq_mode) * 2 + o->a_exact) * 1024 + tile_code(g)) * 1024 + o->mg_post) * 1024 +
       o->mg_pre) * 32 + (long long)sizeof(T) * 2 + (fp32 ? 1 : 0);
  while (true) {
    if (use_graph) {
      if (!w->gexec || w->gkey != key) {
        if (w->gexec) { cudaGraphExecDestroy(w->gexec); w->gexec = nullptr; }
        cudaGraph_t graph = nullptr, body = nullptr;
        cudaGraphConditionalHandle cond = 0;
        if (device_loop) {
          // a WHILE conditional node whose body is two MINRES iterations and the loop test
          ETH_CUDA(cudaGraphCreate(&graph, 0));
          cudaError_t ge = cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault);
          cudaGraphNodeParams cp{};
          cp.type = cudaGraphNodeTypeConditional;
          cp.conditional.handle = cond;
          cp.conditional.type = cudaGraphCondTypeWhile;
          cp.conditional.size = 1;
          cudaGraphNode_t cnode;
          if (ge == cudaSuccess) ge = cudaGraphAddNode(&cnode, graph, nullptr, nullptr, 0, &cp);
          if (ge == cudaSuccess) {
            body = cp.conditional.phGraph_out[0];
            ge = cudaStreamBeginCaptureToGraph(g->s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
          }
          if (ge != cudaSuccess) {   // no conditional nodes here: fall back to host-replayed graphs
            cudaGraphDestroy(graph);
            cudaGetLastError();
            w->no_cond_nodes = true;
            device_loop = false;
            continue;
          }
        } else {
          ETH_CUDA(cudaStreamBeginCapture(g->s, cudaStreamCaptureModeThreadLocal));
        }
        const long l0 = g->launches;
        eth_status st = minres_iter<T>(g, w, o, fp32, 1);
        if (st == ETH_OK) st = minres_iter<T>(g, w, o, fp32, 2);
        if (st == ETH_OK && device_loop) {
          k_minres_loop<<<1, 1, 0, g->s>>>(cond, g->sc);
          if (cudaGetLastError() != cudaSuccess) st = ETH_ECUDA;
        }
        cudaGraph_t captured = nullptr;
        cudaError_t ce = cudaStreamEndCapture(g->s, &captured);
        w->glaunch = g->launches - l0;
        g->launches = l0;
        if (!device_loop) graph = captured;
        if (st != ETH_OK || ce != cudaSuccess) {
          if (graph) cudaGraphDestroy(graph);
          if (st != ETH_OK) return st;
          ETH_CUDA(ce);
        }
        if (pdl_enabled()) {
          const eth_status ps = make_programmatic(device_loop ? body : graph);
          if (ps != ETH_OK) { cudaGraphDestroy(graph); return ps; }
        }
        const cudaError_t ie = cudaGraphInstantiate(&w->gexec, graph, 0);
        cudaGraphDestroy(graph);
        ETH_CUDA(ie);
        w->gkey = key;
      }
      ETH_CUDA(cudaGraphLaunch(w->gexec, g->s));
      if (device_loop) {
        ETH_TRY(read_scalars(g));
        g->launches += (long)g->sch->loops * w->glaunch;
        break;
      }
      g->launches += w->glaunch;
    } else {
      ETH_TRY(minres_iter<T>(g, w, o, fp32, j));
      ETH_TRY(minres_iter<T>(g, w, o, fp32, j + 1));
    }
    j += 2;
    ETH_TRY(read_scalars(g));
    if (g->sch->done || (int)g->sch->v[S_ITS] >= maxit) break;
  }
  {
    const int J = (int)g->sch->v[S_ITS];   // last iteration with a Givens step
    k_minres_wx_tail<<<vblocks(nt), 256, 0, g->s>>>(nt, w->Z[J & 1], w->W[(J + 1) & 1], w->W[J & 1], w->d, g->sc);
    k_minres_wx_clear<<<1, 1, 0, g->s>>>(g->sc);
    ETH_CUDA(cudaGetLastError());
    g->launches += 2;
  }
  *its = (int)g->sch->v[S_ITS];
  *dstat = g->sch->status;
  return ETH_OK;
}

template <class T>
eth_status ensure_hier(eth_grid* g, Work* w, const eth_opts* o) {
  const int nmin = o->mg_min_n > 0 ? std::max(2, o->mg_min_n) : (g->kind == ETH_OSEEN ? 8 : 4);
  if (w->nmin_built != nmin) {
    mg_free(w->vf); mg_free(w->qf); mg_free(w->vd); mg_free(w->qd); mg_free(w->vft); mg_free(w->vdt);
    if (w->gexec) { cudaGraphExecDestroy(w->gexec); w->gexec = nullptr; w->gkey = -1; }
    w->nmin_built = nmin;
  }
  Hier<T>& V = vel_hier<T>(w);
  Hier<T>& Q = q1_hier<T>(w);
  if (!V.built) ETH_TRY(mg_build_vel<T>(g, V, nmin, g->kind == ETH_OSEEN ? 0.5 : 0.0, false));
  const double om = o->mg_omega > 0.0 ? o->mg_omega : 0.9;   // 0.9: fewest iterations, Stokes 256^2 / 512^2
  if (V.omega != om) {   // the captured graph holds the damping as a kernel argument
    V.omega = om;
    if (w->gexec) { cudaGraphExecDestroy(w->gexec); w->gexec = nullptr; w->gkey = -1; }
  }
  if (g->kind == ETH_OSEEN && w->need_adj) {
    Hier<T>& Vt = vel_hier_t<T>(w);
    if (!Vt.built) ETH_TRY(mg_build_vel<T>(g, Vt, nmin, 0.5, true));
    Vt.omega = om;
  }
  if (!Q.built) ETH_TRY(mg_build_q1<T>(g, Q, nmin));
  return ETH_OK;
}

// ||b - K x||^2 in FP64 (K applied with FP64 element arithmetic); result to host.
eth_status true_residual(eth_grid* g, Work* w, const double* b, double* rr, bool trans) {
  ETH_TRY(op_apply_K(g, false, trans, w->x, w->Kz, nullptr));
  const int nb = vblocks(g->nt);
  k_residual<<<nb, 256, 0, g->s>>>((size_t)g->nt, b, w->Kz, w->r, slot_of(g, SL_NORM, nb, FIN_STORE));
  ETH_CUDA(cudaGetLastError());
  ETH_CUDA(cudaMemcpyAsync(&g->sch->dots[SL_NORM], &g->sc->dots[SL_NORM], 8, cudaMemcpyDeviceToHost, g->s));
  ETH_CUDA(cudaStreamSynchronize(g->s));
  *rr = g->sch->dots[SL_NORM];
  g->launches += 1;
  return ETH_OK;
}

// remove the e1 / e0 components of the pressure block of x (Euclidean)
eth_status canonicalize(eth_grid* g, double* x) {
  const int nb = vblocks((size_t)g->n1 + g->n0);
  const size_t off = 2 * (size_t)g->nv;
  k_psums<0><<<nb, 256, 0, g->s>>>(off, (size_t)g->n1, (size_t)g->n0, x, slot_of(g, SL_PSUM, nb, FIN_STORE));
  ETH_CUDA(cudaGetLastError());
  k_psub<<<nb, 256, 0, g->s>>>(off, (size_t)g->n1, (size_t)g->n0, x, &g->sc->dots[SL_PSUM]);
  ETH_CUDA(cudaGetLastError());
  g->launches += 2;
  return ETH_OK;
}

// After canonicalize(g, bp): the size of the null-space component that was removed,
// sqrt(s1^2 / n1 + s0^2 / n0) with s1, s0 the removed block sums, and ||bp||.
eth_status rhs_inconsistency(eth_grid* g, Work* w, const double* bp, double* incons, double* nbp) {
  const size_t nt = g->nt;
  const int nb = vblocks(nt);
  ETH_CUDA(cudaMemsetAsync(w->Kz, 0, nt * 8, g->s));
  k_residual<<<nb, 256, 0, g->s>>>(nt, bp, w->Kz, w->r, slot_of(g, SL_NORM, nb, FIN_STORE));
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  ETH_CUDA(cudaMemcpyAsync(g->sch->dots, g->sc->dots, sizeof(g->sc->dots), cudaMemcpyDeviceToHost, g->s));
  ETH_CUDA(cudaStreamSynchronize(g->s));
  *nbp = std::sqrt(g->sch->dots[SL_NORM]);
  *incons = std::sqrt(g->sch->dots[SL_PSUM] * g->sch->dots[SL_PSUM] / g->n1 +
                      g->sch->dots[SL_PSUM + 1] * g->sch->dots[SL_PSUM + 1] / g->n0);
  return ETH_OK;
}

// Attaches the grid's Lanczos buffers to its scalars and restarts the recording.
__global__ void k_lz_begin(Scalars* sc, double* lz, int cap) {
  ETH_GRID_DEP_WAIT();
  sc->lz_delta = lz;
  sc->lz_gamma = lz + cap;
  sc->lz_cap = cap;
  sc->lz_runs = 0;
  sc->lz_n = 0;
}

template <class T>
static eth_status stokes_solve(eth_grid* g, Work* w, const eth_opts* o, eth_stats* st, const double* bsrc) {
  const size_t nt = g->nt;
  const bool fp32 = o->precision == ETH_MIXED;
  k_lz_begin<<<1, 1, 0, g->s>>>(g->sc, g->lz, ETH_LANCZOS_CAP);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  // consistent right-hand side: b with its e1 / e0 components removed
  ETH_CUDA(cudaMemcpyAsync(w->bp, bsrc, nt * 8, cudaMemcpyDeviceToDevice, g->s));
  ETH_TRY(canonicalize(g, w->bp));
  ETH_CUDA(cudaMemcpyAsync(g->sch->dots, g->sc->dots, sizeof(g->sc->dots), cudaMemcpyDeviceToHost, g->s));
  double bb = 0.0;
  {
    const int nb = vblocks(nt);
    ETH_CUDA(cudaMemsetAsync(w->Kz, 0, nt * 8, g->s));
    k_residual<<<nb, 256, 0, g->s>>>(nt, w->bp, w->Kz, w->r, slot_of(g, SL_NORM, nb, FIN_STORE));
    ETH_CUDA(cudaGetLastError());
    g->launches++;
    ETH_CUDA(cudaMemcpyAsync(&g->sch->dots[SL_NORM], &g->sc->dots[SL_NORM], 8, cudaMemcpyDeviceToHost, g->s));
    ETH_CUDA(cudaStreamSynchronize(g->s));
    bb = g->sch->dots[SL_NORM];
  }
  const double nb2 = std::sqrt(bb);
  const double incons = std::sqrt(g->sch->dots[SL_PSUM] * g->sch->dots[SL_PSUM] / g->n1 +
                                  g->sch->dots[SL_PSUM + 1] * g->sch->dots[SL_PSUM + 1] / g->n0);
  eth_status result = ETH_OK;
  if (!std::isfinite(nb2)) {  // NaN or Inf in the right-hand side: nothing to solve
    st->relres_true = nb2;
    return ETH_ENAN;
  }
  if (nb2 > 0 && incons > 1e-8 * nb2) result = ETH_EINCONSISTENT;
  if (!(nb2 > 0.0)) {  // zero right-hand side: x = 0
    ETH_CUDA(cudaMemsetAsync(w->x, 0, nt * 8, g->s));
    st->relres_true = 0.0;
    return ETH_OK;
  }
  double rr;
  ETH_TRY(true_residual(g, w, w->bp, &rr));
  st->relres0 = std::sqrt(rr) / nb2;
  double rel = st->relres0;
  int total = 0, passes = 0;
  const double inner_floor = fp32 ? o->refine_inner_tol : 0.0;
  while (rel > o->tol && total < o->maxit) {
    if (!std::isfinite(rel)) { result = ETH_ENAN; break; }
    double itol = 0.3 * o->tol / rel;
    itol = std::max(itol, inner_floor);
    itol = std::min(itol, 0.5);
    int its = 0, ds = 0;
    ETH_TRY(minres_solve<T>(g, w, o, fp32, itol, o->maxit - total, &its, &ds));
    total += its;
    passes++;
    const int nb = vblocks(nt);
    k_add<<<nb, 256, 0, g->s>>>(nt, w->x, w->d);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
    ETH_TRY(canonicalize(g, w->x));
    ETH_TRY(true_residual(g, w, w->bp, &rr));
    rel = std::sqrt(rr) / nb2;
    if (o->verbose) fprintf(stderr, "[eth] pass %d: inner its %d (tol %.1e) relres %.3e status %d\n", passes, its, itol, rel, ds);
    if (ds == ETH_EBREAKDOWN && its == 0) { result = ETH_EBREAKDOWN; break; }
    if (its == 0) break;
  }
  st->iters_total = total;
  st->iters_stage1 = total;
  st->refine_passes = passes;
  st->relres_true = rel;
  if (result == ETH_OK && rel > o->tol) result = std::isfinite(rel) ? ETH_ENOTCONV : ETH_ENAN;
  return result;
}

template eth_status ensure_hier<float>(eth_grid*, Work*, const eth_opts*);
template eth_status ensure_hier<double>(eth_grid*, Work*, const eth_opts*);

eth_status adjoint_gradients(eth_grid* g, Work* w, const double* lu, const double* u, double* grad_f, double* grad_nu) {
  return grad_kernels(g, lu, u, grad_f, w->r, w->Kz, grad_nu);
}

}  // namespace eth

using namespace eth;

extern "C" {

eth_status eth_solve(eth_grid* g, const eth_opts* opts, double* u, double* p, eth_stats* stats) {
  if (!g || !u || !p) { set_error("eth_solve: NULL argument"); return ETH_EINVAL; }
  if (!g->has_rhs) { set_error("eth_solve: no right-hand side (eth_set_rhs)"); return ETH_EINVAL; }
  eth_opts o;
  if (opts) o = *opts; else eth_default_opts(&o);
  if (!(o.tol > 0) || o.maxit < 1 || o.mg_pre < 1 || o.mg_post < 1 || o.mg_pre > 64 || o.mg_post > 64 ||
      !(o.mg_omega >= 0.0 && o.mg_omega < 2.0)) {
    set_error("eth_solve: bad options");
    return ETH_EINVAL;
  }
  if ((o.a_exact || o.mq_mode == ETH_MQ_EXACT) && !(o.inner_tol > 0)) { set_error("eth_solve: bad inner_tol"); return ETH_EINVAL; }
  if (o.mq_mode < 0 || o.mq_mode > 2 || o.mq_cheb_steps < 0 || o.mq_cheb_steps > 1000 || !(o.mq_cheb_a >= 0.0 && o.mq_cheb_a < 1.0)) {
    set_error("eth_solve: bad mq_mode / mq_cheb_steps / mq_cheb_a");
    return ETH_EINVAL;
  }
  if (o.precision != ETH_FP64 && o.precision != ETH_MIXED) { set_error("eth_solve: bad precision"); return ETH_EINVAL; }
  if (o.oseen_prec < 0 || o.oseen_prec > 1 || o.lsc_cg < 0 || o.lsc_cg > 100) {
    set_error("eth_solve: oseen_prec must be 0 or 1 and lsc_cg in 0..100");
    return ETH_EINVAL;
  }
  ETH_ON_DEVICE(g);
  eth_stats st;
  std::memset(&st, 0, sizeof(st));
  Work* w;
  ETH_TRY(work_get(g, &w));
  StreamSwap guard(g, w);
  if (o.precision == ETH_MIXED) ETH_TRY(ensure_hier<float>(g, w, &o)); else ETH_TRY(ensure_hier<double>(g, w, &o));
  if (o.a_exact || o.mq_mode == ETH_MQ_EXACT) ETH_TRY(ensure_pcg(g, w));
  if (o.mq_mode == ETH_MQ_CHEB)   // workspace before the solver graph is captured
    ETH_TRY(o.precision == ETH_MIXED ? mqcheb_prepare<float>(g, w) : mqcheb_prepare<double>(g, w));
  if (o.autotune) ETH_TRY(tune_tiles(g, o.precision == ETH_MIXED));
  const long l0 = g->launches;
  ETH_CUDA(cudaEventRecord(w->t0, g->s));
  const size_t nu2 = 2 * (size_t)g->nv;
  ETH_CUDA(cudaMemcpyAsync(w->x, u, nu2 * 8, cudaMemcpyDeviceToDevice, g->s));
  ETH_CUDA(cudaMemcpyAsync(w->x + nu2, p, (size_t)(g->n1 + g->n0) * 8, cudaMemcpyDeviceToDevice, g->s));
  k_set_boundary<<<vblocks(nu2), 256, 0, g->s>>>(g->n, w->x, g->ubc);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  eth_status r;
  if (g->kind == ETH_OSEEN) r = oseen_solve(g, w, &o, &st, false, g->b);
  else r = o.precision == ETH_MIXED ? stokes_solve<float>(g, w, &o, &st, g->b) : stokes_solve<double>(g, w, &o, &st, g->b);
  if (r == ETH_ECUDA || r == ETH_ENOMEM || r == ETH_EINVAL) return r;
  ETH_CUDA(cudaMemcpyAsync(u, w->x, nu2 * 8, cudaMemcpyDeviceToDevice, g->s));
  ETH_CUDA(cudaMemcpyAsync(p, w->x + nu2, (size_t)(g->n1 + g->n0) * 8, cudaMemcpyDeviceToDevice, g->s));
  ETH_CUDA(cudaEventRecord(w->t1, g->s));
  ETH_CUDA(cudaEventSynchronize(w->t1));
  float ms = 0.f;
  ETH_CUDA(cudaEventElapsedTime(&ms, w->t0, w->t1));
  st.seconds = ms * 1e-3;
  st.status = r;
  st.kernel_launches = (int)(g->launches - l0);
  st.tile_rows = tile_rows(g);
  st.tile_persistent = tile_strip(g) ? 2 : (tile_persistent(g) && o.precision == ETH_MIXED);
  if (stats) *stats = st;
  return r;
}

eth_status eth_solve_host(eth_grid* g, const eth_opts* opts, const double* f, const double* ub, double* u, double* p,
                          eth_stats* stats) {
  if (!g || !f || !ub || !u || !p) { set_error("eth_solve_host: NULL argument"); return ETH_EINVAL; }
  ETH_ON_DEVICE(g);
  Work* w;
  ETH_TRY(work_get(g, &w));
  const size_t nu2 = 2 * (size_t)g->nv, np = (size_t)g->n1 + g->n0;
  double *fd = w->Kz, *ud = w->r;   // staging: f and u_b (re-used scratch)
  ETH_CUDA(cudaMemcpyAsync(fd, f, nu2 * 8, cudaMemcpyHostToDevice, g->s));
  ETH_CUDA(cudaMemcpyAsync(ud, ub, nu2 * 8, cudaMemcpyHostToDevice, g->s));
  ETH_TRY(eth_set_rhs(g, fd, ud));
  double* uo = w->V[0];
  double* po = w->V[1];
  ETH_CUDA(cudaMemsetAsync(uo, 0, nu2 * 8, g->s));
  ETH_CUDA(cudaMemsetAsync(po, 0, np * 8, g->s));
  eth_status r = eth_solve(g, opts, uo, po, stats);
  if (r != ETH_OK && r != ETH_ENOTCONV) return r;
  ETH_CUDA(cudaMemcpyAsync(u, uo, nu2 * 8, cudaMemcpyDeviceToHost, g->s));
  ETH_CUDA(cudaMemcpyAsync(p, po, np * 8, cudaMemcpyDeviceToHost, g->s));
  ETH_CUDA(cudaStreamSynchronize(g->s));
  return r;
}

eth_status eth_solve_adjoint(eth_grid* g, const eth_opts* opts, const double* ru, const double* rp, double* lu, double* lp,
                             eth_stats* stats) {
  if (!g || !ru || !rp || !lu || !lp) { set_error("eth_solve_adjoint: NULL argument"); return ETH_EINVAL; }
  if (!g->has_coef) { set_error("eth_solve_adjoint: call eth_set_coefficients first"); return ETH_EINVAL; }
  eth_opts o;
  if (opts) o = *opts; else eth_default_opts(&o);
  if (!(o.tol > 0) || o.maxit < 1 || o.mg_pre < 1 || o.mg_post < 1 || o.mg_pre > 64 || o.mg_post > 64 ||
      !(o.mg_omega >= 0.0 && o.mg_omega < 2.0) || o.oseen_prec < 0 || o.oseen_prec > 1 || o.lsc_cg < 0 ||
      o.lsc_cg > 100) {
    set_error("eth_solve_adjoint: bad options");
    return ETH_EINVAL;
  }
  ETH_ON_DEVICE(g);
  eth_stats st;
  std::memset(&st, 0, sizeof(st));
  Work* w;
  ETH_TRY(work_get(g, &w));
  StreamSwap guard(g, w);
  w->need_adj = true;
  if (o.precision == ETH_MIXED) ETH_TRY(ensure_hier<float>(g, w, &o)); else ETH_TRY(ensure_hier<double>(g, w, &o));
  if (o.autotune) ETH_TRY(tune_tiles(g, o.precision == ETH_MIXED));
  const long l0 = g->launches;
  ETH_CUDA(cudaEventRecord(w->t0, g->s));
  const size_t nu2 = 2 * (size_t)g->nv, np = (size_t)g->n1 + g->n0;
  // right-hand side [r_u; r_p] (boundary rows of K^T are identity rows: l_B = r_B)
  ETH_CUDA(cudaMemcpyAsync(w->d, ru, nu2 * 8, cudaMemcpyDeviceToDevice, g->s));
  ETH_CUDA(cudaMemcpyAsync(w->d + nu2, rp, np * 8, cudaMemcpyDeviceToDevice, g->s));
  ETH_CUDA(cudaMemsetAsync(w->x, 0, (size_t)g->nt * 8, g->s));
  k_set_boundary<<<vblocks(nu2), 256, 0, g->s>>>(g->n, w->x, w->d);
  ETH_CUDA(cudaGetLastError());
  ETH_CUDA(cudaMemcpyAsync(w->Kz, w->d, (size_t)g->nt * 8, cudaMemcpyDeviceToDevice, g->s));
  eth_status r;
  if (g->kind == ETH_OSEEN) r = oseen_solve(g, w, &o, &st, true, w->Kz);
  else r = o.precision == ETH_MIXED ? stokes_solve<float>(g, w, &o, &st, w->Kz) : stokes_solve<double>(g, w, &o, &st, w->Kz);
  if (r == ETH_ECUDA || r == ETH_ENOMEM || r == ETH_EINVAL) return r;
  ETH_CUDA(cudaMemcpyAsync(lu, w->x, nu2 * 8, cudaMemcpyDeviceToDevice, g->s));
  ETH_CUDA(cudaMemcpyAsync(lp, w->x + nu2, np * 8, cudaMemcpyDeviceToDevice, g->s));
  ETH_CUDA(cudaEventRecord(w->t1, g->s));
  ETH_CUDA(cudaEventSynchronize(w->t1));
  float ms = 0.f;
  ETH_CUDA(cudaEventElapsedTime(&ms, w->t0, w->t1));
  st.seconds = ms * 1e-3;
  st.status = r;
  st.kernel_launches = (int)(g->launches - l0);
  st.tile_rows = tile_rows(g);
  st.tile_persistent = tile_strip(g) ? 2 : (tile_persistent(g) && o.precision == ETH_MIXED);
  if (stats) *stats = st;
  return r;
}

eth_status eth_adjoint_gradients(eth_grid* g, const double* lu, const double* u, double* grad_f, double* grad_nu) {
  if (!g || !lu || !u || !grad_f || !grad_nu) { set_error("eth_adjoint_gradients: NULL argument"); return ETH_EINVAL; }
  ETH_ON_DEVICE(g);
  Work* w;
  ETH_TRY(work_get(g, &w));
  StreamSwap guard(g, w);
  ETH_TRY(adjoint_gradients(g, w, lu, u, grad_f, grad_nu));
  return ETH_OK;
}

eth_status eth_batch_create(int count, eth_grid* const* grids, eth_batch** out) {
  if (!out) { set_error("eth_batch_create: out is NULL"); return ETH_EINVAL; }
  *out = nullptr;
  if (count < 1 || !grids) { set_error("eth_batch_create: empty batch"); return ETH_EINVAL; }
  for (int i = 0; i < count; ++i)
    if (!grids[i]) { set_error("eth_batch_create: grid %d is NULL", i); return ETH_EINVAL; }
  eth_batch* b = new eth_batch();
  b->grids.assign(grids, grids + count);
  *out = b;
  return ETH_OK;
}

// Independent instances run concurrently: one host worker per instance slot
// drives that instance's captured-graph solve on its own internal streams, so
// the GPU overlaps the instances' kernels.  Instances are handed out largest
// first (cost ~ N_t) to balance the workers.
eth_status eth_batch_solve(eth_batch* b, const eth_opts* opts, double* const* u, double* const* p, eth_stats* stats) {
  if (!b || !u || !p) { set_error("eth_batch_solve: NULL argument"); return ETH_EINVAL; }
  const int count = (int)b->grids.size();
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int c) { return b->grids[a]->nt > b->grids[c]->nt; });
  std::vector<eth_status> st(count, ETH_OK);
  std::vector<eth_stats> ss(count);
  std::atomic<int> next{0};
  const int nw = std::max(1, std::min(count, b->workers > 0 ? b->workers : 16));
  // the autotuner times kernels: run it for every instance before the workers overlap them
  eth_opts o;
  if (opts) o = *opts; else eth_default_opts(&o);
  if (o.autotune)
    for (int i : order) {
      eth_grid* g = b->grids[i];
      ETH_ON_DEVICE(g);
      ETH_TRY(tune_tiles(g, o.precision == ETH_MIXED));
      if (g->kind == ETH_OSEEN) {   // the Gram-Schmidt tuner as well (GMRES workspace first)
        Work* w;
        ETH_TRY(work_get(g, &w));
        ETH_TRY(oseen_prepare(g, w, &o));
      }
    }
  auto worker = [&]() {   // eth_solve makes each instance's device current
    while (true) {
      const int k = next.fetch_add(1);
      if (k >= count) break;
      const int i = order[k];
      std::memset(&ss[i], 0, sizeof(eth_stats));
      st[i] = eth_solve(b->grids[i], opts, u[i], p[i], &ss[i]);
    }
  };
  std::vector<std::thread> th;
  for (int t = 0; t < nw; ++t) th.emplace_back(worker);
  for (auto& t : th) t.join();
  eth_status r = ETH_OK;
  for (int i = 0; i < count; ++i) {
    if (stats) stats[i] = ss[i];
    if (st[i] != ETH_OK && r == ETH_OK) r = st[i];
  }
  if (r != ETH_OK) set_error("eth_batch_solve: at least one instance returned %s", eth_status_string(r));
  return r;
}

void eth_batch_destroy(eth_batch* b) { delete b; }

// Picard iteration for steady Navier-Stokes (Sec. 3): each step is an Oseen solve
// whose wind is the previous velocity (zero wind first, i.e. the Stokes problem).
// After each step the coefficients are set to the new velocity, so the next step's
// system is in place, and the nonlinear residual ||b(u) - K(u)[u; p]|| / ||b(u)||
// is evaluated with FP64 element arithmetic.
eth_status eth_picard(eth_grid* g, const eth_opts* opts, const double* f_nodal, const double* ubc, int steps,
                      double* u, double* p, double* nlres, eth_stats* stats) {
  if (!g || !f_nodal || !ubc || !u || !p) { set_error("eth_picard: NULL argument"); return ETH_EINVAL; }
  if (g->kind != ETH_OSEEN) { set_error("eth_picard: the grid must be created as ETH_OSEEN"); return ETH_EINVAL; }
  if (!g->has_coef) { set_error("eth_picard: call eth_set_coefficients first (viscosity)"); return ETH_EINVAL; }
  if (steps < 1) { set_error("eth_picard: steps=%d must be >= 1", steps); return ETH_EINVAL; }
  ETH_ON_DEVICE(g);
  const size_t nu2 = 2 * (size_t)g->nv, np = (size_t)g->n1 + g->n0, nt = g->nt;
  const double nu = g->nu;
  ETH_CUDA(cudaMemsetAsync(u, 0, nu2 * 8, g->s));
  ETH_CUDA(cudaMemsetAsync(p, 0, np * 8, g->s));
  ETH_CUDA(cudaMemsetAsync(g->tmp, 0, nu2 * 8, g->s));   // zero wind of the first step
  ETH_TRY(eth_set_coefficients(g, nu, g->tmp));
  ETH_TRY(eth_set_rhs(g, f_nodal, ubc));
  Work* w;
  ETH_TRY(work_get(g, &w));
  for (int k = 0; k < steps; ++k) {
    eth_stats st;
    std::memset(&st, 0, sizeof(st));
    const eth_status r = eth_solve(g, opts, u, p, &st);
    if (stats) stats[k] = st;
    if (r != ETH_OK && r != ETH_ENOTCONV && r != ETH_EINCONSISTENT) return r;
    // linearise at the new iterate (this is also the next step's system) and measure it there
    ETH_TRY(eth_set_coefficients(g, nu, u));
    ETH_TRY(eth_set_rhs(g, f_nodal, ubc));
    if (nlres) {
      ETH_CUDA(cudaMemcpyAsync(g->tmp, u, nu2 * 8, cudaMemcpyDeviceToDevice, g->s));
      ETH_CUDA(cudaMemcpyAsync(g->tmp + nu2, p, np * 8, cudaMemcpyDeviceToDevice, g->s));
      ETH_TRY(op_apply(g, ETH_OP_K, false, g->tmp, g->tmp2));
      double incons = 0.0, nb = 0.0;
      ETH_TRY(rhs_inconsistency(g, w, g->b, &incons, &nb));
      const int nbk = vblocks(nt);
      k_residual<<<nbk, 256, 0, g->s>>>(nt, g->b, g->tmp2, w->r, slot_of(g, SL_NORM, nbk, FIN_STORE));
      ETH_CUDA(cudaGetLastError());
      ETH_CUDA(cudaMemcpyAsync(&g->sch->dots[SL_NORM], &g->sc->dots[SL_NORM], 8, cudaMemcpyDeviceToHost, g->s));
      ETH_CUDA(cudaStreamSynchronize(g->s));
      nlres[k] = nb > 0.0 ? std::sqrt(g->sch->dots[SL_NORM]) / nb : 0.0;
    }
  }
  return ETH_OK;
}
}
