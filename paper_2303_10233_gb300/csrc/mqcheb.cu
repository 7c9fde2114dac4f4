// Chebyshev semi-iteration on multicolour symmetric Gauss-Seidel for the singular
// two-level pressure mass matrix M_Q = [Qk R^T; R Q0]: the cheap M_Q block of the
// preconditioner P_2 (Sec. 2.3-2.4; 20 steps in the paper).
//
// Symmetric Gauss-Seidel P = (D + L) D^{-1} (D + L^T) in the order of five colours:
// the four parity classes (I mod 2, J mod 2) of the Q1 nodes (colour 2 (J mod 2) +
// (I mod 2)), then every P0 element.  Unknowns of one colour are not coupled in M_Q,
// so one kernel per colour performs its part of the sweep exactly: forward over the
// colours (each node uses the already updated nodes of earlier colours), then back
// (each node uses the result of later colours).  A Q1 node couples to its eight Q1
// neighbours through Qk (element masses |T| m_a m_b, 1D linear mass (1/3, 1/6)) and to
// its four elements through R (|T| / 4); an element couples to its four vertices.
//
// Chebyshev on [a, b] for the eigenvalues of P^{-1} M_Q (0 along k excluded; b = 1):
// x += d, r -= M_Q d, d = rho_{k+1} rho_k d + (2 rho_{k+1} / delta) P^{-1} r, with
// theta = (a + b)/2, delta = (b - a)/2, rho_0 = delta / theta, rho_{k+1} =
// 1 / (2 theta / delta - rho_k), d_0 = P^{-1} r / theta.  The right-hand side loses
// its k component first and the output is projected orthogonal to k (Euclidean).
#include <algorithm>
#include <cmath>
#include "solve.cuh"

namespace eth {

// Q1-Q1 coupling of M_Q between nodes (I, J) and (I + dx, J + dy), dx, dy in {-1, 0, 1}:
// the sum over the shared elements of |T| m(c, c') m(d, d') (c, c' the local x corners)
__device__ __forceinline__ int mc_colour(int I, int J) { return 2 * (J & 1) + (I & 1); }

// forward sweep over the Q1 colour col: y = (r - sum_{earlier colours} Qk y) / Qk_diag
template <class T>
__global__ void k_sgs_f1(int n, int col, T area, const T* __restrict__ r, T* __restrict__ y, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  const int M = n + 1, ci = col & 1, cj = col >> 1;
  const int nx = (M - ci + 1) / 2, ny = (M - cj + 1) / 2;   // nodes of this colour per direction
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nx * ny; k += gridDim.x * blockDim.x) {
    const int J = 2 * (k / nx) + cj, I = 2 * (k % nx) + ci;
    T s = 0, dg = 0;
    Q1_FOR_ELEMENTS(n, I, J, {
#pragma unroll
      for (int dd = 0; dd < 2; ++dd)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const T mij = area * (T)(q1m(c, cc) * q1m(d, dd));
          if (cc == c && dd == d) { dg += mij; continue; }
          const int In = I + cc - c, Jn = J + dd - d;
          if (mc_colour(In, Jn) < col) s += mij * y[Jn * M + In];
        }
    })
    const int node = J * M + I;
    y[node] = (r[node] - s) / dg;
  }
}

// forward sweep over the P0 elements (last colour): y0 = (r0 - R y) / |T| =
// r0 / |T| - (sum of the four vertex values) / 4; the backward sweep leaves P0
// unchanged (no later colour), so the result goes to z as well
template <class T>
__global__ void k_sgs_f0(int n, T area, const T* __restrict__ r, T* __restrict__ y, T* __restrict__ z, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  const int M = n + 1, n1 = M * M;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int ey = e / n, ex = e - ey * n;
    const T s = y[ey * M + ex] + y[ey * M + ex + 1] + y[(ey + 1) * M + ex] + y[(ey + 1) * M + ex + 1];
    const T v = r[n1 + e] / area - T(0.25) * s;
    y[n1 + e] = v;
    z[n1 + e] = v;
  }
}

// backward sweep over the Q1 colour col: z = y - (sum_{later Q1 colours} Qk z + R^T z0) / Qk_diag
template <class T>
__global__ void k_sgs_b1(int n, int col, T area, const T* __restrict__ y, T* __restrict__ z, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  const int M = n + 1, n1 = M * M, ci = col & 1, cj = col >> 1;
  const int nx = (M - ci + 1) / 2, ny = (M - cj + 1) / 2;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nx * ny; k += gridDim.x * blockDim.x) {
    const int J = 2 * (k / nx) + cj, I = 2 * (k % nx) + ci;
    T s = 0, dg = 0;
    Q1_FOR_ELEMENTS(n, I, J, {
      s += T(0.25) * area * z[n1 + ey * n + ex];
#pragma unroll
      for (int dd = 0; dd < 2; ++dd)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const T mij = area * (T)(q1m(c, cc) * q1m(d, dd));
          if (cc == c && dd == d) { dg += mij; continue; }
          const int In = I + cc - c, Jn = J + dd - d;
          if (mc_colour(In, Jn) > col) s += mij * z[Jn * M + In];
        }
    })
    const int node = J * M + I;
    z[node] = y[node] - s / dg;
  }
}

// r = [v_k - beta; v_0 + beta] (the right-hand side without its k component), x = 0
template <class T>
__global__ void k_mc_init(int n1, int m, const double* __restrict__ v, const double* beta_p, T* __restrict__ r,
                          T* __restrict__ x, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  const double beta = *beta_p;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    r[k] = (T)(k < n1 ? v[k] - beta : v[k] + beta);
    x[k] = 0;
  }
}

// x += d ; r -= q
template <class T>
__global__ void k_mc_xr(int m, const T* __restrict__ d, const T* __restrict__ q, T* __restrict__ x, T* __restrict__ r,
                        const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    x[k] += d[k];
    r[k] -= q[k];
  }
}

// d = c1 d + c2 w (c1 = 0: d = c2 w without reading d, which may hold anything on the first step)
template <class T>
__global__ void k_mc_d(int m, T c1, T c2, const T* __restrict__ w, T* __restrict__ d, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x)
    d[k] = (c1 == T(0) ? T(0) : c1 * d[k]) + c2 * w[k];
}

// k^T x = sum over Q1 - sum over P0 -> sl
template <class T>
__global__ void k_mc_ksum(int n1, int m, const T* __restrict__ x, Slot sl, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  double s = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) s += k < n1 ? (double)x[k] : -(double)x[k];
  double v[1] = {s};
  if (slot_arrive<1>(sl, blockIdx.x, v)) finish_slot(sl, v[0]);
}

// zp = scale (x - (k^T x / k^T k) k) in FP64; with gsl, <zp, v> partials at goff (the
// fused gamma of MINRES)
template <class T>
__global__ void k_mc_out(int n1, int m, const T* __restrict__ x, const double* ksum, const double* scale_p, double scale,
                         double* __restrict__ zp, const double* __restrict__ v, Slot gsl, int goff, int dot, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  const double mu = *ksum / m, sc = scale_p ? *scale_p : scale;
  double acc = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    const double z = sc * ((double)x[k] - (k < n1 ? mu : -mu));
    zp[k] = z;
    if (dot) acc += z * v[k];
  }
  if (dot) {
    double a[1] = {acc};
    if (slot_arrive<1>(gsl, goff + blockIdx.x, a)) finish_slot(gsl, a[0]);
  }
}

// beta = k^T r / k^T k for an FP64 frame vector r (k = [1; -1]) -> sl.out[0]
__global__ void k_mc_load_beta(int n1, int m, const double* __restrict__ r, Slot sl) {
  ETH_GRID_DEP_WAIT();
  double s = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) s += k < n1 ? r[k] : -r[k];
  double v[1] = {s};
  if (slot_arrive<1>(sl, blockIdx.x, v)) sl.out[0] = v[0] / m;
}

template <class T>
struct McWork {
  T *r = nullptr, *x = nullptr, *d = nullptr, *w = nullptr, *y = nullptr, *q = nullptr;
};

template <class T>
static void mc_free_t(McWork<T>* M) {
  if (!M) return;
  cudaFree(M->r); cudaFree(M->x); cudaFree(M->d); cudaFree(M->w); cudaFree(M->y); cudaFree(M->q);
  delete M;
}

void mqcheb_free(Work* w) {
  mc_free_t(static_cast<McWork<float>*>(w->mcw[0]));
  mc_free_t(static_cast<McWork<double>*>(w->mcw[1]));
  w->mcw[0] = w->mcw[1] = nullptr;
}

template <class T>
static eth_status mc_get(eth_grid* g, Work* w, McWork<T>** out) {
  void*& slot = w->mcw[sizeof(T) == 4 ? 0 : 1];
  if (!slot) {
    McWork<T>* M = new McWork<T>();
    slot = M;
    const size_t m = (size_t)g->n1 + g->n0;
    ETH_CUDA(cudaMalloc((void**)&M->r, m * sizeof(T)));
    ETH_CUDA(cudaMalloc((void**)&M->x, m * sizeof(T)));
    ETH_CUDA(cudaMalloc((void**)&M->d, m * sizeof(T)));
    ETH_CUDA(cudaMalloc((void**)&M->w, m * sizeof(T)));
    ETH_CUDA(cudaMalloc((void**)&M->y, m * sizeof(T)));
    ETH_CUDA(cudaMalloc((void**)&M->q, m * sizeof(T)));
  }
  *out = static_cast<McWork<T>*>(slot);
  return ETH_OK;
}

template <class T>
eth_status mqcheb_prepare(eth_grid* g, Work* w) {
  McWork<T>* M = nullptr;
  return mc_get<T>(g, w, &M);
}

// z = P^{-1} r (one multicolour symmetric Gauss-Seidel sweep pair), y scratch
template <class T>
static eth_status sgs(eth_grid* g, const T* r, T* y, T* z, const int* done, cudaStream_t s) {
  const T area = (T)(g->hx * g->hy);
  const int nq = std::max(1, vblocks((size_t)(g->n1 + 3) / 4)), n0b = vblocks((size_t)g->n0);
  for (int col = 0; col < 4; ++col) k_sgs_f1<T><<<nq, 256, 0, s>>>(g->n, col, area, r, y, done);
  k_sgs_f0<T><<<n0b, 256, 0, s>>>(g->n, area, r, y, z, done);
  for (int col = 3; col >= 0; --col) k_sgs_b1<T><<<nq, 256, 0, s>>>(g->n, col, area, y, z, done);
  ETH_CUDA(cudaGetLastError());
  g->launches += 9;
  return ETH_OK;
}

// q = M_Q d
template <class T>
static eth_status mq_apply(eth_grid* g, const T* d, T* q, const int* done, cudaStream_t s) {
  Q1Params<T, T, T> P{};
  P.n = g->n; P.hx = (T)g->hx; P.hy = (T)g->hy;
  P.cm = 1; P.ck = 0; P.c1 = 0; P.x = d; P.x0 = d + g->n1; P.r0 = 1; P.y = q; P.done = done;
  k_q1node<T, T, T, Q1E_APPLY><<<q1_blocks(g->n), 256, 0, s>>>(P);
  k_p0rows<T, T, T><<<vblocks((size_t)g->n0), 256, 0, s>>>(g->n, (T)(g->hx * g->hy), (T)1, (T)1, d, d + g->n1, q + g->n1, done);
  ETH_CUDA(cudaGetLastError());
  g->launches += 2;
  return ETH_OK;
}

// x = `steps` Chebyshev-SGS steps for M_Q x = r on [a, b], x_0 = 0 (M->r holds r and
// ends as the residual)
template <class T>
static eth_status mc_chebyshev(eth_grid* g, McWork<T>* M, int steps, double a, double b, const int* done, cudaStream_t s) {
  const int m = g->n1 + g->n0, nb = vblocks((size_t)m);
  const double theta = 0.5 * (b + a), delta = 0.5 * (b - a), sigma = theta / delta;
  double rho = 1.0 / sigma;
  ETH_TRY(sgs<T>(g, M->r, M->y, M->w, done, s));
  k_mc_d<T><<<nb, 256, 0, s>>>(m, T(0), (T)(1.0 / theta), M->w, M->d, done);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  for (int k = 0; k < steps; ++k) {
    ETH_TRY(mq_apply<T>(g, M->d, M->q, done, s));
    k_mc_xr<T><<<nb, 256, 0, s>>>(m, M->d, M->q, M->x, M->r, done);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
    if (k + 1 == steps) break;
    const double rn = 1.0 / (2.0 * sigma - rho);
    ETH_TRY(sgs<T>(g, M->r, M->y, M->w, done, s));
    k_mc_d<T><<<nb, 256, 0, s>>>(m, (T)(rn * rho), (T)(2.0 * rn / delta), M->w, M->d, done);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
    rho = rn;
  }
  return ETH_OK;
}

// Smallest nonzero eigenvalue of P^{-1} M_Q used when none is given: it scales like
// h^2; on square elements of an n x n grid it is close to 0.655 / n^2 (computed by a
// dense generalised eigen-solve at n = 8, 16, 32: 0.666, 0.666, 0.655 times 1/n^2)
double mqcheb_default_a(const eth_grid* g) { return 0.655 / ((double)g->n * g->n); }

// MINRES pressure block with M_Q^+ replaced by M_cheb: zp = nu M_cheb^{-1}(v_p - beta k),
// projected orthogonal to k, <zp, v_p> partials into gsl at goff (the P_2 form)
template <class T>
eth_status precond_pressure_cheb(eth_grid* g, Work* w, const eth_opts* o, const double* vp, double* zp, const Slot& gsl,
                                 int goff, const int* done, cudaStream_t s) {
  McWork<T>* M = nullptr;
  ETH_TRY(mc_get<T>(g, w, &M));
  const int m = g->n1 + g->n0, nb = vblocks((size_t)m);
  const double a = o->mq_cheb_a > 0.0 ? o->mq_cheb_a : mqcheb_default_a(g);
  k_mc_init<T><<<nb, 256, 0, s>>>(g->n1, m, vp, &g->sc->v[S_BETA], M->r, M->x, done);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  ETH_TRY(mc_chebyshev<T>(g, M, o->mq_cheb_steps > 0 ? o->mq_cheb_steps : 20, a, 1.0, done, s));
  Slot ks = slot_of(g, SL_MQ, nb, FIN_STORE);
  k_mc_ksum<T><<<nb, 256, 0, s>>>(g->n1, m, M->x, ks, done);
  k_mc_out<T><<<nb, 256, 0, s>>>(g->n1, m, M->x, &g->sc->dots[SL_MQ], &g->sc->v[S_MQNU], 0.0, zp, vp, gsl, goff, 1, done);
  ETH_CUDA(cudaGetLastError());
  g->launches += 2;
  return ETH_OK;
}

template eth_status precond_pressure_cheb<float>(eth_grid*, Work*, const eth_opts*, const double*, double*, const Slot&, int,
                                                 const int*, cudaStream_t);
template eth_status precond_pressure_cheb<double>(eth_grid*, Work*, const eth_opts*, const double*, double*, const Slot&,
                                                  int, const int*, cudaStream_t);
template eth_status mqcheb_prepare<float>(eth_grid*, Work*);
template eth_status mqcheb_prepare<double>(eth_grid*, Work*);

// the entry point's body: z = M_cheb^{-1} r with the k component of r removed and z orthogonal to k
template <class T>
static eth_status apply_mqcheb_t(eth_grid* g, Work* w, int steps, double a, double b, const double* r, double* z) {
  McWork<T>* M = nullptr;
  ETH_TRY(mc_get<T>(g, w, &M));
  const int m = g->n1 + g->n0, nb = vblocks((size_t)m);
  // beta = k^T r / k^T k into the grid scalars' generic slot
  Slot bs = slot_of(g, SL_GEN, nb, FIN_STORE);
  k_mc_load_beta<<<nb, 256, 0, g->s>>>(g->n1, m, r, bs);
  k_mc_init<T><<<nb, 256, 0, g->s>>>(g->n1, m, r, &g->sc->dots[SL_GEN], M->r, M->x, nullptr);
  ETH_CUDA(cudaGetLastError());
  g->launches += 2;
  ETH_TRY(mc_chebyshev<T>(g, M, steps, a, b, nullptr, g->s));
  Slot ks = slot_of(g, SL_MQ, nb, FIN_STORE);
  k_mc_ksum<T><<<nb, 256, 0, g->s>>>(g->n1, m, M->x, ks, nullptr);
  Slot none{};
  k_mc_out<T><<<nb, 256, 0, g->s>>>(g->n1, m, M->x, &g->sc->dots[SL_MQ], nullptr, 1.0, z, r, none, 0, 0, nullptr);
  ETH_CUDA(cudaGetLastError());
  g->launches += 2;
  return ETH_OK;
}

}  // namespace eth

using namespace eth;

extern "C" eth_status eth_apply_mqcheb(eth_grid* g, int fp32, int steps, double a, double b, const double* r_dev,
                                       double* z_dev) {
  if (!g || !r_dev || !z_dev) { set_error("eth_apply_mqcheb: NULL argument"); return ETH_EINVAL; }
  if (steps < 1 || steps > 10000) { set_error("eth_apply_mqcheb: steps=%d out of 1..10000", steps); return ETH_EINVAL; }
  if (a <= 0.0) a = mqcheb_default_a(g);
  if (b <= 0.0) b = 1.0;
  if (!(a < b) || !std::isfinite(a) || !std::isfinite(b)) { set_error("eth_apply_mqcheb: interval [%g, %g]", a, b); return ETH_EINVAL; }
  ETH_ON_DEVICE(g);
  Work* w;
  ETH_TRY(work_get(g, &w));
  StreamSwap guard(g, w);
  return fp32 ? apply_mqcheb_t<float>(g, w, steps, a, b, r_dev, z_dev)
              : apply_mqcheb_t<double>(g, w, steps, a, b, r_dev, z_dev);
}
