// Oseen solver: right-preconditioned flexible GMRES(m) with classical
// Gram-Schmidt applied twice (FP64 basis, FP64 Givens recurrence on the
// device), and the two-stage pressure convection-diffusion method of Sec. 3.1:
//
//   Step I   GMRES on the reduced system [F B1^T; B1 0] (Eq. reduced-system)
//            with [M B1^T; 0 -M_S]^{-1}, M_S^{-1} = Ap^{-1} F1 Q1^{-1}
//            (Eq. discrete-commutator1x), to a residual <= c*eta*||b_red||;
//   Step II  GMRES on the full system from [u1*, q1*, 0] with
//            M_1 = [M B^T; 0 -(1/nu) M_Q] (Eq. nse-precon-ref) to eta*||b||.
//
// M is one GMG V-cycle on F (coarse levels stabilised by streamline
// diffusion), M_Q^+ the block-elimination approximation with k projected out,
// Q1^{-1} a fixed Chebyshev-Jacobi polynomial, Ap^{-1} a few PCG steps on
// Ap = B1 Md^{-1} B1^T preconditioned by the Q1 Laplacian V-cycle.  Inside a
// GMRES cycle the operator is applied with FP32 element arithmetic; every
// restart recomputes the residual with FP64 element arithmetic, which makes
// the restarts an FP64 iterative refinement.
#include <map>
#include <mutex>
#include <cmath>
#include <cstring>
#include "solve.cuh"

namespace eth {

constexpr int GM_MAX = 160;
constexpr int GM_CHUNK = 4;   // graph-replayed Arnoldi steps between host convergence checks

struct GScalars {
  double H[GM_MAX + 1][GM_MAX];
  double cs[GM_MAX], sn[GM_MAX], g[GM_MAX + 1], y[GM_MAX];
  double h1[GM_MAX + 1], h2[GM_MAX + 1];
  double res, tol_abs, wnorm, beta;
  double pcg[8];       // inner PCG scalars: rz, pAp, alpha, beta
  int k, done, bdown, skip2;   // skip2: the second Gram-Schmidt pass is not needed
  int jcur;                    // Arnoldi column of the iteration in flight (graph-replayed loop)
};

struct GMRESWork {
  int m = 0;
  size_t cap = 0;
  double* V = nullptr;     // (m+1) x cap
  double* Z = nullptr;     // m x cap
  double* w = nullptr;
  double* b = nullptr;
  double* t = nullptr;     // velocity scratch (FP64)
  GScalars* gs = nullptr;
  GScalars* gsh = nullptr;
  double* part = nullptr;
  unsigned* ticket = nullptr;
  int nbmax = 0;
  // PCD data (both precisions, built lazily)
  float* c1f = nullptr; double* c1d = nullptr;     // Q1 convection element matrices
  float* mdf = nullptr; double* mdd = nullptr;     // inverse velocity-mass diagonal (interior)
  float* q1df = nullptr; double* q1dd = nullptr;   // inverse Q1-mass diagonal
  void* pv[8] = {};                                // Q1 / velocity scratch (type T)
  int pcd_prec = -1;
  int grp = 16;        // basis vectors per pass of the Gram-Schmidt dot kernel (autotuned)
  bool grp_tuned = false;
  double* vin = nullptr;   // fixed in/out vectors of the graph-replayed Arnoldi step
  double* zout = nullptr;
};

void gmres_free(Work* w) {
  GMRESWork* G = w->gm;
  if (!G) return;
  cudaFree(G->V); cudaFree(G->Z); cudaFree(G->w); cudaFree(G->b); cudaFree(G->t);
  cudaFree(G->vin); cudaFree(G->zout);
  cudaFree(G->gs); if (G->gsh) cudaFreeHost(G->gsh);
  cudaFree(G->part); cudaFree(G->ticket);
  cudaFree(G->c1f); cudaFree(G->c1d); cudaFree(G->mdf); cudaFree(G->mdd); cudaFree(G->q1df); cudaFree(G->q1dd);
  for (void* p : G->pv) cudaFree(p);
  delete G;
  w->gm = nullptr;
}

// ---------------------------------------------------------------------------
// multi-vector kernels: h_i = <V_i, w> (i < nvec) and w -= sum_i h_i V_i
// ---------------------------------------------------------------------------
constexpr int MG_GRP_MAX = 16;

// last-block sum of partials part[i*nb + b] into out[i]
__device__ __forceinline__ bool multi_finish(int nvec, int nb, double* part, unsigned* ticket, double* out) {
  __shared__ bool last;
  __threadfence();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == (unsigned)nb - 1u);
  __syncthreads();
  if (!last) return false;
  __threadfence();
  for (int i = threadIdx.x / 32; i < nvec; i += blockDim.x / 32) {
    double a = 0.0;
    for (int b = threadIdx.x & 31; b < nb; b += 32) a += ((volatile double*)part)[(size_t)i * nb + b];
    a = warp_sum(a);
    if ((threadIdx.x & 31) == 0) out[i] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// h_i = <V_i, w> for i < nvec; with wnorm, also out[nvec] = <w, w> (grouped MG_GRP vectors per
// pass over w: more vectors per pass read w fewer times but hold more accumulators)
template <int MG_GRP>
__global__ void k_mdot(size_t n, const double* __restrict__ V, size_t ld, int nvec, const double* __restrict__ w,
                       double* part, unsigned* ticket, double* out, const int* done, const int* skip, int wnorm,
                       const int* jp) {
  ETH_GRID_DEP_WAIT();
  if ((done && *done) || (skip && *skip)) return;
  if (jp) nvec = *jp + 1;   // column index read on the device (graph-replayed loop)
  const int nb = gridDim.x;
  const int nout = nvec + (wnorm ? 1 : 0);
  for (int g0 = 0; g0 < nout; g0 += MG_GRP) {
    double acc[MG_GRP];
#pragma unroll
    for (int i = 0; i < MG_GRP; ++i) acc[i] = 0.0;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
      const double wk = w[k];
#pragma unroll
      for (int i = 0; i < MG_GRP; ++i) {
        if (g0 + i < nvec) acc[i] += V[(size_t)(g0 + i) * ld + k] * wk;
        else if (g0 + i == nvec && wnorm) acc[i] += wk * wk;
      }
    }
    block_sum<MG_GRP>(acc);
    if (threadIdx.x == 0)
      for (int i = 0; i < MG_GRP && g0 + i < nout; ++i) part[(size_t)(g0 + i) * nb + blockIdx.x] = acc[i];
  }
  multi_finish(nout, nb, part, ticket, out);
}

// w -= sum_i h_i V_i ; optionally ||w||^2 -> finisher (Arnoldi column j)
__device__ __forceinline__ void arnoldi_finish(GScalars* gs, int j, double wn2) {
  for (int i = 0; i <= j; ++i) gs->H[i][j] = gs->h1[i] + gs->h2[i];
  const double wn = sqrt(fmax(wn2, 0.0));
  gs->wnorm = wn;
  gs->H[j + 1][j] = wn;
  for (int i = 0; i < j; ++i) {
    const double a = gs->H[i][j], b = gs->H[i + 1][j];
    gs->H[i][j] = gs->cs[i] * a + gs->sn[i] * b;
    gs->H[i + 1][j] = -gs->sn[i] * a + gs->cs[i] * b;
  }
  const double a = gs->H[j][j], b = wn;
  const double den = sqrt(a * a + b * b);
  const double c = den > 0.0 ? a / den : 1.0, s = den > 0.0 ? b / den : 0.0;
  gs->cs[j] = c; gs->sn[j] = s;
  gs->H[j][j] = den;
  gs->g[j + 1] = -s * gs->g[j];
  gs->g[j] = c * gs->g[j];
  gs->res = fabs(gs->g[j + 1]);
  gs->k = j + 1;
  if (!isfinite(gs->res)) { gs->done = 1; gs->bdown = 8; }
  else if (gs->res <= gs->tol_abs || wn == 0.0) gs->done = 1;
}

// w -= sum_i h_i V_i.  mode 0: nothing else; mode 1: ||w||^2 and the Arnoldi/Givens
// finisher; mode 2 (after the first Gram-Schmidt pass): the DGKS test
// ||w_new|| >= 0.7 ||w_old|| accepts the column (h2 = 0, finisher, skip the
// second pass), otherwise the second pass runs.
__global__ void k_mupd(size_t n, const double* __restrict__ V, size_t ld, int nvec, const double* __restrict__ h,
                       double* __restrict__ w, int norm, double* part, unsigned* ticket, GScalars* gs, int j, const int* done,
                       const int* skip, const int* jp) {
  ETH_GRID_DEP_WAIT();
  if ((done && *done) || (skip && *skip)) return;
  if (jp) { j = *jp; nvec = j + 1; }
  double acc = 0.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    double v = w[k];
    for (int i = 0; i < nvec; ++i) v -= h[i] * V[(size_t)i * ld + k];
    w[k] = v;
    acc += v * v;
  }
  if (!norm) return;
  double a[1] = {acc};
  block_sum<1>(a);
  if (threadIdx.x == 0) part[blockIdx.x] = a[0];
  if (multi_finish(1, gridDim.x, part, ticket, &gs->pcg[7])) {
    if (threadIdx.x == 0) {
      if (norm == 2) {
        const double before = gs->h1[nvec];   // ||w||^2 before the first pass
        if (gs->pcg[7] >= 0.49 * before) {
          for (int i = 0; i < nvec; ++i) gs->h2[i] = 0.0;
          gs->skip2 = 1;
          arnoldi_finish(gs, j, gs->pcg[7]);
        } else {
          gs->skip2 = 0;
        }
      } else {
        arnoldi_finish(gs, j, gs->pcg[7]);
      }
    }
  }
}

__global__ void k_vscale(size_t n, const double* __restrict__ w, double* __restrict__ v, const GScalars* gs, int use_beta,
                         size_t ld = 0, const int* jp = nullptr) {
  ETH_GRID_DEP_WAIT();
  if (gs->done && !use_beta) return;
  if (jp) v += (size_t)(*jp + 1) * ld;   // next basis column, index read on the device
  const double s = 1.0 / (use_beta ? gs->beta : gs->wnorm);
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) v[k] = s * w[k];
}

// r = b - y, ||r||^2 -> gs->beta (sqrt), cycle initialisation of the Givens state
__global__ void k_gm_resid(size_t n, const double* __restrict__ b, const double* __restrict__ y, double* __restrict__ r,
                           double* part, unsigned* ticket, GScalars* gs, double tol_abs) {
  ETH_GRID_DEP_WAIT();
  double acc = 0.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    const double v = b[k] - y[k];
    r[k] = v;
    acc += v * v;
  }
  double a[1] = {acc};
  block_sum<1>(a);
  if (threadIdx.x == 0) part[blockIdx.x] = a[0];
  if (multi_finish(1, gridDim.x, part, ticket, &gs->pcg[6])) {
    if (threadIdx.x == 0) {
      const double beta = sqrt(gs->pcg[6]);
      gs->beta = beta;
      gs->g[0] = beta;
      for (int i = 1; i <= GM_MAX; ++i) gs->g[i] = 0.0;
      gs->res = beta;
      gs->tol_abs = tol_abs;
      gs->k = 0;
      gs->jcur = 0;
      gs->done = (beta <= tol_abs || !isfinite(beta)) ? 1 : 0;
      gs->bdown = isfinite(beta) ? 0 : 8;
    }
  }
}

// column jcur of a basis <-> a fixed vector (graph-replayed Arnoldi loop)
__global__ void k_gm_col_in(size_t n, const double* __restrict__ V, size_t ld, const GScalars* gs, double* __restrict__ out) {
  ETH_GRID_DEP_WAIT();
  if (gs->done) return;
  const double* src = V + (size_t)gs->jcur * ld;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) out[k] = src[k];
}
__global__ void k_gm_col_out(size_t n, const double* __restrict__ in, double* __restrict__ Z, size_t ld, const GScalars* gs) {
  ETH_GRID_DEP_WAIT();
  if (gs->done) return;
  double* dst = Z + (size_t)gs->jcur * ld;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) dst[k] = in[k];
}
__global__ void k_gm_next(GScalars* gs) {
  ETH_GRID_DEP_WAIT();
  if (!gs->done) gs->jcur += 1;
}

// y = H(0:k,0:k)^{-1} g(0:k) by back substitution (one thread)
__global__ void k_gm_solve(GScalars* gs) {
  ETH_GRID_DEP_WAIT();
  const int k = gs->k;
  for (int i = k - 1; i >= 0; --i) {
    double s = gs->g[i];
    for (int l = i + 1; l < k; ++l) s -= gs->H[i][l] * gs->y[l];
    gs->y[i] = s / gs->H[i][i];
  }
}

// x += sum_{i<k} y_i Z_i  (k read on the device)
__global__ void k_zupd(size_t n, const double* __restrict__ Z, size_t ld, const GScalars* gs, double* __restrict__ x) {
  ETH_GRID_DEP_WAIT();
  const int kk = gs->k;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    double v = x[k];
    for (int i = 0; i < kk; ++i) v += gs->y[i] * Z[(size_t)i * ld + k];
    x[k] = v;
  }
}

// ---------------------------------------------------------------------------
// PCD set-up kernels
// ---------------------------------------------------------------------------
// Q1 convection element matrices C_T[a][b] = int_T psi_a (w_h . grad psi_b) (3x3 Gauss, Q2 wind)
template <class T>
__global__ void k_q1_conv_mats(int n, double hx, double hy, const double* __restrict__ w, T* __restrict__ C, int trans) {
  ETH_GRID_DEP_WAIT();
  const int N = 2 * n + 1;
  const size_t nv = (size_t)N * N;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const int ey = e / n, ex = e - ey * n;
  double c[4][4] = {};
  for (int qy = 0; qy < 3; ++qy)
    for (int qx = 0; qx < 3; ++qx) {
      double wx = 0, wy = 0;
      for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) {
          const double f = q2v(a, gq(qx)) * q2v(b, gq(qy));
          const size_t gn = (size_t)(2 * ey + b) * N + 2 * ex + a;
          wx += f * w[gn];
          wy += f * w[gn + nv];
        }
      const double W = gw(qx) * gw(qy) * hx * hy;
      for (int li = 0; li < 4; ++li) {
        const int ci = li & 1, di = li >> 1;
        const double psi = q1v(ci, gq(qx)) * q1v(di, gq(qy));
        for (int lj = 0; lj < 4; ++lj) {
          const int cj = lj & 1, dj = lj >> 1;
          const double dx = q1d(cj) * q1v(dj, gq(qy)) / hx, dy = q1v(cj, gq(qx)) * q1d(dj) / hy;
          c[li][lj] += W * psi * (wx * dx + wy * dy);
        }
      }
    }
  for (int li = 0; li < 4; ++li)
    for (int lj = 0; lj < 4; ++lj) C[(size_t)e * 16 + li * 4 + lj] = (T)(trans ? c[lj][li] : c[li][lj]);
}

// inverse of the diagonal of the velocity mass matrix (interior nodes), 0 on the boundary
template <class T>
__global__ void k_q2_mass_diag(int n, double hx, double hy, T* __restrict__ md) {
  ETH_GRID_DEP_WAIT();
  const int N = 2 * n + 1;
  for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < N * N; node += gridDim.x * blockDim.x) {
    const int j = node / N, i = node - j * N;
    if (i == 0 || j == 0 || i == N - 1 || j == N - 1) { md[node] = 0; continue; }
    // 1D lumped diagonal of the quadratic mass: vertex 4/30 per element side, midpoint 16/30
    const double dx = (i & 1) ? 16.0 / 30.0 * hx : 2.0 * 4.0 / 30.0 * hx;
    const double dy = (j & 1) ? 16.0 / 30.0 * hy : 2.0 * 4.0 / 30.0 * hy;
    md[node] = (T)(1.0 / (dx * dy));
  }
}

template <class T>
__global__ void k_q1_mass_diag(int n, double hx, double hy, T* __restrict__ d) {
  ETH_GRID_DEP_WAIT();
  const int M = n + 1;
  for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < M * M; node += gridDim.x * blockDim.x) {
    const int J = node / M, I = node - J * M;
    const double dx = ((I > 0) + (I < n)) * hx / 3.0, dy = ((J > 0) + (J < n)) * hy / 3.0;
    d[node] = (T)(1.0 / (dx * dy));
  }
}

// Chebyshev step on the Q1 mass: x += d; r -= Q d; d' = c1 d + c2 D^{-1} r
template <class T>
__global__ void k_cheb_step(int n, T area, const T* __restrict__ d_in, T* __restrict__ r, T* __restrict__ x, T* __restrict__ dn,
                            const T* __restrict__ dinv, T c1, T c2, const int* done) {
  ETH_GRID_DEP_WAIT();
  const T* d = d_in;
  if (done && *done) return;
  const int M = n + 1;
  for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < M * M; node += gridDim.x * blockDim.x) {
    const int J = node / M, I = node - J * M;
    T q = 0;
    Q1_FOR_ELEMENTS(n, I, J, {
#pragma unroll
      for (int dd = 0; dd < 2; ++dd)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc)
          q += area * (T)(q1m(c, cc) * q1m(d, dd)) * d_in[(size_t)(ey + dd) * M + ex + cc];
    })
    const T rn = r[node] - q;
    r[node] = rn;
    x[node] += d[node];
    dn[node] = c1 * d[node] + c2 * dinv[node] * rn;
  }
}

template <class TI, class T>
__global__ void k_cheb_init(int m, T theta, const TI* __restrict__ b, const T* __restrict__ dinv, T* __restrict__ r,
                            T* __restrict__ x, T* __restrict__ d, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    const T v = (T)b[k];
    r[k] = v;
    x[k] = 0;
    d[k] = dinv[k] * v / theta;
  }
}

// generic small vector kernels on type T (Q1 lattice)
template <class T>
__global__ void k_axpy_t(int m, T a, const T* __restrict__ x, T* __restrict__ y) {
  ETH_GRID_DEP_WAIT();
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) y[k] += a * x[k];
}

// PCG pieces with device scalars (gs->pcg: [0] rz, [1] pAp, [2] sum r)
template <class T>
__global__ void k_pcg_dot(int m, const T* __restrict__ a, const T* __restrict__ b, double* part, unsigned* ticket, double* out,
                          const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  double acc = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) acc += (double)a[k] * (double)b[k];
  double v[1] = {acc};
  block_sum<1>(v);
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
  multi_finish(1, gridDim.x, part, ticket, out);
}

// (<r, z>, sum z) -> out[0], out[1]: the PCG inner product and the constant
// component of the preconditioned residual (the Q1 V-cycle of a singular operator
// may return one; it is removed from the search direction below)
template <class T>
__global__ void k_pcg_dot_sum(int m, const T* __restrict__ r, const T* __restrict__ z, double* part, unsigned* ticket,
                              double* out, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  double a = 0.0, c = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    const double zk = (double)z[k];
    a += (double)r[k] * zk;
    c += zk;
  }
  double v[2] = {a, c};
  block_sum<2>(v);
  if (threadIdx.x == 0) { part[blockIdx.x] = v[0]; part[gridDim.x + blockIdx.x] = v[1]; }
  multi_finish(2, gridDim.x, part, ticket, out);
}

// p = z - mean(z)   (first PCG direction, mean from gs->pcg[1]); keeps the initial
// <r, z> in gs->pcg[6] for the convergence guard of k_pcg_xr
template <class T>
__global__ void k_pcg_p0(int m, const T* __restrict__ z, T* __restrict__ p, GScalars* gs, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  const T mu = (T)(gs->pcg[1] / m);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) p[k] = z[k] - mu;
  if (blockIdx.x == 0 && threadIdx.x == 0) gs->pcg[6] = gs->pcg[0];
}

// x += alpha p ; r -= alpha q   (alpha = rz / pAp).  Once <r, z> has fallen to the
// rounding level of T relative to its initial value the iterate is left alone:
// further steps of a converged CG on the singular Ap only amplify rounding noise.
template <class T>
__global__ void k_pcg_xr(int m, const T* __restrict__ p, const T* __restrict__ q, T* __restrict__ x, T* __restrict__ r,
                         const GScalars* gs, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  const double pap = gs->pcg[1], rz = gs->pcg[0];
  const double floor_rz = (sizeof(T) == 4 ? 1e-13 : 1e-28) * gs->pcg[6];
  const T a = (T)((pap > 0.0 && rz > floor_rz) ? rz / pap : 0.0);   // zero right-hand side: stay at zero
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    x[k] += a * p[k];
    r[k] -= a * q[k];
  }
}

// p = (z - mean z) + (rz_new / rz) p ; rz = rz_new   (rz_new in gs->pcg[2], sum z in gs->pcg[3]).
// Keeping p free of constants keeps the iterate's constant component from drifting
// when many steps run on the singular Ap.
template <class T>
__global__ void k_pcg_p(int m, const T* __restrict__ z, T* __restrict__ p, GScalars* gs, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  const T bt = (T)(gs->pcg[0] != 0.0 ? gs->pcg[2] / gs->pcg[0] : 0.0);
  const T mu = (T)(gs->pcg[3] / m);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) p[k] = (z[k] - mu) + bt * p[k];
  __syncthreads();
}
__global__ void k_pcg_shift(GScalars* gs) {
  ETH_GRID_DEP_WAIT(); gs->pcg[0] = gs->pcg[2]; }

template <class T>
__global__ void k_copy_t(int m, const T* __restrict__ a, T* __restrict__ b) {
  ETH_GRID_DEP_WAIT();
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) b[k] = a[k];
}

// z_p = -(x - mean x) written as FP64 (mean from gs->pcg[3])
template <class T>
__global__ void k_pcd_out(int m, const T* __restrict__ x, double* __restrict__ zp, const GScalars* gs, double scale) {
  ETH_GRID_DEP_WAIT();
  const double mean = gs->pcg[3] / m;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) zp[k] = scale * ((double)x[k] - mean);
}

template <class T>
__global__ void k_sum_t(int m, const T* __restrict__ a, double* part, unsigned* ticket, double* out) {
  ETH_GRID_DEP_WAIT();
  double acc = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) acc += (double)a[k];
  double v[1] = {acc};
  block_sum<1>(v);
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
  multi_finish(1, gridDim.x, part, ticket, out);
}

template <class T>
__global__ void k_sub_mean_t(int m, T* __restrict__ a, const double* sum) {
  ETH_GRID_DEP_WAIT();
  const T mu = (T)(*sum / m);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) a[k] -= mu;
}

__global__ void k_oseen_scalars(Scalars* sc, double n1, double n0, double mqc, double nuq) {
  ETH_GRID_DEP_WAIT();
  sc->v[S_NP1] = n1; sc->v[S_NP0] = n0; sc->v[S_MQC] = mqc; sc->v[S_MQNU] = nuq;
  sc->done = 0;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int gb(size_t m) { return vblocks(m); }

static eth_status launch_mdot(GMRESWork* G, int nb, cudaStream_t s, size_t ntv, size_t ld, int nvec, double* out,
                              const int* done, const int* skip, int wnorm, const int* jp = nullptr) {
  switch (G->grp) {
    case 4: k_mdot<4><<<nb, 256, 0, s>>>(ntv, G->V, ld, nvec, G->w, G->part, G->ticket + 3, out, done, skip, wnorm, jp); break;
    case 8: k_mdot<8><<<nb, 256, 0, s>>>(ntv, G->V, ld, nvec, G->w, G->part, G->ticket + 3, out, done, skip, wnorm, jp); break;
    default: k_mdot<16><<<nb, 256, 0, s>>>(ntv, G->V, ld, nvec, G->w, G->part, G->ticket + 3, out, done, skip, wnorm, jp); break;
  }
  ETH_CUDA(cudaGetLastError());
  return ETH_OK;
}

// Autotuner of the Gram-Schmidt dot kernel: times the vectors-per-pass choices
// {4, 8, 16} on a 32-vector dot against the basis storage (its contents do not
// matter for the timing) and keeps the fastest; cached per vector length.
static eth_status tune_cgs(eth_grid* g, GMRESWork* G) {
  static std::mutex mu;
  static std::map<size_t, int> cache;
  const size_t ntv = g->nt;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(ntv);
    if (it != cache.end()) { G->grp = it->second; G->grp_tuned = true; return ETH_OK; }
  }
  const int nvec = std::min(G->m, 32);
  const int nb = gb(ntv);
  cudaEvent_t e0, e1;
  ETH_CUDA(cudaEventCreate(&e0));
  ETH_CUDA(cudaEventCreate(&e1));
  int best = 16;
  float best_ms = 1e30f;
  for (int grp : {4, 8, 16}) {
    G->grp = grp;
    ETH_TRY(launch_mdot(G, nb, g->s, ntv, G->cap, nvec, &G->gs->h1[0], nullptr, nullptr, 1));
    cudaEventRecord(e0, g->s);
    for (int r = 0; r < 3; ++r) ETH_TRY(launch_mdot(G, nb, g->s, ntv, G->cap, nvec, &G->gs->h1[0], nullptr, nullptr, 1));
    cudaEventRecord(e1, g->s);
    ETH_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) { best_ms = ms; best = grp; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  G->grp = best;
  G->grp_tuned = true;
  std::lock_guard<std::mutex> lk(mu);
  cache[ntv] = best;
  return ETH_OK;
}

static eth_status gm_alloc(eth_grid* g, Work* w, int m) {
  GMRESWork* G = w->gm;
  if (G && G->m == m) return ETH_OK;
  if (G) gmres_free(w);
  G = new GMRESWork();
  w->gm = G;
  G->m = m;
  G->cap = ((size_t)g->nt + 31) & ~(size_t)31;
  ETH_CUDA(cudaMalloc((void**)&G->V, (size_t)(m + 1) * G->cap * 8));
  ETH_CUDA(cudaMalloc((void**)&G->Z, (size_t)m * G->cap * 8));
  ETH_CUDA(cudaMalloc((void**)&G->w, G->cap * 8));
  ETH_CUDA(cudaMalloc((void**)&G->b, G->cap * 8));
  ETH_CUDA(cudaMalloc((void**)&G->t, G->cap * 8));
  ETH_CUDA(cudaMalloc((void**)&G->vin, G->cap * 8));
  ETH_CUDA(cudaMalloc((void**)&G->zout, G->cap * 8));
  ETH_CUDA(cudaMalloc((void**)&G->gs, sizeof(GScalars)));
  ETH_CUDA(cudaMallocHost((void**)&G->gsh, sizeof(GScalars)));
  G->nbmax = 152 * 8;
  ETH_CUDA(cudaMalloc((void**)&G->part, (size_t)(GM_MAX + 1) * G->nbmax * 8));
  ETH_CUDA(cudaMalloc((void**)&G->ticket, 8 * sizeof(unsigned)));
  ETH_CUDA(cudaMemsetAsync(G->ticket, 0, 8 * sizeof(unsigned), g->s));
  ETH_CUDA(cudaMemsetAsync(G->gs, 0, sizeof(GScalars), g->s));
  return ETH_OK;
}

template <class T> struct PcdPtr;
template <> struct PcdPtr<float> {
  static float*& c1(GMRESWork* G) { return G->c1f; }
  static float*& md(GMRESWork* G) { return G->mdf; }
  static float*& q1d(GMRESWork* G) { return G->q1df; }
};
template <> struct PcdPtr<double> {
  static double*& c1(GMRESWork* G) { return G->c1d; }
  static double*& md(GMRESWork* G) { return G->mdd; }
  static double*& q1d(GMRESWork* G) { return G->q1dd; }
};

// scratch layout (type T): 0..5 Q1 vectors (r, x, d, dn, p, q), 6 velocity (2 nv), 7 Q1 (z)
template <class T>
static T* pv(GMRESWork* G, int i) { return (T*)G->pv[i]; }

template <class T>
static eth_status pcd_setup(eth_grid* g, Work* w, bool adjoint) {
  GMRESWork* G = w->gm;
  const int key = (int)sizeof(T) + (adjoint ? 100 : 0);
  if (G->pcd_prec == key) return ETH_OK;
  const size_t n1 = g->n1, nv = g->nv, ne = (size_t)g->n * g->n;
  T*& c1 = PcdPtr<T>::c1(G);
  T*& md = PcdPtr<T>::md(G);
  T*& q1d = PcdPtr<T>::q1d(G);
  if (!c1) ETH_CUDA(cudaMalloc((void**)&c1, ne * 16 * sizeof(T)));
  if (!md) ETH_CUDA(cudaMalloc((void**)&md, nv * sizeof(T)));
  if (!q1d) ETH_CUDA(cudaMalloc((void**)&q1d, n1 * sizeof(T)));
  for (int i = 0; i < 8; ++i) {
    if (G->pv[i]) { cudaFree(G->pv[i]); G->pv[i] = nullptr; }
    const size_t len = (i == 6) ? 2 * nv : n1;
    ETH_CUDA(cudaMalloc(&G->pv[i], len * sizeof(T)));
    ETH_CUDA(cudaMemsetAsync(G->pv[i], 0, len * sizeof(T), g->s));
  }
  k_q1_conv_mats<T><<<cdiv((long)ne, 128), 128, 0, g->s>>>(g->n, g->hx, g->hy, g->wind, c1, adjoint ? 1 : 0);
  k_q2_mass_diag<T><<<gb(nv), 256, 0, g->s>>>(g->n, g->hx, g->hy, md);
  k_q1_mass_diag<T><<<gb(n1), 256, 0, g->s>>>(g->n, g->hx, g->hy, q1d);
  ETH_CUDA(cudaGetLastError());
  G->pcd_prec = key;
  return ETH_OK;
}

// q = Ap p = B1 Md^{-1} B1^T p (matrix free, two tile launches); fused <q, p> into gs->pcg[1]
template <class T>
static eth_status ap_apply(eth_grid* g, GMRESWork* G, const T* p, T* q, const int* done) {
  T* vel = pv<T>(G, 6);
  {
    Q2Params<T, T, T> P{};
    P.n = g->n; P.hx = (T)g->hx; P.hy = (T)g->hy; P.nu = 0;
    P.p = p; P.y = vel; P.dinv = PcdPtr<T>::md(G); P.done = done;
    ETH_CUDA((launch_q2<T, T, T, QF_PIN | QF_UOUT, EPI_SCALE>(P, g->s)));
  }
  {
    Q2Params<T, T, T> P{};
    P.n = g->n; P.hx = (T)g->hx; P.hy = (T)g->hy; P.nu = 0;
    P.x = vel; P.yp = q; P.done = done;
    ETH_CUDA((launch_q2<T, T, T, QF_XIN | QF_POUT, EPI_APPLY>(P, g->s)));
  }
  const int m = g->n1;
  k_pcg_dot<T><<<gb(m), 256, 0, g->s>>>(m, q, p, G->part, G->ticket + 1, &G->gs->pcg[1], done);
  ETH_CUDA(cudaGetLastError());
  g->launches += 3;
  return ETH_OK;
}

// z = V_K1(r) using the Q1 hierarchy (level-0 b := r, first Jacobi sweep from zero)
template <class T>
__global__ void k_q1_j0(int m, T omega, const T* __restrict__ dinv, const T* __restrict__ r, T* __restrict__ b,
                        T* __restrict__ x, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    const T v = r[k];
    b[k] = v;
    x[k] = omega * dinv[k] * v;
  }
}

template <class T>
static eth_status q1_vcycle(eth_grid* g, Work* w, const T* r, T* z, const int* done) {
  Hier<T>& Q = q1_hier<T>(w);
  Level<T>& L0 = Q.lv[0];
  const int m = g->n1;
  k_q1_j0<T><<<gb(m), 256, 0, g->s>>>(m, (T)Q.omega, L0.dinv, r, L0.b, L0.x, done);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  const T* res = nullptr;
  ETH_TRY(vcycle_q1_from<T>(g, Q, 1, 1, done, &res));
  k_copy_t<T><<<gb(m), 256, 0, g->s>>>(m, res, z);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  return ETH_OK;
}

// x ~= Ap^+ b (b: Q1, type T, consistent up to its mean); `its` PCG steps
template <class T>
static eth_status ap_solve(eth_grid* g, Work* w, const T* b, T* x, int its, const int* done) {
  GMRESWork* G = w->gm;
  const int m = g->n1;
  T *r = pv<T>(G, 0), *z = pv<T>(G, 7), *p = pv<T>(G, 4), *q = pv<T>(G, 5);
  double* gsum = &G->gs->pcg[4];
  k_copy_t<T><<<gb(m), 256, 0, g->s>>>(m, b, r);
  k_sum_t<T><<<gb(m), 256, 0, g->s>>>(m, r, G->part, G->ticket + 2, gsum);
  k_sub_mean_t<T><<<gb(m), 256, 0, g->s>>>(m, r, gsum);
  ETH_CUDA(cudaMemsetAsync(x, 0, m * sizeof(T), g->s));
  ETH_CUDA(cudaGetLastError());
  g->launches += 3;
  ETH_TRY(q1_vcycle<T>(g, w, r, z, done));
  k_pcg_dot_sum<T><<<gb(m), 256, 0, g->s>>>(m, r, z, G->part, G->ticket + 1, &G->gs->pcg[0], done);
  k_pcg_p0<T><<<gb(m), 256, 0, g->s>>>(m, z, p, G->gs, done);
  ETH_CUDA(cudaGetLastError());
  g->launches += 2;
  for (int it = 0; it < its; ++it) {
    ETH_TRY(ap_apply<T>(g, G, p, q, done));
    k_pcg_xr<T><<<gb(m), 256, 0, g->s>>>(m, p, q, x, r, G->gs, done);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
    if (it + 1 == its) break;
    ETH_TRY(q1_vcycle<T>(g, w, r, z, done));
    k_pcg_dot_sum<T><<<gb(m), 256, 0, g->s>>>(m, r, z, G->part, G->ticket + 1, &G->gs->pcg[2], done);
    k_pcg_p<T><<<gb(m), 256, 0, g->s>>>(m, z, p, G->gs, done);
    k_pcg_shift<<<1, 1, 0, g->s>>>(G->gs);
    ETH_CUDA(cudaGetLastError());
    g->launches += 3;
  }
  return ETH_OK;
}

// Q1^{-1} b by a fixed Chebyshev polynomial on D^{-1} Q1 (spectrum in [1/4, 9/4]); b FP64 -> x (T)
template <class T>
static eth_status q1_mass_inv(eth_grid* g, GMRESWork* G, const double* b, T* x, int steps, const int* done) {
  const int m = g->n1;
  const double lmin = 0.25, lmax = 2.25, theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
  const double sigma = theta / delta;
  T *r = pv<T>(G, 0), *d = pv<T>(G, 2), *dn = pv<T>(G, 3);
  k_cheb_init<double, T><<<gb(m), 256, 0, g->s>>>(m, (T)theta, b, PcdPtr<T>::q1d(G), r, x, d, done);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  double rho = 1.0 / sigma;
  for (int k = 0; k < steps; ++k) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    k_cheb_step<T><<<gb(m), 256, 0, g->s>>>(g->n, (T)(g->hx * g->hy), d, r, x, dn, PcdPtr<T>::q1d(G), (T)(rn * rho),
                                           (T)(2.0 * rn / delta), done);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
    std::swap(d, dn);
    rho = rn;
  }
  return ETH_OK;
}

// velocity part of a block-triangular preconditioner: z_u = V_F(r_u - B^T z_p)
template <class T>
static eth_status vel_part(eth_grid* g, Work* w, const eth_opts* o, const double* ru, const double* zp, bool p0, double* zu,
                           const int* done, bool adj) {
  GMRESWork* G = w->gm;
  Q2Params<double, double, T> P{};
  P.n = g->n; P.hx = (T)g->hx; P.hy = (T)g->hy; P.nu = 0;
  P.p = zp; P.y = G->t; P.bsrc = ru; P.done = done;
  if (p0) ETH_CUDA((launch_q2<double, double, T, QF_PIN | QF_P0 | QF_UOUT, EPI_BSUB>(P, g->s)));
  else ETH_CUDA((launch_q2<double, double, T, QF_PIN | QF_UOUT, EPI_BSUB>(P, g->s)));
  g->launches++;
  return vcycle_vel<T>(g, adj ? vel_hier_t<T>(w) : vel_hier<T>(w), G->t, zu, o->mg_pre, o->mg_post, done, nullptr, 0);
}

// Q1 PCD Schur approximation (Sec. 3.1, Eq. discrete-commutator1x):
// zp = scale * M_S^{-1} rp = scale * Ap^+ F1 Q1^{-1} rp (mean-free), Q1^{-1} by
// `cheb` Chebyshev steps, Ap^+ by `its` PCG steps; F1 (or F1^T, adjoint set-up)
// with the element convection matrices of pcd_setup.
template <class T>
static eth_status pcd_schur(eth_grid* g, Work* w, const double* rp, double* zp, double scale, int cheb, int its,
                            const int* done) {
  GMRESWork* G = w->gm;
  const int m = g->n1;
  T* a = pv<T>(G, 1);
  T* fa = pv<T>(G, 5);
  ETH_TRY(q1_mass_inv<T>(g, G, rp, a, cheb, done));
  {
    Q1Params<T, T, T> P{};
    P.n = g->n; P.hx = (T)g->hx; P.hy = (T)g->hy; P.cm = 0; P.ck = (T)g->nu; P.c1 = 0;
    P.conv = PcdPtr<T>::c1(G); P.x = a; P.y = fa; P.done = done;
    k_q1node<T, T, T, Q1E_APPLY><<<q1_blocks(g->n), 256, 0, g->s>>>(P);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
  }
  T* sol = pv<T>(G, 1);   // a no longer needed
  // ap_solve uses pv 0,4,5,7: copy the right-hand side out of slot 5 first
  T* rhs = pv<T>(G, 3);
  k_copy_t<T><<<gb(m), 256, 0, g->s>>>(m, fa, rhs);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  ETH_TRY(ap_solve<T>(g, w, rhs, sol, its, done));
  k_sum_t<T><<<gb(m), 256, 0, g->s>>>(m, sol, G->part, G->ticket + 2, &G->gs->pcg[3]);
  k_pcd_out<T><<<gb(m), 256, 0, g->s>>>(m, sol, zp, G->gs, scale);
  ETH_CUDA(cudaGetLastError());
  g->launches += 2;
  return ETH_OK;
}

// Step I preconditioner on [r_u; r_p1]: z_p = -Ap^+ F1 Q1^{-1} r_p, z_u = V_F(r_u - B1^T z_p)
template <class T>
static eth_status precond_pcd(eth_grid* g, Work* w, const eth_opts* o, const double* r, double* z, const int* done, bool adj) {
  const size_t nu2 = 2 * (size_t)g->nv;
  ETH_TRY(pcd_schur<T>(g, w, r + nu2, z + nu2, -1.0, 10, 2, done));
  return vel_part<T>(g, w, o, r, z + nu2, false, z, done, adj);
}

// Step II preconditioner M_1: z_p = -nu M_Q^+ r_p (k projected out), z_u = V_F(r_u - B^T z_p)
template <class T>
static eth_status precond_m1(eth_grid* g, Work* w, const eth_opts* o, const double* r, double* z, const int* done, bool adj) {
  const size_t nu2 = 2 * (size_t)g->nv;
  const int nb = vblocks((size_t)g->n1 + g->n0);
  k_psums<0><<<nb, 256, 0, g->s>>>(nu2, (size_t)g->n1, (size_t)g->n0, r, slot_of(g, SL_VSUM, nb, FIN_VSUMS));
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  Slot gs = slot_of(g, SL_GEN, mq_blocks(g), FIN_STORE);
  ETH_TRY(precond_pressure<T>(g, q1_hier<T>(w), r + nu2, z + nu2, gs, 0, done, g->s));
  return vel_part<T>(g, w, o, r, z + nu2, true, z, done, adj);
}

// y = K x for the active system (stage 1: reduced [F B1^T; B1 0], stages 2 and 3: full)
static eth_status sys_apply(eth_grid* g, int stage, bool fp32, bool trans, const double* x, double* y) {
  const eth_op op = stage == 1 ? (trans ? ETH_OP_K1T : ETH_OP_K1) : (trans ? ETH_OP_KT : ETH_OP_K);
  return op_apply(g, op, fp32, x, y);
}

// One Arnoldi step (preconditioner, operator, Gram-Schmidt, normalisation) with the
// column index read on the device (GScalars::jcur), so the same launches serve
// every column: this is what the graph-replayed loop captures once per stage.
template <class T>
static eth_status gm_iter_kernels(eth_grid* g, Work* w, const eth_opts* o, int stage, bool fp32, bool adj, size_t ntv) {
  GMRESWork* G = w->gm;
  const size_t ld = G->cap;
  const int nb = gb(ntv);
  const int* done = &G->gs->done;
  const int* jp = &G->gs->jcur;
  const int* sk = &G->gs->skip2;
  double* h1 = &G->gs->h1[0];
  double* h2 = &G->gs->h2[0];
  k_gm_col_in<<<nb, 256, 0, g->s>>>(ntv, G->V, ld, G->gs, G->vin);
  ETH_CUDA(cudaGetLastError());
  if (stage == 1) ETH_TRY(precond_pcd<T>(g, w, o, G->vin, G->zout, done, adj));
  else if (stage == 3) ETH_TRY(precond_lsc<T>(g, w, o, G->vin, G->zout, done, adj));
  else ETH_TRY(precond_m1<T>(g, w, o, G->vin, G->zout, done, adj));
  k_gm_col_out<<<nb, 256, 0, g->s>>>(ntv, G->zout, G->Z, ld, G->gs);
  ETH_CUDA(cudaGetLastError());
  ETH_TRY(sys_apply(g, stage, fp32, adj, G->zout, G->w));
  ETH_TRY(launch_mdot(G, nb, g->s, ntv, ld, 1, h1, done, nullptr, 1, jp));
  k_mupd<<<nb, 256, 0, g->s>>>(ntv, G->V, ld, 1, h1, G->w, 2, G->part, G->ticket + 4, G->gs, 0, done, nullptr, jp);
  ETH_TRY(launch_mdot(G, nb, g->s, ntv, ld, 1, h2, done, sk, 0, jp));
  k_mupd<<<nb, 256, 0, g->s>>>(ntv, G->V, ld, 1, h2, G->w, 1, G->part, G->ticket + 4, G->gs, 0, done, sk, jp);
  k_vscale<<<nb, 256, 0, g->s>>>(ntv, G->w, G->V, G->gs, 0, ld, jp);
  k_gm_next<<<1, 1, 0, g->s>>>(G->gs);
  ETH_CUDA(cudaGetLastError());
  g->launches += 8;
  return ETH_OK;
}

template <class T>
// Restarted flexible GMRES; every cycle starts from the FP64 residual of the
// current iterate (a refinement step).  In mixed precision the Arnoldi
// products K z run in FP32; a cycle can then only reduce the FP64 residual
// as far as the FP32 products represent K z, and when the preconditioned
// vectors z are large against K z (poor preconditioning at high cell Peclet
// number) the FP64 residual can even grow.  After such a cycle the products
// of the remaining cycles run in FP64 (*escalated = 1).
static eth_status gmres_run(eth_grid* g, Work* w, const eth_opts* o, int stage, bool adj, const double* b, double* x,
                            size_t ntv, double tol_abs, int maxit, int* its_out, double* res_out, int* status,
                            int* escalated) {
  GMRESWork* G = w->gm;
  int m = std::max(1, std::min(o->restart, G->m));   // cycle length (adaptive up to G->m)
  const size_t ld = G->cap;
  bool fp32 = o->precision == ETH_MIXED;
  const int nb = gb(ntv);
  int its = 0;
  *status = 0;
  *escalated = 0;
  double res = 0.0, res_prev = -1.0;
  const bool use_graph = o->graph != 0;
  cudaGraphExec_t gexec = nullptr;
  int gfp32 = -1;
  long glaunch = 0;
  struct GraphGuard {
    cudaGraphExec_t* e;
    ~GraphGuard() { if (*e) cudaGraphExecDestroy(*e); }
  } guard{&gexec};
  while (true) {
    ETH_TRY(sys_apply(g, stage, false, adj, x, G->w));
    k_gm_resid<<<nb, 256, 0, g->s>>>(ntv, b, G->w, G->V, G->part, G->ticket, G->gs, tol_abs);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
    ETH_CUDA(cudaMemcpyAsync(G->gsh, G->gs, sizeof(GScalars), cudaMemcpyDeviceToHost, g->s));
    ETH_CUDA(cudaStreamSynchronize(g->s));
    res = G->gsh->beta;
    if (o->verbose) fprintf(stderr, "[eth] stage %d restart: its %d res %.3e (tol %.3e)\n", stage, its, res, tol_abs);
    if (!std::isfinite(res)) { *status = ETH_ENAN; break; }
    if (res <= tol_abs || its >= maxit) break;
    if (fp32 && res_prev >= 0.0 && res > res_prev) {
      fp32 = false;
      *escalated = 1;
      if (o->verbose) fprintf(stderr, "[eth] stage %d: FP64 residual grew, Arnoldi products now FP64\n", stage);
    }
    if (res_prev >= 0.0 && res > 0.5 * res_prev && m < G->m) {
      m = std::min(2 * m, G->m);
      if (o->verbose) fprintf(stderr, "[eth] stage %d: slow restart cycle, restart length now %d\n", stage, m);
    }
    res_prev = res;
    k_vscale<<<nb, 256, 0, g->s>>>(ntv, G->V, G->V, G->gs, 1);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
    const int* done = &G->gs->done;
    if (use_graph) {
      // the captured Arnoldi step, replayed in chunks; the host checks convergence after
      // each chunk (steps after the converged one return at once: every kernel checks done)
      if (!gexec || gfp32 != (int)fp32) {
        if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
        cudaGraph_t graph;
        const long l0 = g->launches;
        ETH_CUDA(cudaStreamBeginCapture(g->s, cudaStreamCaptureModeThreadLocal));
        const eth_status cs = gm_iter_kernels<T>(g, w, o, stage, fp32, adj, ntv);
        const cudaError_t ce = cudaStreamEndCapture(g->s, &graph);
        glaunch = g->launches - l0;
        g->launches = l0;
        if (cs != ETH_OK) { if (ce == cudaSuccess) cudaGraphDestroy(graph); return cs; }
        ETH_CUDA(ce);
        const cudaError_t ie = cudaGraphInstantiate(&gexec, graph, 0);
        cudaGraphDestroy(graph);
        ETH_CUDA(ie);
        gfp32 = (int)fp32;
      }
      int j = 0;
      while (j < m && its < maxit) {
        const int ch = std::min(GM_CHUNK, std::min(m - j, maxit - its));
        for (int c = 0; c < ch; ++c) ETH_CUDA(cudaGraphLaunch(gexec, g->s));
        g->launches += ch * glaunch;
        ETH_CUDA(cudaMemcpyAsync(&G->gsh->res, &G->gs->res, 4 * sizeof(double), cudaMemcpyDeviceToHost, g->s));
        ETH_CUDA(cudaMemcpyAsync(&G->gsh->k, &G->gs->k, 4 * sizeof(int), cudaMemcpyDeviceToHost, g->s));
        ETH_CUDA(cudaStreamSynchronize(g->s));
        if (G->gsh->done) { its += G->gsh->k - j; break; }
        j += ch;
        its += ch;
      }
    }
    for (int j = 0; !use_graph && j < m && its < maxit; ++j) {
      double* Vj = G->V + (size_t)j * ld;
      double* Zj = G->Z + (size_t)j * ld;
      if (stage == 1) ETH_TRY(precond_pcd<T>(g, w, o, Vj, Zj, done, adj));
      else if (stage == 3) ETH_TRY(precond_lsc<T>(g, w, o, Vj, Zj, done, adj));
      else ETH_TRY(precond_m1<T>(g, w, o, Vj, Zj, done, adj));
      ETH_TRY(sys_apply(g, stage, fp32, adj, Zj, G->w));
      double* h1 = &G->gs->h1[0];
      double* h2 = &G->gs->h2[0];
      // classical Gram-Schmidt with selective reorthogonalisation (DGKS, 0.7)
      const int* sk = &G->gs->skip2;
      ETH_TRY(launch_mdot(G, nb, g->s, ntv, ld, j + 1, h1, done, nullptr, 1));
      k_mupd<<<nb, 256, 0, g->s>>>(ntv, G->V, ld, j + 1, h1, G->w, 2, G->part, G->ticket + 4, G->gs, j, done, nullptr, nullptr);
      ETH_TRY(launch_mdot(G, nb, g->s, ntv, ld, j + 1, h2, done, sk, 0));
      k_mupd<<<nb, 256, 0, g->s>>>(ntv, G->V, ld, j + 1, h2, G->w, 1, G->part, G->ticket + 4, G->gs, j, done, sk, nullptr);
      k_vscale<<<nb, 256, 0, g->s>>>(ntv, G->w, G->V + (size_t)(j + 1) * ld, G->gs, 0);
      ETH_CUDA(cudaGetLastError());
      g->launches += 5;
      its++;
      ETH_CUDA(cudaMemcpyAsync(&G->gsh->res, &G->gs->res, 4 * sizeof(double), cudaMemcpyDeviceToHost, g->s));
      ETH_CUDA(cudaMemcpyAsync(&G->gsh->k, &G->gs->k, 4 * sizeof(int), cudaMemcpyDeviceToHost, g->s));
      ETH_CUDA(cudaStreamSynchronize(g->s));
      if (G->gsh->done) break;
    }
    k_gm_solve<<<1, 1, 0, g->s>>>(G->gs);
    k_zupd<<<nb, 256, 0, g->s>>>(ntv, G->Z, ld, G->gs, x);
    ETH_CUDA(cudaGetLastError());
    g->launches += 2;
    if (G->gsh->bdown) { *status = G->gsh->bdown; }
  }
  *its_out = its;
  *res_out = res;
  return ETH_OK;
}

__global__ void k_copy_d(size_t m, const double* __restrict__ a, double* __restrict__ b) {
  ETH_GRID_DEP_WAIT();
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) b[k] = a[k];
}

// Prop. 2 quantities at the stage switch: ||z*||^2 and ||r0*||^2 (P0 block)
__global__ void k_prop2(size_t nt, size_t off0, const double* __restrict__ r, double* part, unsigned* ticket, double* out) {
  ETH_GRID_DEP_WAIT();
  double a = 0.0, c = 0.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < nt; k += (size_t)gridDim.x * blockDim.x) {
    const double v = r[k] * r[k];
    a += v;
    if (k >= off0) c += v;
  }
  double v[2] = {a, c};
  block_sum<2>(v);
  if (threadIdx.x == 0) { part[blockIdx.x] = v[0]; part[gridDim.x + blockIdx.x] = v[1]; }
  multi_finish(2, gridDim.x, part, ticket, out);
}

template <class T>
static eth_status two_stage(eth_grid* g, Work* w, const eth_opts* o, eth_stats* st, bool adj, const double* b) {
  const size_t nt = g->nt, nu2 = 2 * (size_t)g->nv, nt1 = nu2 + g->n1;
  GMRESWork* G = w->gm;
  ETH_TRY(pcd_setup<T>(g, w, adj));
  k_oseen_scalars<<<1, 1, 0, g->s>>>(g->sc, (double)g->n1, (double)g->n0, 16.0 / (g->hx * g->hy), -g->nu);
  ETH_CUDA(cudaGetLastError());
  // norms of b and of the reduced right-hand side
  k_prop2<<<gb(nt), 256, 0, g->s>>>(nt, nt1, b, G->part, G->ticket + 5, &G->gs->pcg[0]);
  ETH_CUDA(cudaMemcpyAsync(G->gsh, G->gs, sizeof(GScalars), cudaMemcpyDeviceToHost, g->s));
  ETH_CUDA(cudaStreamSynchronize(g->s));
  const double nb2 = std::sqrt(G->gsh->pcg[0]);
  const double nbred = std::sqrt(std::max(G->gsh->pcg[0] - G->gsh->pcg[1], 0.0));
  if (!std::isfinite(nb2)) { st->relres_true = nb2; return ETH_ENAN; }   // NaN or Inf in the right-hand side
  if (!(nb2 > 0.0)) { ETH_CUDA(cudaMemsetAsync(w->x, 0, nt * 8, g->s)); st->relres_true = 0; return ETH_OK; }
  const double eta = o->tol;
  int its1 = 0, its2 = 0, s1 = 0, s2 = 0, e1 = 0, e2 = 0;
  double res1 = 0, res2 = 0;
  // Step I: reduced system on [u; p1], p0 = 0
  ETH_TRY(gmres_run<T>(g, w, o, 1, adj, b, w->x, nt1, o->c_stage * eta * nbred, o->maxit, &its1, &res1, &s1, &e1));
  ETH_CUDA(cudaMemsetAsync(w->x + nt1, 0, (nt - nt1) * 8, g->s));
  // Prop. 2 at the switch (FP64 residual of the full system)
  ETH_TRY(sys_apply(g, 2, false, adj, w->x, G->w));
  k_gm_resid<<<gb(nt), 256, 0, g->s>>>(nt, b, G->w, G->t, G->part, G->ticket, G->gs, 0.0);
  k_prop2<<<gb(nt), 256, 0, g->s>>>(nt, nt1, G->t, G->part, G->ticket + 5, &G->gs->pcg[0]);
  ETH_CUDA(cudaMemcpyAsync(G->gsh, G->gs, sizeof(GScalars), cudaMemcpyDeviceToHost, g->s));
  ETH_CUDA(cudaStreamSynchronize(g->s));
  st->prop2_lhs = G->gsh->pcg[0];
  st->prop2_bound = std::pow(o->c_stage * eta * nbred, 2) + G->gsh->pcg[1];
  // Step II: full system with M_1
  ETH_TRY(gmres_run<T>(g, w, o, 2, adj, b, w->x, nt, eta * nb2, o->maxit - its1, &its2, &res2, &s2, &e2));
  ETH_TRY(canonicalize(g, w->x));
  double rr;
  ETH_TRY(true_residual(g, w, b, &rr, adj));
  st->iters_stage1 = its1;
  st->iters_stage2 = its2;
  st->iters_total = its1 + its2;
  st->refine_passes = 0;
  st->escalations = e1 + e2;
  st->relres_true = std::sqrt(rr) / nb2;
  if (s1 == ETH_ENAN || s2 == ETH_ENAN || !std::isfinite(st->relres_true)) return ETH_ENAN;
  return st->relres_true <= eta * (1.0 + 1e-9) ? ETH_OK : ETH_ENOTCONV;
}

// One flexible GMRES run on the full system with the LSC preconditioner M_3 (Sec. 3.2)
// from the lifted boundary data to eta ||b||; the stage statistics report it as Step II.
template <class T>
static eth_status lsc_solve(eth_grid* g, Work* w, const eth_opts* o, eth_stats* st, bool adj, const double* b) {
  const size_t nt = g->nt;
  GMRESWork* G = w->gm;
  ETH_TRY(lsc_prepare<T>(g, w));   // allocations before the Arnoldi step is captured
  k_oseen_scalars<<<1, 1, 0, g->s>>>(g->sc, (double)g->n1, (double)g->n0, 16.0 / (g->hx * g->hy), -g->nu);
  k_prop2<<<gb(nt), 256, 0, g->s>>>(nt, nt, b, G->part, G->ticket + 5, &G->gs->pcg[0]);
  ETH_CUDA(cudaGetLastError());
  ETH_CUDA(cudaMemcpyAsync(G->gsh, G->gs, sizeof(GScalars), cudaMemcpyDeviceToHost, g->s));
  ETH_CUDA(cudaStreamSynchronize(g->s));
  const double nb2 = std::sqrt(G->gsh->pcg[0]);
  if (!std::isfinite(nb2)) { st->relres_true = nb2; return ETH_ENAN; }
  if (!(nb2 > 0.0)) { ETH_CUDA(cudaMemsetAsync(w->x, 0, nt * 8, g->s)); st->relres_true = 0; return ETH_OK; }
  int its = 0, s2 = 0, e2 = 0;
  double res = 0;
  ETH_TRY(gmres_run<T>(g, w, o, 3, adj, b, w->x, nt, o->tol * nb2, o->maxit, &its, &res, &s2, &e2));
  ETH_TRY(canonicalize(g, w->x));
  double rr;
  ETH_TRY(true_residual(g, w, b, &rr, adj));
  st->iters_stage1 = 0;
  st->iters_stage2 = its;
  st->iters_total = its;
  st->refine_passes = 0;
  st->escalations = e2;
  st->relres_true = std::sqrt(rr) / nb2;
  if (s2 == ETH_ENAN || !std::isfinite(st->relres_true)) return ETH_ENAN;
  return st->relres_true <= o->tol * (1.0 + 1e-9) ? ETH_OK : ETH_ENOTCONV;
}

// M_S^{-1} rp alone, with chosen inner step counts (eth_apply_pcd).
template <class T>
static eth_status apply_pcd_t(eth_grid* g, Work* w, bool adjoint, int cheb, int its, const double* rp, double* zp) {
  eth_opts o;
  eth_default_opts(&o);
  o.precision = sizeof(T) == 4 ? ETH_MIXED : ETH_FP64;
  ETH_TRY(ensure_hier<T>(g, w, &o));
  if (!w->gm) ETH_TRY(gm_alloc(g, w, 1));
  ETH_TRY(pcd_setup<T>(g, w, adjoint));
  return pcd_schur<T>(g, w, rp, zp, 1.0, cheb, its, nullptr);
}

// GMRES workspace and the Gram-Schmidt autotuning of an Oseen grid ahead of its solve
// (the batch driver runs this for every instance before the instances overlap, so the
// tuner times its kernels on an otherwise idle GPU)
eth_status oseen_prepare(eth_grid* g, Work* w, const eth_opts* o) {
  const int m = std::max(1, std::min(std::max(o->restart, o->restart_max), GM_MAX));
  ETH_TRY(gm_alloc(g, w, m));
  if (o->autotune && !w->gm->grp_tuned) ETH_TRY(tune_cgs(g, w->gm));
  return ETH_OK;
}

eth_status oseen_solve(eth_grid* g, Work* w, const eth_opts* o, eth_stats* st, bool adjoint, const double* bsrc) {
  ETH_TRY(oseen_prepare(g, w, o));
  // consistent right-hand side (e1 / e0 components removed)
  ETH_CUDA(cudaMemcpyAsync(w->bp, bsrc, (size_t)g->nt * 8, cudaMemcpyDeviceToDevice, g->s));
  ETH_TRY(canonicalize(g, w->bp));
  double incons = 0.0, nbp = 0.0;
  ETH_TRY(rhs_inconsistency(g, w, w->bp, &incons, &nbp));
  eth_status r;
  if (o->precision == ETH_MIXED) {
    ETH_TRY(ensure_hier<float>(g, w, o));
    r = o->oseen_prec == 1 ? lsc_solve<float>(g, w, o, st, adjoint, w->bp) : two_stage<float>(g, w, o, st, adjoint, w->bp);
  } else {
    ETH_TRY(ensure_hier<double>(g, w, o));
    r = o->oseen_prec == 1 ? lsc_solve<double>(g, w, o, st, adjoint, w->bp) : two_stage<double>(g, w, o, st, adjoint, w->bp);
  }
  // the solve used the projected right-hand side; report a removed component as for Stokes
  if (r == ETH_OK && std::isfinite(nbp) && nbp > 0.0 && incons > 1e-8 * nbp) r = ETH_EINCONSISTENT;
  return r;
}

}  // namespace eth

using namespace eth;

extern "C" eth_status eth_apply_pcd(eth_grid* g, int adjoint, int fp32, int cheb_steps, int ap_its, const double* rp_dev,
                                    double* zp_dev) {
  if (!g || !rp_dev || !zp_dev) { set_error("eth_apply_pcd: NULL argument"); return ETH_EINVAL; }
  if (g->kind != ETH_OSEEN) { set_error("eth_apply_pcd: the PCD block belongs to ETH_OSEEN grids"); return ETH_EINVAL; }
  if (!g->has_coef) { set_error("eth_apply_pcd: call eth_set_coefficients first"); return ETH_EINVAL; }
  if (cheb_steps < 0 || cheb_steps > 1000 || ap_its < 1 || ap_its > 1000) {
    set_error("eth_apply_pcd: cheb_steps=%d (0..1000) or ap_its=%d (1..1000) out of range", cheb_steps, ap_its);
    return ETH_EINVAL;
  }
  ETH_ON_DEVICE(g);
  Work* w;
  ETH_TRY(work_get(g, &w));
  StreamSwap guard(g, w);
  return fp32 ? apply_pcd_t<float>(g, w, adjoint != 0, cheb_steps, ap_its, rp_dev, zp_dev)
              : apply_pcd_t<double>(g, w, adjoint != 0, cheb_steps, ap_its, rp_dev, zp_dev);
}
