// Least-squares commutator (LSC) preconditioner M_3 for the Oseen system with the
// two-field pressure (Sec. 3.2, Eq. lsc-definition and Eq. nse-precon-lsc):
//
//   M_3 = [ F  B^T ; 0  -M_S ],
//   M_S^{-1} = (B M^{-1} B^T)^+ (B M^{-1} F H^{-1} B^T) (B H^{-1} B^T)^+,
//
// with B = [B1; B0] on the whole frame Q1 + P0 (interior velocity columns), M the
// diagonal of the Q2 velocity mass and H = M (plain LSC: D = I).  Both outer
// factors are then solves with the frame operator S = B M^{-1} B^T, singular on
// span{e1, e0} (constant Q1 and constant P0 pressure).  They run as a fixed
// number of conjugate-gradient steps on the complement of span{e1, e0} with a
// block-diagonal preconditioner: the Q1 block of S is spectrally equivalent to
// the Q1 Laplacian (the existing Q1 V-cycle), the P0 block to 3.8 times the
// cell-centred 5-point Laplacian (a cell-centred V-cycle defined here: damped
// Jacobi, bilinear cell-centred prolongation with weights 9/16, 3/16, 3/16,
// 1/16, restriction its transpose, the 5-point operator rediscretised on every
// level, damped Jacobi sweeps on the coarsest grid).  The middle factor is one
// B^T, two diagonal scalings, one F apply and one B.  The velocity block of M_3
// is the F V-cycle of the two-stage solver.  A fixed step count makes M_3 a
// fixed (if nonlinear) map per application, which flexible GMRES accepts, and
// keeps every launch capturable in the replayed Arnoldi step.
#include <algorithm>
#include <cmath>
#include <vector>
#include "solve.cuh"

namespace eth {

// ---------------------------------------------------------------------------
// cell-centred 5-point Laplacian on an n x n cell grid (natural boundary):
// (L x)_c = sum over existing edge neighbours (x_c - x_nb), diagonal d_c = count
// ---------------------------------------------------------------------------
// bilinear cell-centred prolongation, 1D: fine cell f = 2I + a takes 3/4 of coarse
// cell I and 1/4 of its neighbour on the side of f (I - 1 for a = 0, I + 1 for a = 1),
// or all of I when that neighbour lies outside the grid
__device__ __forceinline__ void p0_pw(int f, int nc, int& i0, int& i1, float& w0, float& w1) {
  const int I = f >> 1, nb = (f & 1) ? I + 1 : I - 1;
  i0 = I;
  if (nb >= 0 && nb < nc) { i1 = nb; w0 = 0.75f; w1 = 0.25f; }
  else { i1 = I; w0 = 1.0f; w1 = 0.0f; }
}

// first Jacobi sweep from zero and its residual: x = om b / d, r = b - L x
template <class T>
__global__ void k_p0_down(int n, T om, const T* __restrict__ b, T* __restrict__ x, T* __restrict__ r, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n * n; c += gridDim.x * blockDim.x) {
    const int ey = c / n, ex = c - ey * n;
    int cnt = 0;
    T nbs = 0;
    auto nbx = [&](int i, int j) {
      const int e = j * n + i;
      const int d = (i > 0) + (i < n - 1) + (j > 0) + (j < n - 1);
      nbs += om * b[e] / (T)d;
      ++cnt;
    };
    if (ex > 0) nbx(ex - 1, ey);
    if (ex < n - 1) nbx(ex + 1, ey);
    if (ey > 0) nbx(ex, ey - 1);
    if (ey < n - 1) nbx(ex, ey + 1);
    const T xc = om * b[c] / (T)cnt;
    x[c] = xc;
    r[c] = b[c] - ((T)cnt * xc - nbs);
  }
}

// restriction (transpose of the prolongation): bc(I, J) = sum_f P(f, I) P(g, J) r(f, g)
template <class T>
__global__ void k_p0_restrict(int nc, const T* __restrict__ r, T* __restrict__ bc, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  const int nf = 2 * nc;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc * nc; c += gridDim.x * blockDim.x) {
    const int J = c / nc, I = c - J * nc;
    T wx[4], wy[4];
    int fx[4], fy[4];
    // fine cells 2I-1 .. 2I+2 and their weights toward coarse cell I
    auto w1d = [&](int K, int (&f)[4], T (&w)[4]) {
      f[0] = 2 * K - 1; w[0] = K >= 1 ? T(0.25) : T(0);
      f[1] = 2 * K;     w[1] = K >= 1 ? T(0.75) : T(1);
      f[2] = 2 * K + 1; w[2] = K + 1 < nc ? T(0.75) : T(1);
      f[3] = 2 * K + 2; w[3] = K + 1 < nc ? T(0.25) : T(0);
    };
    w1d(I, fx, wx);
    w1d(J, fy, wy);
    T acc = 0;
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (wx[u] != T(0) && wy[v] != T(0) && fx[u] >= 0 && fx[u] < nf && fy[v] >= 0 && fy[v] < nf)
          acc += wx[u] * wy[v] * r[fy[v] * nf + fx[u]];
    bc[c] = acc;
  }
}

// coarse-grid correction and one Jacobi sweep: xo = s * (y + om (b - L y) / d) with
// y = x + P xc, evaluated at the cell and its neighbours
template <class T>
__global__ void k_p0_up(int n, T om, const T* __restrict__ b, const T* __restrict__ x, const T* __restrict__ xc,
                        T* __restrict__ xo, T s, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  const int nc = n / 2;
  auto y = [&](int i, int j) -> T {
    int ix0, ix1, iy0, iy1;
    float ax0, ax1, ay0, ay1;
    p0_pw(i, nc, ix0, ix1, ax0, ax1);
    p0_pw(j, nc, iy0, iy1, ay0, ay1);
    T v = x[j * n + i];
    v += (T)(ax0 * ay0) * xc[iy0 * nc + ix0];
    if (ax1 != 0.f) v += (T)(ax1 * ay0) * xc[iy0 * nc + ix1];
    if (ay1 != 0.f) v += (T)(ax0 * ay1) * xc[iy1 * nc + ix0];
    if (ax1 != 0.f && ay1 != 0.f) v += (T)(ax1 * ay1) * xc[iy1 * nc + ix1];
    return v;
  };
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n * n; c += gridDim.x * blockDim.x) {
    const int ey = c / n, ex = c - ey * n;
    const T yc = y(ex, ey);
    int cnt = 0;
    T nbs = 0;
    if (ex > 0) { nbs += y(ex - 1, ey); ++cnt; }
    if (ex < n - 1) { nbs += y(ex + 1, ey); ++cnt; }
    if (ey > 0) { nbs += y(ex, ey - 1); ++cnt; }
    if (ey < n - 1) { nbs += y(ex, ey + 1); ++cnt; }
    xo[c] = s * (yc + om * (b[c] - ((T)cnt * yc - nbs)) / (T)cnt);
  }
}

// coarsest grid: `sweeps` damped Jacobi sweeps from zero in one CTA (a fixed
// polynomial in D^{-1} L, so the V-cycle stays a symmetric linear map), output scaled by s
template <class T>
__global__ void k_p0_coarse(int n, T om, int sweeps, const T* __restrict__ b, T* __restrict__ x, T s, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char p0_smem[];
  T* xs = reinterpret_cast<T*>(p0_smem);
  T* xt = xs + n * n;
  const int m = n * n;
  for (int c = threadIdx.x; c < m; c += blockDim.x) xs[c] = 0;
  __syncthreads();
  for (int it = 0; it < sweeps; ++it) {
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
      const int ey = c / n, ex = c - ey * n;
      int cnt = 0;
      T nbs = 0;
      if (ex > 0) { nbs += xs[c - 1]; ++cnt; }
      if (ex < n - 1) { nbs += xs[c + 1]; ++cnt; }
      if (ey > 0) { nbs += xs[c - n]; ++cnt; }
      if (ey < n - 1) { nbs += xs[c + n]; ++cnt; }
      xt[c] = xs[c] + om * (b[c] - ((T)cnt * xs[c] - nbs)) / (T)cnt;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < m; c += blockDim.x) xs[c] = xt[c];
    __syncthreads();
  }
  for (int c = threadIdx.x; c < m; c += blockDim.x) x[c] = s * xs[c];
}

// ---------------------------------------------------------------------------
// frame vectors [q1 (m1); q0 (m - m1)] of type T
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_l_load(int m, const double* __restrict__ a, T* __restrict__ b, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) b[k] = (T)a[k];
}

// block sums of a -> out[0] (Q1), out[1] (P0)
template <class T>
__global__ void k_l_sums(int m1, int m, const T* __restrict__ a, Slot sl, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  double s1 = 0.0, s0 = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    if (k < m1) s1 += (double)a[k]; else s0 += (double)a[k];
  }
  double v[2] = {s1, s0};
  if (slot_arrive<2>(sl, blockIdx.x, v)) finish_slot_n<2>(sl, v);
}

// a -= block means (sums in s[0], s[1])
template <class T>
__global__ void k_l_center(int m1, int m, T* __restrict__ a, const double* s, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  const T mu1 = (T)(s[0] / m1), mu0 = (T)(s[1] / (m - m1));
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) a[k] -= k < m1 ? mu1 : mu0;
}

// (<r, z>, sum z_1, sum z_0) -> out[0..2]
template <class T>
__global__ void k_l_dot3(int m1, int m, const T* __restrict__ r, const T* __restrict__ z, Slot sl, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  double a = 0.0, s1 = 0.0, s0 = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    const double zk = (double)z[k];
    a += (double)r[k] * zk;
    if (k < m1) s1 += zk; else s0 += zk;
  }
  double v[3] = {a, s1, s0};
  if (slot_arrive<3>(sl, blockIdx.x, v)) finish_slot_n<3>(sl, v);
}

// p = (z - block means of z) + beta p, beta = cur[0] / prev[0] (0 on the first step,
// which also keeps cur[0] as the initial <r, z> in *rz0)
template <class T>
__global__ void k_l_p(int m1, int m, const T* __restrict__ z, T* __restrict__ p, const double* cur, const double* prev,
                      double* rz0, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  const T bt = (T)(prev ? (prev[0] != 0.0 ? cur[0] / prev[0] : 0.0) : 0.0);
  const T mu1 = (T)(cur[1] / m1), mu0 = (T)(cur[2] / (m - m1));
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x)
    p[k] = (z[k] - (k < m1 ? mu1 : mu0)) + (prev ? bt * p[k] : T(0));
  if (!prev && blockIdx.x == 0 && threadIdx.x == 0) *rz0 = cur[0];
}

// x += alpha p, r -= alpha q with alpha = rz / pAp; a converged CG (rz at the rounding
// level of T relative to its initial value) leaves x alone
template <class T>
__global__ void k_l_xr(int m, const T* __restrict__ p, const T* __restrict__ q, T* __restrict__ x, T* __restrict__ r,
                       const double* rz, const double* pap, const double* rz0, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  const double fl = (sizeof(T) == 4 ? 1e-13 : 1e-28) * *rz0;
  const T a = (T)((*pap > 0.0 && *rz > fl) ? *rz / *pap : 0.0);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    x[k] += a * p[k];
    r[k] -= a * q[k];
  }
}

template <class T>
__global__ void k_l_out(int m, const T* __restrict__ x, double* __restrict__ y, double s, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) y[k] = s * (double)x[k];
}

template <class T>
__global__ void k_l_copy(int m, const T* __restrict__ a, T* __restrict__ b, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) b[k] = a[k];
}

// level-0 right-hand side of the Q1 V-cycle and its first Jacobi step from zero
template <class T>
__global__ void k_l_q1j0(int m, T om, const T* __restrict__ dinv, const T* __restrict__ r, T* __restrict__ b,
                         T* __restrict__ x, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done && *done) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    const T v = r[k];
    b[k] = v;
    x[k] = om * dinv[k] * v;
  }
}

// inverse of the diagonal of the Q2 velocity mass (M of Eq. lsc-definition), 0 on the boundary
template <class T>
__global__ void k_l_mdiag(int n, double hx, double hy, T* __restrict__ md) {
  ETH_GRID_DEP_WAIT();
  const int N = 2 * n + 1;
  for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < N * N; node += gridDim.x * blockDim.x) {
    const int j = node / N, i = node - j * N;
    if (i == 0 || j == 0 || i == N - 1 || j == N - 1) { md[node] = 0; continue; }
    // per direction: 16/30 h at a midpoint (one element), 2 x 4/30 h at a vertex (two elements)
    const double dx = (i & 1) ? 16.0 / 30.0 * hx : 8.0 / 30.0 * hx;
    const double dy = (j & 1) ? 16.0 / 30.0 * hy : 8.0 / 30.0 * hy;
    md[node] = (T)(1.0 / (dx * dy));
  }
}

// ---------------------------------------------------------------------------
// workspace (per precision), owned by the solver workspace of a grid
// ---------------------------------------------------------------------------
constexpr float P0_OMEGA = 0.8f;       // damped Jacobi of the cell-centred V-cycle
constexpr int P0_COARSE_SWEEPS = 40;   // Jacobi sweeps on the coarsest cell grid
constexpr float P0_SCALE = 1.0f / 3.8f;   // P0 block of S ~ 3.8 x the 5-point Laplacian

template <class T>
struct LscWork {
  int n = 0;
  T* md = nullptr;                    // inverse velocity-mass diagonal (N_v)
  T *v1 = nullptr, *v2 = nullptr;     // velocity scratch (2 N_v each)
  double* vt = nullptr;               // FP64 velocity scratch (2 N_v): r_u - B^T z_p
  T *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *x = nullptr, *y = nullptr, *t = nullptr;   // frame
  std::vector<int> ln;                // cell-grid sizes of the P0 hierarchy (ln[0] = n)
  std::vector<T*> lb, lx, lr, lo;     // per level: rhs, first sweep, residual, output
  double* sc = nullptr;               // device scalars (see lsc_cg)
  double* part = nullptr;             // reduction partials
  unsigned* ticket = nullptr;
};

template <class T>
static void lsc_free_t(LscWork<T>* L) {
  if (!L) return;
  cudaFree(L->md); cudaFree(L->v1); cudaFree(L->v2); cudaFree(L->vt);
  cudaFree(L->r); cudaFree(L->z); cudaFree(L->p); cudaFree(L->q); cudaFree(L->x); cudaFree(L->y); cudaFree(L->t);
  for (size_t l = 0; l < L->ln.size(); ++l) {   // level 0 has no rhs / output arrays of its own (nullptr)
    cudaFree(L->lb[l]); cudaFree(L->lx[l]); cudaFree(L->lr[l]); cudaFree(L->lo[l]);
  }
  cudaFree(L->sc); cudaFree(L->part); cudaFree(L->ticket);
  delete L;
}

void lsc_free(Work* w) {
  lsc_free_t(static_cast<LscWork<float>*>(w->lscw[0]));
  lsc_free_t(static_cast<LscWork<double>*>(w->lscw[1]));
  w->lscw[0] = w->lscw[1] = nullptr;
}

constexpr int LSC_PART = 152 * 4;   // partial sums per reduction (the largest vblocks grid)

template <class T>
static eth_status lsc_get(eth_grid* g, Work* w, LscWork<T>** out) {
  void*& slot = w->lscw[sizeof(T) == 4 ? 0 : 1];
  if (slot) { *out = static_cast<LscWork<T>*>(slot); return ETH_OK; }
  LscWork<T>* L = new LscWork<T>();
  slot = L;
  L->n = g->n;
  const size_t nv = g->nv, m = (size_t)g->n1 + g->n0;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
  A((void**)&L->md, nv * sizeof(T));
  A((void**)&L->v1, 2 * nv * sizeof(T));
  A((void**)&L->v2, 2 * nv * sizeof(T));
  A((void**)&L->vt, 2 * nv * sizeof(double));
  A((void**)&L->r, m * sizeof(T)); A((void**)&L->z, m * sizeof(T)); A((void**)&L->p, m * sizeof(T));
  A((void**)&L->q, m * sizeof(T)); A((void**)&L->x, m * sizeof(T)); A((void**)&L->y, m * sizeof(T));
  A((void**)&L->t, m * sizeof(T));
  A((void**)&L->sc, 32 * sizeof(double));
  // partials: three sums per block of a vector reduction, or one per tile of the fused <p, S p>
  A((void**)&L->part, std::max((size_t)3 * LSC_PART, (size_t)q2_blocks(g->n)) * sizeof(double));
  A((void**)&L->ticket, 8 * sizeof(unsigned));
  // P0 hierarchy: halve while even and above 4 cells per side
  int k = g->n;
  L->ln.push_back(k);
  while (k % 2 == 0 && k > 4) { k /= 2; L->ln.push_back(k); }
  const int nl = (int)L->ln.size();
  L->lb.assign(nl, nullptr); L->lx.assign(nl, nullptr); L->lr.assign(nl, nullptr); L->lo.assign(nl, nullptr);
  for (int l = 0; l < nl; ++l) {
    const size_t c = (size_t)L->ln[l] * L->ln[l];
    if (l > 0) { A((void**)&L->lb[l], c * sizeof(T)); A((void**)&L->lo[l], c * sizeof(T)); }
    if (l + 1 < nl) { A((void**)&L->lx[l], c * sizeof(T)); A((void**)&L->lr[l], c * sizeof(T)); }
  }
  if (e != cudaSuccess) return cuda_status(e, "LSC workspace");
  ETH_CUDA(cudaMemsetAsync(L->ticket, 0, 8 * sizeof(unsigned), g->s));
  ETH_CUDA(cudaMemsetAsync(L->sc, 0, 32 * sizeof(double), g->s));
  k_l_mdiag<T><<<vblocks(nv), 256, 0, g->s>>>(g->n, g->hx, g->hy, L->md);
  ETH_CUDA(cudaGetLastError());
  const int Lc = L->ln.back();
  if (2 * (size_t)Lc * Lc * sizeof(T) > 48 * 1024) {
    set_error("LSC: coarsest cell grid %d x %d too large", Lc, Lc);
    return ETH_EINVAL;
  }
  *out = L;
  return ETH_OK;
}

template <class T>
static Slot lsc_slot(LscWork<T>* L, int ticket, double* out, int total) {
  Slot s{};
  s.part = L->part;
  s.ticket = L->ticket + ticket;
  s.out = out;
  s.total = total;
  s.op = FIN_STORE;
  s.sc = nullptr;
  return s;
}

// z0 = P0_SCALE * V(r0): one cell-centred V(1,1) cycle from zero on the P0 block
template <class T>
static eth_status p0_vcycle(eth_grid* g, LscWork<T>* L, const T* r0, T* z0, const int* done) {
  const int nl = (int)L->ln.size();
  const T om = (T)P0_OMEGA;
  for (int l = 0; l + 1 < nl; ++l) {
    const int n = L->ln[l];
    const T* b = l == 0 ? r0 : L->lb[l];
    k_p0_down<T><<<vblocks((size_t)n * n), 256, 0, g->s>>>(n, om, b, L->lx[l], L->lr[l], done);
    const int nc = L->ln[l + 1];
    k_p0_restrict<T><<<vblocks((size_t)nc * nc), 256, 0, g->s>>>(nc, L->lr[l], L->lb[l + 1], done);
  }
  {
    const int n = L->ln[nl - 1];
    const T* b = nl == 1 ? r0 : L->lb[nl - 1];
    T* o = nl == 1 ? z0 : L->lo[nl - 1];
    k_p0_coarse<T><<<1, 256, 2 * n * n * sizeof(T), g->s>>>(n, om, P0_COARSE_SWEEPS, b, o,
                                                               nl == 1 ? (T)P0_SCALE : T(1), done);
  }
  for (int l = nl - 2; l >= 0; --l) {
    const int n = L->ln[l];
    const T* b = l == 0 ? r0 : L->lb[l];
    T* o = l == 0 ? z0 : L->lo[l];
    k_p0_up<T><<<vblocks((size_t)n * n), 256, 0, g->s>>>(n, om, b, L->lx[l], L->lo[l + 1], o,
                                                          l == 0 ? (T)P0_SCALE : T(1), done);
  }
  ETH_CUDA(cudaGetLastError());
  g->launches += 3 * (nl - 1) + 1;
  return ETH_OK;
}

template <class T>
static const T* lsc_wind(eth_grid* g);
template <>
const float* lsc_wind<float>(eth_grid* g) { return g->windf; }
template <>
const double* lsc_wind<double>(eth_grid* g) { return g->wind; }

// z = blockdiag(V_K1, P0_SCALE V_L5) r: the preconditioner of the frame solves
template <class T>
static eth_status lsc_prec(eth_grid* g, Work* w, LscWork<T>* L, const T* r, T* z, const int* done) {
  Hier<T>& Q = q1_hier<T>(w);
  Level<T>& L0 = Q.lv[0];
  const int m1 = g->n1;
  k_l_q1j0<T><<<vblocks(m1), 256, 0, g->s>>>(m1, (T)Q.omega, L0.dinv, r, L0.b, L0.x, done);
  ETH_CUDA(cudaGetLastError());
  const T* res = nullptr;
  ETH_TRY(vcycle_q1_from<T>(g, Q, 1, 1, done, &res));
  k_l_copy<T><<<vblocks(m1), 256, 0, g->s>>>(m1, res, z, done);
  ETH_CUDA(cudaGetLastError());
  g->launches += 2;
  return p0_vcycle<T>(g, L, r + m1, z + m1, done);
}

// q = S p = B M^{-1} B^T p (frame operator); with pap, <p, q> fused into *pap
template <class T>
static eth_status lsc_S(eth_grid* g, LscWork<T>* L, const T* p, T* q, double* pap, const int* done) {
  {
    Q2Params<T, T, T> P{};
    P.n = g->n; P.hx = (T)g->hx; P.hy = (T)g->hy; P.nu = 0;
    P.p = p; P.y = L->v1; P.dinv = L->md; P.done = done;
    ETH_CUDA((launch_q2<T, T, T, QF_PIN | QF_P0 | QF_UOUT, EPI_SCALE>(P, g->s)));
  }
  {
    Q2Params<T, T, T> P{};
    P.n = g->n; P.hx = (T)g->hx; P.hy = (T)g->hy; P.nu = 0;
    P.x = L->v1; P.yp = q; P.done = done;
    P.slot = lsc_slot(L, 1, pap, q2_blocks(g->n));
    P.dvp = p;
    ETH_CUDA((launch_q2<T, T, T, QF_XIN | QF_P0 | QF_POUT | QF_DOT, EPI_APPLY>(P, g->s)));
  }
  g->launches += 2;
  return ETH_OK;
}

// x = S^+ b by `its` preconditioned CG steps on the complement of span{e1, e0};
// L->r holds b (block sums zero) on entry and the residual on exit.  Scalars in
// L->sc: [0..2] and [4..6] the alternating (<r, z>, sum z_1, sum z_0), [8] <p, S p>,
// [9] the initial <r, z>.
template <class T>
static eth_status lsc_cg(eth_grid* g, Work* w, LscWork<T>* L, T* x, int its, const int* done) {
  const int m1 = g->n1, m = g->n1 + g->n0, nb = vblocks(m);
  double *cur = L->sc, *nxt = L->sc + 4, *pap = L->sc + 8, *rz0 = L->sc + 9;
  ETH_CUDA(cudaMemsetAsync(x, 0, (size_t)m * sizeof(T), g->s));
  ETH_TRY(lsc_prec<T>(g, w, L, L->r, L->z, done));
  k_l_dot3<T><<<nb, 256, 0, g->s>>>(m1, m, L->r, L->z, lsc_slot(L, 0, cur, nb), done);
  k_l_p<T><<<nb, 256, 0, g->s>>>(m1, m, L->z, L->p, cur, nullptr, rz0, done);
  ETH_CUDA(cudaGetLastError());
  g->launches += 2;
  for (int k = 0; k < its; ++k) {
    ETH_TRY(lsc_S<T>(g, L, L->p, L->q, pap, done));
    k_l_xr<T><<<nb, 256, 0, g->s>>>(m, L->p, L->q, x, L->r, cur, pap, rz0, done);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
    if (k + 1 == its) break;
    ETH_TRY(lsc_prec<T>(g, w, L, L->r, L->z, done));
    k_l_dot3<T><<<nb, 256, 0, g->s>>>(m1, m, L->r, L->z, lsc_slot(L, 0, nxt, nb), done);
    k_l_p<T><<<nb, 256, 0, g->s>>>(m1, m, L->z, L->p, nxt, cur, rz0, done);
    ETH_CUDA(cudaGetLastError());
    g->launches += 2;
    std::swap(cur, nxt);
  }
  return ETH_OK;
}

// L->r -= its block means
template <class T>
static eth_status lsc_center(eth_grid* g, LscWork<T>* L, const int* done) {
  const int m1 = g->n1, m = g->n1 + g->n0, nb = vblocks(m);
  k_l_sums<T><<<nb, 256, 0, g->s>>>(m1, m, L->r, lsc_slot(L, 2, L->sc + 10, nb), done);
  k_l_center<T><<<nb, 256, 0, g->s>>>(m1, m, L->r, L->sc + 10, done);
  ETH_CUDA(cudaGetLastError());
  g->launches += 2;
  return ETH_OK;
}

// z = M_3^{-1} r (Eq. nse-precon-lsc): z_p = -M_S^{-1} r_p, z_u = V_F(r_u - B^T z_p);
// adj: the same for K^T (F^T in the middle factor and the F^T V-cycle).
template <class T>
eth_status precond_lsc(eth_grid* g, Work* w, const eth_opts* o, const double* r, double* z, const int* done, bool adj) {
  LscWork<T>* L = nullptr;
  ETH_TRY(lsc_get<T>(g, w, &L));
  const size_t nu2 = 2 * (size_t)g->nv;
  const int m = g->n1 + g->n0;
  const int its = o->lsc_cg > 0 ? o->lsc_cg : 6;
  // y = (B H^{-1} B^T)^+ r_p
  k_l_load<T><<<vblocks(m), 256, 0, g->s>>>(m, r + nu2, L->r, done);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  ETH_TRY(lsc_center<T>(g, L, done));
  ETH_TRY(lsc_cg<T>(g, w, L, L->y, its, done));
  // t = B M^{-1} F H^{-1} B^T y, the right-hand side of the second frame solve
  {
    Q2Params<T, T, T> P{};
    P.n = g->n; P.hx = (T)g->hx; P.hy = (T)g->hy; P.nu = 0;
    P.p = L->y; P.y = L->v1; P.dinv = L->md; P.done = done;
    ETH_CUDA((launch_q2<T, T, T, QF_PIN | QF_P0 | QF_UOUT, EPI_SCALE>(P, g->s)));
  }
  {
    Q2Params<T, T, T> P{};
    P.n = g->n; P.hx = (T)g->hx; P.hy = (T)g->hy; P.nu = (T)g->nu;
    P.x = L->v1; P.w = lsc_wind<T>(g); P.y = L->v2; P.dinv = L->md; P.done = done;
    if (adj) ETH_CUDA((launch_q2<T, T, T, QF_DIFF | QF_CONV | QF_TRANS | QF_XIN | QF_UOUT, EPI_SCALE>(P, g->s)));
    else ETH_CUDA((launch_q2<T, T, T, QF_DIFF | QF_CONV | QF_XIN | QF_UOUT, EPI_SCALE>(P, g->s)));
  }
  {
    Q2Params<T, T, T> P{};
    P.n = g->n; P.hx = (T)g->hx; P.hy = (T)g->hy; P.nu = 0;
    P.x = L->v2; P.yp = L->r; P.done = done;
    ETH_CUDA((launch_q2<T, T, T, QF_XIN | QF_P0 | QF_POUT, EPI_APPLY>(P, g->s)));
  }
  g->launches += 3;
  ETH_TRY(lsc_center<T>(g, L, done));
  // x = (B M^{-1} B^T)^+ t ; z_p = -x
  ETH_TRY(lsc_cg<T>(g, w, L, L->x, its, done));
  k_l_out<T><<<vblocks(m), 256, 0, g->s>>>(m, L->x, z + nu2, -1.0, done);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  // z_u = V_F(r_u - B^T z_p)
  {
    Q2Params<double, double, T> P{};
    P.n = g->n; P.hx = (T)g->hx; P.hy = (T)g->hy; P.nu = 0;
    P.p = z + nu2; P.y = L->vt; P.bsrc = r; P.done = done;
    ETH_CUDA((launch_q2<double, double, T, QF_PIN | QF_P0 | QF_UOUT, EPI_BSUB>(P, g->s)));
    g->launches++;
  }
  return vcycle_vel<T>(g, adj ? vel_hier_t<T>(w) : vel_hier<T>(w), L->vt, z, o->mg_pre, o->mg_post, done, nullptr, 0);
}

// allocates the workspace (before any stream capture of precond_lsc)
template <class T>
eth_status lsc_prepare(eth_grid* g, Work* w) {
  LscWork<T>* L = nullptr;
  return lsc_get<T>(g, w, &L);
}

template eth_status lsc_prepare<float>(eth_grid*, Work*);
template eth_status lsc_prepare<double>(eth_grid*, Work*);
template eth_status precond_lsc<float>(eth_grid*, Work*, const eth_opts*, const double*, double*, const int*, bool);
template eth_status precond_lsc<double>(eth_grid*, Work*, const eth_opts*, const double*, double*, const int*, bool);

}  // namespace eth
