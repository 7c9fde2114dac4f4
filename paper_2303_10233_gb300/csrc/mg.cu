// Geometric multigrid hierarchies and V-cycles (see mg.cuh).
#include <cmath>
#include <vector>
#include "mg.cuh"

namespace eth {

// ---------------------------------------------------------------------------
// velocity (Q2) level kernels
// ---------------------------------------------------------------------------
// Inverse diagonal of nu*A + N(w) at interior nodes (3x3 Gauss), 0 on the boundary.
template <class T>
__device__ __forceinline__ void wind_at(int N, size_t nv, int ex, int ey, const T* __restrict__ w, int qx, int qy, double& wx, double& wy) {
  wx = 0; wy = 0;
  for (int bb = 0; bb < 3; ++bb)
    for (int aa = 0; aa < 3; ++aa) {
      const double f = q2v(aa, gq(qx)) * q2v(bb, gq(qy));
      const size_t gn = (size_t)(2 * ey + bb) * N + 2 * ex + aa;
      wx += f * (double)w[gn];
      wy += f * (double)w[gn + nv];
    }
}

// streamline-diffusion parameter of an element (matches the tile kernel)
template <class T>
__device__ __forceinline__ double sd_delta(int N, size_t nv, int ex, int ey, const T* __restrict__ w, double h, double nu, double sdc) {
  if (w == nullptr || sdc <= 0.0) return 0.0;
  double wn = 0.0;
  for (int qy = 0; qy < 3; ++qy)
    for (int qx = 0; qx < 3; ++qx) {
      double a, b;
      wind_at<T>(N, nv, ex, ey, w, qx, qy, a, b);
      wn += sqrt(a * a + b * b);
    }
  wn /= 9.0;
  const double pe = wn * h / (2.0 * nu);
  return pe > 1.0 ? sdc * h / (2.0 * wn) * (1.0 - 1.0 / pe) : 0.0;
}

template <class T>
__global__ void k_q2_diag(int n, double hx, double hy, double nu, double sdc, const T* __restrict__ w, T* __restrict__ dinv) {
  ETH_GRID_DEP_WAIT();
  const int N = 2 * n + 1;
  const size_t nv = (size_t)N * N;
  for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < N * N; node += gridDim.x * blockDim.x) {
    const int j = node / N, i = node - j * N;
    if (i == 0 || j == 0 || i == N - 1 || j == N - 1) { dinv[node] = 0; continue; }
    double diag = 0.0;
    for (int ey = (j - 2) / 2; ey <= j / 2; ++ey) {
      const int b = j - 2 * ey;
      if (ey < 0 || ey >= n || b < 0 || b > 2) continue;
      for (int ex = (i - 2) / 2; ex <= i / 2; ++ex) {
        const int a = i - 2 * ex;
        if (ex < 0 || ex >= n || a < 0 || a > 2) continue;
        const double dl = sd_delta<T>(N, nv, ex, ey, w, fmax(hx, hy), nu, sdc);
        for (int qy = 0; qy < 3; ++qy)
          for (int qx = 0; qx < 3; ++qx) {
            const double W = gw(qx) * gw(qy) * hx * hy;
            const double ph = q2v(a, gq(qx)) * q2v(b, gq(qy));
            const double dx = q2d(a, gq(qx)) * q2v(b, gq(qy)) / hx;
            const double dy = q2v(a, gq(qx)) * q2d(b, gq(qy)) / hy;
            double wx = 0, wy = 0;
            if (w != nullptr) wind_at<T>(N, nv, ex, ey, w, qx, qy, wx, wy);
            const double wg = wx * dx + wy * dy;
            diag += W * (nu * (dx * dx + dy * dy) + wg * ph + dl * wg * wg);
          }
      }
    }
    dinv[node] = (T)(1.0 / diag);
  }
}

// x = omega D^{-1} b on the interior (first sweep from a zero guess), b copied.
template <class TI, class T>
__global__ void k_q2_jacobi0(int n, T omega, const T* __restrict__ dinv, const TI* __restrict__ bin, T* __restrict__ bc,
                             T* __restrict__ x, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done != nullptr && *done) return;
  const int N = 2 * n + 1;
  const size_t nv = (size_t)N * N;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < 2 * nv; k += (size_t)gridDim.x * blockDim.x) {
    const size_t g = k < nv ? k : k - nv;
    const int j = (int)(g / N), i = (int)(g - (size_t)j * N);
    const bool bnd = i == 0 || j == 0 || i == N - 1 || j == N - 1;
    const T b = bnd ? T(0) : cvt<T, TI>(bin[k]);
    if (bc != (const T*)bin) bc[k] = b;
    x[k] = omega * dinv[g] * b;
  }
}

// 1D Q2 restriction weight of the fine node at offset o in [-3, 3] from 2I
// (coarse midpoint I odd: 3/4, 1, 3/4 on o = -1, 0, 1; coarse vertex I even:
// -1/8, 3/8, 1, 3/8, -1/8 on o = -3, -1, 0, 1, 3; every other offset 0).
__device__ __forceinline__ float q2_rw(int odd, int o) {
  if (o == 0) return 1.f;
  if (odd) return (o == -1 || o == 1) ? 0.75f : 0.f;
  return (o == -1 || o == 1) ? 0.375f : ((o == -3 || o == 3) ? -0.125f : 0.f);
}
// 1D Q2 prolongation to fine index i: coarse base index and three weights
// (even i: injection; i = 4E+1: 3/8, 3/4, -1/8; i = 4E+3: -1/8, 3/4, 3/8).
__device__ __forceinline__ int q2_pw(int i, float& w0, float& w1, float& w2) {
  if (!(i & 1)) { w0 = 1.f; w1 = 0.f; w2 = 0.f; return i >> 1; }
  const int E = i >> 2;
  if ((i & 3) == 1) { w0 = 0.375f; w1 = 0.75f; w2 = -0.125f; }
  else { w0 = -0.125f; w1 = 0.75f; w2 = 0.375f; }
  return 2 * E;
}

template <class T>
__global__ void k_q2_restrict(int nc, const T* __restrict__ rf, T* __restrict__ bc, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done != nullptr && *done) return;
  const int Nc = 2 * nc + 1, Nf = 4 * nc + 1;
  const size_t nvc = (size_t)Nc * Nc, nvf = (size_t)Nf * Nf;
  for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < Nc * Nc; node += gridDim.x * blockDim.x) {
    const int J = node / Nc, I = node - J * Nc;
    if (I == 0 || J == 0 || I == Nc - 1 || J == Nc - 1) { bc[node] = 0; bc[node + nvc] = 0; continue; }
    const int ox = I & 1, oy = J & 1;
    T s0 = 0, s1 = 0;
#pragma unroll
    for (int u = -3; u <= 3; ++u) {
      const float wyv = q2_rw(oy, u);
      if (wyv == 0.f) continue;
      const size_t row = (size_t)(2 * J + u) * Nf;
      T t0 = 0, t1 = 0;
#pragma unroll
      for (int v = -3; v <= 3; ++v) {
        const float wxv = q2_rw(ox, v);
        if (wxv == 0.f) continue;
        const size_t f = row + 2 * I + v;
        t0 += (T)wxv * rf[f];
        t1 += (T)wxv * rf[f + nvf];
      }
      s0 += (T)wyv * t0;
      s1 += (T)wyv * t1;
    }
    bc[node] = s0;
    bc[node + nvc] = s1;
  }
}

template <class T>
__global__ void k_q2_prolong_add(int nc, const T* __restrict__ xc, T* __restrict__ xf, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done != nullptr && *done) return;
  const int Nc = 2 * nc + 1, Nf = 4 * nc + 1;
  const size_t nvc = (size_t)Nc * Nc, nvf = (size_t)Nf * Nf;
  for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < Nf * Nf; node += gridDim.x * blockDim.x) {
    const int j = node / Nf, i = node - j * Nf;
    if (i == 0 || j == 0 || i == Nf - 1 || j == Nf - 1) continue;
    float wx[3], wy[3];
    const int cx = q2_pw(i, wx[0], wx[1], wx[2]), cy = q2_pw(j, wy[0], wy[1], wy[2]);
    T s0 = 0, s1 = 0;
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        if (wx[v] == 0.f || wy[u] == 0.f) continue;
        const size_t c = (size_t)(cy + u) * Nc + cx + v;
        const T f = (T)(wx[v] * wy[u]);
        s0 += f * xc[c];
        s1 += f * xc[c + nvc];
      }
    xf[node] += s0;
    xf[node + nvf] += s1;
  }
}

template <class T>
__global__ void k_q2_inject(int nc, const T* __restrict__ wf, T* __restrict__ wc) {
  ETH_GRID_DEP_WAIT();
  const int Nc = 2 * nc + 1, Nf = 4 * nc + 1;
  const size_t nvc = (size_t)Nc * Nc, nvf = (size_t)Nf * Nf;
  for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < Nc * Nc; node += gridDim.x * blockDim.x) {
    const int J = node / Nc, I = node - J * Nc;
    const size_t f = (size_t)(2 * J) * Nf + 2 * I;
    wc[node] = wf[f];
    wc[node + nvc] = wf[f + nvf];
  }
}

template <class TI>
__global__ void k_f64_from(size_t m, const TI* __restrict__ a, double* __restrict__ b) {
  ETH_GRID_DEP_WAIT();
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) b[k] = (double)a[k];
}
template <class TO>
__global__ void k_cast_from_f64(size_t m, const double* __restrict__ a, TO* __restrict__ b) {
  ETH_GRID_DEP_WAIT();
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) b[k] = (TO)a[k];
}

// Dense matrix of the interior scalar operator on the coarsest grid (FP64 atomics, set-up only).
__global__ void k_q2_coarse_mat(int n, double hx, double hy, double nu, double sdc, const double* __restrict__ w, double* __restrict__ D) {
  ETH_GRID_DEP_WAIT();
  const int N = 2 * n + 1, m = (N - 2) * (N - 2);
  const size_t nv = (size_t)N * N;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const int ey = e / n, ex = e - ey * n;
  double wq[2][9];
  for (int qy = 0; qy < 3; ++qy)
    for (int qx = 0; qx < 3; ++qx) {
      double a0 = 0, a1 = 0;
      if (w != nullptr)
        for (int b = 0; b < 3; ++b)
          for (int a = 0; a < 3; ++a) {
            const double f = q2v(a, gq(qx)) * q2v(b, gq(qy));
            const size_t gn = (size_t)(2 * ey + b) * N + 2 * ex + a;
            a0 += f * w[gn];
            a1 += f * w[gn + nv];
          }
      wq[0][qy * 3 + qx] = a0;
      wq[1][qy * 3 + qx] = a1;
    }
  const double dl = sd_delta<double>(N, nv, ex, ey, w, fmax(hx, hy), nu, sdc);
  for (int ti = 0; ti < 9; ++ti) {
    const int ai = ti % 3, bi = ti / 3;
    const int gi = 2 * ex + ai, gj = 2 * ey + bi;
    if (gi == 0 || gj == 0 || gi == N - 1 || gj == N - 1) continue;
    const int row = (gj - 1) * (N - 2) + (gi - 1);
    for (int tj = 0; tj < 9; ++tj) {
      const int aj = tj % 3, bj = tj / 3;
      const int hi = 2 * ex + aj, hj = 2 * ey + bj;
      if (hi == 0 || hj == 0 || hi == N - 1 || hj == N - 1) continue;
      const int col = (hj - 1) * (N - 2) + (hi - 1);
      double s = 0;
      for (int qy = 0; qy < 3; ++qy)
        for (int qx = 0; qx < 3; ++qx) {
          const double W = gw(qx) * gw(qy) * hx * hy;
          const double phi = q2v(ai, gq(qx)) * q2v(bi, gq(qy));
          const double dxi = q2d(ai, gq(qx)) * q2v(bi, gq(qy)) / hx, dyi = q2v(ai, gq(qx)) * q2d(bi, gq(qy)) / hy;
          const double dxj = q2d(aj, gq(qx)) * q2v(bj, gq(qy)) / hx, dyj = q2v(aj, gq(qx)) * q2d(bj, gq(qy)) / hy;
          const double wgj = wq[0][qy * 3 + qx] * dxj + wq[1][qy * 3 + qx] * dyj;
          const double wgi = wq[0][qy * 3 + qx] * dxi + wq[1][qy * 3 + qx] * dyi;
          s += W * (nu * (dxi * dxj + dyi * dyj) + wgj * phi + dl * wgi * wgj);
        }
      atomicAdd(&D[(size_t)row * m + col], s);
    }
  }
}

// x(interior) = Ainv * b(interior) per component (blockIdx.y), Q2 lattice.
// Dense inverses are stored column-major (entry (r, k) at k * m + r), so the
// threads of a warp (consecutive rows r) read consecutive addresses.
template <class T>
__global__ void k_q2_dense_mv(int n, const T* __restrict__ Ainv, const T* __restrict__ b, T* __restrict__ x, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done != nullptr && *done) return;
  extern __shared__ __align__(16) unsigned char sm[];
  T* sb = reinterpret_cast<T*>(sm);
  const int N = 2 * n + 1, M = N - 2, m = M * M;
  const size_t off = (size_t)blockIdx.y * N * N;
  for (int k = threadIdx.x; k < m; k += blockDim.x) sb[k] = b[off + (size_t)(k / M + 1) * N + (k % M + 1)];
  __syncthreads();
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
    T s = 0;
    for (int k = 0; k < m; ++k) s += Ainv[(size_t)k * m + r] * sb[k];
    x[off + (size_t)(r / M + 1) * N + (r % M + 1)] = s;
  }
}

// ---------------------------------------------------------------------------
// pressure (Q1 Laplacian) level kernels
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_q1_diag_lap(int n, double hx, double hy, T* __restrict__ dinv) {
  ETH_GRID_DEP_WAIT();
  const int M = n + 1;
  for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < M * M; node += gridDim.x * blockDim.x) {
    const int J = node / M, I = node - J * M;
    const int ne = ((I > 0) + (I < n)) * ((J > 0) + (J < n));
    dinv[node] = (T)(1.0 / (ne * (hy / hx + hx / hy) / 3.0));
  }
}

template <class T>
__global__ void k_q1_restrict(int nc, const T* __restrict__ rf, T* __restrict__ bc, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done != nullptr && *done) return;
  const int Mc = nc + 1, Mf = 2 * nc + 1;
  for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < Mc * Mc; node += gridDim.x * blockDim.x) {
    const int J = node / Mc, I = node - J * Mc;
    T s = 0;
    for (int dy = -1; dy <= 1; ++dy) {
      const int j = 2 * J + dy;
      if (j < 0 || j >= Mf) continue;
      const T wyv = dy == 0 ? T(1) : T(0.5);
      for (int dx = -1; dx <= 1; ++dx) {
        const int i = 2 * I + dx;
        if (i < 0 || i >= Mf) continue;
        s += wyv * (dx == 0 ? T(1) : T(0.5)) * rf[(size_t)j * Mf + i];
      }
    }
    bc[node] = s;
  }
}

template <class T>
__global__ void k_q1_prolong_add(int nc, const T* __restrict__ xc, T* __restrict__ xf, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done != nullptr && *done) return;
  const int Mc = nc + 1, Mf = 2 * nc + 1;
  for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < Mf * Mf; node += gridDim.x * blockDim.x) {
    const int j = node / Mf, i = node - j * Mf;
    const int I0 = i >> 1, I1 = (i + 1) >> 1, J0 = j >> 1, J1 = (j + 1) >> 1;
    const T v = T(0.25) * (xc[(size_t)J0 * Mc + I0] + xc[(size_t)J0 * Mc + I1] + xc[(size_t)J1 * Mc + I0] + xc[(size_t)J1 * Mc + I1]);
    xf[node] += v;
  }
}

template <class T>
__global__ void k_q1_jacobi0(int n, T omega, const T* __restrict__ dinv, const T* __restrict__ b, T* __restrict__ x, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done != nullptr && *done) return;
  const int tot = (n + 1) * (n + 1);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < tot; k += gridDim.x * blockDim.x) x[k] = omega * dinv[k] * b[k];
}

template <class T>
__global__ void k_dense_mv(int m, const T* __restrict__ Ainv, const T* __restrict__ b, T* __restrict__ x, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done != nullptr && *done) return;
  extern __shared__ __align__(16) unsigned char sm[];
  T* sb = reinterpret_cast<T*>(sm);
  for (int k = threadIdx.x; k < m; k += blockDim.x) sb[k] = b[k];
  __syncthreads();
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
    T s = 0;
    for (int k = 0; k < m; ++k) s += Ainv[(size_t)k * m + r] * sb[k];
    x[r] = s;
  }
}

// ---------------------------------------------------------------------------
// host: in-place transpose of a dense m x m matrix (row-major <-> column-major)
static void transpose_sq(std::vector<double>& h, int m) {
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j) std::swap(h[(size_t)i * m + j], h[(size_t)j * m + i]);
}

// host: dense inverse by Gauss-Jordan with partial pivoting (set-up only)
// ---------------------------------------------------------------------------
static bool invert(std::vector<double>& A, int m) {
  std::vector<double> I((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) I[(size_t)i * m + i] = 1.0;
  for (int c = 0; c < m; ++c) {
    int p = c;
    double best = std::fabs(A[(size_t)c * m + c]);
    for (int r = c + 1; r < m; ++r)
      if (std::fabs(A[(size_t)r * m + c]) > best) { best = std::fabs(A[(size_t)r * m + c]); p = r; }
    if (best == 0.0) return false;
    if (p != c)
      for (int k = 0; k < m; ++k) { std::swap(A[(size_t)p * m + k], A[(size_t)c * m + k]); std::swap(I[(size_t)p * m + k], I[(size_t)c * m + k]); }
    const double inv = 1.0 / A[(size_t)c * m + c];
    for (int k = 0; k < m; ++k) { A[(size_t)c * m + k] *= inv; I[(size_t)c * m + k] *= inv; }
    for (int r = 0; r < m; ++r) {
      if (r == c) continue;
      const double f = A[(size_t)r * m + c];
      if (f == 0.0) continue;
      for (int k = 0; k < m; ++k) { A[(size_t)r * m + k] -= f * A[(size_t)c * m + k]; I[(size_t)r * m + k] -= f * I[(size_t)c * m + k]; }
    }
  }
  A.swap(I);
  return true;
}

template <class T>
static eth_status upload(const std::vector<double>& h, T** d, cudaStream_t s) {
  std::vector<T> t(h.begin(), h.end());
  ETH_CUDA(cudaMalloc((void**)d, t.size() * sizeof(T)));
  ETH_CUDA(cudaMemcpyAsync(*d, t.data(), t.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  ETH_CUDA(cudaStreamSynchronize(s));
  return ETH_OK;
}

template <class T>
void mg_free(Hier<T>& H) {
  for (auto& L : H.lv) {
    cudaFree(L.w); cudaFree(L.dinv); cudaFree(L.x); cudaFree(L.b); cudaFree(L.r); cudaFree(L.t); cudaFree(L.conv);
  }
  H.lv.clear();
  cudaFree(H.coarse_inv);
  H.coarse_inv = nullptr;
  H.built = false;
}

static int gsize(size_t work) {
  size_t b = (work + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

// levels n, n/2, ... while the size stays even and above nmin
static std::vector<int> level_sizes(int n, int nmin) {
  std::vector<int> ns{n};
  while (ns.back() % 2 == 0 && ns.back() / 2 >= nmin && ns.back() / 2 >= 2) ns.push_back(ns.back() / 2);
  return ns;
}

template <class T>
eth_status mg_build_vel(eth_grid* g, Hier<T>& H, int nmin, double art, bool trans) {
  mg_free(H);
  H.trans = trans;
  const std::vector<int> ns = level_sizes(g->n, nmin);
  if (ns.back() > 32) { set_error("multigrid: n=%d does not coarsen to <= 32 (n must be c*2^k, c <= 32)", g->n); return ETH_EINVAL; }
  const bool conv = g->kind == ETH_OSEEN;
  double wmax = 0.0;
  if (conv) {
    std::vector<double> wh(2 * (size_t)g->nv);
    ETH_CUDA(cudaMemcpyAsync(wh.data(), g->wind, wh.size() * 8, cudaMemcpyDeviceToHost, g->s));
    ETH_CUDA(cudaStreamSynchronize(g->s));
    for (size_t k = 0; k < (size_t)g->nv; ++k) wmax = std::fmax(wmax, std::sqrt(wh[k] * wh[k] + wh[k + g->nv] * wh[k + g->nv]));
  }
  H.q1 = false;
  H.omega = 0.85;
  for (size_t l = 0; l < ns.size(); ++l) {
    Level<T> L;
    L.n = ns[l];
    L.hx = g->hx * (g->n / L.n);
    L.hy = g->hy * (g->n / L.n);
    L.nu = g->nu;
    // streamline diffusion on every level of the preconditioner's hierarchy (only
    // where the cell Peclet number exceeds 1); the Krylov method applies the exact F
    L.sd = conv ? art : 0.0;
    L.trans = trans && conv;
    const size_t N = 2 * (size_t)L.n + 1, nv = N * N;
    ETH_CUDA(cudaMalloc((void**)&L.dinv, nv * sizeof(T)));
    ETH_CUDA(cudaMalloc((void**)&L.x, 2 * nv * sizeof(T)));
    ETH_CUDA(cudaMalloc((void**)&L.b, 2 * nv * sizeof(T)));
    ETH_CUDA(cudaMalloc((void**)&L.r, 2 * nv * sizeof(T)));
    ETH_CUDA(cudaMalloc((void**)&L.t, 2 * nv * sizeof(T)));
    ETH_CUDA(cudaMemsetAsync(L.x, 0, 2 * nv * sizeof(T), g->s));
    ETH_CUDA(cudaMemsetAsync(L.t, 0, 2 * nv * sizeof(T), g->s));
    if (conv) {
      ETH_CUDA(cudaMalloc((void**)&L.w, 2 * nv * sizeof(T)));
      if (l == 0) {
        k_cast_from_f64<T><<<gsize(2 * nv), 256, 0, g->s>>>(2 * nv, g->wind, L.w);
      } else {
        k_q2_inject<T><<<gsize(nv), 256, 0, g->s>>>(L.n, H.lv[l - 1].w, L.w);
      }
      ETH_CUDA(cudaGetLastError());
    }
    k_q2_diag<T><<<gsize(nv), 256, 0, g->s>>>(L.n, L.hx, L.hy, L.nu, L.sd, L.w, L.dinv);
    ETH_CUDA(cudaGetLastError());
    H.lv.push_back(L);
  }
  // coarsest: dense inverse of the interior scalar operator
  Level<T>& C = H.lv.back();
  const int Nc = 2 * C.n + 1, m = (Nc - 2) * (Nc - 2);
  double* D = nullptr;
  double* wd = nullptr;
  ETH_CUDA(cudaMalloc((void**)&D, (size_t)m * m * 8));
  ETH_CUDA(cudaMemsetAsync(D, 0, (size_t)m * m * 8, g->s));
  if (conv) {
    ETH_CUDA(cudaMalloc((void**)&wd, 2 * (size_t)Nc * Nc * 8));
    k_f64_from<T><<<gsize(2 * (size_t)Nc * Nc), 256, 0, g->s>>>(2 * (size_t)Nc * Nc, C.w, wd);
  }
  k_q2_coarse_mat<<<cdiv((long)C.n * C.n, 64), 64, 0, g->s>>>(C.n, C.hx, C.hy, C.nu, C.sd, wd, D);
  ETH_CUDA(cudaGetLastError());
  std::vector<double> h((size_t)m * m);
  ETH_CUDA(cudaMemcpyAsync(h.data(), D, h.size() * 8, cudaMemcpyDeviceToHost, g->s));
  ETH_CUDA(cudaStreamSynchronize(g->s));
  cudaFree(D);
  cudaFree(wd);
  if (trans)
    for (int i = 0; i < m; ++i)
      for (int j = i + 1; j < m; ++j) std::swap(h[(size_t)i * m + j], h[(size_t)j * m + i]);
  if (!invert(h, m)) { set_error("multigrid: singular coarse operator"); return ETH_EINVAL; }
  transpose_sq(h, m);   // stored column-major
  ETH_TRY(upload<T>(h, &H.coarse_inv, g->s));
  H.ncoarse = m;
  H.built = true;
  return ETH_OK;
}

template <class T>
eth_status mg_build_q1(eth_grid* g, Hier<T>& H, int nmin) {
  mg_free(H);
  const std::vector<int> ns = level_sizes(g->n, nmin);
  if (ns.back() > 32) { set_error("multigrid: n=%d does not coarsen to <= 32", g->n); return ETH_EINVAL; }
  H.q1 = true;
  H.omega = 0.85;
  for (size_t l = 0; l < ns.size(); ++l) {
    Level<T> L;
    L.n = ns[l];
    L.hx = g->hx * (g->n / L.n);
    L.hy = g->hy * (g->n / L.n);
    const size_t M = (size_t)L.n + 1, tot = M * M;
    ETH_CUDA(cudaMalloc((void**)&L.dinv, tot * sizeof(T)));
    ETH_CUDA(cudaMalloc((void**)&L.x, tot * sizeof(T)));
    ETH_CUDA(cudaMalloc((void**)&L.b, tot * sizeof(T)));
    ETH_CUDA(cudaMalloc((void**)&L.r, tot * sizeof(T)));
    ETH_CUDA(cudaMalloc((void**)&L.t, tot * sizeof(T)));
    k_q1_diag_lap<T><<<gsize(tot), 256, 0, g->s>>>(L.n, L.hx, L.hy, L.dinv);
    ETH_CUDA(cudaGetLastError());
    H.lv.push_back(L);
  }
  // coarsest: pseudo-inverse of K1 = (K1 + J/m)^{-1} - J/m, J = ones
  const Level<T>& C = H.lv.back();
  const int nc = C.n, M = nc + 1, m = M * M;
  std::vector<double> K((size_t)m * m, 0.0);
  const double rxy = C.hy / C.hx, ryx = C.hx / C.hy;
  auto km = [](int a, int b) { return a == b ? 1.0 / 3.0 : 1.0 / 6.0; };
  auto kk = [](int a, int b) { return a == b ? 1.0 : -1.0; };
  for (int ey = 0; ey < nc; ++ey)
    for (int ex = 0; ex < nc; ++ex)
      for (int d = 0; d < 2; ++d)
        for (int c = 0; c < 2; ++c)
          for (int dd = 0; dd < 2; ++dd)
            for (int cc = 0; cc < 2; ++cc) {
              const int r = (ey + d) * M + ex + c, q = (ey + dd) * M + ex + cc;
              K[(size_t)r * m + q] += rxy * kk(c, cc) * km(d, dd) + ryx * km(c, cc) * kk(d, dd);
            }
  for (size_t k = 0; k < K.size(); ++k) K[k] += 1.0 / m;
  if (!invert(K, m)) { set_error("multigrid: singular Q1 coarse operator"); return ETH_EINVAL; }
  for (size_t k = 0; k < K.size(); ++k) K[k] -= 1.0 / m;
  transpose_sq(K, m);   // stored column-major
  ETH_TRY(upload<T>(K, &H.coarse_inv, g->s));
  H.ncoarse = m;
  H.built = true;
  return ETH_OK;
}

// ---------------------------------------------------------------------------
// Single-CTA V-cycle over the coarsest levels, entirely in shared memory.
// One launch replaces the (smoothing, residual, transfer) launches of every
// level with n <= the coarse threshold; each operator application is an
// element loop in four colour phases (elements of one colour share no node).
// ---------------------------------------------------------------------------
constexpr int CMAXL = 6;
template <class T>
struct CoarseQ2 {
  int nlev;
  int n[CMAXL];
  T hx[CMAXL], hy[CMAXL], nu[CMAXL], sd[CMAXL];
  const T* dinv[CMAXL];
  const T* w[CMAXL];
};

template <class T, int FL>
__device__ void cq2_residual(int n, T hx, T hy, T nu, T sd, const T* __restrict__ w, const T* X, const T* B, T* R) {
  const int N = 2 * n + 1, nv = N * N;
  for (int k = threadIdx.x; k < 2 * nv; k += blockDim.x) R[k] = B[k];
  __syncthreads();
  const T ihx = T(1) / hx, ihy = T(1) / hy, area = hx * hy;
  for (int col = 0; col < 4; ++col) {
    const int cx = col & 1, cy = col >> 1;
    const int nx = (n - cx + 1) / 2, ny = (n - cy + 1) / 2;
    for (int e = threadIdx.x; e < nx * ny; e += blockDim.x) {
      const int ex = 2 * (e % nx) + cx, ey = 2 * (e / nx) + cy;
      T U[2][9], Wn[2][9], P1[4] = {0, 0, 0, 0}, Y[2][9], YP1[4], YP0;
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const int g = (2 * ey + b) * N + 2 * ex + a;
          U[0][b * 3 + a] = X[g];
          U[1][b * 3 + a] = X[g + nv];
          if (FL & QF_CONV) { Wn[0][b * 3 + a] = w[g]; Wn[1][b * 3 + a] = w[g + nv]; }
        }
      q2_elem<T, FL>(U, Wn, P1, T(0), nu, ihx, ihy, area, sd, Y, YP1, YP0);
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const int g = (2 * ey + b) * N + 2 * ex + a;
          R[g] -= Y[0][b * 3 + a];
          R[g + nv] -= Y[1][b * 3 + a];
        }
    }
    __syncthreads();
  }
}

// Node-parallel residual R = B - nu A X for the Stokes levels of the coarse
// kernel: every interior node sums its (up to four) element rows from the
// closed-form element matrix (tables KM, MK in shared memory), so all threads
// work on every pass (no colour phases).
template <class T>
__device__ void cq2_residual_node(int n, T hx, T hy, T nu, const T* KM, const T* MK, const T* X, const T* B, T* R) {
  const int N = 2 * n + 1, nv = N * N;
  const T skm = nu * hy / hx, smk = nu * hx / hy;
  for (int node = threadIdx.x; node < nv; node += blockDim.x) {
    const int j = node / N, i = node - j * N;
    if (i == 0 || j == 0 || i == N - 1 || j == N - 1) { R[node] = 0; R[node + nv] = 0; continue; }
    int ex0, ex1, a0, a1, nx, ey0, ey1, b0, b1, ny;
    if (i & 1) { ex0 = i >> 1; a0 = 1; ex1 = ex0; a1 = a0; nx = 1; } else { ex0 = (i >> 1) - 1; a0 = 2; ex1 = i >> 1; a1 = 0; nx = 2; }
    if (j & 1) { ey0 = j >> 1; b0 = 1; ey1 = ey0; b1 = b0; ny = 1; } else { ey0 = (j >> 1) - 1; b0 = 2; ey1 = j >> 1; b1 = 0; ny = 2; }
    T acc0 = 0, acc1 = 0;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (u >= ny) break;
      const int ey = u ? ey1 : ey0, bb = u ? b1 : b0;
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        if (v >= nx) break;
        const int ex = v ? ex1 : ex0, aa = v ? a1 : a0;
        const int row = (bb * 3 + aa) * 9;
        const int g0 = 2 * ey * N + 2 * ex;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          const T cf = skm * KM[row + q] + smk * MK[row + q];
          const int gq = g0 + (q / 3) * N + (q % 3);
          acc0 += cf * X[gq];
          acc1 += cf * X[gq + nv];
        }
      }
    }
    R[node] = B[node] - acc0;
    R[node + nv] = B[node + nv] - acc1;
  }
  __syncthreads();
}

// Threads of the single-CTA coarse V-cycle: 1024 for the FP32 Stokes levels (64
// registers, no spills), 512 where the convection terms need more registers.
template <class T, int FL>
__host__ __device__ constexpr int q2_coarse_threads() { return (sizeof(T) == 4 && !(FL & QF_CONV)) ? 1024 : 512; }

template <class T, int FL>
__global__ void __launch_bounds__(q2_coarse_threads<T, FL>()) k_q2_coarse_vc(CoarseQ2<T> L, const T* __restrict__ Ainv, int m,
                                                        const T* __restrict__ bin, T* __restrict__ xout, T omega,
                                                        int pre, int post, const int* done, int ainv_smem) {
  ETH_GRID_DEP_WAIT();
  if (done != nullptr && *done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  constexpr bool CONVL = FL & QF_CONV;
  // per level: X, B, R (2 N^2 each), the inverse diagonal (N^2) and the wind (2 N^2) staged
  // from global memory once, so the sweeps below touch shared memory only
  T *X[CMAXL], *B[CMAXL], *R[CMAXL], *D[CMAXL], *Wl[CMAXL];
  size_t off = 0;
  for (int l = 0; l < L.nlev; ++l) {
    const int N = 2 * L.n[l] + 1;
    X[l] = sm + off; off += 2 * N * N;
    B[l] = sm + off; off += 2 * N * N;
    R[l] = sm + off; off += 2 * N * N;
    D[l] = sm + off; off += N * N;
    Wl[l] = sm + off; off += CONVL ? 2 * N * N : 0;
    for (int k = threadIdx.x; k < N * N; k += blockDim.x) D[l][k] = L.dinv[l][k];
    if (CONVL)
      for (int k = threadIdx.x; k < 2 * N * N; k += blockDim.x) Wl[l][k] = L.w[l][k];
  }
  const T* Ai = Ainv;   // dense coarse inverse: staged too when it fits (ainv_smem)
  if (ainv_smem) {
    T* sa = sm + off;
    for (int k = threadIdx.x; k < m * m; k += blockDim.x) sa[k] = Ainv[k];
    Ai = sa;
  }
  constexpr bool NODE = !CONVL;
  __shared__ T KM[81], MK[81];
  if (NODE) {
    for (int k = threadIdx.x; k < 81; k += blockDim.x) {
      const int i = k / 9, q = k % 9;
      KM[k] = (T)(k1d(i % 3, q % 3) * m1d(i / 3, q / 3));
      MK[k] = (T)(m1d(i % 3, q % 3) * k1d(i / 3, q / 3));
    }
  }
  auto resid = [&](int l) {
    if (NODE) cq2_residual_node<T>(L.n[l], L.hx[l], L.hy[l], L.nu[l], KM, MK, X[l], B[l], R[l]);
    else cq2_residual<T, FL>(L.n[l], L.hx[l], L.hy[l], L.nu[l], L.sd[l], Wl[l], X[l], B[l], R[l]);
  };
  {
    const int N = 2 * L.n[0] + 1;
    for (int k = threadIdx.x; k < 2 * N * N; k += blockDim.x) B[0][k] = bin[k];
  }
  __syncthreads();
  for (int l = 0; l < L.nlev - 1; ++l) {
    const int n = L.n[l], N = 2 * n + 1, nv = N * N;
    for (int k = threadIdx.x; k < 2 * nv; k += blockDim.x) {
      const int g = k < nv ? k : k - nv;
      X[l][k] = omega * D[l][g] * B[l][k];   // dinv and B vanish on the boundary
    }
    __syncthreads();
    for (int s = 1; s < pre; ++s) {
      resid(l);
      for (int k = threadIdx.x; k < 2 * nv; k += blockDim.x) X[l][k] += omega * D[l][k < nv ? k : k - nv] * R[l][k];
      __syncthreads();
    }
    resid(l);
    const int nc = L.n[l + 1], Nc = 2 * nc + 1, nvc = Nc * Nc;
    for (int node = threadIdx.x; node < nvc; node += blockDim.x) {
      const int J = node / Nc, I = node - J * Nc;
      T s0 = 0, s1 = 0;
      if (!(I == 0 || J == 0 || I == Nc - 1 || J == Nc - 1)) {
        const int ox = I & 1, oy = J & 1;
#pragma unroll
        for (int u = -3; u <= 3; ++u) {
          const float wyv = q2_rw(oy, u);
          if (wyv == 0.f) continue;
#pragma unroll
          for (int v = -3; v <= 3; ++v) {
            const float wxv = q2_rw(ox, v);
            if (wxv == 0.f) continue;
            const int f = (2 * J + u) * N + 2 * I + v;
            const T cf = (T)(wxv * wyv);
            s0 += cf * R[l][f];
            s1 += cf * R[l][f + nv];
          }
        }
      }
      B[l + 1][node] = s0;
      B[l + 1][node + nvc] = s1;
    }
    __syncthreads();
  }
  {
    const int l = L.nlev - 1, n = L.n[l], N = 2 * n + 1, M = N - 2, nv = N * N;
    for (int k = threadIdx.x; k < 2 * nv; k += blockDim.x) X[l][k] = 0;
    __syncthreads();
    // both components per row; column-major inverse: coalesced over r, B read as a broadcast
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
      T acc0 = 0, acc1 = 0;
      const T* col = Ai + r;
      for (int ky = 0; ky < M; ++ky) {
        const T* b0 = B[l] + (ky + 1) * N + 1;
        for (int kx = 0; kx < M; ++kx, col += m) {
          const T a = *col;
          acc0 += a * b0[kx];
          acc1 += a * b0[kx + nv];
        }
      }
      const int o = (r / M + 1) * N + (r % M + 1);
      X[l][o] = acc0;
      X[l][o + nv] = acc1;
    }
    __syncthreads();
  }
  for (int l = L.nlev - 2; l >= 0; --l) {
    const int n = L.n[l], N = 2 * n + 1, nv = N * N;
    const int nc = L.n[l + 1], Nc = 2 * nc + 1, nvc = Nc * Nc;
    for (int node = threadIdx.x; node < nv; node += blockDim.x) {
      const int j = node / N, i = node - j * N;
      if (i == 0 || j == 0 || i == N - 1 || j == N - 1) continue;
      float wx[3], wy[3];
      const int cx = q2_pw(i, wx[0], wx[1], wx[2]), cy = q2_pw(j, wy[0], wy[1], wy[2]);
      T s0 = 0, s1 = 0;
#pragma unroll
      for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          if (wx[v] == 0.f || wy[u] == 0.f) continue;
          const int c = (cy + u) * Nc + cx + v;
          const T f = (T)(wx[v] * wy[u]);
          s0 += f * X[l + 1][c];
          s1 += f * X[l + 1][c + nvc];
        }
      X[l][node] += s0;
      X[l][node + nv] += s1;
    }
    __syncthreads();
    for (int s = 0; s < post; ++s) {
      resid(l);
      for (int k = threadIdx.x; k < 2 * nv; k += blockDim.x) X[l][k] += omega * D[l][k < nv ? k : k - nv] * R[l][k];
      __syncthreads();
    }
  }
  {
    const int N = 2 * L.n[0] + 1;
    for (int k = threadIdx.x; k < 2 * N * N; k += blockDim.x) xout[k] = X[0][k];
  }
}

// Q1 Laplacian counterpart (natural boundary; pseudo-inverse on the coarsest grid)
template <class T>
struct CoarseQ1 {
  int nlev;
  int n[CMAXL];
  T hx[CMAXL], hy[CMAXL];
  const T* dinv[CMAXL];
};

template <class T>
__device__ void cq1_residual(int n, T hx, T hy, const T* X, const T* B, T* R) {
  const int M = n + 1;
  const T rxy = hy / hx, ryx = hx / hy;
  for (int node = threadIdx.x; node < M * M; node += blockDim.x) {
    const int J = node / M, I = node - J * M;
    T acc = 0;
    Q1_FOR_ELEMENTS(n, I, J, {
#pragma unroll
      for (int dd = 0; dd < 2; ++dd)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const T kc = rxy * (T)(q1k(c, cc) * q1m(d, dd)) + ryx * (T)(q1m(c, cc) * q1k(d, dd));
          acc += kc * X[(ey + dd) * M + ex + cc];
        }
    })
    R[node] = B[node] - acc;
  }
  __syncthreads();
}

template <class T>
__global__ void __launch_bounds__(1024) k_q1_coarse_vc(CoarseQ1<T> L, const T* __restrict__ Apinv, int m,
                                                        const T* __restrict__ bin, T* __restrict__ xout, T omega,
                                                        const int* done, int ainv_smem) {
  ETH_GRID_DEP_WAIT();
  if (done != nullptr && *done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  // per level X, B, R and the inverse diagonal (staged once), then the dense pseudo-inverse when it fits
  T *X[CMAXL], *B[CMAXL], *R[CMAXL], *D[CMAXL];
  size_t off = 0;
  for (int l = 0; l < L.nlev; ++l) {
    const int M = L.n[l] + 1;
    X[l] = sm + off; off += M * M;
    B[l] = sm + off; off += M * M;
    R[l] = sm + off; off += M * M;
    D[l] = sm + off; off += M * M;
    for (int k = threadIdx.x; k < M * M; k += blockDim.x) D[l][k] = L.dinv[l][k];
  }
  const T* Apinv_s = Apinv;
  if (ainv_smem) {
    T* sa = sm + off;
    for (int k = threadIdx.x; k < m * m; k += blockDim.x) sa[k] = Apinv[k];
    Apinv_s = sa;
  }
  {
    const int M = L.n[0] + 1;
    for (int k = threadIdx.x; k < M * M; k += blockDim.x) B[0][k] = bin[k];
  }
  __syncthreads();
  for (int l = 0; l < L.nlev - 1; ++l) {
    const int n = L.n[l], M = n + 1;
    for (int k = threadIdx.x; k < M * M; k += blockDim.x) X[l][k] = omega * D[l][k] * B[l][k];
    __syncthreads();
    cq1_residual<T>(n, L.hx[l], L.hy[l], X[l], B[l], R[l]);
    const int Mc = L.n[l + 1] + 1;
    for (int node = threadIdx.x; node < Mc * Mc; node += blockDim.x) {
      const int J = node / Mc, I = node - J * Mc;
      T s = 0;
      for (int dy = -1; dy <= 1; ++dy) {
        const int j = 2 * J + dy;
        if (j < 0 || j >= M) continue;
        for (int dx = -1; dx <= 1; ++dx) {
          const int i = 2 * I + dx;
          if (i < 0 || i >= M) continue;
          s += (dy == 0 ? T(1) : T(0.5)) * (dx == 0 ? T(1) : T(0.5)) * R[l][j * M + i];
        }
      }
      B[l + 1][node] = s;
    }
    __syncthreads();
  }
  {
    const int l = L.nlev - 1;
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
      T acc = 0;
      for (int k = 0; k < m; ++k) acc += Apinv_s[(size_t)k * m + r] * B[l][k];
      X[l][r] = acc;
    }
    __syncthreads();
  }
  for (int l = L.nlev - 2; l >= 0; --l) {
    const int n = L.n[l], M = n + 1, Mc = L.n[l + 1] + 1;
    for (int node = threadIdx.x; node < M * M; node += blockDim.x) {
      const int j = node / M, i = node - j * M;
      const int I0 = i >> 1, I1 = (i + 1) >> 1, J0 = j >> 1, J1 = (j + 1) >> 1;
      X[l][node] += T(0.25) * (X[l + 1][J0 * Mc + I0] + X[l + 1][J0 * Mc + I1] + X[l + 1][J1 * Mc + I0] + X[l + 1][J1 * Mc + I1]);
    }
    __syncthreads();
    cq1_residual<T>(n, L.hx[l], L.hy[l], X[l], B[l], R[l]);
    for (int k = threadIdx.x; k < M * M; k += blockDim.x) X[l][k] += omega * D[l][k] * R[l][k];
    __syncthreads();
  }
  {
    const int M = L.n[0] + 1;
    for (int k = threadIdx.x; k < M * M; k += blockDim.x) xout[k] = X[0][k];
  }
}

// Q1 first sweep from zero fused with the residual: x = omega D^{-1} b, r = b - K1 x
template <class T>
__global__ void k_q1_jr(int n, T hx, T hy, T omega, const T* __restrict__ dinv, const T* __restrict__ b,
                        T* __restrict__ x, T* __restrict__ r, const int* done) {
  ETH_GRID_DEP_WAIT();
  if (done != nullptr && *done) return;
  const int M = n + 1;
  const T rxy = hy / hx, ryx = hx / hy;
  for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < M * M; node += gridDim.x * blockDim.x) {
    const int J = node / M, I = node - J * M;
    T acc = 0;
    Q1_FOR_ELEMENTS(n, I, J, {
#pragma unroll
      for (int dd = 0; dd < 2; ++dd)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const int q = (ey + dd) * M + ex + cc;
          const T kc = rxy * (T)(q1k(c, cc) * q1m(d, dd)) + ryx * (T)(q1m(c, cc) * q1k(d, dd));
          acc += kc * omega * dinv[q] * b[q];
        }
    })
    const T xv = omega * dinv[node] * b[node];
    x[node] = xv;
    r[node] = b[node] - acc;
  }
}

// Q1 prolongation fused with the smoothing sweep: x' = x + P xc ; y = x' + omega D^{-1} (b - K1 x')
template <class T>
__global__ void k_q1_ps(int n, T hx, T hy, T omega, const T* __restrict__ dinv, const T* __restrict__ b,
                        const T* __restrict__ x, const T* __restrict__ xc, T* __restrict__ y, const int* done,
                        int sums, Slot sl, int soff) {
  ETH_GRID_DEP_WAIT();
  if (done != nullptr && *done) return;
  T s0 = 0, s1 = 0;
  const int M = n + 1, Mc = n / 2 + 1;
  const T rxy = hy / hx, ryx = hx / hy;
  auto xcorr = [&](int jj, int ii) -> T {
    const int I0 = ii >> 1, I1 = (ii + 1) >> 1, J0 = jj >> 1, J1 = (jj + 1) >> 1;
    return x[jj * M + ii] + T(0.25) * (xc[J0 * Mc + I0] + xc[J0 * Mc + I1] + xc[J1 * Mc + I0] + xc[J1 * Mc + I1]);
  };
  for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < M * M; node += gridDim.x * blockDim.x) {
    const int J = node / M, I = node - J * M;
    T acc = 0;
    Q1_FOR_ELEMENTS(n, I, J, {
#pragma unroll
      for (int dd = 0; dd < 2; ++dd)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const T kc = rxy * (T)(q1k(c, cc) * q1m(d, dd)) + ryx * (T)(q1m(c, cc) * q1k(d, dd));
          acc += kc * xcorr(ey + dd, ex + cc);
        }
    })
    const T xv = xcorr(J, I);
    const T yv = xv + omega * dinv[node] * (b[node] - acc);
    y[node] = yv;
    if (sums) {
      s0 += yv;
      s1 += (T)(((I > 0) + (I < n)) * ((J > 0) + (J < n))) * yv;
    }
  }
  if (sums) {   // (sum y, sum_I (#elements at I) y_I, 0) for the M_Q constant
    double v[3] = {(double)s0, (double)s1, 0.0};
    if (slot_arrive<3>(sl, soff + blockIdx.x, v)) finish_slot_n<3>(sl, v);
  }
}

// ---------------------------------------------------------------------------
// V-cycles
// ---------------------------------------------------------------------------
template <class T, class TO, int EPI, int CF>
static eth_status q2_level(eth_grid* g, const Level<T>& L, const T* x, TO* y, T omega, const TO* bsrc,
                           const int* done, const Slot* slot, int slot_off, const TO* dv) {
  constexpr int F0 = QF_DIFF | QF_XIN | QF_UOUT | CF;
  Q2Params<T, TO, T> P{};
  P.n = L.n; P.hx = (T)L.hx; P.hy = (T)L.hy; P.nu = (T)L.nu; P.sd = (T)L.sd;
  P.x = x; P.w = L.w; P.y = y; P.b = L.b; P.dinv = L.dinv; P.omega = omega; P.bsrc = bsrc; P.done = done;
  if (slot) {
    P.slot = *slot; P.slot_off = slot_off; P.dv = dv;
    ETH_CUDA((launch_q2<T, TO, T, F0 | QF_DOT, EPI>(P, g->s)));
  } else {
    ETH_CUDA((launch_q2<T, TO, T, F0, EPI>(P, g->s)));
  }
  g->launches++;
  return ETH_OK;
}

template <class T, class TO, int EPI>
static eth_status q2_level_d(eth_grid* g, const Level<T>& L, const T* x, TO* y, T omega, const TO* bsrc,
                             const int* done, const Slot* slot = nullptr, int slot_off = 0, const TO* dv = nullptr) {
  if (L.w != nullptr && L.trans && L.sd > 0.0) return q2_level<T, TO, EPI, QF_CONV | QF_TRANS | QF_SD>(g, L, x, y, omega, bsrc, done, slot, slot_off, dv);
  if (L.w != nullptr && L.trans) return q2_level<T, TO, EPI, QF_CONV | QF_TRANS>(g, L, x, y, omega, bsrc, done, slot, slot_off, dv);
  if (L.w != nullptr && L.sd > 0.0) return q2_level<T, TO, EPI, QF_CONV | QF_SD>(g, L, x, y, omega, bsrc, done, slot, slot_off, dv);
  if (L.w != nullptr) return q2_level<T, TO, EPI, QF_CONV>(g, L, x, y, omega, bsrc, done, slot, slot_off, dv);
  return q2_level<T, TO, EPI, 0>(g, L, x, y, omega, bsrc, done, slot, slot_off, dv);
}

int vel_final_blocks(int n) { return q2_blocks(n); }

template <class T> static int vel_fused_start(const Hier<T>& H);
template <class T>
static eth_status vcycle_vel_fused(eth_grid* g, Hier<T>& H, const double* v, double* z, int pre, int post,
                                   const int* done, const Slot* slot, int slot_off, int Lc);

template <class T>
eth_status vcycle_vel(eth_grid* g, Hier<T>& H, const double* v, double* z, int pre, int post, const int* done,
                      const Slot* slot, int slot_off) {
  const int nl = (int)H.lv.size();
  const T om = (T)H.omega;
  if (nl < 2) { set_error("vcycle: hierarchy needs two levels"); return ETH_EINVAL; }
  if (H.fused) {
    const int Lc = vel_fused_start(H);
    if (Lc >= 1) return vcycle_vel_fused<T>(g, H, v, z, pre, post, done, slot, slot_off, Lc);
  }
  // descend
  for (int l = 0; l < nl - 1; ++l) {
    Level<T>& L = H.lv[l];
    const size_t N = 2 * (size_t)L.n + 1, nv = N * N;
    if (l == 0)
      k_q2_jacobi0<double, T><<<gsize(2 * nv), 256, 0, g->s>>>(L.n, om, L.dinv, v, L.b, L.x, done);
    else
      k_q2_jacobi0<T, T><<<gsize(2 * nv), 256, 0, g->s>>>(L.n, om, L.dinv, L.b, L.b, L.x, done);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
    T* cur = L.x;
    T* oth = L.t;
    for (int s = 1; s < pre; ++s) {
      ETH_TRY((q2_level_d<T, T, EPI_SMOOTH>(g, L, cur, oth, om, nullptr, done)));
      std::swap(cur, oth);
    }
    if (cur != L.x) {  // keep the iterate in L.x
      ETH_CUDA(cudaMemcpyAsync(L.x, cur, 2 * nv * sizeof(T), cudaMemcpyDeviceToDevice, g->s));
    }
    ETH_TRY((q2_level_d<T, T, EPI_RESID>(g, L, L.x, L.r, om, nullptr, done)));
    const Level<T>& Cn = H.lv[l + 1];
    const size_t Nc = 2 * (size_t)Cn.n + 1;
    k_q2_restrict<T><<<gsize(Nc * Nc), 256, 0, g->s>>>(Cn.n, L.r, Cn.b, done);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
  }
  {  // coarse solve
    Level<T>& C = H.lv[nl - 1];
    const int m = H.ncoarse;
    k_q2_dense_mv<T><<<dim3(cdiv(m, 128), 2), 128, m * sizeof(T), g->s>>>(C.n, H.coarse_inv, C.b, C.x, done);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
  }
  // ascend
  for (int l = nl - 2; l >= 0; --l) {
    Level<T>& L = H.lv[l];
    const Level<T>& Cn = H.lv[l + 1];
    const size_t N = 2 * (size_t)L.n + 1;
    k_q2_prolong_add<T><<<gsize(N * N), 256, 0, g->s>>>(Cn.n, Cn.x, L.x, done);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
    T* cur = L.x;
    T* oth = L.t;
    for (int s = 0; s < post; ++s) {
      const bool last = (l == 0 && s == post - 1);
      if (last) {
        ETH_TRY((q2_level_d<T, double, EPI_SMOOTH>(g, L, cur, z, om, v, done, slot, slot_off, v)));
      } else {
        ETH_TRY((q2_level_d<T, T, EPI_SMOOTH>(g, L, cur, oth, om, nullptr, done)));
        std::swap(cur, oth);
      }
    }
    if (l > 0 && cur != L.x) {
      const size_t nv = N * N;
      ETH_CUDA(cudaMemcpyAsync(L.x, cur, 2 * nv * sizeof(T), cudaMemcpyDeviceToDevice, g->s));
    }
  }
  return ETH_OK;
}

template <class T>
static eth_status q1_level(eth_grid* g, const Level<T>& L, const T* x, T* y, int epi, T omega, const int* done) {
  Q1Params<T, T, T> P{};
  P.n = L.n; P.hx = (T)L.hx; P.hy = (T)L.hy; P.cm = 0; P.ck = 1; P.c1 = 0;
  P.x = x; P.y = y; P.b = L.b; P.dinv = L.dinv; P.omega = omega; P.done = done;
  if (epi == Q1E_SMOOTH) k_q1node<T, T, T, Q1E_SMOOTH><<<q1_blocks(L.n), 256, 0, g->s>>>(P);
  else k_q1node<T, T, T, Q1E_RESID><<<q1_blocks(L.n), 256, 0, g->s>>>(P);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  return ETH_OK;
}

template <class T> static int q1_fused_start(const Hier<T>& H);
template <class T>
static eth_status q1_coarse_launch(eth_grid* g, Hier<T>& H, int Lc, const int* done);

template <class T>
bool q1_vcycle_fused(const Hier<T>& H, int pre, int post) { return H.fused && pre == 1 && post == 1 && q1_fused_start(H) >= 1; }

template <class T>
eth_status vcycle_q1_from(eth_grid* g, Hier<T>& H, int pre, int post, const int* done, const T** result,
                          const Slot* sums, int soff) {
  const int nl = (int)H.lv.size();
  const T om = (T)H.omega;
  *result = H.lv[0].x;
  if (H.fused && pre == 1 && post == 1) {
    const int Lc = q1_fused_start(H);
    if (Lc >= 1) {
      std::vector<const T*> res(nl, nullptr);
      for (int l = 0; l < Lc; ++l) {
        Level<T>& L = H.lv[l];
        k_q1_jr<T><<<q1_blocks(L.n), 256, 0, g->s>>>(L.n, (T)L.hx, (T)L.hy, om, L.dinv, L.b, L.x, L.r, done);
        const Level<T>& Cn = H.lv[l + 1];
        k_q1_restrict<T><<<gsize((size_t)(Cn.n + 1) * (Cn.n + 1)), 256, 0, g->s>>>(Cn.n, L.r, Cn.b, done);
        ETH_CUDA(cudaGetLastError());
        g->launches += 2;
      }
      ETH_TRY(q1_coarse_launch<T>(g, H, Lc, done));
      res[Lc] = H.lv[Lc].x;
      for (int l = Lc - 1; l >= 0; --l) {
        Level<T>& L = H.lv[l];
        const bool s0 = (l == 0 && sums != nullptr);
        k_q1_ps<T><<<q1_blocks(L.n), 256, 0, g->s>>>(L.n, (T)L.hx, (T)L.hy, om, L.dinv, L.b, L.x, res[l + 1], L.t, done,
                                                     s0 ? 1 : 0, s0 ? *sums : Slot{}, soff);
        ETH_CUDA(cudaGetLastError());
        g->launches++;
        res[l] = L.t;
      }
      *result = res[0];
      return ETH_OK;
    }
  }
  for (int l = 0; l < nl - 1; ++l) {
    Level<T>& L = H.lv[l];
    const size_t tot = (size_t)(L.n + 1) * (L.n + 1);
    if (l > 0) {
      k_q1_jacobi0<T><<<gsize(tot), 256, 0, g->s>>>(L.n, om, L.dinv, L.b, L.x, done);
      ETH_CUDA(cudaGetLastError());
      g->launches++;
    }
    for (int s = 1; s < pre; ++s) {
      ETH_TRY(q1_level<T>(g, L, L.x, L.t, Q1E_SMOOTH, om, done));
      ETH_CUDA(cudaMemcpyAsync(L.x, L.t, tot * sizeof(T), cudaMemcpyDeviceToDevice, g->s));
    }
    ETH_TRY(q1_level<T>(g, L, L.x, L.r, Q1E_RESID, om, done));
    const Level<T>& Cn = H.lv[l + 1];
    k_q1_restrict<T><<<gsize((size_t)(Cn.n + 1) * (Cn.n + 1)), 256, 0, g->s>>>(Cn.n, L.r, Cn.b, done);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
  }
  {
    Level<T>& C = H.lv[nl - 1];
    const int m = H.ncoarse;
    k_dense_mv<T><<<cdiv(m, 128), 128, m * sizeof(T), g->s>>>(m, H.coarse_inv, C.b, C.x, done);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
  }
  for (int l = nl - 2; l >= 0; --l) {
    Level<T>& L = H.lv[l];
    const Level<T>& Cn = H.lv[l + 1];
    const size_t tot = (size_t)(L.n + 1) * (L.n + 1);
    k_q1_prolong_add<T><<<gsize(tot), 256, 0, g->s>>>(Cn.n, Cn.x, L.x, done);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
    for (int s = 0; s < post; ++s) {
      ETH_TRY(q1_level<T>(g, L, L.x, L.t, Q1E_SMOOTH, om, done));
      ETH_CUDA(cudaMemcpyAsync(L.x, L.t, tot * sizeof(T), cudaMemcpyDeviceToDevice, g->s));
    }
  }
  return ETH_OK;
}


// ---------------------------------------------------------------------------
// fused V-cycles: (Jacobi-from-zero + residual) and (prolongation + smoothing)
// in one tile launch per level, single-CTA shared-memory V-cycle below the
// coarse threshold.
// ---------------------------------------------------------------------------
#ifndef ETH_Q2_COARSE
#define ETH_Q2_COARSE 16
#endif
#ifndef ETH_Q1_COARSE
#define ETH_Q1_COARSE 32
#endif
template <class T> static int q2_coarse_threshold() { return ETH_Q2_COARSE; }
template <class T> static int q1_coarse_threshold() { return ETH_Q1_COARSE; }

template <class T, class TI, int CF>
static eth_status q2_jr(eth_grid* g, Level<T>& L, const TI* b, T* bcopy, T omega, const int* done) {
  Q2Params<TI, T, T> P{};
  P.n = L.n; P.hx = (T)L.hx; P.hy = (T)L.hy; P.nu = (T)L.nu; P.sd = (T)L.sd;
  P.w = L.w; P.dinv = L.dinv; P.omega = omega; P.done = done;
  P.bx = b; P.y = L.r; P.y2 = L.x; P.bcopy = bcopy;
  ETH_CUDA((launch_q2<TI, T, T, QF_DIFF | QF_XIN | QF_UOUT | QF_SRC_JB | CF, EPI_JR>(P, g->s)));
  g->launches++;
  return ETH_OK;
}

// the first sweep of a coarser level whose right-hand side is the restriction of
// the finer level's residual rf, formed on the fly (b written to L.b)
template <class T, int CF>
static eth_status q2_rjr(eth_grid* g, Level<T>& L, const T* rf, T omega, const int* done) {
  Q2Params<T, T, T> P{};
  P.n = L.n; P.hx = (T)L.hx; P.hy = (T)L.hy; P.nu = (T)L.nu; P.sd = (T)L.sd;
  P.w = L.w; P.dinv = L.dinv; P.omega = omega; P.done = done;
  P.bx = rf; P.y = L.r; P.y2 = L.x; P.bcopy = L.b;
  ETH_CUDA((launch_q2<T, T, T, QF_DIFF | QF_XIN | QF_UOUT | QF_SRC_JB | QF_SRC_RJB | CF, EPI_JR>(P, g->s)));
  g->launches++;
  return ETH_OK;
}

template <class T, class TO, int CF>
static eth_status q2_ps(eth_grid* g, Level<T>& L, const T* x, const T* xc, TO* y, T omega, const TO* bsrc,
                        const int* done, const Slot* slot, int slot_off, const TO* dv) {
  Q2Params<T, TO, T> P{};
  P.n = L.n; P.hx = (T)L.hx; P.hy = (T)L.hy; P.nu = (T)L.nu; P.sd = (T)L.sd;
  P.w = L.w; P.dinv = L.dinv; P.omega = omega; P.done = done;
  P.x = x; P.xc = xc; P.b = L.b; P.y = y; P.bsrc = bsrc;
  constexpr int F0 = QF_DIFF | QF_XIN | QF_UOUT | QF_SRC_XPC | CF;
  if (slot) {
    P.slot = *slot; P.slot_off = slot_off; P.dv = dv;
    ETH_CUDA((launch_q2<T, TO, T, F0 | QF_DOT, EPI_SMOOTH>(P, g->s)));
  } else {
    ETH_CUDA((launch_q2<T, TO, T, F0, EPI_SMOOTH>(P, g->s)));
  }
  g->launches++;
  return ETH_OK;
}

template <class T, int FL>
static eth_status q2_coarse_launch(eth_grid* g, Hier<T>& H, int Lc, int pre, int post, const int* done) {
  CoarseQ2<T> C{};
  C.nlev = (int)H.lv.size() - Lc;
  if (C.nlev > CMAXL) { set_error("multigrid: too many coarse levels"); return ETH_EINVAL; }
  size_t smem = 0;
  for (int l = 0; l < C.nlev; ++l) {
    const Level<T>& L = H.lv[Lc + l];
    C.n[l] = L.n; C.hx[l] = (T)L.hx; C.hy[l] = (T)L.hy; C.nu[l] = (T)L.nu; C.sd[l] = (T)L.sd;
    C.dinv[l] = L.dinv; C.w[l] = L.w;
    const size_t N = 2 * (size_t)L.n + 1;
    smem += (3 * 2 + 1 + ((FL & QF_CONV) ? 2 : 0)) * N * N * sizeof(T);
  }
  const size_t ainv_bytes = (size_t)H.ncoarse * H.ncoarse * sizeof(T);
  const int ainv_smem = (ainv_bytes <= 48 * 1024 && smem + ainv_bytes <= 200 * 1024) ? 1 : 0;
  if (ainv_smem) smem += ainv_bytes;
  static SmemAttr attr;   // largest dynamic shared memory enabled so far, per device
  if (smem > 200 * 1024) { set_error("multigrid: coarse levels exceed shared memory"); return ETH_EINVAL; }
  ETH_CUDA(smem_attr(k_q2_coarse_vc<T, FL>, smem, attr));
  k_q2_coarse_vc<T, FL><<<1, q2_coarse_threads<T, FL>(), smem, g->s>>>(C, H.coarse_inv, H.ncoarse, H.lv[Lc].b, H.lv[Lc].x, (T)H.omega, pre, post, done,
                                                  ainv_smem);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  return ETH_OK;
}

template <class T, int CF>
static eth_status vcycle_vel_fused_cf(eth_grid* g, Hier<T>& H, const double* v, double* z, int pre, int post,
                                      const int* done, const Slot* slot, int slot_off, int Lc) {
  const T om = (T)H.omega;
  std::vector<T*> res(H.lv.size(), nullptr);
  // level 0 from v; each coarser multi-CTA level restricts the finer level's residual
  // inside its first sweep (no separate restriction launch); the coarse V-cycle
  // kernel's level gets an explicit restriction
  for (int l = 0; l < Lc; ++l) {
    Level<T>& L = H.lv[l];
    const size_t N = 2 * (size_t)L.n + 1, nv = N * N;
    if (l == 0) ETH_TRY((q2_jr<T, double, CF>(g, L, v, L.b, om, done)));
    else ETH_TRY((q2_rjr<T, CF>(g, L, H.lv[l - 1].r, om, done)));
    for (int s = 1; s < pre; ++s) {
      ETH_TRY((q2_level<T, T, EPI_SMOOTH, CF>(g, L, L.x, L.t, om, nullptr, done, nullptr, 0, nullptr)));
      ETH_CUDA(cudaMemcpyAsync(L.x, L.t, 2 * nv * sizeof(T), cudaMemcpyDeviceToDevice, g->s));
      ETH_TRY((q2_level<T, T, EPI_RESID, CF>(g, L, L.x, L.r, om, nullptr, done, nullptr, 0, nullptr)));
    }
    if (l + 1 < Lc) continue;
    const Level<T>& Cn = H.lv[l + 1];
    const size_t Nc = 2 * (size_t)Cn.n + 1;
    k_q2_restrict<T><<<gsize(Nc * Nc), 256, 0, g->s>>>(Cn.n, L.r, Cn.b, done);
    ETH_CUDA(cudaGetLastError());
    g->launches++;
  }
  constexpr int FL = QF_DIFF | QF_XIN | QF_UOUT | CF;
  ETH_TRY((q2_coarse_launch<T, FL>(g, H, Lc, pre, post, done)));
  res[Lc] = H.lv[Lc].x;
  for (int l = Lc - 1; l >= 0; --l) {
    Level<T>& L = H.lv[l];
    const bool last0 = (l == 0 && post == 1);
    if (last0) {
      ETH_TRY((q2_ps<T, double, CF>(g, L, L.x, res[l + 1], z, om, v, done, slot, slot_off, v)));
      continue;
    }
    ETH_TRY((q2_ps<T, T, CF>(g, L, L.x, res[l + 1], L.t, om, nullptr, done, nullptr, 0, nullptr)));
    T* cur = L.t;
    T* oth = L.x;
    for (int s = 1; s < post; ++s) {
      if (l == 0 && s == post - 1) {
        ETH_TRY((q2_level<T, double, EPI_SMOOTH, CF>(g, L, cur, z, om, v, done, slot, slot_off, v)));
        cur = nullptr;
        break;
      }
      ETH_TRY((q2_level<T, T, EPI_SMOOTH, CF>(g, L, cur, oth, om, nullptr, done, nullptr, 0, nullptr)));
      std::swap(cur, oth);
    }
    res[l] = cur;
  }
  return ETH_OK;
}

template <class T>
static eth_status vcycle_vel_fused(eth_grid* g, Hier<T>& H, const double* v, double* z, int pre, int post,
                                   const int* done, const Slot* slot, int slot_off, int Lc) {
  const Level<T>& L0 = H.lv[0];
  // every level carries the streamline-diffusion coefficient (delta_T = 0 where the cell
  // Peclet number is <= 1), so one instantiation with QF_SD serves all levels.
  const bool sd = L0.w != nullptr && L0.sd > 0.0;
  if (L0.w != nullptr && H.trans && sd) return vcycle_vel_fused_cf<T, QF_CONV | QF_TRANS | QF_SD>(g, H, v, z, pre, post, done, slot, slot_off, Lc);
  if (L0.w != nullptr && H.trans) return vcycle_vel_fused_cf<T, QF_CONV | QF_TRANS>(g, H, v, z, pre, post, done, slot, slot_off, Lc);
  if (sd) return vcycle_vel_fused_cf<T, QF_CONV | QF_SD>(g, H, v, z, pre, post, done, slot, slot_off, Lc);
  if (L0.w != nullptr) return vcycle_vel_fused_cf<T, QF_CONV>(g, H, v, z, pre, post, done, slot, slot_off, Lc);
  return vcycle_vel_fused_cf<T, 0>(g, H, v, z, pre, post, done, slot, slot_off, Lc);
}

template <class T>
static eth_status q1_coarse_launch(eth_grid* g, Hier<T>& H, int Lc, const int* done) {
  CoarseQ1<T> C{};
  C.nlev = (int)H.lv.size() - Lc;
  if (C.nlev > CMAXL) { set_error("multigrid: too many Q1 coarse levels"); return ETH_EINVAL; }
  size_t smem = 0;
  for (int l = 0; l < C.nlev; ++l) {
    const Level<T>& L = H.lv[Lc + l];
    C.n[l] = L.n; C.hx[l] = (T)L.hx; C.hy[l] = (T)L.hy; C.dinv[l] = L.dinv;
    const size_t M = (size_t)L.n + 1;
    smem += 4 * M * M * sizeof(T);
  }
  const size_t ainv_bytes = (size_t)H.ncoarse * H.ncoarse * sizeof(T);
  const int ainv_smem = (ainv_bytes <= 48 * 1024 && smem + ainv_bytes <= 200 * 1024) ? 1 : 0;
  if (ainv_smem) smem += ainv_bytes;
  static SmemAttr attr;
  if (smem > 200 * 1024) { set_error("multigrid: Q1 coarse levels exceed shared memory"); return ETH_EINVAL; }
  ETH_CUDA(smem_attr(k_q1_coarse_vc<T>, smem, attr));
  k_q1_coarse_vc<T><<<1, 1024, smem, g->s>>>(C, H.coarse_inv, H.ncoarse, H.lv[Lc].b, H.lv[Lc].x, (T)H.omega, done,
                                              ainv_smem);
  ETH_CUDA(cudaGetLastError());
  g->launches++;
  return ETH_OK;
}

template <class T>
static int vel_fused_start(const Hier<T>& H) {
  const int thr = q2_coarse_threshold<T>();
  for (int l = 0; l < (int)H.lv.size(); ++l)
    if (H.lv[l].n <= thr) return ((int)H.lv.size() - l > CMAXL) ? -1 : l;
  return -1;
}
template <class T>
static int q1_fused_start(const Hier<T>& H) {
  const int thr = q1_coarse_threshold<T>();
  for (int l = 0; l < (int)H.lv.size(); ++l)
    if (H.lv[l].n <= thr) return ((int)H.lv.size() - l > CMAXL) ? -1 : l;
  return -1;
}

#define ETH_MG_INST(T)                                                                                    \
  template eth_status mg_build_vel<T>(eth_grid*, Hier<T>&, int, double, bool);                                 \
  template eth_status mg_build_q1<T>(eth_grid*, Hier<T>&, int);                                          \
  template void mg_free<T>(Hier<T>&);                                                                    \
  template eth_status vcycle_vel<T>(eth_grid*, Hier<T>&, const double*, double*, int, int, const int*,   \
                                    const Slot*, int);                                                   \
  template eth_status vcycle_q1_from<T>(eth_grid*, Hier<T>&, int, int, const int*, const T**, const Slot*, int); \
  template bool q1_vcycle_fused<T>(const Hier<T>&, int, int);
ETH_MG_INST(float)
ETH_MG_INST(double)

}  // namespace eth
