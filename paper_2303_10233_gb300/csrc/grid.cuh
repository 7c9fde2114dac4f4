// Internal state of an eth_grid handle (host side) and the device pools.
#pragma once
#include <vector>
#include "common.cuh"

struct eth_grid;

namespace eth {

// One level of the velocity (Q2) or pressure (Q1) multigrid hierarchy.
template <class T>
struct Level {
  int n = 0;
  double hx = 0, hy = 0;
  double nu = 1.0;       // viscosity of the level operator
  double sd = 0.0;       // streamline-diffusion coefficient of the level (coarse Oseen levels)
  bool trans = false;    // transposed convection (adjoint operator F^T)
  T* w = nullptr;        // Q2 wind (2 N_v), velocity levels with convection
  T* dinv = nullptr;     // inverse diagonal (N_v for velocity, (n+1)^2 for Q1)
  T* x = nullptr;        // iterate
  T* b = nullptr;        // right-hand side
  T* r = nullptr;        // residual / scratch
  T* t = nullptr;        // smoother ping-pong
  T* conv = nullptr;     // Q1 levels: per-element 4x4 convection matrices
};

template <class T>
struct Hier {
  std::vector<Level<T>> lv;
  T* coarse_inv = nullptr;   // dense inverse of the coarsest interior operator
  int* coarse_idx = nullptr; // lattice index of each coarse unknown
  int ncoarse = 0;
  bool q1 = false;           // pressure (Q1 Laplacian) hierarchy
  bool trans = false;        // velocity hierarchy of F^T (adjoint)
  bool built = false;
  bool fused = true;         // fused level kernels + single-CTA coarse V-cycle
  double omega = 0.8;
};

}  // namespace eth

struct eth_grid {
  int n = 0;
  int dev = 0;                // CUDA device current at creation (owns every allocation below)
  double x0 = -1, x1 = 1, y0 = -1, y1 = 1, hx = 0, hy = 0;
  eth_kind kind = ETH_STOKES;
  cudaStream_t s = nullptr;
  int nv = 0, n1 = 0, n0 = 0, nt = 0;
  double nu = 1.0;
  bool has_coef = false, has_rhs = false;
  double* wind = nullptr;     // 2 nv FP64
  float* windf = nullptr;     // 2 nv FP32
  double* b = nullptr;        // assembled right-hand side (nt)
  double* ubc = nullptr;      // Dirichlet data (2 nv), boundary entries only
  double* tmp = nullptr;      // scratch (nt)
  double* tmp2 = nullptr;     // scratch (nt)
  eth::Scalars* sc = nullptr; // device scalars
  eth::Scalars* sch = nullptr;// pinned host mirror
  double* part = nullptr;     // reduction partials
  unsigned* ticket = nullptr; // reduction tickets (16)
  int part_cap = 0;
  double* lz = nullptr;       // Lanczos coefficients of MINRES (2 x ETH_LANCZOS_CAP)
  // solver workspaces are created lazily by the solvers
  void* ws = nullptr;
  void (*ws_free)(void*) = nullptr;
  long launches = 0;
  int tile_rows = 0;          // element rows per CTA of the fused K apply (0: default shape)
  bool tuned = false;         // tile_rows chosen by the autotuner
};

struct eth_batch {
  std::vector<eth_grid*> grids;
  int workers = 0;   // host workers (0: min(count, 16))
};
