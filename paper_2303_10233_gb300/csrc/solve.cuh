// Solver entry points (MINRES / GMRES drivers, multigrid, pressure blocks).
#pragma once
#include "ops.cuh"
#include "mg.cuh"

namespace eth {

enum : int { SL_DELTA = 0, SL_VSUM = 1, SL_GAMMA = 2, SL_MQ = 3, SL_DONE = 4, SL_NORM = 5, SL_PSUM = 6, SL_GEN = 7 };

// Solver workspace owned by a handle (created on the first solve).
struct GMRESWork;
struct Work {
  Hier<float> vf, qf, vft;     // velocity (F), Q1 Laplacian, velocity (F^T) hierarchies
  Hier<double> vd, qd, vdt;
  bool need_adj = false;       // build the F^T hierarchy (adjoint solves)
  double *x = nullptr, *d = nullptr, *r = nullptr, *Kz = nullptr, *bp = nullptr;
  double *V[2] = {nullptr, nullptr}, *Z[2] = {nullptr, nullptr}, *W[2] = {nullptr, nullptr};
  cudaStream_t s2 = nullptr;   // second branch (pressure block)
  cudaStream_t s3 = nullptr;   // third branch (MINRES w/x update beside the K apply)
  cudaEvent_t evw = nullptr, evx = nullptr;
  cudaStream_t sm = nullptr;   // internal main stream (capturable), joined to the user stream
  cudaEvent_t evf = nullptr, evj = nullptr, evu = nullptr, t0 = nullptr, t1 = nullptr;
  cudaGraphExec_t gexec = nullptr;
  long long gkey = -1;
  long glaunch = 0;            // kernels in one replay of gexec
  bool no_cond_nodes = false;  // the driver refused a conditional graph node: host-replayed graphs
  int nmin_built = -1;
  GMRESWork* gm = nullptr;     // GMRES / PCD workspace (Oseen)
  double* pcg = nullptr;       // exact-block inner PCG vectors (4 x 2 N_v + 6 x N_1)
  void* lscw[2] = {nullptr, nullptr};   // LSC preconditioner workspaces (FP32, FP64; lsc.cu)
  void* mcw[2] = {nullptr, nullptr};    // Chebyshev-SGS M_Q workspaces (FP32, FP64; mqcheb.cu)
};


// sums of the Q1 and P0 pressure blocks of x (offset off): FIN_* of (sum p1, sum p0)
template <int D>
__global__ void k_psums(size_t off, size_t n1, size_t n0, const double* __restrict__ x, Slot sl) {
  ETH_GRID_DEP_WAIT();
  double a1 = 0.0, a0 = 0.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n1 + n0; k += (size_t)gridDim.x * blockDim.x) {
    if (k < n1) a1 += x[off + k]; else a0 += x[off + k];
  }
  double v[2] = {a1, a0};
  if (slot_arrive<2>(sl, blockIdx.x, v)) finish_slot_n<2>(sl, v);
}

void solver_free(eth_grid* g);
eth_status solver_coefficients_changed(eth_grid* g);
eth_status work_get(eth_grid* g, Work** out);
int vblocks(size_t m);
Slot slot_of(eth_grid* g, int which, int total, int op);
eth_status read_scalars(eth_grid* g);
eth_status canonicalize(eth_grid* g, double* x);
eth_status rhs_inconsistency(eth_grid* g, Work* w, const double* bp, double* incons, double* nbp);
eth_status true_residual(eth_grid* g, Work* w, const double* b, double* rr, bool trans = false);
int mq_blocks(eth_grid* g);
template <class T>
eth_status precond_pressure(eth_grid* g, Hier<T>& Q, const double* vp, double* zp, const Slot& gsl, int goff,
                            const int* done, cudaStream_t s);
template <class T>
eth_status ensure_hier(eth_grid* g, Work* w, const eth_opts* o);
template <class T>
Hier<T>& vel_hier(Work* w);
template <class T>
Hier<T>& q1_hier(Work* w);
template <class T>
Hier<T>& vel_hier_t(Work* w);
eth_status adjoint_gradients(eth_grid* g, Work* w, const double* lu, const double* u, double* grad_f, double* grad_nu);
void gmres_free(Work* w);
void lsc_free(Work* w);
void mqcheb_free(Work* w);
double mqcheb_default_a(const eth_grid* g);
template <class T>
eth_status mqcheb_prepare(eth_grid* g, Work* w);
// MINRES pressure block nu M_cheb^{-1} (the cheap M_Q of P_2, Sec. 2.3-2.4), mqcheb.cu
template <class T>
eth_status precond_pressure_cheb(eth_grid* g, Work* w, const eth_opts* o, const double* vp, double* zp, const Slot& gsl,
                                 int goff, const int* done, cudaStream_t s);
// z = M_3^{-1} r, the LSC block-triangular preconditioner (Sec. 3.2) of the full Oseen system
template <class T>
eth_status lsc_prepare(eth_grid* g, Work* w);
template <class T>
eth_status precond_lsc(eth_grid* g, Work* w, const eth_opts* o, const double* r, double* z, const int* done, bool adj);
eth_status oseen_solve(eth_grid* g, Work* w, const eth_opts* o, eth_stats* st, bool adjoint, const double* b);
eth_status oseen_prepare(eth_grid* g, Work* w, const eth_opts* o);

// Runs the solver body on the handle's internal stream (capturable even when
// the user stream is the legacy default stream), ordered after and before the
// user stream's work.
struct StreamSwap {
  eth_grid* g;
  Work* w;
  cudaStream_t user;
  StreamSwap(eth_grid* g_, Work* w_) : g(g_), w(w_), user(g_->s) {
    cudaEventRecord(w->evu, user);
    cudaStreamWaitEvent(w->sm, w->evu, 0);
    g->s = w->sm;
  }
  ~StreamSwap() {
    cudaEventRecord(w->evu, w->sm);
    cudaStreamWaitEvent(user, w->evu, 0);
    g->s = user;
  }
};

}  // namespace eth
