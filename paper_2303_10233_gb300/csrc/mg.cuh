// Geometric multigrid on nested uniform grids n -> n/2 -> ... -> n_c.
//
// Velocity hierarchy (Q2): operator nu_l*A + N(w_l) with Dirichlet rows, wind
// injected at the coarse nodes (coarse Q2 nodes are fine Q2 nodes), Q2
// interpolation P (tensor product of the 1D quadratic interpolation from the
// coarse element to the fine nodes at t = 1/4, 1/2, 3/4), restriction P^T,
// damped Jacobi smoothing, dense exact solve on the coarsest grid.  With
// equal pre/post sweeps the V-cycle is symmetric, as MINRES requires.
//
// Pressure hierarchy (Q1): Q1 Laplacian K1 (natural boundary, singular with
// the constants), bilinear interpolation, damped Jacobi, pseudo-inverse on the
// coarsest grid.  Used as the preconditioner of the Schur complement
// S = Qk - R^T Q0^{-1} R of M_Q (element-wise h^2/24 K1 <= S <= h^2/12 K1) and
// of the PCD matrices.
#pragma once
#include "ops.cuh"

namespace eth {

template <class T>
eth_status mg_build_vel(eth_grid* g, Hier<T>& H, int nmin, double art, bool trans = false);
template <class T>
eth_status mg_build_q1(eth_grid* g, Hier<T>& H, int nmin);
template <class T>
void mg_free(Hier<T>& H);

// z_u = V(v_u): one V-cycle on both velocity components.  v and z are FP64
// (2 N_v); boundary rows copy v.  If slot != nullptr the final smoothing adds
// <z_u, v_u> partials at slot_off.
template <class T>
eth_status vcycle_vel(eth_grid* g, Hier<T>& H, const double* v, double* z, int pre, int post, const int* done,
                      const Slot* slot, int slot_off);
// Q1 V-cycle on level 0 whose b (and, for the unfused path, x after the first
// sweep) are already set; *result points to the level-0 result (type T).
template <class T>
eth_status vcycle_q1_from(eth_grid* g, Hier<T>& H, int pre, int post, const int* done, const T** result,
                          const Slot* sums = nullptr, int soff = 0);
// true when vcycle_q1_from takes the fused path (and can fold the level-0 sums)
template <class T>
bool q1_vcycle_fused(const Hier<T>& H, int pre, int post);
int vel_final_blocks(int n);

}  // namespace eth
