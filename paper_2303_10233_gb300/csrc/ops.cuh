// Declarations shared by the translation units of the library.
#pragma once
#include "common.cuh"
#include "grid.cuh"
#include "q2tile.cuh"
#include "q1ops.cuh"
#include "q2persist.cuh"
#include "q2strip.cuh"

namespace eth {
Slot make_slot(eth_grid* g, int which, int total);
eth_status op_apply(eth_grid* g, eth_op op, bool fp32, const double* x, double* y);
eth_status op_apply_K_dot(eth_grid* g, bool fp32, bool trans, const double* x, double* y, Slot s, const int* done);
eth_status op_apply_K(eth_grid* g, bool fp32, bool trans, const double* x, double* y, const int* done);
constexpr int TILE_PERSIST = 100;   // tile code offset of the persistent K apply
// (TILE_STRIP = 200 in q2strip.cuh: tile code offset of the warp-strip K apply)
int tile_code(const eth_grid* g);
int tile_rows(const eth_grid* g);
bool tile_persistent(const eth_grid* g);
bool tile_strip(const eth_grid* g);
eth_status op_apply_tiles(eth_grid* g, bool fp32, const double* x, double* y, Slot s, int ty);
eth_status tune_tiles(eth_grid* g, bool fp32);
eth_status assemble_rhs(eth_grid* g, const double* f, const double* ubc);
eth_status grad_kernels(eth_grid* g, const double* lu, const double* u, double* grad_f, double* scratch_lm,
                        double* scratch_au, double* grad_nu);
}  // namespace eth
