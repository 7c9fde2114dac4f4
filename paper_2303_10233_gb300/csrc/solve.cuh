// Solver entry points (MINRES / GMRES drivers, multigrid, pressure blocks).
#pragma once
#include "ops.cuh"

namespace eth {
void solver_free(eth_grid* g);
eth_status solver_coefficients_changed(eth_grid* g);
}  // namespace eth
