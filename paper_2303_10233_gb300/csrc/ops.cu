// Operator applies of the public ABI (eth_apply) and right-hand-side assembly.
#include <map>
#include <mutex>
#include <tuple>
#include <cstdio>
#include <cstdlib>
#include "ops.cuh"

namespace eth {

Slot make_slot(eth_grid* g, int which, int total) {
  Slot s;
  s.part = g->part + (size_t)which * g->part_cap;
  s.ticket = g->ticket + which;
  s.out = &g->sc->dots[which];
  s.total = total;
  s.op = FIN_STORE;
  s.sc = g->sc;
  return s;
}

template <class CT>
static const CT* wind_ptr(eth_grid* g);
template <>
const float* wind_ptr<float>(eth_grid* g) { return g->windf; }
template <>
const double* wind_ptr<double>(eth_grid* g) { return g->wind; }

// y = K x with the velocity block F (Stokes: nu*A, Oseen: nu*A + N) --------
// TUNED: the fused K apply, launched with the grid's (autotuned) tile: 32 x rows
// elements, one tile per CTA, or (FP32 element arithmetic only) the persistent
// pipelined 32 x 8 kernel.  A tile code is rows, or rows + TILE_PERSIST.
int tile_code(const eth_grid* g) { return g->tile_rows ? g->tile_rows : TILE_STRIP + 8; }
int tile_rows(const eth_grid* g) { return tile_code(g) % TILE_PERSIST; }
bool tile_persistent(const eth_grid* g) { return tile_code(g) >= TILE_PERSIST && tile_code(g) < TILE_STRIP; }
bool tile_strip(const eth_grid* g) { return tile_code(g) >= TILE_STRIP; }

template <class CT, int F, bool TUNED = false>
static eth_status run_q2(eth_grid* g, const double* x, const double* p, double* y, double* yp,
                         const int* done = nullptr, Slot* slot = nullptr, int slot_off = 0, int code = 0) {
  Q2Params<double, double, CT> P{};
  P.n = g->n; P.hx = (CT)g->hx; P.hy = (CT)g->hy; P.nu = (CT)g->nu;
  P.x = x; P.p = p; P.w = wind_ptr<CT>(g); P.y = y; P.yp = yp;
  P.done = done;
  if (slot) { P.slot = *slot; P.slot_off = slot_off; P.dv = x; P.dvp = p; }
  if (TUNED) {
    if (!code) code = tile_code(g);
    const int ty = code % TILE_PERSIST;
    if constexpr ((F & QF_XIN) && (F & QF_UOUT) && !(F & (QF_NOBC | QF_MASS))) {
      if (code >= TILE_STRIP) {
        const int rows = code - TILE_STRIP;
        if (slot) P.slot.total = q2s_blocks(g->n, rows);
        ETH_CUDA((launch_q2s<CT, F>(P, g->s, rows)));
        g->launches++;
        return ETH_OK;
      }
    }
    if constexpr (sizeof(CT) == 4 && (F & QF_XIN) && !(F & (QF_NOBC | QF_MASS))) {
      if (code >= TILE_PERSIST) {
        if (slot) P.slot.total = q2p_blocks<F>(g->n);
        ETH_CUDA((launch_q2p<F>(P, g->s)));
        g->launches++;
        return ETH_OK;
      }
    }
    if (slot) P.slot.total = q2_blocks(g->n, ty);
    ETH_CUDA((launch_q2_ty<double, double, CT, F, EPI_APPLY>(P, g->s, ty)));
  } else {
    ETH_CUDA((launch_q2<double, double, CT, F, EPI_APPLY>(P, g->s)));
  }
  g->launches++;
  return ETH_OK;
}

template <class CT>
static eth_status apply_t(eth_grid* g, eth_op op, const double* x, double* y) {
  const bool conv = g->kind == ETH_OSEEN;
  const size_t nu2 = 2 * (size_t)g->nv;
  switch (op) {
    case ETH_OP_K:
      if (conv) return run_q2<CT, QF_DIFF | QF_CONV | QF_XIN | QF_PIN | QF_P0 | QF_UOUT | QF_POUT, true>(g, x, x + nu2, y, y + nu2);
      return run_q2<CT, QF_DIFF | QF_XIN | QF_PIN | QF_P0 | QF_UOUT | QF_POUT, true>(g, x, x + nu2, y, y + nu2);
    case ETH_OP_KT:
      if (conv) return run_q2<CT, QF_DIFF | QF_CONV | QF_TRANS | QF_XIN | QF_PIN | QF_P0 | QF_UOUT | QF_POUT, true>(g, x, x + nu2, y, y + nu2);
      return run_q2<CT, QF_DIFF | QF_XIN | QF_PIN | QF_P0 | QF_UOUT | QF_POUT, true>(g, x, x + nu2, y, y + nu2);
    case ETH_OP_K1:
      if (conv) return run_q2<CT, QF_DIFF | QF_CONV | QF_XIN | QF_PIN | QF_UOUT | QF_POUT, true>(g, x, x + nu2, y, y + nu2);
      return run_q2<CT, QF_DIFF | QF_XIN | QF_PIN | QF_UOUT | QF_POUT, true>(g, x, x + nu2, y, y + nu2);
    case ETH_OP_K1T:
      if (conv) return run_q2<CT, QF_DIFF | QF_CONV | QF_TRANS | QF_XIN | QF_PIN | QF_UOUT | QF_POUT, true>(g, x, x + nu2, y, y + nu2);
      return run_q2<CT, QF_DIFF | QF_XIN | QF_PIN | QF_UOUT | QF_POUT, true>(g, x, x + nu2, y, y + nu2);
    case ETH_OP_A:
      return run_q2<CT, QF_DIFF | QF_XIN | QF_UOUT>(g, x, nullptr, y, nullptr);
    case ETH_OP_F:
      if (conv) return run_q2<CT, QF_DIFF | QF_CONV | QF_XIN | QF_UOUT>(g, x, nullptr, y, nullptr);
      return run_q2<CT, QF_DIFF | QF_XIN | QF_UOUT>(g, x, nullptr, y, nullptr);
    case ETH_OP_B:
      return run_q2<CT, QF_XIN | QF_P0 | QF_POUT>(g, x, nullptr, nullptr, y);
    case ETH_OP_BT:
      return run_q2<CT, QF_PIN | QF_P0 | QF_UOUT>(g, nullptr, x, y, nullptr);
    case ETH_OP_MV:
      return run_q2<CT, QF_MASS | QF_XIN | QF_UOUT | QF_NOBC>(g, x, nullptr, y, nullptr);
    case ETH_OP_MQ: {
      Q1Params<double, double, CT> P{};
      P.n = g->n; P.hx = (CT)g->hx; P.hy = (CT)g->hy;
      P.cm = 1; P.ck = 0; P.c1 = 0; P.x = x; P.x0 = x + g->n1; P.r0 = 1; P.y = y;
      k_q1node<double, double, CT, Q1E_APPLY><<<q1_blocks(g->n), 256, 0, g->s>>>(P);
      ETH_CUDA(cudaGetLastError());
      k_p0rows<double, double, CT><<<cdiv((long)g->n0, 256), 256, 0, g->s>>>(
          g->n, (CT)(g->hx * g->hy), (CT)1, (CT)1, x, x + g->n1, y + g->n1, nullptr);
      ETH_CUDA(cudaGetLastError());
      g->launches += 2;
      return ETH_OK;
    }
  }
  set_error("eth_apply: unknown operator %d", (int)op);
  return ETH_EINVAL;
}

eth_status op_apply(eth_grid* g, eth_op op, bool fp32, const double* x, double* y) {
  return fp32 ? apply_t<float>(g, op, x, y) : apply_t<double>(g, op, x, y);
}

// K z with the fused FP64 dot <Kz, z> into slot `which` (MINRES delta) ----
template <class CT>
static eth_status apply_dot_t(eth_grid* g, bool trans, const double* x, double* y, Slot s, const int* done, int ty) {
  const bool conv = g->kind == ETH_OSEEN;
  const size_t nu2 = 2 * (size_t)g->nv;
  if (conv && trans)
    return run_q2<CT, QF_DIFF | QF_CONV | QF_TRANS | QF_XIN | QF_PIN | QF_P0 | QF_UOUT | QF_POUT | QF_DOT, true>(g, x, x + nu2, y, y + nu2, done, &s, 0, ty);
  if (conv)
    return run_q2<CT, QF_DIFF | QF_CONV | QF_XIN | QF_PIN | QF_P0 | QF_UOUT | QF_POUT | QF_DOT, true>(g, x, x + nu2, y, y + nu2, done, &s, 0, ty);
  return run_q2<CT, QF_DIFF | QF_XIN | QF_PIN | QF_P0 | QF_UOUT | QF_POUT | QF_DOT, true>(g, x, x + nu2, y, y + nu2, done, &s, 0, ty);
}

eth_status op_apply_K_dot(eth_grid* g, bool fp32, bool trans, const double* x, double* y, Slot s, const int* done) {
  return fp32 ? apply_dot_t<float>(g, trans, x, y, s, done, 0) : apply_dot_t<double>(g, trans, x, y, s, done, 0);
}

eth_status op_apply_K(eth_grid* g, bool fp32, bool trans, const double* x, double* y, const int* done) {
  const bool conv = g->kind == ETH_OSEEN;
  const size_t nu2 = 2 * (size_t)g->nv;
  if (fp32) {
    if (conv && trans) return run_q2<float, QF_DIFF | QF_CONV | QF_TRANS | QF_XIN | QF_PIN | QF_P0 | QF_UOUT | QF_POUT, true>(g, x, x + nu2, y, y + nu2, done);
    if (conv) return run_q2<float, QF_DIFF | QF_CONV | QF_XIN | QF_PIN | QF_P0 | QF_UOUT | QF_POUT, true>(g, x, x + nu2, y, y + nu2, done);
    return run_q2<float, QF_DIFF | QF_XIN | QF_PIN | QF_P0 | QF_UOUT | QF_POUT, true>(g, x, x + nu2, y, y + nu2, done);
  }
  if (conv && trans) return run_q2<double, QF_DIFF | QF_CONV | QF_TRANS | QF_XIN | QF_PIN | QF_P0 | QF_UOUT | QF_POUT, true>(g, x, x + nu2, y, y + nu2, done);
  if (conv) return run_q2<double, QF_DIFF | QF_CONV | QF_XIN | QF_PIN | QF_P0 | QF_UOUT | QF_POUT, true>(g, x, x + nu2, y, y + nu2, done);
  return run_q2<double, QF_DIFF | QF_XIN | QF_PIN | QF_P0 | QF_UOUT | QF_POUT, true>(g, x, x + nu2, y, y + nu2, done);
}

// ---------------------------------------------------------------------------
// Tile-height autotuner: times the fused K apply with its dot (the form the
// Krylov loops launch) for every tile height whose block count fits the
// reduction partials, on the grid's right-hand side, and keeps the fastest.
// Results are cached per (n, operator kind, precision) for the process.
// ---------------------------------------------------------------------------
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int> g_tune_cache;
}  // namespace

eth_status tune_tiles(eth_grid* g, bool fp32) {
  if (g->tuned) return ETH_OK;
  const auto key = std::make_tuple(g->n, (int)g->kind, fp32 ? 1 : 0);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) { g->tile_rows = it->second; g->tuned = true; return ETH_OK; }
  }
  // Each candidate is timed as a captured graph of REPS back-to-back launches on a
  // private stream, the way the solvers replay it: timing stream launches would
  // measure the host's launch rate (about 2 us per launch) for the small grids.
  // Three rounds over all candidates, the minimum per candidate; a strip form
  // within 10 % of the fastest wins the tie: inside the solvers' graphs, between
  // the shared-memory-heavy multigrid kernels, the strip forms (no shared memory)
  // measured relatively faster than alone (256^2 Stokes solve 5.83 ms with 2-row
  // strips against 6.03 ms with 32 x 8 tiles, which alone time 14.2 and 13.4 us).
  // ETH_TUNE_VERBOSE=1 in the environment prints every candidate's time.
  cudaEvent_t e0, e1, ej;
  cudaStream_t ts;
  ETH_CUDA(cudaEventCreate(&e0));
  ETH_CUDA(cudaEventCreate(&e1));
  ETH_CUDA(cudaEventCreateWithFlags(&ej, cudaEventDisableTiming));
  ETH_CUDA(cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking));
  ETH_CUDA(cudaEventRecord(ej, g->s));
  ETH_CUDA(cudaStreamWaitEvent(ts, ej, 0));
  const cudaStream_t keep = g->s;
  g->s = ts;
  eth_status st = ETH_OK;
  const int cands[9] = {4, 8, 16, 8 + TILE_PERSIST, 2 + TILE_STRIP, 4 + TILE_STRIP, 6 + TILE_STRIP, 8 + TILE_STRIP, 16 + TILE_STRIP};
  constexpr int NC = 9, REPS = 16, ROUNDS = 3;
  cudaGraphExec_t exec[NC] = {};
  float tmin[NC];
  for (int c = 0; c < NC; ++c) tmin[c] = 1e30f;
  for (int c = 0; c < NC && st == ETH_OK; ++c) {
    const int ty = cands[c];
    if (ty >= TILE_PERSIST && ty < TILE_STRIP && !fp32) continue;
    if (ty < TILE_PERSIST && q2_blocks(g->n, ty) > g->part_cap) continue;
    if (ty >= TILE_STRIP && q2s_blocks(g->n, ty - TILE_STRIP) > g->part_cap) continue;
    Slot s = make_slot(g, 11, 0);
    for (int r = 0; r < 2 && st == ETH_OK; ++r) st = op_apply_tiles(g, fp32, g->b, g->tmp, s, ty);   // warm (attributes set)
    if (st != ETH_OK) break;
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(ts, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) { st = cuda_status(ce, "autotune capture"); break; }
    for (int r = 0; r < REPS && st == ETH_OK; ++r) st = op_apply_tiles(g, fp32, g->b, g->tmp, s, ty);
    ce = cudaStreamEndCapture(ts, &graph);
    if (st != ETH_OK) { if (graph) cudaGraphDestroy(graph); break; }
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec[c], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (ce != cudaSuccess) { exec[c] = nullptr; st = cuda_status(ce, "autotune graph"); break; }
  }
  for (int round = 0; round < ROUNDS && st == ETH_OK; ++round)
    for (int c = 0; c < NC && st == ETH_OK; ++c) {
      if (!exec[c]) continue;
      cudaGraphLaunch(exec[c], ts);   // warm
      cudaEventRecord(e0, ts);
      for (int r = 0; r < 2; ++r) cudaGraphLaunch(exec[c], ts);
      cudaEventRecord(e1, ts);
      const cudaError_t ce = cudaEventSynchronize(e1);
      if (ce != cudaSuccess) { st = cuda_status(ce, "autotune"); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      tmin[c] = std::min(tmin[c], ms);
      if (std::getenv("ETH_TUNE_VERBOSE"))
        std::fprintf(stderr, "autotune n=%d fp32=%d code=%d us=%.3f\n", g->n, (int)fp32, cands[c], ms * 1e3 / (2 * REPS));
    }
  for (cudaGraphExec_t& e : exec)
    if (e) cudaGraphExecDestroy(e);
  int best = TILE_STRIP + 8;
  float best_ms = 1e30f;
  for (int c = 0; c < NC; ++c)
    if (tmin[c] < best_ms) { best_ms = tmin[c]; best = cands[c]; }
  if (best < TILE_STRIP)   // tie-break toward the strip forms
    for (int c = 0; c < NC; ++c)
      if (cands[c] >= TILE_STRIP && tmin[c] <= 1.10f * best_ms) { best = cands[c]; break; }
  g->s = keep;
  cudaEventRecord(ej, ts);
  cudaStreamWaitEvent(keep, ej, 0);
  cudaStreamSynchronize(ts);
  cudaStreamDestroy(ts);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(ej);
  if (st != ETH_OK) return st;
  g->tile_rows = best;
  g->tuned = true;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = best;
  return ETH_OK;
}

}  // namespace eth

extern "C" eth_status eth_grid_set_tile(eth_grid* g, int rows, int persistent) {
  using namespace eth;
  if (!g) { set_error("eth_grid_set_tile: NULL grid"); return ETH_EINVAL; }
  ETH_ON_DEVICE(g);
  if (rows == 0) { g->tile_rows = 0; g->tuned = false; return ETH_OK; }
  if (persistent == 2) {   // warp-strip kernel, `rows` element rows per warp
    if (!q2s_rows_ok(rows)) { set_error("eth_grid_set_tile: strip rows=%d not in 2..32", rows); return ETH_EINVAL; }
    if (q2s_blocks(g->n, rows) > g->part_cap) { set_error("eth_grid_set_tile: too many strips for n=%d", g->n); return ETH_EINVAL; }
    g->tile_rows = rows + TILE_STRIP;
    g->tuned = true;
    return ETH_OK;
  }
  if (!q2_tile_ok(rows)) { set_error("eth_grid_set_tile: rows=%d not in {4, 8, 16}", rows); return ETH_EINVAL; }
  if (persistent && rows != 8) { set_error("eth_grid_set_tile: the persistent kernel has 8 rows"); return ETH_EINVAL; }
  if (!persistent && q2_blocks(g->n, rows) > g->part_cap) { set_error("eth_grid_set_tile: too many tiles for n=%d", g->n); return ETH_EINVAL; }
  g->tile_rows = rows + (persistent ? TILE_PERSIST : 0);
  g->tuned = true;
  return ETH_OK;
}

namespace eth {

eth_status op_apply_tiles(eth_grid* g, bool fp32, const double* x, double* y, Slot s, int ty) {
  return fp32 ? apply_dot_t<float>(g, false, x, y, s, nullptr, ty) : apply_dot_t<double>(g, false, x, y, s, nullptr, ty);
}

// ---------------------------------------------------------------------------
// adjoint gradients: grad_f = M_v D_I l_u ; grad_nu = -(D_I l_u)^T A u
// ---------------------------------------------------------------------------
__global__ void k_keep_interior(int n, const double* __restrict__ src, double* __restrict__ dst) {
  ETH_GRID_DEP_WAIT();
  const int N = 2 * n + 1;
  const size_t nv = (size_t)N * N;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < 2 * nv; k += (size_t)gridDim.x * blockDim.x) {
    const size_t gg = k < nv ? k : k - nv;
    const int j = (int)(gg / N), i = (int)(gg - (size_t)j * N);
    dst[k] = (i == 0 || j == 0 || i == N - 1 || j == N - 1) ? 0.0 : src[k];
  }
}

eth_status grad_kernels(eth_grid* g, const double* lu, const double* u, double* grad_f, double* scratch_lm,
                        double* scratch_au, double* grad_nu) {
  const size_t nu2 = 2 * (size_t)g->nv;
  const unsigned nb = cdiv((long)nu2, 256) > 4096 ? 4096 : cdiv((long)nu2, 256);
  k_keep_interior<<<nb, 256, 0, g->s>>>(g->n, lu, scratch_lm);
  ETH_CUDA(cudaGetLastError());
  ETH_TRY((run_q2<double, QF_MASS | QF_XIN | QF_UOUT | QF_NOBC>(g, scratch_lm, nullptr, grad_f, nullptr)));
  // A u on the full lattice (no Dirichlet treatment), unit viscosity, fused dot with D_I l_u
  Q2Params<double, double, double> P{};
  P.n = g->n; P.hx = g->hx; P.hy = g->hy; P.nu = 1.0;
  P.x = u; P.y = scratch_au;
  Slot s = make_slot(g, 8, q2_blocks(g->n));
  P.slot = s; P.slot_off = 0; P.dv = scratch_lm;
  ETH_CUDA((launch_q2<double, double, double, QF_DIFF | QF_XIN | QF_UOUT | QF_NOBC | QF_DOT, EPI_APPLY>(P, g->s)));
  ETH_CUDA(cudaMemcpyAsync(&g->sch->dots[8], &g->sc->dots[8], 8, cudaMemcpyDeviceToHost, g->s));
  ETH_CUDA(cudaStreamSynchronize(g->s));
  *grad_nu = -g->sch->dots[8];
  g->launches += 3;
  return ETH_OK;
}

// ---------------------------------------------------------------------------
// right-hand side: b = [D_I (M f - F u_b) + D_B u_b ; -B u_b]
// ---------------------------------------------------------------------------
__global__ void k_rhs_combine(int n, const double* __restrict__ mf, const double* __restrict__ fub,
                              const double* __restrict__ ub, double* __restrict__ bu) {
  ETH_GRID_DEP_WAIT();
  const int N = 2 * n + 1;
  const size_t nv = (size_t)N * N;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < 2 * nv; k += (size_t)gridDim.x * blockDim.x) {
    const size_t g = k < nv ? k : k - nv;
    const int j = (int)(g / N), i = (int)(g - (size_t)j * N);
    const bool bnd = i == 0 || j == 0 || i == N - 1 || j == N - 1;
    bu[k] = bnd ? ub[k] : mf[k] - fub[k];
  }
}

__global__ void k_keep_boundary(int n, const double* __restrict__ src, double* __restrict__ dst) {
  ETH_GRID_DEP_WAIT();
  const int N = 2 * n + 1;
  const size_t nv = (size_t)N * N;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < 2 * nv; k += (size_t)gridDim.x * blockDim.x) {
    const size_t g = k < nv ? k : k - nv;
    const int j = (int)(g / N), i = (int)(g - (size_t)j * N);
    const bool bnd = i == 0 || j == 0 || i == N - 1 || j == N - 1;
    dst[k] = bnd ? src[k] : 0.0;
  }
}

__global__ void k_scale(size_t m, double a, double* __restrict__ x) {
  ETH_GRID_DEP_WAIT();
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) x[k] *= a;
}

eth_status assemble_rhs(eth_grid* g, const double* f, const double* ubc) {
  const size_t nu2 = 2 * (size_t)g->nv;
  const unsigned nb = cdiv((long)nu2, 256) > 4096 ? 4096 : cdiv((long)nu2, 256);
  k_keep_boundary<<<nb, 256, 0, g->s>>>(g->n, ubc, g->ubc);
  ETH_CUDA(cudaGetLastError());
  double* mf = g->tmp;
  double* fub = g->tmp2;
  // M f (no Dirichlet masking)
  ETH_TRY((run_q2<double, QF_MASS | QF_XIN | QF_UOUT | QF_NOBC>(g, f, nullptr, mf, nullptr)));
  // F u_b with the boundary-only field (no masking of the input)
  if (g->kind == ETH_OSEEN) {
    ETH_TRY((run_q2<double, QF_DIFF | QF_CONV | QF_XIN | QF_UOUT | QF_NOBC>(g, g->ubc, nullptr, fub, nullptr)));
  } else {
    ETH_TRY((run_q2<double, QF_DIFF | QF_XIN | QF_UOUT | QF_NOBC>(g, g->ubc, nullptr, fub, nullptr)));
  }
  k_rhs_combine<<<nb, 256, 0, g->s>>>(g->n, mf, fub, g->ubc, g->b);
  ETH_CUDA(cudaGetLastError());
  // g = -B u_b
  ETH_TRY((run_q2<double, QF_XIN | QF_P0 | QF_POUT | QF_NOBC>(g, g->ubc, nullptr, nullptr, g->b + nu2)));
  k_scale<<<cdiv((long)(g->n1 + g->n0), 256), 256, 0, g->s>>>((size_t)(g->n1 + g->n0), -1.0, g->b + nu2);
  ETH_CUDA(cudaGetLastError());
  g->launches += 4;
  return ETH_OK;
}

}  // namespace eth
