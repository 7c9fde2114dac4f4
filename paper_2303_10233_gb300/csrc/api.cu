// C ABI entry points: handles, coefficients, right-hand side, operator applies.
#include <cstdarg>
#include <cstring>
#include <cmath>
#include "ops.cuh"
#include "solve.cuh"

namespace eth {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

eth_status cuda_status(cudaError_t e, const char* what) {
  set_error("CUDA error %s (%s) in %s", cudaGetErrorName(e), cudaGetErrorString(e), what);
  return e == cudaErrorMemoryAllocation ? ETH_ENOMEM : ETH_ECUDA;
}

__global__ void k_f64_to_f32(size_t m, const double* __restrict__ a, float* __restrict__ b) {
  ETH_GRID_DEP_WAIT();
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x) b[k] = (float)a[k];
}

}  // namespace eth

using namespace eth;

extern "C" {

int eth_sizes(int n, int* nv, int* n1, int* n0) {
  if (n < 1) return -1;
  const int a = (2 * n + 1) * (2 * n + 1), b = (n + 1) * (n + 1), c = n * n;
  if (nv) *nv = a;
  if (n1) *n1 = b;
  if (n0) *n0 = c;
  return 2 * a + b + c;
}

const char* eth_status_string(eth_status s) {
  switch (s) {
    case ETH_OK: return "ok";
    case ETH_EINVAL: return "invalid argument";
    case ETH_ENOMEM: return "out of device memory";
    case ETH_ECUDA: return "CUDA error";
    case ETH_ENOTCONV: return "not converged";
    case ETH_EBREAKDOWN: return "Krylov breakdown";
    case ETH_EINCONSISTENT: return "inconsistent right-hand side";
    case ETH_ETIMEOUT: return "device wait timed out";
    case ETH_ENAN: return "NaN or Inf in residual";
  }
  return "unknown status";
}

const char* eth_last_error(void) { return eth::g_err; }

void eth_default_opts(eth_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-6;
  o->maxit = 2000;
  o->restart = 50;
  o->c_stage = 10.0;
  o->precision = ETH_MIXED;
  o->mg_pre = 1;
  o->mg_post = 1;
  o->mg_min_n = 0;
  o->mq_mode = ETH_MQ_VCYCLE;
  o->a_exact = 0;
  o->inner_tol = 1e-12;
  o->refine_inner_tol = 1e-4;
  o->graph = 1;
  o->verbose = 0;
  o->autotune = 1;
}

eth_status eth_grid_create(int n, double x0, double x1, double y0, double y1, eth_kind kind, void* cuda_stream,
                           eth_grid** out) {
  if (!out) { set_error("eth_grid_create: out is NULL"); return ETH_EINVAL; }
  *out = nullptr;
  if (n < 2 || (n & 1) || n > 8192) { set_error("eth_grid_create: n=%d must be even, 2 <= n <= 8192", n); return ETH_EINVAL; }
  if (!(x1 > x0) || !(y1 > y0)) { set_error("eth_grid_create: empty domain"); return ETH_EINVAL; }
  if (kind != ETH_STOKES && kind != ETH_OSEEN) { set_error("eth_grid_create: bad kind"); return ETH_EINVAL; }
  int dev = 0;
  ETH_CUDA(cudaGetDevice(&dev));
  eth_grid* g = new eth_grid();
  g->dev = dev;
  g->n = n; g->x0 = x0; g->x1 = x1; g->y0 = y0; g->y1 = y1;
  g->hx = (x1 - x0) / n; g->hy = (y1 - y0) / n;
  g->kind = kind;
  g->s = (cudaStream_t)cuda_stream;
  g->nt = eth_sizes(n, &g->nv, &g->n1, &g->n0);
  const size_t nt = g->nt, nu2 = 2 * (size_t)g->nv;
  // reduction partials per slot: one per CTA of the largest launch (the 32 x 4 tile grid)
  g->part_cap = std::max(1 << 16, q2_blocks(n, 4));
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
  A((void**)&g->b, nt * 8);
  A((void**)&g->ubc, nu2 * 8);
  A((void**)&g->tmp, nt * 8);
  A((void**)&g->tmp2, nt * 8);
  A((void**)&g->sc, sizeof(Scalars));
  A((void**)&g->part, (size_t)16 * g->part_cap * 8);
  A((void**)&g->ticket, 16 * sizeof(unsigned));
  A((void**)&g->lz, 2 * (size_t)ETH_LANCZOS_CAP * 8);
  if (kind == ETH_OSEEN) { A((void**)&g->wind, nu2 * 8); A((void**)&g->windf, nu2 * 4); }
  if (e == cudaSuccess) e = cudaMallocHost((void**)&g->sch, sizeof(Scalars));
  if (e == cudaSuccess) e = cudaMemsetAsync(g->ticket, 0, 16 * sizeof(unsigned), g->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->sc, 0, sizeof(Scalars), g->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->b, 0, nt * 8, g->s);
  if (e != cudaSuccess) {
    eth_status st = cuda_status(e, "eth_grid_create");
    eth_grid_destroy(g);
    return st;
  }
  *out = g;
  return ETH_OK;
}

void eth_grid_destroy(eth_grid* g) {
  if (!g) return;
  DeviceGuard guard(g->dev);
  if (g->s) cudaStreamSynchronize(g->s); else cudaDeviceSynchronize();
  solver_free(g);
  cudaFree(g->b); cudaFree(g->ubc); cudaFree(g->tmp); cudaFree(g->tmp2);
  cudaFree(g->sc); cudaFree(g->part); cudaFree(g->ticket); cudaFree(g->lz);
  cudaFree(g->wind); cudaFree(g->windf);
  if (g->sch) cudaFreeHost(g->sch);
  delete g;
}

eth_status eth_set_coefficients(eth_grid* g, double nu, const double* wind_dev) {
  if (!g) { set_error("eth_set_coefficients: NULL handle"); return ETH_EINVAL; }
  if (!(nu > 0.0) || !std::isfinite(nu)) { set_error("eth_set_coefficients: nu=%g must be > 0", nu); return ETH_EINVAL; }
  if (g->kind == ETH_OSEEN && !wind_dev) { set_error("eth_set_coefficients: Oseen needs a wind"); return ETH_EINVAL; }
  if (g->kind == ETH_STOKES && wind_dev) { set_error("eth_set_coefficients: Stokes takes no wind"); return ETH_EINVAL; }
  ETH_ON_DEVICE(g);
  g->nu = nu;
  if (wind_dev) {
    const size_t nu2 = 2 * (size_t)g->nv;
    ETH_CUDA(cudaMemcpyAsync(g->wind, wind_dev, nu2 * 8, cudaMemcpyDeviceToDevice, g->s));
    k_f64_to_f32<<<cdiv((long)nu2, 256) > 4096 ? 4096 : cdiv((long)nu2, 256), 256, 0, g->s>>>(nu2, g->wind, g->windf);
    ETH_CUDA(cudaGetLastError());
  }
  g->has_coef = true;
  g->has_rhs = false;
  return solver_coefficients_changed(g);
}

eth_status eth_set_rhs(eth_grid* g, const double* f, const double* ubc) {
  if (!g || !f || !ubc) { set_error("eth_set_rhs: NULL argument"); return ETH_EINVAL; }
  if (!g->has_coef) { set_error("eth_set_rhs: call eth_set_coefficients first"); return ETH_EINVAL; }
  ETH_ON_DEVICE(g);
  ETH_TRY(assemble_rhs(g, f, ubc));
  g->has_rhs = true;
  return ETH_OK;
}

eth_status eth_get_rhs(eth_grid* g, double* b_dev) {
  if (!g || !b_dev) { set_error("eth_get_rhs: NULL argument"); return ETH_EINVAL; }
  if (!g->has_rhs) { set_error("eth_get_rhs: no right-hand side set"); return ETH_EINVAL; }
  ETH_ON_DEVICE(g);
  ETH_CUDA(cudaMemcpyAsync(b_dev, g->b, (size_t)g->nt * 8, cudaMemcpyDeviceToDevice, g->s));
  return ETH_OK;
}

eth_status eth_apply(eth_grid* g, eth_op op, int fp32, const double* x, double* y) {
  if (!g || !x || !y) { set_error("eth_apply: NULL argument"); return ETH_EINVAL; }
  if (!g->has_coef && op != ETH_OP_MV && op != ETH_OP_MQ && op != ETH_OP_B && op != ETH_OP_BT) {
    set_error("eth_apply: call eth_set_coefficients first");
    return ETH_EINVAL;
  }
  if ((int)op < 0 || (int)op > (int)ETH_OP_K1T) { set_error("eth_apply: bad operator %d", (int)op); return ETH_EINVAL; }
  ETH_ON_DEVICE(g);
  return op_apply(g, op, fp32 != 0, x, y);
}

}  // extern "C"
