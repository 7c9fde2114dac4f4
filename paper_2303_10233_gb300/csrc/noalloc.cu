// Allocation-free variant of the fused Stokes K apply with its FP64 dot product.
//
// Some callers cannot allocate device memory: code that runs inside another
// framework's memory pool or under a strict memory budget, a host that only
// hands out pre-registered buffers, or a process that must not call cudaMalloc
// after start-up.  They cannot create an eth_grid (whose workspace is
// allocated), so this entry point takes the grid description by value and
// keeps its reduction scratch (per-block partial sums and the arrival ticket)
// in a file-scope __device__ array of fixed size instead.
//
// The array belongs to the library image: every GPU that loads the library
// holds it until the process exits.  Every call shares it and it keeps the
// previous call's contents, so each call clears the ticket first; two calls
// whose kernels overlap on the GPU race on it.
#include <mutex>
#include "ops.cuh"

namespace eth {

// at most ETH_NOALLOC_MAX_BLOCKS tile CTAs per call: ceil(n/31) * ceil(n/7) tiles of
// 32 x 8 elements, e.g. 67 * 293 = 19,631 at n = 2048; the largest even n that fits is 2666
// (86 * 381 = 32,766)
constexpr int ETH_NOALLOC_MAX_BLOCKS = 32768;
struct NoAllocScratch {
  double partials[ETH_NOALLOC_MAX_BLOCKS];
  unsigned ticket;
  unsigned pad[63];
};
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device address of the scratch array, looked up once per device (with that
// device current) by cudaGetSymbolAddress; the host-side symbol itself is not a
// device address.
static std::mutex g_noalloc_mu;
static NoAllocScratch* g_noalloc_ptr[64] = {};

static eth_status noalloc_scratch(NoAllocScratch** out) {
  int dev = 0;
  ETH_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) { set_error("eth_apply_k_dot_static: device index %d out of range", dev); return ETH_EINVAL; }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_ptr[dev] = (NoAllocScratch*)p;
  }
  *out = g_noalloc_ptr[dev];
  return ETH_OK;
}

template <class CT>
static eth_status noalloc_run(int n, double hx, double hy, double nu, const double* x, double* y, double* dot,
                              NoAllocScratch* sc, cudaStream_t s) {
  constexpr int F = QF_DIFF | QF_XIN | QF_PIN | QF_P0 | QF_UOUT | QF_POUT | QF_DOT;
  const int nv = (2 * n + 1) * (2 * n + 1);
  Q2Params<double, double, CT> P{};
  P.n = n; P.hx = (CT)hx; P.hy = (CT)hy; P.nu = (CT)nu;
  P.x = x; P.p = x + 2 * (size_t)nv; P.y = y; P.yp = y + 2 * (size_t)nv;
  P.dv = x; P.dvp = x + 2 * (size_t)nv;
  P.slot.part = sc->partials;
  P.slot.ticket = &sc->ticket;
  P.slot.out = dot;
  P.slot.total = q2_blocks(n);
  P.slot.op = FIN_STORE;
  P.slot.sc = nullptr;
  ETH_CUDA(cudaMemsetAsync(&sc->ticket, 0, sizeof(unsigned), s));
  ETH_CUDA((launch_q2<double, double, CT, F, EPI_APPLY>(P, s)));
  return ETH_OK;
}

}  // namespace eth

using namespace eth;

extern "C" eth_status eth_apply_k_dot_static(int n, double x0, double x1, double y0, double y1, double nu, int fp32,
                                             const double* x_dev, double* y_dev, double* dot_dev, void* cuda_stream) {
  if (!x_dev || !y_dev || !dot_dev) { set_error("eth_apply_k_dot_static: NULL argument"); return ETH_EINVAL; }
  if (n < 2 || (n & 1)) { set_error("eth_apply_k_dot_static: n=%d must be even and >= 2", n); return ETH_EINVAL; }
  if (!(x1 > x0) || !(y1 > y0) || !(nu > 0.0)) { set_error("eth_apply_k_dot_static: bad domain or viscosity"); return ETH_EINVAL; }
  if (q2_blocks(n) > ETH_NOALLOC_MAX_BLOCKS) {
    set_error("eth_apply_k_dot_static: n=%d needs %d element tiles, the static scratch holds %d (even n <= 2666)", n,
              q2_blocks(n), ETH_NOALLOC_MAX_BLOCKS);
    return ETH_EINVAL;
  }
  NoAllocScratch* sc = nullptr;
  ETH_TRY(noalloc_scratch(&sc));
  const cudaStream_t s = (cudaStream_t)cuda_stream;
  const double hx = (x1 - x0) / n, hy = (y1 - y0) / n;
  return fp32 ? noalloc_run<float>(n, hx, hy, nu, x_dev, y_dev, dot_dev, sc, s)
              : noalloc_run<double>(n, hx, hy, nu, x_dev, y_dev, dot_dev, sc, s);
}
