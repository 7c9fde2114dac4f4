// Persistent, software-pipelined form of the fused K apply (FP32 element
// arithmetic, FP64 input and output, tiles of 32 x 8 elements).
//
// The one-tile-per-CTA kernel of q2tile.cuh loads a tile, waits, computes and
// stores; the loads of a CTA are only overlapped by the other CTAs on the SM.
// Here a CTA walks over tiles t, t + G, t + 2G, ... (G = grid size) and issues
// the asynchronous global->shared copies (cp.async, zero-filled where the
// velocity is a Dirichlet node or outside the domain) of its next tile before
// it converts, computes and stores the current one, so the HBM reads of the
// next tile are in flight during the arithmetic of this one.  The FP64 input
// stays in shared memory, which also gives the exact FP64 partner of the fused
// dot <Kx, x> without a second read of x.  Arithmetic and summation order per
// node are those of k_q2 (same q2_elem, same gather), so the outputs are
// bitwise identical to it.
#pragma once
#include <algorithm>
#include "q2tile.cuh"

namespace eth {

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int NPEND>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(NPEND) : "memory"); }

// default tile shape (TEY rows): staged node counts
constexpr int QP_NQ = SQY * SQX;                       // Q2 nodes of a tile
constexpr int QP_NP1 = SPY * SPX;                      // Q1 nodes
constexpr int QP_NP0 = TEY * TEX;                      // elements (P0)
constexpr int QP_NLD = (QP_NQ + Q2T - 1) / Q2T;        // velocity slots per thread
constexpr int QP_NLP = (QP_NP1 + Q2T - 1) / Q2T;       // Q1 slots per thread
constexpr int QP_RAWD = 2 * QP_NQ + QP_NP1 + QP_NP0;   // FP64 values per staged tile
static_assert(QP_NLD <= 8 && QP_NLP <= 4 && QP_NP0 == Q2T, "slot masks");
static_assert(2 * QP_NQ + QP_NP1 + QP_NP0 <= NEO * Q2T, "FP32 staging aliases the element outputs");

constexpr size_t q2p_buf_bytes(bool conv) {
  return ((size_t)QP_RAWD * 8 + (conv ? (size_t)2 * QP_NQ * 4 : 0) + 15) / 16 * 16;
}
constexpr size_t q2p_smem_bytes(bool conv) { return 2 * q2p_buf_bytes(conv) + (size_t)NEO * Q2T * 4; }

template <int F>
__global__ void __launch_bounds__(Q2T) k_q2p(Q2Params<double, double, float> P, int ntx, int ntiles) {
  ETH_GRID_DEP_WAIT();
  using CT = float;
  constexpr bool CONV = F & QF_CONV, XIN = F & QF_XIN, PIN = F & QF_PIN, HP0 = F & QF_P0, UOUT = F & QF_UOUT,
                 POUT = F & QF_POUT, DOT = F & QF_DOT;
  static_assert(!(F & (QF_NOBC | QF_SRC_JB | QF_SRC_XPC | QF_MASS | QF_SD)), "K apply flags only");
  static_assert(XIN, "velocity input required");
  if (P.done != nullptr && *P.done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr size_t BUFB = q2p_buf_bytes(CONV);
  float* eo = reinterpret_cast<float*>(smem_raw + 2 * BUFB);   // [NEO][Q2T]
  float* sx = eo;                                              // [2][QP_NQ]  (aliases eo)
  float* sp1 = sx + 2 * QP_NQ;                                 // [QP_NP1]
  float* sp0 = sp1 + QP_NP1;                                   // [QP_NP0]

  const int n = P.n, N = 2 * n + 1;
  const size_t nv = (size_t)N * N;
  const int n1 = (n + 1) * (n + 1);
  const int tid = threadIdx.x;

  // copies of tile t into buffer b; returns this thread's validity bits
  // (bits 0..7 velocity slots, 8..11 Q1 slots, 12 the P0 slot)
  auto issue = [&](int t, int b) -> unsigned {
    const int by = t / ntx, bx = t - by * ntx;
    const int ex0 = bx * OEX, ey0 = by * OEY;
    const int gi0 = 2 * (ex0 - 1), gj0 = 2 * (ey0 - 1);
    double* rv = reinterpret_cast<double*>(smem_raw + b * BUFB);
    float* rw = reinterpret_cast<float*>(smem_raw + b * BUFB + (size_t)QP_RAWD * 8);
    unsigned m = 0;
#pragma unroll
    for (int r = 0; r < QP_NLD; ++r) {
      const int k = tid + r * Q2T;
      if (k < QP_NQ) {
        const int lj = k / SQX, li = k - lj * SQX;
        const int i = gi0 + li, j = gj0 + lj;
        const bool inside = i >= 0 && i < N && j >= 0 && j < N;
        const bool ok = inside && !(i == 0 || j == 0 || i == N - 1 || j == N - 1);
        const size_t g = inside ? (size_t)j * N + i : 0;
        cp_async8(&rv[k], P.x + g, ok);
        cp_async8(&rv[QP_NQ + k], P.x + g + nv, ok);
        if (CONV) {
          cp_async4(&rw[k], P.w + g, inside);
          cp_async4(&rw[QP_NQ + k], P.w + g + nv, inside);
        }
        if (ok) m |= 1u << r;
      }
    }
    if (PIN) {
#pragma unroll
      for (int r = 0; r < QP_NLP; ++r) {
        const int k = tid + r * Q2T;
        if (k < QP_NP1) {
          const int lj = k / SPX, li = k - lj * SPX;
          const int I = ex0 - 1 + li, J = ey0 - 1 + lj;
          const bool ok = I >= 0 && I <= n && J >= 0 && J <= n;
          cp_async8(&rv[2 * QP_NQ + k], P.p + (ok ? (size_t)J * (n + 1) + I : 0), ok);
          if (ok) m |= 1u << (8 + r);
        }
      }
      if (HP0) {
        const int ly = tid / TEX, lx = tid - ly * TEX;
        const int ex = ex0 - 1 + lx, ey = ey0 - 1 + ly;
        const bool ok = ex >= 0 && ex < n && ey >= 0 && ey < n;
        cp_async8(&rv[2 * QP_NQ + QP_NP1 + tid], P.p + n1 + (ok ? (size_t)ey * n + ex : 0), ok);
        if (ok) m |= 1u << 12;
      }
    }
    return m;
  };

  double dacc = 0.0;
  int t = blockIdx.x;
  unsigned mcur = 0, mnext = 0;
  if (t < ntiles) mcur = issue(t, 0);
  cp_async_commit();
  for (int it = 0; t < ntiles; ++it, t += gridDim.x) {
    const int b = it & 1;
    const int tn = t + gridDim.x;
    cp_async_wait<0>();   // this thread's copies of tile t have landed
    __syncthreads();      // ... and every thread's; the previous tile (buffer b^1, eo) is consumed
    if (tn < ntiles) mnext = issue(tn, b ^ 1);   // in flight during this tile's work
    cp_async_commit();
    const double* rv = reinterpret_cast<const double*>(smem_raw + b * BUFB);
    const float* rw = reinterpret_cast<const float*>(smem_raw + b * BUFB + (size_t)QP_RAWD * 8);
    // FP64 -> FP32 of this thread's own slots (warp-collective conversion: all lanes call it)
#pragma unroll
    for (int r = 0; r < QP_NLD; ++r) {
      const int k = tid + r * Q2T;
      const int kk = k < QP_NQ ? k : 0;
      const bool ok = (mcur >> r) & 1u;
      const float c0 = cvt_stage<float, double>(rv[kk], ok);
      const float c1 = cvt_stage<float, double>(rv[QP_NQ + kk], ok);
      if (k < QP_NQ) { sx[k] = c0; sx[QP_NQ + k] = c1; }
    }
    if (PIN) {
#pragma unroll
      for (int r = 0; r < QP_NLP; ++r) {
        const int k = tid + r * Q2T;
        const int kk = k < QP_NP1 ? k : 0;
        const float c = cvt_stage<float, double>(rv[2 * QP_NQ + kk], (mcur >> (8 + r)) & 1u);
        if (k < QP_NP1) sp1[k] = c;
      }
      if (HP0) sp0[tid] = cvt_stage<float, double>(rv[2 * QP_NQ + QP_NP1 + tid], (mcur >> 12) & 1u);
    }
    __syncthreads();

    const int by = t / ntx, bx = t - by * ntx;
    const int ex0 = bx * OEX, ey0 = by * OEY;
    const int gi0 = 2 * (ex0 - 1), gj0 = 2 * (ey0 - 1);
    const int lx = tid % TEX, ly = tid / TEX;
    const int ex = ex0 - 1 + lx, ey = ey0 - 1 + ly;
    const bool in = ex >= 0 && ex < n && ey >= 0 && ey < n;
    // ---- phase 1: element inputs to registers, then (after a barrier, sx aliases eo) the element
    CT U[2][9], Wn[2][9], P1[4], P0v = 0;
    if (in) {
#pragma unroll
      for (int bb = 0; bb < 3; ++bb)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const int s = (2 * ly + bb) * SQX + 2 * lx + a;
          U[0][bb * 3 + a] = sx[s];
          U[1][bb * 3 + a] = sx[QP_NQ + s];
          if (CONV) { Wn[0][bb * 3 + a] = rw[s]; Wn[1][bb * 3 + a] = rw[QP_NQ + s]; }
        }
      if (PIN) {
#pragma unroll
        for (int d = 0; d < 2; ++d)
#pragma unroll
          for (int c = 0; c < 2; ++c) P1[d * 2 + c] = sp1[(ly + d) * SPX + lx + c];
        if (HP0) P0v = sp0[ly * TEX + lx];
      }
    }
    __syncthreads();
    {
      CT Y[2][9], YP1[4], YP0 = 0;
      if (in) {
        const CT ihx = CT(1) / P.hx, ihy = CT(1) / P.hy, area = P.hx * P.hy;
        q2_elem<CT, F>(U, Wn, P1, P0v, P.nu, ihx, ihy, area, P.sd, Y, YP1, YP0);
      } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) { Y[0][k] = 0; Y[1][k] = 0; }
#pragma unroll
        for (int k = 0; k < 4; ++k) YP1[k] = 0;
      }
      if (UOUT) {
#pragma unroll
        for (int k = 0; k < 9; ++k) { eo[k * Q2T + tid] = Y[0][k]; eo[(9 + k) * Q2T + tid] = Y[1][k]; }
      }
      if (POUT) {
#pragma unroll
        for (int k = 0; k < 4; ++k) eo[(18 + k) * Q2T + tid] = YP1[k];
        eo[22 * Q2T + tid] = YP0;
      }
    }
    __syncthreads();
    // ---- phase 2: owned nodes gather their element sums (order as in k_q2) and store
    const bool own = lx >= 1 && ly >= 1 && ex < n && ey < n;
    const int tL = tid - 1, tB = tid - TEX, tLB = tid - TEX - 1;
    auto E = [&](int a, int bb, int tt, int c) -> CT { return eo[(c * 9 + bb * 3 + a) * Q2T + tt]; };
    auto emit = [&](int i, int j, CT s0, CT s1) {
      const size_t g = (size_t)j * N + i;
      const bool bnd = i == 0 || j == 0 || i == N - 1 || j == N - 1;
      double o0, o1, d0, d1;
      if (bnd) {
        o0 = P.x[g]; o1 = P.x[g + nv];
        d0 = o0; d1 = o1;
      } else {
        o0 = cvt_out<double, CT>(s0); o1 = cvt_out<double, CT>(s1);
        const int sI = (j - gj0) * SQX + (i - gi0);
        d0 = rv[sI]; d1 = rv[QP_NQ + sI];
      }
      P.y[g] = o0;
      P.y[g + nv] = o1;
      if (DOT) dacc += o0 * d0 + o1 * d1;
    };
    if (UOUT && own) {
      const int i0 = 2 * ex, j0 = 2 * ey;
      const bool lastx = ex == n - 1, lasty = ey == n - 1;
      emit(i0, j0, E(2, 2, tLB, 0) + E(0, 2, tB, 0) + E(2, 0, tL, 0) + E(0, 0, tid, 0),
                   E(2, 2, tLB, 1) + E(0, 2, tB, 1) + E(2, 0, tL, 1) + E(0, 0, tid, 1));
      emit(i0 + 1, j0, E(1, 2, tB, 0) + E(1, 0, tid, 0), E(1, 2, tB, 1) + E(1, 0, tid, 1));
      emit(i0, j0 + 1, E(2, 1, tL, 0) + E(0, 1, tid, 0), E(2, 1, tL, 1) + E(0, 1, tid, 1));
      emit(i0 + 1, j0 + 1, E(1, 1, tid, 0), E(1, 1, tid, 1));
      if (lastx) {
        emit(i0 + 2, j0, E(2, 2, tB, 0) + E(2, 0, tid, 0), E(2, 2, tB, 1) + E(2, 0, tid, 1));
        emit(i0 + 2, j0 + 1, E(2, 1, tid, 0), E(2, 1, tid, 1));
      }
      if (lasty) {
        emit(i0, j0 + 2, E(2, 2, tL, 0) + E(0, 2, tid, 0), E(2, 2, tL, 1) + E(0, 2, tid, 1));
        emit(i0 + 1, j0 + 2, E(1, 2, tid, 0), E(1, 2, tid, 1));
      }
      if (lastx && lasty) emit(i0 + 2, j0 + 2, E(2, 2, tid, 0), E(2, 2, tid, 1));
    }
    if (POUT && own) {
      auto Q = [&](int cc, int dd, int tt) -> CT { return eo[(18 + dd * 2 + cc) * Q2T + tt]; };
      auto pemit = [&](int I, int J, CT v) {
        const size_t gp = (size_t)J * (n + 1) + I;
        const double so = cvt_out<double, CT>(v);
        P.yp[gp] = so;
        if (DOT) dacc += so * rv[2 * QP_NQ + (J - (ey0 - 1)) * SPX + (I - (ex0 - 1))];
      };
      pemit(ex, ey, Q(1, 1, tLB) + Q(0, 1, tB) + Q(1, 0, tL) + Q(0, 0, tid));
      if (ex == n - 1) pemit(ex + 1, ey, Q(1, 1, tB) + Q(1, 0, tid));
      if (ey == n - 1) pemit(ex, ey + 1, Q(1, 1, tL) + Q(0, 1, tid));
      if (ex == n - 1 && ey == n - 1) pemit(ex + 1, ey + 1, Q(1, 1, tid));
      if (HP0) {
        const size_t ge = (size_t)n1 + (size_t)ey * n + ex;
        const double so = cvt_out<double, CT>(eo[22 * Q2T + tid]);
        P.yp[ge] = so;
        if (DOT) dacc += so * rv[2 * QP_NQ + QP_NP1 + tid];
      }
    }
    mcur = mnext;
  }
  cp_async_wait<0>();
  if (DOT) {
    double v[1] = {dacc};
    if (slot_arrive<1>(P.slot, P.slot_off + blockIdx.x, v)) finish_slot(P.slot, v[0]);
  }
}

// CTAs of the persistent launch on the current device: resident CTAs per SM x
// SMs, at most one per tile (the occupancy figure is cached per device; the
// shared-memory attribute is set on each device before its first launch).
template <int F>
static int q2p_blocks(int n) {   // per translation unit, like launch_q2
  static SmemAttr attr;
  static std::atomic<int> caps[ETH_MAX_DEVICES];
  int dev = 0;
  cudaGetDevice(&dev);
  const bool tracked = dev >= 0 && dev < ETH_MAX_DEVICES;
  int cap = tracked ? caps[dev].load(std::memory_order_acquire) : 0;
  if (cap == 0) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    smem_attr(k_q2p<F>, q2p_smem_bytes(F & QF_CONV), attr);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_q2p<F>, Q2T, q2p_smem_bytes(F & QF_CONV));
    cap = std::max(1, sms) * std::max(1, per);
    if (tracked) caps[dev].store(cap, std::memory_order_release);
  }
  const int ntiles = (int)(cdiv(n, OEX) * cdiv(n, OEY));
  return std::min(ntiles, cap);
}

template <int F>
static cudaError_t launch_q2p(const Q2Params<double, double, float>& P, cudaStream_t s) {
  const int grid = q2p_blocks<F>(P.n);   // also sets the shared-memory attribute
  const int ntx = (int)cdiv(P.n, OEX), ntiles = ntx * (int)cdiv(P.n, OEY);
  k_q2p<F><<<grid, Q2T, q2p_smem_bytes(F & QF_CONV), s>>>(P, ntx, ntiles);
  return cudaGetLastError();
}

}  // namespace eth
