// Device kernels of the nsamg solve phase (sm_103a).
//
// Design notes (B300): the path is HBM-bound sparse/vector work, and FP64 arithmetic on this
// part issues at ~1.6 FMA/clk/SM (1/73 of FP32), so the FP64 kernels keep exactly one FP64
// operation per matrix entry (pre-scaled matrices remove per-entry D^-1 multiplies) and put
// all whole-vector reductions into a single deterministic pass with a last-block finalise.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace nsamg {

constexpr int kMaxM = 64;  // largest restart length (matches NSAMG_MAX_RESTART)

// A vector argument: either a plain pointer or column `*sel` of a column-major block with
// leading dimension ld (used to aim V-cycle kernels at V[:, i] / Z[:, i] inside a CUDA graph).
template <typename T>
struct VRef {
  T* p = nullptr;
  const int* sel = nullptr;
  int64_t ld = 0;
  __device__ __forceinline__ T* get() const { return sel ? p + (int64_t)(*sel) * ld : p; }
};

template <typename T>
__host__ __device__ inline VRef<T> vref(T* p) { VRef<T> r; r.p = p; return r; }

// ------------------------------------------------------------------------------------------
// Generic fused row kernel:
//   acc_i = sum_j M_ij src_j                              (skipped when M is absent)
//   c_i   = bscale_i * base_i  (bscale optional; base absent = 0)
//   t_i   = neg ? c_i - acc_i : c_i + acc_i
//   out2_i = t_i (optional), t_i *= scale_i (optional), t_i += add_i (optional), out_i = t_i
// Every SpMV, residual, smoother pass, restriction and prolongation is one launch of this.
// TM: matrix value type, TX: source vector type, TY: type of all other vectors / accumulation.
// G threads cooperate on one row (G = 1, 2, 4, 8, 16, 32).
// ------------------------------------------------------------------------------------------
template <typename TM, typename TX, typename TY>
struct RowOp {
  int n = 0;
  const int* rp = nullptr;
  const int* ci = nullptr;
  const TM* v = nullptr;
  VRef<const TX> src;
  VRef<const TY> base;
  const TY* bscale = nullptr;
  const TY* scale = nullptr;
  VRef<const TY> add;
  VRef<TY> out;
  VRef<TY> out2;
  int neg = 0;
  const int* skip = nullptr;  // if set and *skip != 0 the launch does nothing (stopped solve)
};

template <int G, typename TM, typename TX, typename TY>
__global__ void __launch_bounds__(256) k_row(RowOp<TM, TX, TY> op) {
  if (op.skip && *op.skip) return;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int row = (int)(gid / G);
  if (row >= op.n) return;  // uniform over the G lanes of a row
  TY acc = TY(0);
  if (op.v) {
    const TX* __restrict__ src = op.src.get();
    const int lane = (int)(gid & (G - 1));
    const int b = __ldg(op.rp + row), e = __ldg(op.rp + row + 1);
#pragma unroll 4
    for (int p = b + lane; p < e; p += G) {
      const int c = __ldg(op.ci + p);
      acc = fma((TY)__ldg(op.v + p), (TY)__ldg(src + c), acc);
    }
    if constexpr (G > 1) {
      const unsigned seg = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(seg, acc, o, G);
    }
    if (lane != 0) return;
  }
  const TY* base = op.base.get();
  TY c = TY(0);
  if (base) c = op.bscale ? op.bscale[row] * base[row] : base[row];
  TY t = op.neg ? c - acc : c + acc;
  if (op.out2.p) op.out2.get()[row] = t;
  if (op.scale) t *= op.scale[row];
  if (op.add.p) t += op.add.get()[row];
  op.out.get()[row] = t;
}

// ------------------------------------------------------------------------------------------
// Small helpers
// ------------------------------------------------------------------------------------------
template <typename TA, typename TB>
__global__ void k_cast(int64_t n, VRef<const TA> a, VRef<TB> b, const int* skip) {
  if (skip && *skip) return;
  const TA* pa = a.get();
  TB* pb = b.get();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    pb[i] = (TB)pa[i];
}

template <typename T>
__global__ void k_fill(int64_t n, T* a, T v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) a[i] = v;
}

// Dense coarse solve z = C b with C the row-major inverse of the coarsest operator; one warp
// per row, fixed-order reduction.
template <typename TC, typename T>
__global__ void k_dense_gemv(int n, const TC* __restrict__ C, VRef<const T> bref, VRef<T> zref, const int* skip) {
  if (skip && *skip) return;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const T* b = bref.get();
  T acc = T(0);
  for (int j = lane; j < n; j += 32) acc = fma((T)C[(int64_t)warp * n + j], b[j], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) zref.get()[warp] = acc;
}

// ------------------------------------------------------------------------------------------
// GMRES device state (one per handle, in device memory).
// ------------------------------------------------------------------------------------------
struct GState {
  // per-solve inputs (written by the host before each solve)
  const double* b;
  double* x;
  double rtol;
  int maxit;
  int m;
  int t_exact;
  int pad0;
  // loop control
  int i;          // current Arnoldi step within the cycle (column index of vt)
  int k;          // columns completed in this cycle
  int stop;       // inner loop must stop (cycle finished)
  int done;       // solve finished
  int iters;      // total Arnoldi columns
  int cycles;     // restart cycles started
  int status;     // 0 ok, 1 not converged, <0 error
  int converged;
  double bnorm;
  double relres_true;
  double relres_implicit;
  // Arnoldi / least-squares data (row-major with stride kMaxM + 1)
  double beta[kMaxM + 1];
  double invbeta[kMaxM + 1];
  double h[kMaxM + 1];      // projection coefficients of the current step
  double coef[kMaxM];       // x-update coefficients y_j / beta_j
  double cs[kMaxM], sn[kMaxM], g[kMaxM + 1];
  double R[(kMaxM + 1) * kMaxM];  // Hessenberg columns, rotated in place (column-major, ld kMaxM+1)
  double L[(kMaxM + 1) * (kMaxM + 1)];  // strictly lower part of V^T V (row-major)
};

}  // namespace nsamg
