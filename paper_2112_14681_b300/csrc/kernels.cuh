// Device kernels of the nsamg solve phase (sm_103a).
//
// Design notes (B300): the path is HBM-bound sparse/vector work, and FP64 arithmetic on this
// part issues at ~1.6 FMA/clk/SM (1/73 of FP32), so the FP64 kernels keep exactly one FP64
// operation per matrix entry (pre-scaled matrices remove per-entry D^-1 multiplies) and put
// all whole-vector reductions into a single deterministic pass with a last-block finalise.
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>
#include <cooperative_groups.h>

namespace nsamg {

constexpr int kMaxM = 64;  // largest restart length (matches NSAMG_MAX_RESTART)

// A vector argument: either a plain pointer or column `*sel` of a column-major block with
// leading dimension ld (used to aim V-cycle kernels at V[:, i] / Z[:, i] inside a CUDA graph).
// Programmatic dependent launch: wait until the predecessor grid has completed and its writes
// are visible, then allow the successor grid to be scheduled.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename T>
struct VRef {
  T* p = nullptr;
  const int* sel = nullptr;
  int64_t ld = 0;
  __device__ __forceinline__ T* get() const { return sel ? p + (int64_t)(*sel) * ld : p; }
};

template <typename T>
__host__ __device__ inline VRef<T> vref(T* p) { VRef<T> r; r.p = p; return r; }

// IEEE 754 binary32 <-> binary64 conversions with integer operations. On this part the hardware
// conversion instructions issue on the FP64 pipe at a fraction of the FMA rate, which made the
// precision casts of the FP32 V-cycle conversion bound; the integer forms run on the integer
// pipe. Widening is exact for every input; narrowing rounds to nearest, ties to even (IEEE 754
// default), and inputs outside the binary32 normal range (results that underflow or overflow,
// infinities, NaN) take the hardware conversion.
__device__ __forceinline__ double widen_f32(float f) {
  // branch-free (it runs per gathered entry inside the mixed-precision SpMV): every class of
  // input is formed with selects; a subnormal m * 2^-149 is renormalised from its leading bit p
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  const uint32_t m = u & 0x7fffffu;
  const int p = 31 - __clz(m | 1u);  // leading bit of a subnormal's field (m > 0)
  const bool sub = (e == 0u) & (m != 0u);
  const uint64_t ed = sub ? (uint64_t)(p + 874) : (e == 0u ? 0ull : (e == 0xffu ? 2047ull : (uint64_t)(e + 896u)));
  const uint64_t md = sub ? (((uint64_t)m << (52 - p)) & 0xfffffffffffffull) : ((uint64_t)m << 29);
  return __longlong_as_double((long long)(((uint64_t)(u >> 31) << 63) | (ed << 52) | md));
}

__device__ __forceinline__ float narrow_f64(double d) {
  const uint64_t u = (uint64_t)__double_as_longlong(d);
  const int e = (int)((u >> 52) & 0x7ff);
  if (e < 897 || e > 1150) return __double2float_rn(d);  // below the binary32 normal range, or beyond it
  const uint64_t m = u & 0xfffffffffffffull;              // 52 mantissa bits
  const uint64_t rem = m & 0x1fffffffull;                 // the 29 bits dropped
  uint32_t bits = ((uint32_t)(e - 896) << 23) | (uint32_t)(m >> 29);
  if (rem > 0x10000000ull || (rem == 0x10000000ull && (bits & 1u))) bits += 1u;  // may carry into the exponent (to infinity at the top)
  return __uint_as_float(((uint32_t)(u >> 63) << 31) | bits);
}

template <typename TB, typename TA>
__device__ __forceinline__ TB convert(TA a) {
  if constexpr (std::is_same<TA, TB>::value) return a;
  else if constexpr (std::is_same<TA, double>::value && std::is_same<TB, float>::value) return narrow_f64(a);
  else if constexpr (std::is_same<TA, float>::value && std::is_same<TB, double>::value) return widen_f32(a);
  else return (TB)a;
}

// ------------------------------------------------------------------------------------------
// Generic fused row kernel:
//   acc_i = sum_j M_ij src_j                              (skipped when M is absent)
//   c_i   = bscale_i * base_i  (bscale optional; base absent = 0)
//   t_i   = neg ? c_i - acc_i : c_i + acc_i
//   t_i *= scale_i (optional), t_i += add_i (optional), out_i = t_i
// Every SpMV, residual, smoother pass, restriction and prolongation is one launch of this.
// TM: matrix value type, TX: source vector type, TY: type of all other vectors / accumulation.
// The matrix is CSR (G threads per row, G = 1..32) or SELL-32-sigma (one thread per row, rows
// sorted by length inside windows, 32 rows per chunk stored column-major so that every load of
// a warp is one contiguous segment). The epilogue form is a compile-time code where it is one of
// the forms the engine uses, so each row costs exactly the FP64 operations it needs.
// ------------------------------------------------------------------------------------------
enum : int { E_NEG = 1, E_BASE = 2, E_BSCALE = 4, E_SCALE = 8, E_ADD = 16, E_RUNTIME = -1 };

template <typename TM>
struct SellView {
  int nchunks = 0;
  // Sorted layout: position -> row (-1 for padding lanes). Null for the plain layout of
  // near-uniform matrices (rows in natural order, chunk c holds rows 32c..32c+31). Either way
  // every row is padded to its chunk's width with zero values.
  const int* perm = nullptr;
  const int64_t* cptr = nullptr;  // chunk offsets, nchunks + 1
  const int* col = nullptr;
  const TM* val = nullptr;
  int width = 0;  // plain layout with every chunk padded to this width: chunk c starts at 32 width c
};

template <typename TM, typename TX, typename TY>
struct RowOp {
  int n = 0;
  const int* rp = nullptr;
  const int* ci = nullptr;
  const TM* v = nullptr;
  SellView<TM> sell;              // used instead of rp/ci/v when sell.nchunks > 0
  int sell_k = 1;                 // SELL chunks per warp (host-side launch choice)
  int sell_u = 1;                 // SELL entries staged per chunk and round (host-side launch choice)
  VRef<const TX> src;
  VRef<const TY> base;
  const TY* bscale = nullptr;
  const TY* scale = nullptr;
  VRef<const TY> add;
  VRef<TY> out;
  int neg = 0;
  const int* skip = nullptr;  // if set and *skip != 0 the launch does nothing (stopped solve)
  int src_n = 0;              // length of the source vector (columns of the matrix)
  int mat_stream = 0;         // large matrix: entries loaded evict-first in L2 (ld_stream)
};

// Matrix entries of a large FP64 matrix in a row pass: each stored entry is read once per pass,
// and a matrix streamed with the default L2 priority pushes out the vector that the pass gathers
// from (each entry of it is gathered by several rows) and the vectors that the next pass reads
// again. Such matrices are loaded evict-first in L2. (Bypassing L1 as well, or giving the FP32
// matrices of the mixed-precision V-cycle the same path, measured slower.)
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ int ld_stream(const int* p, uint64_t pol) {
  int v;
  asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double ld_stream(const double* p, uint64_t pol) {
  double v;
  asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float ld_stream(const float* p, uint64_t pol) {
  float v;
  asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}

template <typename TM, typename TX, typename TY>
__host__ __device__ inline int epi_code(const RowOp<TM, TX, TY>& op) {
  return (op.neg ? E_NEG : 0) | (op.base.p ? E_BASE : 0) | (op.bscale ? E_BSCALE : 0) | (op.scale ? E_SCALE : 0) |
         (op.add.p ? E_ADD : 0);
}

template <int EPI, typename TM, typename TX, typename TY>
__device__ __forceinline__ void row_epilogue(const RowOp<TM, TX, TY>& op, int row, TY acc) {
  constexpr bool rt = EPI < 0;
  const bool neg = rt ? op.neg != 0 : (EPI & E_NEG) != 0;
  const bool hb = rt ? op.base.p != nullptr : (EPI & E_BASE) != 0;
  const bool hbs = rt ? op.bscale != nullptr : (EPI & E_BSCALE) != 0;
  const bool hs = rt ? op.scale != nullptr : (EPI & E_SCALE) != 0;
  const bool ha = rt ? op.add.p != nullptr : (EPI & E_ADD) != 0;
  TY t;
  if (hb) {
    TY c = op.base.get()[row];
    if (hbs) c *= op.bscale[row];
    t = neg ? c - acc : c + acc;
  } else {
    t = neg ? -acc : acc;
  }
  if (hs) t *= op.scale[row];
  if (ha) t += op.add.get()[row];
  op.out.get()[row] = t;
}

template <bool ST, typename T>
__device__ __forceinline__ T ld_entry(const T* p, uint64_t pol) {
  if constexpr (ST) return ld_stream(p, pol);
  else return __ldg(p);
}

// Entries b + lane, b + lane + G, ... of one CSR row, UR per round: the UR column and value loads
// are issued before the gathers and the gathers before the FMAs, which keep the order of p (so
// the lane's sum is the one of the plain loop). csr_round_loads issues one round's loads; the
// caller issues the first round before it waits for the previous kernel (the matrix does not
// depend on it, only the gathers do).
template <bool ST, int G, int UR, typename TM>
__device__ __forceinline__ void csr_round_loads(const int* __restrict__ ci, const TM* __restrict__ v, int p0, int e,
                                                int (&cj)[UR], TM (&vj)[UR], uint64_t pol) {
#pragma unroll
  for (int u = 0; u < UR; ++u) {
    const int p = p0 + u * G;
    cj[u] = p < e ? ld_entry<ST>(ci + p, pol) : 0;
    vj[u] = p < e ? ld_entry<ST>(v + p, pol) : TM(0);
  }
}

template <bool ST, int G, int UR, typename TM, typename TX, typename TY>
__device__ __forceinline__ TY csr_accumulate(const int* __restrict__ ci, const TM* __restrict__ v, const TX* __restrict__ src,
                                             int b, int e, int lane, TY acc, uint64_t pol, int (&cj)[UR], TM (&vj)[UR]) {
  for (int p0 = b + lane; p0 < e; p0 += UR * G) {
    if (p0 != b + lane) csr_round_loads<ST, G, UR>(ci, v, p0, e, cj, vj, pol);  // round 0: loaded by the caller
    TX xj[UR];
#pragma unroll
    for (int u = 0; u < UR; ++u) xj[u] = p0 + u * G < e ? __ldg(src + cj[u]) : TX(0);
#pragma unroll
    for (int u = 0; u < UR; ++u)
      if (p0 + u * G < e) acc = fma(convert<TY>(vj[u]), convert<TY>(xj[u]), acc);
  }
  return acc;
}

template <int G, int EPI, typename TM, typename TX, typename TY>
__global__ void __launch_bounds__(256) k_row(RowOp<TM, TX, TY> op) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int row = (int)(gid / G);
  if (row >= op.n) {  // uniform over the G lanes of a row
    pdl_enter();
    return;
  }
  constexpr int UR = 4;
  const int lane = (int)(gid & (G - 1));
  int b = 0, e = 0;
  int cj[UR];
  TM vj[UR];
  bool stream = false;
  if constexpr (sizeof(TM) == sizeof(double)) stream = op.mat_stream != 0;  // uniform over the launch
  if (op.v) {  // row bounds and the first round of entries: static data, before the wait
    b = __ldg(op.rp + row);
    e = __ldg(op.rp + row + 1);
    if (stream) {
      if constexpr (sizeof(TM) == sizeof(double)) csr_round_loads<true, G, UR>(op.ci, op.v, b + lane, e, cj, vj, l2_evict_first());
    } else {
      csr_round_loads<false, G, UR>(op.ci, op.v, b + lane, e, cj, vj, 0ull);
    }
  }
  pdl_enter();  // the source vector, epilogue vectors and the skip flag may come from the previous kernel
  if (op.skip && *op.skip) return;
  TY acc = TY(0);
  if (op.v) {
    const TX* __restrict__ src = op.src.get();
    if (stream) {
      if constexpr (sizeof(TM) == sizeof(double))
        acc = csr_accumulate<true, G, UR>(op.ci, op.v, src, b, e, lane, acc, l2_evict_first(), cj, vj);
    } else {
      acc = csr_accumulate<false, G, UR>(op.ci, op.v, src, b, e, lane, acc, 0ull, cj, vj);
    }
    if constexpr (G > 1) {
      const unsigned seg = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(seg, acc, o, G);
    }
    if (lane != 0) return;
  }
  row_epilogue<EPI>(op, row, acc);
}

// Entries j, j+1, ... of K chunks, U at a time per chunk: the column and value loads of all K*U
// entries are issued before any gather and the gathers before any FMA, so a thread has K*U
// entries in flight per memory round trip (longer rows are latency bound with one or two; short
// rows prefer U = 1, which needs fewer registers and keeps more warps resident). Every lane runs
// to its chunk's width (uniform over the warp); padded entries hold zero values and a column of
// their own row, so they add exact zeros. Each row's FMAs keep the order j = 0, 1, 2, ...
// The first round's column and value loads are issued by the caller (sell_round_loads) before
// it waits for the previous kernel: the matrix does not depend on it, only the gathers do.
template <bool ST, int K, int U, typename TM>
__device__ __forceinline__ void sell_round_loads(const SellView<TM>& sv, const int64_t (&off)[K], const int (&len)[K],
                                                 int j, int (&cj)[K][U], TM (&vj)[K][U], uint64_t pol) {
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool in = j + u < len[k];
      const int64_t q = off[k] + 32 * (int64_t)(j + u);
      cj[k][u] = in ? ld_entry<ST>(sv.col + q, pol) : 0;
      vj[k][u] = in ? ld_entry<ST>(sv.val + q, pol) : TM(0);
    }
}

template <bool ST, int K, int U, typename TM, typename TX, typename TY>
__device__ __forceinline__ void sell_accumulate(const SellView<TM>& sv, const TX* __restrict__ src, const int64_t (&off)[K],
                                                const int (&len)[K], int jmax, TY (&acc)[K], uint64_t pol,
                                                int (&cj)[K][U], TM (&vj)[K][U]) {
#pragma unroll(U == 1 ? 2 : 1)
  for (int j = 0; j < jmax; j += U) {
    if (j > 0) sell_round_loads<ST, K, U>(sv, off, len, j, cj, vj, pol);  // round 0: loaded by the caller
    TX xj[K][U];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int u = 0; u < U; ++u) xj[k][u] = j + u < len[k] ? __ldg(src + cj[k][u]) : TX(0);
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (j + u < len[k]) acc[k] = fma(convert<TY>(vj[k][u]), convert<TY>(xj[k][u]), acc[k]);
  }
}

// K chunks of 32 rows per warp, each lane one row of each chunk, U entries of each chunk staged
// per round (sell_accumulate). PLAIN: natural row order (chunk c holds rows 32c..32c+31);
// otherwise rows sorted by length within windows, with a permutation. Chunk widths come from
// cptr, or from sell.width when every chunk has the same width. The chunk geometry and the first
// round of matrix entries are loaded before the wait for the previous kernel.
constexpr int kSellPrefetchRounds = 8;

template <int EPI, int K, int U, bool PLAIN, typename TM, typename TX, typename TY>
__global__ void __launch_bounds__(256) k_sell(RowOp<TM, TX, TY> op) {
  const int lane = threadIdx.x & 31;
  const int c0 = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * K;
  if (c0 >= op.sell.nchunks) {
    pdl_enter();
    return;
  }
  int row[K], len[K];
  int64_t off[K];
  TY acc[K];
  int jmax = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int c = c0 + k;
    const bool ok = c < op.sell.nchunks;
    const int pos = c * 32 + lane;
    if constexpr (PLAIN) {
      row[k] = (ok && pos < op.n) ? pos : -1;
    } else {
      row[k] = ok ? __ldg(op.sell.perm + pos) : -1;
    }
    if (op.sell.width) {  // uniform chunks: no offset load ahead of the entry loads
      len[k] = ok ? op.sell.width : 0;
      off[k] = (int64_t)c * 32 * op.sell.width + lane;
    } else {
      const int64_t c_b = ok ? __ldg(op.sell.cptr + c) : 0;
      len[k] = ok ? (int)((__ldg(op.sell.cptr + c + 1) - c_b) >> 5) : 0;
      off[k] = c_b + lane;
    }
    acc[k] = TY(0);
    jmax = max(jmax, len[k]);
  }
  bool stream = false;
  if constexpr (sizeof(TM) == sizeof(double)) stream = op.mat_stream != 0;  // uniform over the launch
  int cj[K][U];
  TM vj[K][U];
  if (stream) {
    if constexpr (sizeof(TM) == sizeof(double)) sell_round_loads<true, K, U>(op.sell, off, len, 0, cj, vj, l2_evict_first());
  } else {
    sell_round_loads<false, K, U>(op.sell, off, len, 0, cj, vj, 0ull);
  }
  // the later rounds of short chunks into L2 as well (one line request per lane and entry)
  if (jmax <= kSellPrefetchRounds) {
#pragma unroll
    for (int k = 0; k < K; ++k)
      for (int j = U; j < len[k]; ++j) {
        const int64_t q = off[k] + 32 * (int64_t)j;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(op.sell.col + q));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(op.sell.val + q));
      }
  }
  pdl_enter();  // the source vector (and the skip flag) may come from the previous kernel
  if (op.skip && *op.skip) return;
  const TX* __restrict__ src = op.src.get();
  if (stream) {
    if constexpr (sizeof(TM) == sizeof(double))
      sell_accumulate<true, K, U>(op.sell, src, off, len, jmax, acc, l2_evict_first(), cj, vj);
  } else {
    sell_accumulate<false, K, U>(op.sell, src, off, len, jmax, acc, 0ull, cj, vj);
  }
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (row[k] >= 0) row_epilogue<EPI>(op, row[k], acc[k]);
}

// ------------------------------------------------------------------------------------------
// Small helpers
// ------------------------------------------------------------------------------------------
// Four consecutive elements per load/store when both vectors start 16-byte aligned (library
// vectors and basis columns are 256-byte aligned); caller arrays that are not take the scalar loop.
template <typename T>
struct Quad;
template <>
struct Quad<double> {
  double v[4];
  __device__ __forceinline__ void load(const double* p) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
  }
  __device__ __forceinline__ void store(double* p) const {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
};
template <>
struct Quad<float> {
  float v[4];
  __device__ __forceinline__ void load(const float* p) {
    const float4 a = reinterpret_cast<const float4*>(p)[0];
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
  }
  __device__ __forceinline__ void store(float* p) const { reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]); }
};

template <typename TA, typename TB>
__global__ void k_cast(int64_t n, VRef<const TA> a, VRef<TB> b, const int* skip) {
  pdl_enter();
  if (skip && *skip) return;
  const TA* pa = a.get();
  TB* pb = b.get();
  const bool aligned = ((reinterpret_cast<uintptr_t>(pa) | reinterpret_cast<uintptr_t>(pb)) & 15u) == 0;
  const int64_t n4 = aligned ? n / 4 : 0, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += stride) {
    Quad<TA> x;
    x.load(pa + 4 * q);
    Quad<TB> y;
#pragma unroll
    for (int k = 0; k < 4; ++k) y.v[k] = convert<TB>(x.v[k]);
    y.store(pb + 4 * q);
  }
  for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) pb[i] = convert<TB>(pa[i]);
}

template <typename T>
__global__ void k_fill(int64_t n, T* a, T v) {
  pdl_enter();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) a[i] = v;
}

// Dense coarse solve z = C b with C the row-major inverse of the coarsest operator; one warp
// per row, fixed-order reduction.
template <typename TC, typename T>
__global__ void k_dense_gemv(int n, const TC* __restrict__ C, VRef<const T> bref, VRef<T> zref, const int* skip) {
  pdl_enter();
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
// Fused V-cycle tail: every pass of the V-cycle below a level whose vectors fit in shared memory
// (pre-smoothing with all its Neumann terms, residual, restriction, the coarse solve,
// prolongation, post-smoothing) run by ONE thread-block cluster. A cluster barrier separates
// dependent passes; each CTA stages the pass's source vector in its shared memory and gathers
// from there. Rows of a pass are split over the cluster's CTAs, G lanes per row, with the
// accumulation order, shuffle reduction and compile-time epilogue of k_row and k_dense_gemv, so
// the result equals the unfused launches bit for bit.
// ------------------------------------------------------------------------------------------
template <typename T>
struct TailPass {
  RowOp<T, T, T> op;
  int G = 1;       // threads per row (the standalone launch's choice)
  int epi = 0;     // epilogue code
  int dense = 0;   // 1: out = C src, C dense src_n x src_n row-major (coarse solve)
  const T* C = nullptr;
};

constexpr int kTailThreads = 1024;
constexpr int kTailStage = 8192;  // longest staged source vector (elements)

template <int EPI, typename T>
__device__ __forceinline__ void tail_row_pass(const RowOp<T, T, T>& op, int G, const T* __restrict__ xs, int r0, int r1) {
  const int64_t t_end = (int64_t)r1 * G;
  for (int64_t t = (int64_t)r0 * G + threadIdx.x; t < t_end; t += blockDim.x) {
    const int row = (int)(t / G);
    T acc = T(0);
    if (op.v) {
      const int lane = (int)(t & (G - 1));
      const int b = __ldg(op.rp + row), e = __ldg(op.rp + row + 1);
#pragma unroll 4
      for (int p = b + lane; p < e; p += G) {
        const int c = __ldg(op.ci + p);
        acc = fma((T)__ldg(op.v + p), xs[c], acc);
      }
      if (G > 1) {
        const unsigned seg = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(seg, acc, o, G);
      }
      if (lane != 0) continue;
    }
    row_epilogue<EPI>(op, row, acc);
  }
}

template <typename T>
__global__ void __launch_bounds__(kTailThreads) k_tail(const TailPass<T>* __restrict__ passes, int np, const int* skip) {
  pdl_enter();
  if (skip && *skip) return;  // same value in every CTA: the whole cluster leaves
  extern __shared__ __align__(16) unsigned char tail_smem[];
  T* sx = reinterpret_cast<T*>(tail_smem);
  cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
  const int rank = (int)cl.block_rank(), ncl = (int)cl.num_blocks();
  for (int q = 0; q < np; ++q) {
    const TailPass<T>& P = passes[q];
    const RowOp<T, T, T>& op = P.op;
    const T* src = op.src.p;
    const T* xs = src;
    if (src && op.src_n > 0 && op.src_n <= kTailStage) {
      for (int k = threadIdx.x; k < op.src_n; k += blockDim.x) sx[k] = src[k];
      __syncthreads();
      xs = sx;
    }
    if (P.dense) {
      const int n = op.n;
      const int wpb = blockDim.x >> 5, lane = threadIdx.x & 31;
      for (int row = rank * wpb + (threadIdx.x >> 5); row < n; row += ncl * wpb) {
        T acc = T(0);
        for (int j = lane; j < n; j += 32) acc = fma(P.C[(int64_t)row * n + j], xs[j], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) op.out.p[row] = acc;
      }
    } else {
      const int chunk = (op.n + ncl - 1) / ncl;
      const int r0 = min(op.n, rank * chunk), r1 = min(op.n, r0 + chunk);
      const int G = op.v ? P.G : 1;
      switch (P.epi) {
        case 0: tail_row_pass<0>(op, G, xs, r0, r1); break;
        case 2: tail_row_pass<2>(op, G, xs, r0, r1); break;
        case 3: tail_row_pass<3>(op, G, xs, r0, r1); break;
        case 6: tail_row_pass<6>(op, G, xs, r0, r1); break;
        case 7: tail_row_pass<7>(op, G, xs, r0, r1); break;
        case 11: tail_row_pass<11>(op, G, xs, r0, r1); break;
        case 16: tail_row_pass<16>(op, G, xs, r0, r1); break;
        case 18: tail_row_pass<18>(op, G, xs, r0, r1); break;
        case 19: tail_row_pass<19>(op, G, xs, r0, r1); break;
        case 27: tail_row_pass<27>(op, G, xs, r0, r1); break;
        default: tail_row_pass<E_RUNTIME>(op, G, xs, r0, r1); break;
      }
    }
    cl.sync();  // outputs visible to the whole cluster; shared staging free for the next pass
  }
}

// ------------------------------------------------------------------------------------------
// Grid-wide fused V-cycle tail: the same recorded passes as k_tail (every pass below a level of
// at most kGridTailRows rows), run by one cooperative launch over the whole GPU, one block per
// SM, with a grid barrier between dependent passes instead of a kernel boundary. Rows of a pass
// are dealt to all threads of the grid, G lanes per row, with k_row's accumulation order,
// shuffle reduction and epilogue, so the result equals the separate launches bit for bit. The
// source vector of a pass is read through L2 (it was written by other SMs in an earlier pass).
// Every barrier wait is bounded: after `spin_limit` polls the block records NSAMG_ERR_TIMEOUT in
// *status and the kernel returns, leaving the context usable.
// ------------------------------------------------------------------------------------------
constexpr int kGridTailThreads = 512;
constexpr int kGridTailRows = 32768;
constexpr unsigned kGridSpinLimit = 1u << 20;  // polls of ~0.1 us: about 0.1 s before giving up

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Barrier over `nb` co-resident blocks on a monotonic 64-bit counter (zeroed before the launch):
// arrival k of the counter belongs to barrier k / nb. True once every block has arrived; false
// if the wait gave up.
__device__ __forceinline__ bool grid_barrier(unsigned long long* ctr, unsigned nb, unsigned spin_limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();  // the block's writes of this pass before its arrival
    const unsigned long long old = atomicAdd(ctr, 1ull);
    const unsigned long long target = (old / nb + 1) * nb;
    int ok = 1;
    for (unsigned k = 0; ld_acquire_u64(ctr) < target; ++k) {
      if (k >= spin_limit) {
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <int EPI, typename T>
__device__ __forceinline__ void tail_grid_row_pass(const RowOp<T, T, T>& op, int G) {
  const T* __restrict__ src = op.src.p;
  const int64_t t_end = (int64_t)op.n * G, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < t_end; t += stride) {
    const int row = (int)(t / G);
    T acc = T(0);
    if (op.v) {
      const int lane = (int)(t & (G - 1));
      const int b = __ldg(op.rp + row), e = __ldg(op.rp + row + 1);
#pragma unroll 4
      for (int p = b + lane; p < e; p += G) {
        const int c = __ldg(op.ci + p);
        acc = fma((T)__ldg(op.v + p), __ldcg(src + c), acc);
      }
      if (G > 1) {
        const unsigned seg = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(seg, acc, o, G);
      }
      if (lane != 0) continue;
    }
    row_epilogue<EPI>(op, row, acc);
  }
}

template <typename T>
__global__ void __launch_bounds__(kGridTailThreads) k_tail_grid(const TailPass<T>* __restrict__ passes, int np,
                                                               const int* skip, unsigned long long* ctr, int* status,
                                                               unsigned spin_limit) {
  pdl_enter();
  if (skip && *skip) return;  // the same value in every block: the whole grid leaves
  for (int q = 0; q < np; ++q) {
    const TailPass<T>& P = passes[q];
    const RowOp<T, T, T>& op = P.op;
    if (P.dense) {
      const T* __restrict__ src = op.src.p;
      const int n = op.n, lane = threadIdx.x & 31;
      const int warps = (int)(gridDim.x * blockDim.x) >> 5;
      for (int row = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); row < n; row += warps) {
        T acc = T(0);
        for (int j = lane; j < n; j += 32) acc = fma(P.C[(int64_t)row * n + j], __ldcg(src + j), acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) op.out.p[row] = acc;
      }
    } else {
      const int G = op.v ? P.G : 1;
      switch (P.epi) {
        case 0: tail_grid_row_pass<0>(op, G); break;
        case 2: tail_grid_row_pass<2>(op, G); break;
        case 3: tail_grid_row_pass<3>(op, G); break;
        case 6: tail_grid_row_pass<6>(op, G); break;
        case 7: tail_grid_row_pass<7>(op, G); break;
        case 11: tail_grid_row_pass<11>(op, G); break;
        case 16: tail_grid_row_pass<16>(op, G); break;
        case 18: tail_grid_row_pass<18>(op, G); break;
        case 19: tail_grid_row_pass<19>(op, G); break;
        case 27: tail_grid_row_pass<27>(op, G); break;
        default: tail_grid_row_pass<E_RUNTIME>(op, G); break;
      }
    }
    if (q + 1 < np && !grid_barrier(ctr, gridDim.x, spin_limit)) {
      if (threadIdx.x == 0 && status) atomicExch(status, -5);  // NSAMG_ERR_TIMEOUT
      return;
    }
  }
}

// The grid barrier alone, for its tests: `rounds` barriers, each expecting gridDim.x + missing
// arrivals (missing > 0: arrivals that never come, so that every wait runs out); each block adds
// 1 to *passed per barrier it completed, and a block that gave up records NSAMG_ERR_TIMEOUT in
// *status.
__global__ void __launch_bounds__(256) k_grid_barrier_test(unsigned long long* ctr, int rounds, int missing,
                                                            unsigned spin_limit, int* passed, int* status) {
  for (int r = 0; r < rounds; ++r) {
    if (!grid_barrier(ctr, gridDim.x + (unsigned)missing, spin_limit)) {
      if (threadIdx.x == 0) atomicExch(status, -5);
      return;
    }
    if (threadIdx.x == 0) atomicAdd(passed, 1);
  }
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
  int stop_nrbe;  // 1: stop on the backward error nrbe <= rtol instead of the relative residual
  // loop control
  int i;          // current Arnoldi step within the cycle (column index of vt)
  int k;          // columns completed in this cycle
  int stop;       // inner loop must stop (cycle finished)
  int done;       // solve finished
  int iters;      // total Arnoldi columns
  int cycles;     // restart cycles started
  int status;     // 0 ok, 1 not converged, <0 error
  int converged;
  int klast;      // Arnoldi vectors of the last finished cycle (rows of L it filled)
  int pad1;
  double bnorm;
  double relres_true;
  double relres_implicit;
  double anorm_inf;   // ||A||_inf of the finest operator (set at setup)
  double nrbe;        // ||r|| / (||b|| + ||A||_inf ||x||) of the last true residual
  double xnorm;       // ||x|| at the last true residual (the start of the current cycle)
  double rnorm;       // ||b - A x|| at the last true residual
  double r0_scale;    // split basis: column 0 holds r / r0_scale (r0_scale an exact power of two)
  double lsum;        // sum of squares of the L entries of the current cycle
  double orth_loss;   // sqrt(2 lsum): ||I - V^T V||_F of the last cycle (diagonal terms ~ eps)
  double sk_norm;     // ||S_k||_2, S_k = (I + L^T)^-1 L^T, of the last cycle
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
