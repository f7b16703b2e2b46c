// Host engine and C ABI of nsamg: hierarchy upload, V-cycle orchestration, the one-reduce
// GMRES(m) loop (run as one CUDA graph with device-side WHILE conditionals, or as a plain
// launch loop), and the per-kernel entry points.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>
#include <algorithm>
#include <initializer_list>
#include <type_traits>

#include "nsamg.h"
#include "kernels.cuh"
#include "gmres.cuh"
#include "batch.cuh"
#include <functional>
#include <deque>
#include <thread>
#include <condition_variable>
#include <chrono>
#include <unordered_map>
#include <atomic>

using namespace nsamg;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  const int code = (e == cudaErrorMemoryAllocation) ? NSAMG_ERR_OOM : NSAMG_ERR_CUDA;
  return fail(code, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

constexpr int kThreads = 256;

// Kernel launches enqueued by the engine on this thread (used to report launches per step).
thread_local int64_t g_launches = 0;

inline int blocks_for(int64_t threads) { return (int)std::max<int64_t>(1, (threads + kThreads - 1) / kThreads); }

// Every kernel is launched with programmatic dependent launch allowed: each kernel starts by
// waiting for its predecessor grid (griddepcontrol.wait) and then lets its own successor be
// scheduled, so launch latency overlaps the predecessor's last wave. NSAMG_PDL=0 turns it off.
bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("NSAMG_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}

template <typename... KArgs, typename... Args>
void launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

template <typename... KArgs, typename... Args>
void launch_k_smem(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// The bulk-copy Gram's dynamic shared memory exceeds the 48 KB default: raise the limit once per
// device (a host-side attribute; no allocation).
std::mutex g_tma_mu;
std::vector<char> g_tma_ready;
cudaError_t gram_tma_prepare() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_tma_mu);
  if ((int)g_tma_ready.size() <= dev) g_tma_ready.resize(dev + 1, 0);
  if (g_tma_ready[dev]) return cudaSuccess;
  if ((e = cudaFuncSetAttribute(k_gram_tma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGramTmaSmem)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_gram_tma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGramTmaSmem)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_update_tma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGramTmaSmem)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_update_tma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGramTmaSmem)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_gram_s, cudaFuncAttributeMaxDynamicSharedMemorySize, kGramSSmem)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_update_s, cudaFuncAttributeMaxDynamicSharedMemorySize, kGramTmaSmem)) != cudaSuccess)
    return e;
  g_tma_ready[dev] = 1;
  return cudaSuccess;
}

// The bulk-copy path needs every column start of V and w 16-byte aligned.
bool gram_tma_aligned(const double* V, int64_t ldv, const double* w) {
  return ((reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(w)) & 15u) == 0 && (ldv & 1) == 0;
}

// ------------------------------------------------------------------------------------------
// Device CSR
// ------------------------------------------------------------------------------------------
template <typename T>
struct DCSR {
  int n = 0, m = 0;
  int64_t nnz = 0;
  int* rp = nullptr;
  int* ci = nullptr;
  T* v = nullptr;
  int G = 1;
  // SELL-32-sigma copy (matrices with at least kSellMinRows rows); use_sell picks it at launch
  int nchunks = 0;
  int* s_perm = nullptr;
  int64_t* s_cptr = nullptr;
  int* s_col = nullptr;
  T* s_val = nullptr;
  int s_width = 0;  // plain layout with uniform chunk width (0: widths from s_cptr)
  bool use_sell = false;
  int sell_k = 1;  // chunks per warp
  int sell_u = 1;  // entries staged per chunk and round
  bool present() const { return n > 0; }
};

constexpr int kSellMinRows = 16384;
constexpr double kPlainPad = 1.03;  // natural-order chunk padding accepted for the plain layout
constexpr int kSellSigma = 4096;  // rows sorted by length inside windows of this many rows

struct HostCSR {  // host copy used while building derived matrices
  int n = 0, m = 0;
  std::vector<int> rp, ci;
  std::vector<double> v;
};

double norm_inf(const nsamg_csr& A) {
  double mx = 0.0;
  for (int i = 0; i < A.nrows; ++i) {
    double r = 0.0;
    for (int64_t q = A.rowptr[i]; q < A.rowptr[i + 1]; ++q) r += std::fabs(A.val[q]);
    mx = std::max(mx, r);
  }
  return mx;
}

int validate(const nsamg_csr& A, bool square, bool need_diag, const char* name) {
  if (A.nrows <= 0) return fail(NSAMG_ERR_INVALID_ARG, std::string(name) + ": empty matrix");
  if (!A.rowptr || (A.nnz > 0 && (!A.col || !A.val))) return fail(NSAMG_ERR_INVALID_ARG, std::string(name) + ": null array");
  if (A.nnz < 0 || A.nnz > INT32_MAX) return fail(NSAMG_ERR_BAD_MATRIX, std::string(name) + ": nnz out of range");
  if (square && A.ncols != A.nrows) return fail(NSAMG_ERR_BAD_MATRIX, std::string(name) + ": not square");
  if (A.rowptr[0] != 0 || A.rowptr[A.nrows] != A.nnz) return fail(NSAMG_ERR_BAD_MATRIX, std::string(name) + ": bad rowptr ends");
  for (int i = 0; i < A.nrows; ++i) {
    const int b = A.rowptr[i], e = A.rowptr[i + 1];
    if (e < b) return fail(NSAMG_ERR_BAD_MATRIX, std::string(name) + ": rowptr not monotone at row " + std::to_string(i));
    bool diag = false;
    for (int p = b; p < e; ++p) {
      const int c = A.col[p];
      if (c < 0 || c >= A.ncols) return fail(NSAMG_ERR_BAD_MATRIX, std::string(name) + ": column out of range in row " + std::to_string(i));
      if (p > b && c <= A.col[p - 1]) return fail(NSAMG_ERR_BAD_MATRIX, std::string(name) + ": columns not sorted in row " + std::to_string(i));
      if (c == i && A.val[p] != 0.0) diag = true;
      if (!std::isfinite(A.val[p])) return fail(NSAMG_ERR_BAD_MATRIX, std::string(name) + ": non-finite value in row " + std::to_string(i));
    }
    if (need_diag && !diag) return fail(NSAMG_ERR_BAD_MATRIX, std::string(name) + ": missing or zero diagonal in row " + std::to_string(i));
  }
  return NSAMG_OK;
}

// Threads per CSR row before tuning.
int default_group(int n, int64_t nnz) {
  const double avg = n ? (double)nnz / n : 0.0;
  if (n < 16384) {
    // small levels are latency bound: give each row enough lanes that every lane handles about
    // one entry (the FP64 issue cost of idle lanes does not matter at this size)
    int G = 1;
    while (G < 32 && G < avg) G <<= 1;
    return G;
  }
  return avg <= 12 ? 1 : avg <= 24 ? 2 : avg <= 48 ? 4 : avg <= 96 ? 8 : 16;
}

template <typename T>
int upload(const int* rp, const int* ci, const double* v, int n, int m, int64_t nnz, DCSR<T>& d) {
  d.n = n;
  d.m = m;
  d.nnz = nnz;
  CK(cudaMalloc(&d.rp, sizeof(int) * (n + 1)));
  CK(cudaMemcpy(d.rp, rp, sizeof(int) * (n + 1), cudaMemcpyHostToDevice));
  const int64_t cap = std::max<int64_t>(nnz, 1);
  CK(cudaMalloc(&d.ci, sizeof(int) * cap));
  CK(cudaMalloc(&d.v, sizeof(T) * cap));
  if (nnz > 0) {
    CK(cudaMemcpy(d.ci, ci, sizeof(int) * nnz, cudaMemcpyHostToDevice));
    if constexpr (sizeof(T) == sizeof(double)) {
      CK(cudaMemcpy(d.v, v, sizeof(double) * nnz, cudaMemcpyHostToDevice));
    } else {
      std::vector<T> tmp(v, v + nnz);
      CK(cudaMemcpy(d.v, tmp.data(), sizeof(T) * nnz, cudaMemcpyHostToDevice));
    }
  }
  // Near-uniform rows (natural-order chunks padded by at most kPlainPad): the plain layout, rows
  // in their own order, each padded to its chunk's width with zero values (column = the row's last
  // column, or the row itself when empty), so no permutation or row lengths are stored or read.
  bool plain = false;
  if (n >= kSellMinRows && nnz > 0) {
    int64_t slots = 0;
    for (int c = 0; c * 32 < n; ++c) {
      int w = 0;
      for (int i = c * 32; i < std::min(n, c * 32 + 32); ++i) w = std::max(w, rp[i + 1] - rp[i]);
      slots += 32 * (int64_t)w;
    }
    plain = (double)slots <= kPlainPad * (double)nnz;
  }
  if (plain) {
    const int nch = (n + 31) / 32;
    std::vector<int> cw(nch, 0);
    int wmax = 0;
    for (int c = 0; c < nch; ++c) {
      for (int i = c * 32; i < std::min(n, c * 32 + 32); ++i) cw[c] = std::max(cw[c], rp[i + 1] - rp[i]);
      wmax = std::max(wmax, cw[c]);
    }
    // every chunk as wide as the widest when that still pads by at most kPlainPad: the kernel then
    // computes chunk offsets instead of loading them
    d.s_width = 32.0 * wmax * nch <= kPlainPad * (double)nnz ? wmax : 0;
    std::vector<int64_t> cptr(nch + 1, 0);
    for (int c = 0; c < nch; ++c) cptr[c + 1] = cptr[c] + 32 * (int64_t)(d.s_width ? d.s_width : cw[c]);
    std::vector<int> scol(std::max<int64_t>(cptr[nch], 1), 0);
    std::vector<T> sval(std::max<int64_t>(cptr[nch], 1), T(0));
    for (int c = 0; c < nch; ++c) {
      const int w = (int)((cptr[c + 1] - cptr[c]) / 32);
      for (int l = 0; l < 32; ++l) {
        const int row = c * 32 + l;
        const int len = row < n ? rp[row + 1] - rp[row] : 0;
        const int pad_col = len > 0 ? ci[rp[row] + len - 1] : std::min(row, m - 1);
        for (int j = 0; j < w; ++j) {
          const int64_t q = cptr[c] + (int64_t)j * 32 + l;
          scol[q] = j < len ? ci[rp[row] + j] : pad_col;
          sval[q] = j < len ? (T)v[rp[row] + j] : T(0);
        }
      }
    }
    d.nchunks = nch;
    d.sell_k = 1;
    CK(cudaMalloc(&d.s_cptr, sizeof(int64_t) * cptr.size()));
    CK(cudaMemcpy(d.s_cptr, cptr.data(), sizeof(int64_t) * cptr.size(), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&d.s_col, sizeof(int) * scol.size()));
    CK(cudaMemcpy(d.s_col, scol.data(), sizeof(int) * scol.size(), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&d.s_val, sizeof(T) * sval.size()));
    CK(cudaMemcpy(d.s_val, sval.data(), sizeof(T) * sval.size(), cudaMemcpyHostToDevice));
  } else if (n >= kSellMinRows && nnz > 0) {
    // SELL-32-sigma: sort rows by length (descending, stable) inside windows of sigma rows, cut
    // into chunks of 32 positions, store each chunk column-major; every row is padded to its
    // chunk's width with zero values in its own last column (the kernel reads no row lengths).
    const int nch = (n + 31) / 32;
    std::vector<int> perm((size_t)nch * 32, -1), rlen((size_t)nch * 32, 0), order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    for (int w0 = 0; w0 < n; w0 += kSellSigma) {
      const int w1 = std::min(n, w0 + kSellSigma);
      std::stable_sort(order.begin() + w0, order.begin() + w1,
                       [&](int a, int b) { return (rp[a + 1] - rp[a]) > (rp[b + 1] - rp[b]); });
    }
    for (int i = 0; i < n; ++i) {
      perm[i] = order[i];
      rlen[i] = rp[order[i] + 1] - rp[order[i]];
    }
    std::vector<int64_t> cptr(nch + 1, 0);
    for (int c = 0; c < nch; ++c) {
      int w = 0;
      for (int l = 0; l < 32; ++l) w = std::max(w, rlen[(size_t)c * 32 + l]);
      cptr[c + 1] = cptr[c] + 32 * (int64_t)w;
    }
    std::vector<int> scol(std::max<int64_t>(cptr[nch], 1), 0);
    std::vector<T> sval(std::max<int64_t>(cptr[nch], 1), T(0));
    for (int c = 0; c < nch; ++c) {
      const int w = (int)((cptr[c + 1] - cptr[c]) / 32);
      for (int l = 0; l < 32; ++l) {
        const int row = perm[(size_t)c * 32 + l];
        if (row < 0) continue;  // no row at this position: columns 0, values 0
        const int len = rlen[(size_t)c * 32 + l];
        const int pad_col = len > 0 ? ci[rp[row] + len - 1] : std::min(row, m - 1);
        for (int j = 0; j < w; ++j) {
          const int64_t q = cptr[c] + (int64_t)j * 32 + l;
          scol[q] = j < len ? ci[rp[row] + j] : pad_col;
          sval[q] = j < len ? (T)v[rp[row] + j] : T(0);
        }
      }
    }
    d.nchunks = nch;
    const double avg_row = (double)nnz / n;
    // FP64 rows are FP64-issue bound (one chunk per warp keeps registers and occupancy);
    // FP32 rows are latency bound and interleave several chunks
    d.sell_k = sizeof(T) == sizeof(double) ? 1 : (avg_row <= 8 ? 4 : avg_row <= 16 ? 2 : 1);
    CK(cudaMalloc(&d.s_perm, sizeof(int) * perm.size()));
    CK(cudaMemcpy(d.s_perm, perm.data(), sizeof(int) * perm.size(), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&d.s_cptr, sizeof(int64_t) * cptr.size()));
    CK(cudaMemcpy(d.s_cptr, cptr.data(), sizeof(int64_t) * cptr.size(), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&d.s_col, sizeof(int) * scol.size()));
    CK(cudaMemcpy(d.s_col, scol.data(), sizeof(int) * scol.size(), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&d.s_val, sizeof(T) * sval.size()));
    CK(cudaMemcpy(d.s_val, sval.data(), sizeof(T) * sval.size(), cudaMemcpyHostToDevice));
  }
  d.G = default_group(n, nnz);
  return NSAMG_OK;
}

template <typename T>
int upload(const HostCSR& h, DCSR<T>& d) {
  return upload<T>(h.rp.data(), h.ci.data(), h.v.data(), h.n, h.m, (int64_t)h.ci.size(), d);
}

template <typename T>
int upload(const nsamg_csr& c, DCSR<T>& d) {
  return upload<T>(c.rowptr, c.col, c.val, c.nrows, c.ncols, c.nnz, d);
}

template <typename T>
void release(DCSR<T>& d) {
  cudaFree(d.rp);
  cudaFree(d.ci);
  cudaFree(d.v);
  cudaFree(d.s_perm);
  cudaFree(d.s_cptr);
  cudaFree(d.s_col);
  cudaFree(d.s_val);
  d = DCSR<T>();
}

template <typename T>
int upload_vec(const std::vector<double>& h, T** d) {
  CK(cudaMalloc(d, sizeof(T) * std::max<size_t>(h.size(), 1)));
  std::vector<T> tmp(h.begin(), h.end());
  CK(cudaMemcpy(*d, tmp.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
  return NSAMG_OK;
}

// Triangular part of A (strict lower if lower, else strict upper), rows scaled by rs (if given)
// and columns scaled by cs (if given). ranks > 1: only the couplings whose row and column lie in
// the same one of `ranks` contiguous row blocks of ceil(n / ranks) rows (a hybrid smoother's
// local triangle, Sec. 5.2).
HostCSR tri_part(const nsamg_csr& A, bool lower, const std::vector<double>* rs, const std::vector<double>* cs,
                 int ranks = 1) {
  const int64_t bsz = ranks > 1 ? ((int64_t)A.nrows + ranks - 1) / ranks : (int64_t)A.nrows + 1;
  HostCSR h;
  h.n = A.nrows;
  h.m = A.ncols;
  h.rp.assign(A.nrows + 1, 0);
  for (int i = 0; i < A.nrows; ++i) {
    for (int p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p) {
      const int c = A.col[p];
      if ((lower ? c < i : c > i) && c / bsz == i / bsz) {
        double v = A.val[p];
        if (rs) v *= (*rs)[i];
        if (cs) v *= (*cs)[c];
        h.ci.push_back(c);
        h.v.push_back(v);
      }
    }
    h.rp[i + 1] = (int)h.ci.size();
  }
  return h;
}

// ------------------------------------------------------------------------------------------
// Row-kernel launch
// ------------------------------------------------------------------------------------------
// Epilogue codes instantiated at compile time (the forms the engine builds); others fall back to
// the run-time form.
template <int G, typename TM, typename TX, typename TY>
void launch_csr(const RowOp<TM, TX, TY>& op, int nb, cudaStream_t s) {
  if constexpr (std::is_same<TX, TY>::value) {
    switch (epi_code(op)) {
      case 0: launch_k(k_row<G, 0, TM, TX, TY>, nb, kThreads, s, op); return;
      case 2: launch_k(k_row<G, 2, TM, TX, TY>, nb, kThreads, s, op); return;
      case 3: launch_k(k_row<G, 3, TM, TX, TY>, nb, kThreads, s, op); return;
      case 6: launch_k(k_row<G, 6, TM, TX, TY>, nb, kThreads, s, op); return;
      case 7: launch_k(k_row<G, 7, TM, TX, TY>, nb, kThreads, s, op); return;
      case 11: launch_k(k_row<G, 11, TM, TX, TY>, nb, kThreads, s, op); return;
      case 16: launch_k(k_row<G, 16, TM, TX, TY>, nb, kThreads, s, op); return;
      case 18: launch_k(k_row<G, 18, TM, TX, TY>, nb, kThreads, s, op); return;
      case 19: launch_k(k_row<G, 19, TM, TX, TY>, nb, kThreads, s, op); return;
      case 27: launch_k(k_row<G, 27, TM, TX, TY>, nb, kThreads, s, op); return;
      default: break;
    }
  } else {
    if (epi_code(op) == 0) {
      launch_k(k_row<G, 0, TM, TX, TY>, nb, kThreads, s, op);
      return;
    }
  }
  launch_k(k_row<G, E_RUNTIME, TM, TX, TY>, nb, kThreads, s, op);
}

template <int EPI, int K, int U, typename TM, typename TX, typename TY>
void launch_sell_one(const RowOp<TM, TX, TY>& op, cudaStream_t s) {
  const int nb = blocks_for((int64_t)((op.sell.nchunks + K - 1) / K) * 32);
  if (op.sell.perm)
    launch_k(k_sell<EPI, K, U, false, TM, TX, TY>, nb, kThreads, s, op);
  else
    launch_k(k_sell<EPI, K, U, true, TM, TX, TY>, nb, kThreads, s, op);
}

template <int K, int U, typename TM, typename TX, typename TY>
void launch_sell_k(const RowOp<TM, TX, TY>& op, cudaStream_t s) {
  if constexpr (std::is_same<TX, TY>::value) {
    switch (epi_code(op)) {
      case 0: launch_sell_one<0, K, U>(op, s); return;
      case 3: launch_sell_one<3, K, U>(op, s); return;
      case 7: launch_sell_one<7, K, U>(op, s); return;
      case 11: launch_sell_one<11, K, U>(op, s); return;
      case 16: launch_sell_one<16, K, U>(op, s); return;
      case 19: launch_sell_one<19, K, U>(op, s); return;
      case 27: launch_sell_one<27, K, U>(op, s); return;
      default: break;
    }
  } else {
    if (epi_code(op) == 0) {
      launch_sell_one<0, K, U>(op, s);
      return;
    }
  }
  launch_sell_one<E_RUNTIME, K, U>(op, s);
}

// SELL shapes (chunks per warp K, entries staged per chunk U): (1,1), (2,1), (4,1), (1,4), (2,2),
// (1,8). Eight entries a round suit matrices with few chunks and long rows (the coarse levels'
// Galerkin operators), where each warp otherwise walks its rows in many dependent rounds.
template <typename TM, typename TX, typename TY>
void launch_sell(const RowOp<TM, TX, TY>& op, int K, int U, cudaStream_t s) {
  if (K >= 4) launch_sell_k<4, 1>(op, s);
  else if (K == 2) U > 1 ? launch_sell_k<2, 2>(op, s) : launch_sell_k<2, 1>(op, s);
  else if (U >= 8) launch_sell_k<1, 8>(op, s);
  else U > 1 ? launch_sell_k<1, 4>(op, s) : launch_sell_k<1, 1>(op, s);
}

template <typename TM, typename TX, typename TY>
void launch_row(const RowOp<TM, TX, TY>& op, int G, cudaStream_t s) {
  if (op.n <= 0) return;
  ++g_launches;
  if (op.v && op.sell.nchunks > 0) {
    launch_sell(op, op.sell_k, op.sell_u, s);
    return;
  }
  if (!op.v) G = 1;
  const int nb = blocks_for((int64_t)op.n * G);
  switch (G) {
    case 1: launch_csr<1>(op, nb, s); break;
    case 2: launch_csr<2>(op, nb, s); break;
    case 4: launch_csr<4>(op, nb, s); break;
    case 8: launch_csr<8>(op, nb, s); break;
    case 16: launch_csr<16>(op, nb, s); break;
    default: launch_csr<32>(op, nb, s); break;
  }
}

template <typename T>
using VC = VRef<const T>;

template <typename T>
inline VC<T> cref(VRef<T> r) {
  VC<T> c;
  c.p = r.p;
  c.sel = r.sel;
  c.ld = r.ld;
  return c;
}
template <typename T>
inline VC<T> cref(const T* p) {
  VC<T> c;
  c.p = p;
  return c;
}

// out = [add +] [scale *] (bscale*base -/+ M src)  -- builders for the common forms
// Matrices of at least this many stored bytes are streamed evict-first through L2 (ld_stream);
// the smaller coarse-level matrices keep the default priority and can stay in L2 from one
// V-cycle to the next.
constexpr int64_t kStreamMatBytes = 32ll << 20;

template <typename TM, typename TX, typename TY>
void set_matrix(RowOp<TM, TX, TY>& op, const DCSR<TM>& M) {
  op.n = M.n;
  op.src_n = M.m;
  op.mat_stream = M.nnz * (int64_t)(sizeof(TM) + sizeof(int)) >= kStreamMatBytes;
  op.rp = M.rp;
  op.ci = M.ci;
  op.v = M.v;
  if (M.use_sell) {
    op.sell.nchunks = M.nchunks;
    op.sell.perm = M.s_perm;
    op.sell.cptr = M.s_cptr;
    op.sell.col = M.s_col;
    op.sell.val = M.s_val;
    op.sell.width = M.s_width;
    op.sell_k = M.sell_k;
    op.sell_u = M.sell_u;
  }
}

template <typename T>
RowOp<T, T, T> op_mat(const DCSR<T>& M, VC<T> src) {
  RowOp<T, T, T> op;
  set_matrix(op, M);
  op.src = src;
  return op;
}

// ------------------------------------------------------------------------------------------
// Levels
// ------------------------------------------------------------------------------------------
template <typename T>
struct Level {
  int n = 0;
  DCSR<T> A;       // A_l
  DCSR<T> L2, U2;  // D^-1 L D^-1, D^-1 U D^-1 (first pass from a zero initial guess)
  DCSR<T> L1, U1;  // D^-1 L, D^-1 U (later passes)
  DCSR<T> P, R;    // prolongation (n x n_c), restriction (n_c x n)
  DCSR<T> iL, iU;  // ILU(0) L_s, U_s
  bool ilu = false;
  T* dinv = nullptr;
  T* dl1inv = nullptr;
  T* idinv = nullptr;
  T* idc = nullptr;  // column scaling applied to the U-series result (ILUT with Ruiz), or null
  T *b = nullptr, *x = nullptr, *r = nullptr, *t1 = nullptr, *t2 = nullptr, *t3 = nullptr;
  char kind = 'p';  // 'p' poly GS, 'i' ILU, 'j' l1-Jacobi
};

}  // namespace

struct nsamg_handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  nsamg_params p{};
  bool fp32 = false;               // FP32 V-cycle (matrices and vectors) inside FP64 GMRES
  std::vector<Level<double>> lv;    // FP64 levels (only level 0's A when fp32)
  std::vector<Level<float>> lv32;   // FP32 levels (fp32 only)
  double* coarse_inv = nullptr;
  float* coarse_inv32 = nullptr;
  int nc = 0;
  // GMRES workspace
  int n = 0, m = 0;
  int64_t ld = 0;
  double* V = nullptr;  // (m+1) columns (FP64 basis: krylov_fp64 = 1)
  float2* Vs = nullptr; // (m+1) columns of (hi, lo) pairs (split basis: krylov_fp64 = 0)
  double* vin = nullptr;  // split basis: the FP64 residual / next V-cycle input
  bool split = false;     // split basis in use
  double* Z = nullptr;  // m columns (FP64 V-cycle)
  float* Z32 = nullptr; // m columns (FP32 V-cycle)
  double* w = nullptr;
  GState* st = nullptr;
  GState* h_st = nullptr;  // pinned host mirror
  Scratch scr{};
  int gram_blocks = 0, update_blocks = 0, stream_blocks = 0;  // stream_blocks: x-update, column 0
  int64_t partial_cap = 0;
  // graph
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  int launches_per_step = 0;
  struct BatchData* batch = nullptr;  // set for handles made by nsamg_batch_setup
  bool shared_mats = false;           // a solver context: matrices belong to another handle
  double anorm_inf = 0.0;             // ||A_0||_inf (for the backward error)
  // fused V-cycle tail (levels >= tail_l0 run by one cluster kernel, or by one cooperative grid
  // kernel when tail_grid); tail_l0 = 0: off
  int tail_l0 = 0;
  int tail_np = 0;
  int tail_ncl = 0;               // cluster tail: CTAs of the cluster
  int tail_grid = 0;              // grid tail: blocks of the cooperative launch (one per SM)
  unsigned long long* tail_ctr = nullptr;  // grid tail: barrier counter (zeroed before each launch)
  void* tail_passes = nullptr;  // TailPass<double> or TailPass<float> array (device)
  size_t ctx_bytes = 0;               // device bytes of the per-solve workspace (server accounting)
};

// Batched solve data: systems concatenated block-diagonally (system s owns rows off[s]..off[s+1]
// of every concatenated vector), per-system GMRES states and per-kernel block tables.
struct BatchData {
  int nsys = 0;
  std::vector<int64_t> off;       // host copy of the row offsets
  int64_t* d_off = nullptr;
  GState* d_st = nullptr;
  GState* h_st = nullptr;         // pinned
  BatchCtl* d_ctl = nullptr;
  BatchCtl* h_ctl = nullptr;      // pinned
  enum { kGram = 0, kUpdate = 1, kX = 2, kResid = 3 };
  int64_t rpb[4] = {8192, 2048, 2048, 256};
  int* d_bstart[4] = {nullptr, nullptr, nullptr, nullptr};
  int nblocks[4] = {0, 0, 0, 0};
  unsigned* d_sticket = nullptr;  // nsys per kernel kind (4 * nsys)
  unsigned* d_gticket = nullptr;  // 4
  double* partials = nullptr;
  // coarse dense blocks (all systems), row -> system map
  int ncrows = 0;
  int* d_row_sys = nullptr;
  int64_t* d_coff = nullptr;
  int64_t* d_cblk = nullptr;
  double* d_cinv = nullptr;
  float* d_cinv32 = nullptr;
};

namespace {

// ------------------------------------------------------------------------------------------
// Smoothers (Sec. 5.2 / 5.3) as sequences of row-kernel launches on one level.
// b, x: level vectors (VRefs so level 0 can address V[:, i] / Z[:, i]); skip: stop flag.
// ------------------------------------------------------------------------------------------
struct Ctx {
  cudaStream_t s;
  const int* skip;
};

// While a fused tail is being recorded, passes are appended here instead of launched.
template <typename T>
std::vector<TailPass<T>>*& tail_recorder() {
  thread_local std::vector<TailPass<T>>* r = nullptr;
  return r;
}

template <typename T>
void run(RowOp<T, T, T> op, int G, const Ctx& c) {
  op.skip = c.skip;
  if (std::vector<TailPass<T>>* rec = tail_recorder<T>()) {
    if (op.n <= 0) return;
    TailPass<T> P;
    P.op = op;
    P.op.skip = nullptr;
    P.G = op.v ? G : 1;
    P.epi = epi_code(op);
    if (op.v && op.sell.nchunks > 0) P.epi = -100;  // SELL layout: not fusable (flags the recording)
    rec->push_back(P);
    return;
  }
  launch_row(op, G, c.s);
}

template <typename T>
RowOp<T, T, T> op_vec(int n) {
  RowOp<T, T, T> op;
  op.n = n;
  return op;
}

// Polynomial Gauss-Seidel with k terms:
//   x <- x + g,  g = sum_{j<k} (-D^-1 T)^j D^-1 r,  r = b - A x,  T = L (forward) or U (backward),
// evaluated by the Jacobi recurrence g_0 = D^-1 r, g_j = D^-1 r - (D^-1 T) g_{j-1}
// (eqs. jr-initial-guess, jr, jacobi). With a zero initial guess r = b and the first pass uses
// the pre-scaled D^-1 T D^-1 so that g_1 = D^-1 b - (D^-1 T D^-1) b needs no separate g_0.
template <typename T>
void sweep_poly(Level<T>& L, VC<T> b, VRef<T> x, bool backward, bool x_zero, int k, const Ctx& c) {
  const DCSR<T>& M2 = backward ? L.U2 : L.L2;
  const DCSR<T>& M1 = backward ? L.U1 : L.L1;
  T* g[2] = {L.t1, L.t2};
  if (x_zero) {
    if (k == 1) {  // x = D^-1 b
      auto op = op_vec<T>(L.n);
      op.base = b;
      op.bscale = L.dinv;
      op.out = x;
      run(op, 1, c);
      return;
    }
    for (int j = 1; j < k; ++j) {
      const bool last = (j == k - 1);
      auto op = (j == 1) ? op_mat(M2, b) : op_mat(M1, cref(g[(j - 1) & 1]));
      op.base = b;
      op.bscale = L.dinv;
      op.neg = 1;
      op.out = last ? x : vref(g[j & 1]);
      run(op, (j == 1 ? M2 : M1).G, c);
    }
    return;
  }
  // r_hat = D^-1 (b - A x)
  {
    auto op = op_mat(L.A, cref(x));
    op.base = b;
    op.neg = 1;
    op.scale = L.dinv;
    op.out = vref(L.r);
    run(op, L.A.G, c);
  }
  if (k == 1) {  // x += r_hat
    auto op = op_vec<T>(L.n);
    op.base = cref((const T*)L.r);
    op.add = cref(x);
    op.out = x;
    run(op, 1, c);
    return;
  }
  for (int j = 1; j < k; ++j) {
    const bool last = (j == k - 1);
    auto op = op_mat(M1, (j == 1) ? cref((const T*)L.r) : cref(g[(j - 1) & 1]));
    op.base = cref((const T*)L.r);
    op.neg = 1;
    if (last) {
      op.add = cref(x);
      op.out = x;
    } else {
      op.out = vref(g[j & 1]);
    }
    run(op, M1.G, c);
  }
}

// ILU(0) smoother with Neumann-series triangular solves (Sec. 5.3.2, eq. Neumann; Algorithm 2
// with row scaling): x <- x + sum_{j<tU} (-U_s)^j D_U^-1 sum_{j<tL} (-L_s)^j r, r = b - A x,
// evaluated as y_1 = r, y_j = r - L_s y_{j-1}; f = D_U^-1 y; v_1 = f, v_j = f - U_s v_{j-1}.
template <typename T>
void sweep_ilu(Level<T>& L, VC<T> b, VRef<T> x, bool x_zero, int tL, int tU, const Ctx& c) {
  VC<T> r = b;
  if (!x_zero) {
    auto op = op_mat(L.A, cref(x));
    op.base = b;
    op.neg = 1;
    op.out = vref(L.r);
    run(op, L.A.G, c);
    r = cref((const T*)L.r);
  }
  T* y[2] = {L.t1, L.t2};
  T* f = L.t3;
  if (tL == 1) {
    auto op = op_vec<T>(L.n);
    op.base = r;
    op.bscale = L.idinv;
    op.out = vref(f);
    run(op, 1, c);
  } else {
    for (int j = 2; j <= tL; ++j) {
      const bool last = (j == tL);
      auto op = op_mat(L.iL, (j == 2) ? r : cref((const T*)y[j & 1]));
      op.base = r;
      op.neg = 1;
      if (last) {
        op.scale = L.idinv;
        op.out = vref(f);
      } else {
        op.out = vref(y[(j + 1) & 1]);
      }
      run(op, L.iL.G, c);
    }
  }
  if (tU == 1) {
    auto op = op_vec<T>(L.n);
    op.base = cref((const T*)f);
    op.bscale = L.idc;
    if (!x_zero) op.add = cref(x);
    op.out = x;
    run(op, 1, c);
    return;
  }
  for (int j = 2; j <= tU; ++j) {
    const bool last = (j == tU);
    auto op = op_mat(L.iU, (j == 2) ? cref((const T*)f) : cref((const T*)y[j & 1]));
    op.base = cref((const T*)f);
    op.neg = 1;
    if (last) {
      op.scale = L.idc;  // x (+)= D_c v for ILUT with Ruiz scaling
      if (!x_zero) op.add = cref(x);
      op.out = x;
    } else {
      op.out = vref(y[(j + 1) & 1]);
    }
    run(op, L.iU.G, c);
  }
}

// l1-Jacobi: x <- x + D_l1^-1 (b - A x), d_ii = sum_j |a_ij|. `nsw` sweeps, ping-ponging with t1
// so that the last sweep lands in x.
template <typename T>
void sweep_jacobi(Level<T>& L, VC<T> b, VRef<T> x, bool x_zero, int nsw, const Ctx& c) {
  VRef<T> prev;
  for (int s = 0; s < nsw; ++s) {
    const bool to_x = ((nsw - 1 - s) % 2) == 0;
    VRef<T> dst = to_x ? x : vref(L.t1);
    if (s == 0 && x_zero) {
      auto op = op_vec<T>(L.n);
      op.base = b;
      op.bscale = L.dl1inv;
      op.out = dst;
      run(op, 1, c);
    } else {
      VRef<T> src = (s == 0) ? x : prev;
      if (s == 0) {
        // first sweep with a nonzero x: cannot update in place; go through t1 then back
        dst = to_x ? vref(L.t2) : vref(L.t1);
      }
      auto op = op_mat(L.A, cref(src));
      op.base = b;
      op.neg = 1;
      op.scale = L.dl1inv;
      op.add = cref(src);
      op.out = dst;
      run(op, L.A.G, c);
      if (s == 0 && to_x) {  // copy t2 -> x (only when a single in-place sweep is requested)
        auto cp = op_vec<T>(L.n);
        cp.base = cref(dst);
        cp.out = x;
        run(cp, 1, c);
        dst = x;
      }
    }
    prev = dst;
  }
}

template <typename T>
void smooth(nsamg_handle* h, Level<T>& L, VC<T> b, VRef<T> x, bool backward, bool x_zero, int sweeps, const Ctx& c) {
  if (sweeps <= 0) return;
  if (L.kind == 'j') {
    sweep_jacobi(L, b, x, x_zero, sweeps, c);
    return;
  }
  for (int s = 0; s < sweeps; ++s) {
    const bool z = x_zero && s == 0;
    if (L.kind == 'i') sweep_ilu(L, b, x, z, h->p.ilu_terms_L, h->p.ilu_terms_U, c);
    else sweep_poly(L, b, x, backward, z, h->p.neumann_terms, c);
  }
}

inline const double* coarse_ptr(nsamg_handle* h, double*) { return h->coarse_inv; }
inline const float* coarse_ptr(nsamg_handle* h, float*) { return h->coarse_inv32; }

inline const double* bcoarse_ptr(BatchData* B, double*) { return B->d_cinv; }
inline const float* bcoarse_ptr(BatchData* B, float*) { return B->d_cinv32; }

template <typename T>
void coarse_solve(nsamg_handle* h, Level<T>& L, VC<T> b, VRef<T> x, const Ctx& c) {
  const T* C = coarse_ptr(h, (T*)nullptr);
  if (h->batch && bcoarse_ptr(h->batch, (T*)nullptr)) {
    BatchData* B = h->batch;
    ++g_launches;
    const int nb = (B->ncrows * 32 + kThreads - 1) / kThreads;
    launch_k(k_bdense_gemv<T, T>, nb, kThreads, c.s, B->ncrows, B->d_row_sys, B->d_coff, B->d_cblk,
                                                  bcoarse_ptr(B, (T*)nullptr), b, x, c.skip);
  } else if (C) {
    if (std::vector<TailPass<T>>* rec = tail_recorder<T>()) {
      TailPass<T> P;
      P.dense = 1;
      P.C = C;
      P.op.n = L.n;
      P.op.src_n = L.n;
      P.op.src = b;
      P.op.out = x;
      rec->push_back(P);
      return;
    }
    ++g_launches;
    const int nb = (L.n * 32 + kThreads - 1) / kThreads;
    launch_k(k_dense_gemv<T, T>, nb, kThreads, c.s, L.n, C, b, x, c.skip);
  } else {
    smooth(h, L, b, x, false, true, h->p.coarse_sweeps, c);
  }
}

// One V-cycle with zero initial guess on level l (Sec. 5): pre-smooth, residual, restrict,
// recurse, prolongate and correct, post-smooth.
template <typename T>
void launch_tail(nsamg_handle* h, const Ctx& c) {
  ++g_launches;
  if (h->tail_grid) {  // cooperative: every block resident, so the grid barrier can complete
    cudaMemsetAsync(h->tail_ctr, 0, sizeof(unsigned long long), c.s);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(h->tail_grid);
    cfg.blockDim = dim3(kGridTailThreads);
    cfg.stream = c.s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_tail_grid<T>, (const TailPass<T>*)h->tail_passes, h->tail_np, c.skip, h->tail_ctr,
                       &h->st->status, kGridSpinLimit);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(h->tail_ncl);
  cfg.blockDim = dim3(kTailThreads);
  cfg.dynamicSmemBytes = sizeof(T) * kTailStage;
  cfg.stream = c.s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = h->tail_ncl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 2 : 1;
  cudaLaunchKernelEx(&cfg, k_tail<T>, (const TailPass<T>*)h->tail_passes, h->tail_np, c.skip);
}

template <typename T>
void vcycle(nsamg_handle* h, std::vector<Level<T>>& lv, int l, VC<T> b, VRef<T> x, const Ctx& c) {
  Level<T>& L = lv[l];
  if (l > 0 && l == h->tail_l0 && h->tail_passes && !tail_recorder<T>()) {
    launch_tail<T>(h, c);  // every pass of levels >= l in one cluster kernel
    return;
  }
  if (l == (int)lv.size() - 1) {
    coarse_solve(h, L, b, x, c);
    return;
  }
  Level<T>& C = lv[l + 1];
  const int pre = h->p.pre_sweeps, post = h->p.post_sweeps;
  if (pre > 0) {
    smooth(h, L, b, x, false, true, pre, c);
    auto op = op_mat(L.A, cref(x));  // r = b - A x
    op.base = b;
    op.neg = 1;
    op.out = vref(L.r);
    run(op, L.A.G, c);
    auto rs = op_mat(L.R, cref((const T*)L.r));  // b_c = R r
    rs.out = vref(C.b);
    run(rs, L.R.G, c);
  } else {
    auto rs = op_mat(L.R, b);  // x = 0: r = b
    rs.out = vref(C.b);
    run(rs, L.R.G, c);
  }
  vcycle(h, lv, l + 1, cref((const T*)C.b), vref(C.x), c);
  {
    auto op = op_mat(L.P, cref((const T*)C.x));  // x += P e  (x = P e when no pre-smoothing)
    if (pre > 0) op.add = cref(x);
    op.out = x;
    run(op, L.P.G, c);
  }
  smooth(h, L, b, x, true, false, post, c);
}

// ------------------------------------------------------------------------------------------
// Autotuning of threads-per-row for large CSR matrices (timed SpMV with each group size).
// ------------------------------------------------------------------------------------------
// Read sweep over a buffer larger than L2 (no writes: it leaves no dirty lines behind).
__global__ void k_l2_sweep(const double* __restrict__ buf, int64_t n, double* __restrict__ sink) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += buf[i];
  if (acc == -1.0) *sink = acc;  // never true for the zero buffer; keeps the loads
}

struct TuneScratch {
  double* buf = nullptr;
  int64_t n = 0;
  double* sink = nullptr;
  int blocks = 592;
};

// One launch timed after L2 has been swept, as in a V-cycle where the other passes have evicted
// the matrix (a matrix smaller than L2 would otherwise be timed from cache).
template <typename T>
float time_spmv_once(DCSR<T>& M, T* x, T* y, int G, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1,
                     const TuneScratch& fl) {
  auto op = op_mat(M, cref((const T*)x));
  op.out = vref(y);
  if (fl.buf) k_l2_sweep<<<fl.blocks, 256, 0, s>>>(fl.buf, fl.n, fl.sink);
  cudaEventRecord(e0, s);
  launch_row(op, G, s);
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  return ms;
}

// Timed choice among CSR with G = 1, 2, ..., 32 threads per row and the SELL shapes of
// launch_sell. The candidates are timed in interleaved rounds (each round times every candidate
// once, after an L2 sweep), so that a clock or neighbour change during tuning shifts all of them
// alike; each keeps its best of kTuneRounds. A later candidate must beat the best earlier one by
// more than kTuneMargin to be chosen, so shapes the timing cannot separate resolve to the
// simpler one (CSR before SELL, fewer threads, fewer chunks a warp) the same way on every run.
constexpr int kTuneRounds = 9;
constexpr float kTuneMargin = 0.015f;

template <typename T>
int tune(DCSR<T>& M, T* x, T* y, cudaStream_t s, const TuneScratch& fl) {
  if (M.n < 20000 || M.nnz == 0) return NSAMG_OK;
  struct Cand {
    int G, K, U;  // K = 0: CSR with G threads a row; else SELL with K chunks a warp, U-way unrolled
    float best;
  };
  Cand cands[16];
  int nc = 0;
  const double avg = (double)M.nnz / M.n;
  for (int G : {1, 2, 4, 8, 16, 32}) {
    if (G > 2 * avg + 2) break;
    cands[nc++] = {G, 0, 1, 1e30f};
  }
  if (M.nchunks > 0)
    for (const auto& ku : {std::pair<int, int>{1, 1}, {2, 1}, {4, 1}, {1, 4}, {2, 2}, {1, 8}})
      cands[nc++] = {1, ku.first, ku.second, 1e30f};
  auto apply = [&M](const Cand& c) {
    M.use_sell = c.K > 0;
    if (c.K) {
      M.sell_k = c.K;
      M.sell_u = c.U;
    } else {
      M.G = c.G;
    }
  };
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (int c = 0; c < nc; ++c) {  // one untimed launch of each shape (instruction cache, first-launch cost)
    apply(cands[c]);
    time_spmv_once(M, x, y, cands[c].G, s, e0, e1, TuneScratch{});
  }
  for (int round = 0; round < kTuneRounds; ++round)
    for (int c = 0; c < nc; ++c) {
      apply(cands[c]);
      cands[c].best = std::min(cands[c].best, time_spmv_once(M, x, y, cands[c].G, s, e0, e1, fl));
    }
  int pick = 0;
  for (int c = 1; c < nc; ++c)
    if (cands[c].best < cands[pick].best * (1.f - kTuneMargin)) pick = c;
  int pick_csr = 0;  // the CSR group kept for passes that take the CSR arrays of a SELL matrix
  for (int c = 1; c < nc && cands[c].K == 0; ++c)
    if (cands[c].best < cands[pick_csr].best * (1.f - kTuneMargin)) pick_csr = c;
  apply(cands[pick_csr]);
  apply(cands[pick]);
  CK(cudaGetLastError());
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return NSAMG_OK;
}

// Brings the GPU to its working clock before timed tuning (an idle GPU ramps up over the first
// milliseconds of work, which would bias the first candidates).
template <typename T>
void tune_warmup(DCSR<T>& M, T* x, T* y, cudaStream_t s) {
  if (M.n == 0) return;
  auto op = op_mat(M, cref((const T*)x));
  op.out = vref(y);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float total = 0.f;
  for (int it = 0; it < 200 && total < 30.f; ++it) {
    cudaEventRecord(e0, s);
    for (int r = 0; r < 10; ++r) launch_row(op, M.G, s);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    total += ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

// ------------------------------------------------------------------------------------------
// One Arnoldi step (Algorithm 1 steps 5-14) on the handle's stream.
// ------------------------------------------------------------------------------------------
void enqueue_step(nsamg_handle* h, cudaStream_t s, unsigned long long cond_inner) {
  const int* skip = &h->st->stop;
  const int* sel = &h->st->i;
  Ctx c{s, skip};
  VRef<const double> b;
  if (h->split) {  // split basis: the V-cycle input vt_i is the FP64 vector vin
    b.p = h->vin;
  } else {
    b.p = h->V;
    b.sel = sel;
    b.ld = h->ld;
  }
  if (!h->fp32) {
    VRef<double> z;
    z.p = h->Z;
    z.sel = sel;
    z.ld = h->ld;
    vcycle(h, h->lv, 0, b, z, c);  // z_i = M^-1 vt_i
    auto op = op_mat(h->lv[0].A, cref(z));  // w = A z_i
    op.out = vref(h->w);
    run(op, h->lv[0].A.G, c);
  } else {
    // FP32 V-cycle: vt_i rounded to FP32 (round to nearest; the kernel that produced vt_i wrote
    // this copy into the level's input), z_i kept in FP32 (flexible GMRES stores Z), outer product
    // w = A z_i with the FP64 matrix, z widened exactly in registers by integer operations.
    Level<float>& L0 = h->lv32[0];
    VRef<float> z;
    z.p = h->Z32;
    z.sel = sel;
    z.ld = h->ld;
    vcycle(h, h->lv32, 0, cref((const float*)L0.b), z, c);
    const auto& A = h->lv[0].A;
    RowOp<double, float, double> op;
    set_matrix(op, A);
    op.src = cref(z);
    op.out = vref(h->w);
    op.skip = skip;
    launch_row(op, A.G, s);
  }
  GramArgs ga{};
  ga.n = h->n;
  ga.V = h->V;
  ga.Vs = h->Vs;
  ga.ldv = h->ld;
  ga.w = h->w;
  ga.st = h->st;
  ga.scr = h->scr;
  if (h->split) launch_k_smem(k_gram_s, h->gram_blocks, kGramTmaThreads, kGramSSmem, s, ga);
  else launch_k(k_gram, h->gram_blocks, kGramThreads, s, ga);
  g_launches += 2;
  UpdateArgs ua{};
  ua.n = h->n;
  ua.V = h->V;
  ua.ldv = h->ld;
  ua.w = h->w;
  ua.st = h->st;
  ua.cond_inner = cond_inner;
  ua.scr = h->scr;
  ua.scr.ticket = h->scr.ticket + 1;
  ua.v32 = h->fp32 ? h->lv32[0].b : nullptr;
  ua.Vs = h->Vs;
  ua.vin = h->fp32 ? nullptr : h->vin;
  if (h->split) launch_k_smem(k_update_s, h->update_blocks, kGramTmaThreads, kGramTmaSmem, s, ua);
  else launch_k(k_update, h->update_blocks, kRedThreads, s, ua);
}

void enqueue_xupdate(nsamg_handle* h, cudaStream_t s) {
  ++g_launches;
  if (h->fp32) launch_k(k_xupdate<float>, h->stream_blocks, kRedThreads, s, h->n, h->Z32, h->ld, h->st);
  else launch_k(k_xupdate<double>, h->stream_blocks, kRedThreads, s, h->n, h->Z, h->ld, h->st);
}

void enqueue_resid(nsamg_handle* h, cudaStream_t s, int init, unsigned long long co, unsigned long long ci) {
  const auto& A = h->lv[0].A;
  ResidArgs ra{};
  ra.n = A.n;
  ra.rp = A.rp;
  ra.ci = A.ci;
  ra.v = A.v;
  ra.r = h->split ? h->vin : h->V;
  ra.r32 = (h->fp32 && !h->split) ? h->lv32[0].b : nullptr;
  ra.st = h->st;
  ra.init = init;
  ra.cond_outer = co;
  ra.cond_inner = ci;
  ra.scr = h->scr;
  ra.scr.ticket = h->scr.ticket + 2;
  const int G = A.G;
  const int nb = blocks_for((int64_t)A.n * G);
  ++g_launches;
  switch (G) {
    case 1: launch_k(k_resid<1>, nb, kRedThreads, s, ra); break;
    case 2: launch_k(k_resid<2>, nb, kRedThreads, s, ra); break;
    case 4: launch_k(k_resid<4>, nb, kRedThreads, s, ra); break;
    case 8: launch_k(k_resid<8>, nb, kRedThreads, s, ra); break;
    case 16: launch_k(k_resid<16>, nb, kRedThreads, s, ra); break;
    default: launch_k(k_resid<32>, nb, kRedThreads, s, ra); break;
  }
  if (h->split) {  // column 0 of the next cycle (returns at once when the solve is done)
    Col0Args c0{};
    c0.n = h->n;
    c0.r = h->vin;
    c0.r32 = h->fp32 ? h->lv32[0].b : nullptr;
    c0.col = h->Vs;
    c0.st = h->st;
    ++g_launches;
    launch_k(k_col0, h->stream_blocks, kRedThreads, s, c0);
  }
}

// ||S_k||_2 of every solve's last cycle (one block per system).
void enqueue_sknorm(nsamg_handle* h, cudaStream_t s) {
  ++g_launches;
  if (h->batch)
    launch_k(k_sknorm_states, h->batch->nsys, kSkThreads, s, h->batch->d_st);
  else
    launch_k(k_sknorm_states, 1, kSkThreads, s, h->st);
}

using ResidFn = std::function<void(cudaStream_t, int, unsigned long long, unsigned long long)>;
using StepFn = std::function<void(cudaStream_t, unsigned long long)>;
using XFn = std::function<void(cudaStream_t)>;

// One CUDA graph per solve: init residual -> WHILE(outer) { WHILE(inner) { step }, x-update,
// residual }. Kernels set the two conditions from the device.
int build_graph_fn(nsamg_handle* h, const ResidFn& enq_resid, const StepFn& enq_step, const XFn& enq_x,
                   const XFn& enq_final) {
  cudaStream_t cs;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g;
  CK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle hout, hin;
  CK(cudaGraphConditionalHandleCreate(&hout, g, 0, 0));
  CK(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  enq_resid(cs, 1, (unsigned long long)hout, 0ull);
  CK(cudaStreamEndCapture(cs, &g));
  size_t nn = 0;
  CK(cudaGraphGetNodes(g, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  CK(cudaGraphGetNodes(g, nodes.data(), &nn));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hout;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t outer;
  CK(cudaGraphAddNode(&outer, g, nodes.data(), nullptr, nn, &cp));
  cudaGraph_t outer_body = cp.conditional.phGraph_out[0];
  CK(cudaGraphConditionalHandleCreate(&hin, outer_body, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams ip = {};
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = hin;
  ip.conditional.type = cudaGraphCondTypeWhile;
  ip.conditional.size = 1;
  cudaGraphNode_t inner;
  CK(cudaGraphAddNode(&inner, outer_body, nullptr, nullptr, 0, &ip));
  cudaGraph_t inner_body = ip.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(cs, inner_body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  const int64_t before = g_launches;
  enq_step(cs, (unsigned long long)hin);
  h->launches_per_step = (int)(g_launches - before);
  CK(cudaStreamEndCapture(cs, &inner_body));
  CK(cudaStreamBeginCaptureToGraph(cs, outer_body, &inner, nullptr, 1, cudaStreamCaptureModeThreadLocal));
  enq_x(cs);
  enq_resid(cs, 0, (unsigned long long)hout, (unsigned long long)hin);
  CK(cudaStreamEndCapture(cs, &outer_body));
  // after the last cycle: the per-solve diagnostics
  CK(cudaStreamBeginCaptureToGraph(cs, g, &outer, nullptr, 1, cudaStreamCaptureModeThreadLocal));
  enq_final(cs);
  CK(cudaStreamEndCapture(cs, &g));
  CK(cudaGraphInstantiate(&h->exec, g, 0));
  h->graph = g;
  cudaStreamDestroy(cs);
  return NSAMG_OK;
}

int build_graph(nsamg_handle* h) {
  return build_graph_fn(
      h, [h](cudaStream_t s, int init, unsigned long long co, unsigned long long ci) { enqueue_resid(h, s, init, co, ci); },
      [h](cudaStream_t s, unsigned long long ci) { enqueue_step(h, s, ci); }, [h](cudaStream_t s) { enqueue_xupdate(h, s); },
      [h](cudaStream_t s) { enqueue_sknorm(h, s); });
}

// ------------------------------------------------------------------------------------------
// Batched solve: one lock-step Arnoldi step for all systems, x-update, residual.
// ------------------------------------------------------------------------------------------
BatchArgs batch_args(nsamg_handle* h, int kind, unsigned long long co, unsigned long long ci) {
  BatchData* B = h->batch;
  BatchArgs a{};
  a.nsys = B->nsys;
  a.off = B->d_off;
  a.bstart = B->d_bstart[kind];
  a.rpb = B->rpb[kind];
  a.st = B->d_st;
  a.ctl = B->d_ctl;
  a.V = h->V;
  a.ldv = h->ld;
  a.w = h->w;
  a.partials = B->partials;
  a.sticket = B->d_sticket + (int64_t)kind * B->nsys;
  a.gticket = B->d_gticket + kind;
  a.cond_outer = co;
  a.cond_inner = ci;
  if (h->split) {
    a.Vs = h->Vs;
    a.vin = h->vin;
    a.v32 = h->fp32 ? h->lv32[0].b : nullptr;
  }
  return a;
}

void enqueue_bstep(nsamg_handle* h, cudaStream_t s, unsigned long long cond_inner) {
  BatchData* B = h->batch;
  const int* sel = &B->d_ctl->gi;
  Ctx c{s, nullptr};
  VRef<const double> b;
  if (h->split) {  // split basis: the V-cycle input vt_i is the FP64 vector vin (FP32: level 0's b)
    b.p = h->vin;
  } else {
    b.p = h->V;
    b.sel = sel;
    b.ld = h->ld;
  }
  if (!h->fp32) {
    VRef<double> z;
    z.p = h->Z;
    z.sel = sel;
    z.ld = h->ld;
    vcycle(h, h->lv, 0, b, z, c);
    auto op = op_mat(h->lv[0].A, cref(z));
    op.out = vref(h->w);
    run(op, h->lv[0].A.G, c);
  } else {
    Level<float>& L0 = h->lv32[0];
    if (!h->split) {  // the split kernels write the FP32 input themselves
      ++g_launches;
      launch_k(k_cast<double, float>, 8 * 148, kThreads, s, h->n, b, vref(L0.b), nullptr);
    }
    VRef<float> z;
    z.p = h->Z32;
    z.sel = sel;
    z.ld = h->ld;
    vcycle(h, h->lv32, 0, cref((const float*)L0.b), z, c);
    const auto& A = h->lv[0].A;
    RowOp<double, float, double> op;  // z widened exactly in registers
    set_matrix(op, A);
    op.src = cref(z);
    op.out = vref(h->w);
    launch_row(op, A.G, s);
  }
  g_launches += 2;
  if (h->split) {
    launch_k(k_bgram_s, B->nblocks[BatchData::kGram], kGramThreads, s, batch_args(h, BatchData::kGram, 0, 0));
    launch_k(k_bupdate_s, B->nblocks[BatchData::kUpdate], kRedThreads, s,
             batch_args(h, BatchData::kUpdate, 0, cond_inner));
  } else {
    launch_k(k_bgram, B->nblocks[BatchData::kGram], kGramThreads, s, batch_args(h, BatchData::kGram, 0, 0));
    launch_k(k_bupdate, B->nblocks[BatchData::kUpdate], kRedThreads, s, batch_args(h, BatchData::kUpdate, 0, cond_inner));
  }
}

void enqueue_bxupdate(nsamg_handle* h, cudaStream_t s) {
  BatchData* B = h->batch;
  ++g_launches;
  if (h->fp32)
    launch_k(k_bxupdate<float>, B->nblocks[BatchData::kX], kRedThreads, s, batch_args(h, BatchData::kX, 0, 0), h->Z32, h->ld);
  else
    launch_k(k_bxupdate<double>, B->nblocks[BatchData::kX], kRedThreads, s, batch_args(h, BatchData::kX, 0, 0), h->Z, h->ld);
}

void enqueue_bresid(nsamg_handle* h, cudaStream_t s, int init, unsigned long long co, unsigned long long ci) {
  BatchData* B = h->batch;
  const auto& A = h->lv[0].A;
  BResidArgs ra{};
  ra.ba = batch_args(h, BatchData::kResid, co, ci);
  ra.rp = A.rp;
  ra.ci = A.ci;
  ra.v = A.v;
  ra.init = init;
  if (h->split) ra.ba.V = h->vin;  // the residual goes to vin; k_bcol0 scales and splits it
  ++g_launches;
  launch_k(k_bresid, B->nblocks[BatchData::kResid], kRedThreads, s, ra);
  if (h->split) {
    ++g_launches;
    launch_k(k_bcol0, B->nblocks[BatchData::kX], kRedThreads, s, batch_args(h, BatchData::kX, 0, 0));
  }
}

int check_params(const nsamg_params& p) {
  if (p.smoother < 0 || p.smoother > 3) return fail(NSAMG_ERR_INVALID_ARG, "unknown smoother");
  if (p.neumann_terms < 1 || p.ilu_terms_L < 1 || p.ilu_terms_U < 1) return fail(NSAMG_ERR_INVALID_ARG, "series terms must be >= 1");
  if (p.pre_sweeps < 0 || p.post_sweeps < 0 || p.coarse_sweeps < 1) return fail(NSAMG_ERR_INVALID_ARG, "bad sweep counts");
  if (p.restart < 1 || p.restart > NSAMG_MAX_RESTART) return fail(NSAMG_ERR_INVALID_ARG, "restart out of range 1..64");
  if (p.vcycle_fp32 != 0 && p.vcycle_fp32 != 1) return fail(NSAMG_ERR_INVALID_ARG, "vcycle_fp32 must be 0 or 1");
  if (p.t_exact != 0 && p.t_exact != 1) return fail(NSAMG_ERR_INVALID_ARG, "t_exact must be 0 or 1");
  if (p.use_graph != 0 && p.use_graph != 1) return fail(NSAMG_ERR_INVALID_ARG, "use_graph must be 0 or 1");
  if (p.spmv_group < -1 || p.spmv_group > 32 || (p.spmv_group > 0 && (p.spmv_group & (p.spmv_group - 1))))
    return fail(NSAMG_ERR_INVALID_ARG, "spmv_group must be -1, 0 or a power of two <= 32");
  if (p.sell_shape != 0 && p.sell_shape != 11 && p.sell_shape != 21 && p.sell_shape != 41 && p.sell_shape != 14 &&
      p.sell_shape != 22 && p.sell_shape != 18)
    return fail(NSAMG_ERR_INVALID_ARG, "sell_shape must be 0, 11, 21, 41, 14, 18 or 22");
  if (p.fuse_tail < 0 || p.fuse_tail > 2) return fail(NSAMG_ERR_INVALID_ARG, "fuse_tail must be 0, 1 or 2");
  if (p.krylov_fp64 != 0 && p.krylov_fp64 != 1) return fail(NSAMG_ERR_INVALID_ARG, "krylov_fp64 must be 0 or 1");
  if (p.stop_nrbe != 0 && p.stop_nrbe != 1) return fail(NSAMG_ERR_INVALID_ARG, "stop_nrbe must be 0 or 1");
  if (p.ranks < 1 || p.ranks > (1 << 20)) return fail(NSAMG_ERR_INVALID_ARG, "ranks must be in 1..2^20");
  return NSAMG_OK;
}

template <typename T>
int alloc_vec(T** p, int64_t n) {
  CK(cudaMalloc(p, sizeof(T) * std::max<int64_t>(n, 1)));
  CK(cudaMemset(*p, 0, sizeof(T) * std::max<int64_t>(n, 1)));
  return NSAMG_OK;
}

// Upload every level of the host hierarchy at precision T (matrix values and vectors): A, the
// pre-scaled triangles of A for polynomial GS, D^-1, the l1 diagonal, P, R and, where the
// smoother uses it, the ILU(0) factors. `only_A0` uploads just the finest A (the FP64 operator
// of an FP32-V-cycle handle).
// Runs independent host preparation + upload jobs in parallel host threads (each on the caller's
// device); returns the first failure with its message.
int run_parallel(std::vector<std::function<int()>>& jobs) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  std::vector<int> rcs(jobs.size(), NSAMG_OK);
  std::vector<std::string> errs(jobs.size());
  std::vector<std::thread> th;
  th.reserve(jobs.size());
  for (size_t k = 0; k < jobs.size(); ++k)
    th.emplace_back([&, k] {
      cudaSetDevice(dev);
      rcs[k] = jobs[k]();
      if (rcs[k] != NSAMG_OK) errs[k] = g_err;
    });
  for (auto& t : th) t.join();
  for (size_t k = 0; k < jobs.size(); ++k)
    if (rcs[k] != NSAMG_OK) return fail(rcs[k], errs[k]);
  return NSAMG_OK;
}

template <typename T>
int build_levels(const nsamg_hierarchy_desc* H, const nsamg_params& p, std::vector<Level<T>>& lvs, bool only_A0) {
  int rc;
  const int nl = only_A0 ? 1 : H->nlevels;
  lvs.resize(nl);
  for (int l = 0; l < nl; ++l) {
    const nsamg_level_desc& D = H->levels[l];
    Level<T>& L = lvs[l];
    L.n = D.A.nrows;
    if (only_A0) return upload(D.A, L.A);
    std::vector<double> dinv(L.n), dl1(L.n);
    for (int i = 0; i < L.n; ++i) {
      double a = 0, s1 = 0;
      for (int q = D.A.rowptr[i]; q < D.A.rowptr[i + 1]; ++q) {
        if (D.A.col[q] == i) a = D.A.val[q];
        s1 += std::fabs(D.A.val[q]);
      }
      dinv[i] = 1.0 / a;
      dl1[i] = 1.0 / s1;
    }
    if ((rc = upload_vec(dinv, &L.dinv))) return rc;
    if ((rc = upload_vec(dl1, &L.dl1inv))) return rc;
    // the level's matrices are independent: derived copies (scaled triangles), SELL arrays and
    // uploads run in parallel host threads
    std::vector<std::function<int()>> jobs;
    jobs.push_back([&] { return upload(D.A, L.A); });
    const int rk = p.ranks;
    jobs.push_back([&] { return upload(tri_part(D.A, true, &dinv, &dinv, rk), L.L2); });
    jobs.push_back([&] { return upload(tri_part(D.A, false, &dinv, &dinv, rk), L.U2); });
    jobs.push_back([&] { return upload(tri_part(D.A, true, &dinv, nullptr, rk), L.L1); });
    jobs.push_back([&] { return upload(tri_part(D.A, false, &dinv, nullptr, rk), L.U1); });
    if (l < nl - 1) {
      jobs.push_back([&] { return upload(D.P, L.P); });
      jobs.push_back([&] { return upload(D.R, L.R); });
    }
    const bool want_ilu = (p.smoother == NSAMG_SMOOTHER_ILU0) || (p.smoother == NSAMG_SMOOTHER_HYBRID_ILU0 && l == 0);
    const bool ilu_here = want_ilu && D.ilu_L.nrows > 0 && l < nl - 1;
    if (ilu_here) {
      jobs.push_back([&] { return upload(D.ilu_L, L.iL); });
      if (D.ilu_form == 0) jobs.push_back([&] { return upload(D.ilu_U, L.iU); });
    }
    if ((rc = run_parallel(jobs))) return rc;
    if (ilu_here) {
      if (D.ilu_form == 0) {
        std::vector<double> idv(D.ilu_dinv, D.ilu_dinv + L.n);
        if ((rc = upload_vec(idv, &L.idinv))) return rc;
      } else {
        // Algorithm 2: Jacobi on U~ = D_r U D_c with D = diag(U~)^-1, i.e. v <- D D_r y - (D U~_strict) v,
        // then x += D_c v. Pre-scale here: U_hat = D U~_strict, f-scaling D D_r, column scaling D_c.
        const nsamg_csr& U = D.ilu_U;
        std::vector<double> dr(L.n, 1.0), dc(L.n, 1.0), fs(L.n), dg(L.n, 0.0);
        if (D.ilu_dr) dr.assign(D.ilu_dr, D.ilu_dr + L.n);
        if (D.ilu_dc) dc.assign(D.ilu_dc, D.ilu_dc + L.n);
        HostCSR uh;
        uh.n = uh.m = L.n;
        uh.rp.assign(L.n + 1, 0);
        for (int i = 0; i < L.n; ++i) {
          for (int64_t q = U.rowptr[i]; q < U.rowptr[i + 1]; ++q)
            if (U.col[q] == i) dg[i] = dr[i] * U.val[q] * dc[i];
          if (dg[i] == 0.0) return fail(NSAMG_ERR_BAD_MATRIX, "level " + std::to_string(l) + ": zero diagonal in the ILUT factor U");
          fs[i] = dr[i] / dg[i];
          for (int64_t q = U.rowptr[i]; q < U.rowptr[i + 1]; ++q) {
            const int j = U.col[q];
            if (j <= i) continue;
            uh.ci.push_back(j);
            uh.v.push_back(dr[i] * U.val[q] * dc[j] / dg[i]);
          }
          uh.rp[i + 1] = (int)uh.ci.size();
        }
        if ((rc = upload(uh, L.iU))) return rc;
        if ((rc = upload_vec(fs, &L.idinv))) return rc;
        if ((rc = upload_vec(dc, &L.idc))) return rc;
      }
      L.ilu = true;
    }
    L.kind = (p.smoother == NSAMG_SMOOTHER_JACOBI_L1) ? 'j' : (L.ilu ? 'i' : 'p');
    T** vecs[] = {&L.b, &L.x, &L.r, &L.t1, &L.t2, &L.t3};
    for (T** v : vecs)
      if ((rc = alloc_vec(v, L.n))) return rc;
  }
  return NSAMG_OK;
}

template <typename T>
int tune_levels(std::vector<Level<T>>& lvs, T* big_x, T* big_y, int group, int shape, cudaStream_t s) {
  int rc;
  const bool timed = group == 0 && !lvs.empty() && lvs[0].A.n >= 20000;
  if (timed) tune_warmup(lvs[0].A, big_x, big_y, s);
  // L2 sweep buffer (twice the L2 size) for the timed candidates; freed on return
  TuneScratch fl;
  struct FreeScratch {
    TuneScratch& f;
    ~FreeScratch() {
      cudaFree(f.buf);
      cudaFree(f.sink);
    }
  } free_scratch{fl};
  if (timed) {
    int dev = 0, l2 = 0, sms = 148;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    fl.n = std::max<int64_t>(2 * (int64_t)l2 / (int64_t)sizeof(double), 1 << 20);
    fl.blocks = 4 * sms;
    CK(cudaMalloc(&fl.buf, sizeof(double) * fl.n));
    CK(cudaMemsetAsync(fl.buf, 0, sizeof(double) * fl.n, s));
    CK(cudaMalloc(&fl.sink, sizeof(double)));
  }
  for (auto& L : lvs) {
    DCSR<T>* mats[] = {&L.A, &L.L2, &L.U2, &L.L1, &L.U1, &L.P, &L.R, &L.iL, &L.iU};
    for (DCSR<T>* M : mats) {
      if (!M->present()) continue;
      if (group == -1) {  // SELL wherever the matrix has it (the given shape), default CSR shape elsewhere
        M->use_sell = M->nchunks > 0;
        M->sell_k = shape ? shape / 10 : 1;
        M->sell_u = shape ? shape % 10 : 1;
        continue;
      }
      if (group) {
        M->G = group;
        continue;
      }
      T* x = (M->m <= L.n && L.t1) ? L.t1 : big_x;
      T* y = (M->n <= L.n && L.t2) ? L.t2 : big_y;
      if (M == &L.R) { x = L.t1; y = big_y; }
      if (M == &L.P) { x = big_x; y = L.t2; }
      if ((rc = tune(*M, x, y, s, fl))) return rc;
    }
  }
  return NSAMG_OK;
}

template <typename T>
void release_level_vectors(std::vector<Level<T>>& lvs) {
  for (auto& L : lvs) {
    T* vecs[] = {L.b, L.x, L.r, L.t1, L.t2, L.t3};
    for (T* v : vecs) cudaFree(v);
  }
  lvs.clear();
}

template <typename T>
void release_levels(std::vector<Level<T>>& lvs) {
  for (auto& L : lvs) {
    DCSR<T>* mats[] = {&L.A, &L.L2, &L.U2, &L.L1, &L.U1, &L.P, &L.R, &L.iL, &L.iU};
    for (DCSR<T>* M : mats) release(*M);
    T* vecs[] = {L.dinv, L.dl1inv, L.idinv, L.idc, L.b, L.x, L.r, L.t1, L.t2, L.t3};
    for (T* v : vecs) cudaFree(v);
  }
  lvs.clear();
}

// A device buffer of at least n doubles the autotuner may overwrite: the Krylov basis (FP64 or
// split, whichever the handle holds).
double* tuning_scratch(nsamg_handle* h) { return h->split ? reinterpret_cast<double*>(h->Vs) : h->V; }

// GMRES workspace of a handle or solver context: V (m+1 columns), Z (m columns), w, the device
// state and reduction scratch; leading dimension padded to 64 entries.
int alloc_workspace(nsamg_handle* h) {
  int rc;
  h->n = h->lv[0].n;
  h->m = h->p.restart;
  h->ld = ((int64_t)h->n + 63) / 64 * 64;
  h->split = !h->p.krylov_fp64;
  if (h->split) {
    if ((rc = alloc_vec(&h->Vs, h->ld * (h->m + 1)))) return rc;
    if ((rc = alloc_vec(&h->vin, h->ld))) return rc;
  } else {
    if ((rc = alloc_vec(&h->V, h->ld * (h->m + 1)))) return rc;
  }
  if (h->fp32) {
    if ((rc = alloc_vec(&h->Z32, h->ld * h->m))) return rc;
  } else {
    if ((rc = alloc_vec(&h->Z, h->ld * h->m))) return rc;
  }
  if ((rc = alloc_vec(&h->w, h->ld))) return rc;
  CK(cudaMalloc(&h->st, sizeof(GState)));
  CK(cudaMemset(h->st, 0, sizeof(GState)));
  CK(cudaMallocHost(&h->h_st, sizeof(GState)));
  int sms = 148;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  h->gram_blocks = h->split ? kDfGramBlocksPerSM * sms : 2 * sms;
  CK(gram_tma_prepare());
  h->update_blocks = h->split ? sms : 8 * sms;
  h->stream_blocks = 8 * sms;
  const int resid_blocks = blocks_for((int64_t)h->n * 32);
  h->partial_cap = std::max<int64_t>({(int64_t)h->gram_blocks * 2 * (kMaxM + 1), (int64_t)h->update_blocks,
                                      3 * (int64_t)resid_blocks});
  CK(cudaMalloc(&h->scr.partials, sizeof(double) * h->partial_cap));
  CK(cudaMalloc(&h->scr.ticket, sizeof(unsigned) * 4));
  CK(cudaMemset(h->scr.ticket, 0, sizeof(unsigned) * 4));
  h->ctx_bytes = sizeof(double) * h->ld * (h->m + 2 + (h->split ? 1 : 0)) + (h->fp32 ? sizeof(float) : sizeof(double)) * h->ld * h->m +
                 sizeof(GState) + sizeof(double) * h->partial_cap;
  return NSAMG_OK;
}

// Grid tail (fuse_tail = 2): the passes below the first level with at most kGridTailRows rows
// whose passes are all CSR row passes (a SELL pass cannot be recorded; then the next level is
// tried), one block per SM in a cooperative launch. Leaves the tail off when nothing would be
// fused or the device cannot host the grid.
template <typename T>
int build_tail_grid(nsamg_handle* h, std::vector<Level<T>>& lv) {
  const int nl = (int)lv.size();
  std::vector<TailPass<T>> rec;
  int l0 = 0;
  for (int l = 1; l < nl - 1; ++l) {  // at least one smoothed level below the cut
    if (lv[l].n > kGridTailRows) continue;
    rec.clear();
    tail_recorder<T>() = &rec;
    vcycle(h, lv, l, cref((const T*)lv[l].b), vref(lv[l].x), Ctx{h->stream, nullptr});
    tail_recorder<T>() = nullptr;
    bool ok = true;
    for (const auto& P : rec)
      if (P.epi == -100) ok = false;
    if (ok) {
      l0 = l;
      break;
    }
  }
  if (l0 == 0) return NSAMG_OK;
  int occ = 0, sms = 0, coop = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tail_grid<T>, kGridTailThreads, 0));
  if (!coop || occ < 1) return NSAMG_OK;
  if (!h->tail_ctr) CK(cudaMalloc(&h->tail_ctr, sizeof(unsigned long long)));
  CK(cudaMalloc(&h->tail_passes, sizeof(TailPass<T>) * rec.size()));
  CK(cudaMemcpy(h->tail_passes, rec.data(), sizeof(TailPass<T>) * rec.size(), cudaMemcpyHostToDevice));
  h->tail_l0 = l0;
  h->tail_np = (int)rec.size();
  h->tail_grid = sms;
  return NSAMG_OK;
}

// Record the passes of the V-cycle below the first level with at most kTailStage rows and keep
// them on the device for k_tail; picks the largest cluster (16, else 8 CTAs) the device can host.
// Leaves the tail off (separate launches) when nothing would be fused.
template <typename T>
int build_tail(nsamg_handle* h, std::vector<Level<T>>& lv) {
  if (h->tail_passes) {
    cudaFree(h->tail_passes);
    h->tail_passes = nullptr;
  }
  h->tail_l0 = h->tail_np = h->tail_ncl = h->tail_grid = 0;
  if (!h->p.fuse_tail || h->batch) return NSAMG_OK;
  if (h->p.fuse_tail == 2) return build_tail_grid(h, lv);
  const int nl = (int)lv.size();
  int l0 = 0;
  for (int l = 1; l < nl; ++l)
    if (lv[l].n <= kTailStage) {
      l0 = l;
      break;
    }
  if (l0 == 0 || l0 >= nl - 1) return NSAMG_OK;  // at least one smoothed level below the cut
  std::vector<TailPass<T>> rec;
  tail_recorder<T>() = &rec;
  vcycle(h, lv, l0, cref((const T*)lv[l0].b), vref(lv[l0].x), Ctx{h->stream, nullptr});
  tail_recorder<T>() = nullptr;
  for (const auto& P : rec)
    if (P.epi == -100 || P.op.src_n > kTailStage) return NSAMG_OK;
  CK(cudaFuncSetAttribute(k_tail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(T) * kTailStage)));
  CK(cudaFuncSetAttribute(k_tail<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  int want = 16;
  if (const char* e = std::getenv("NSAMG_TAIL_CLUSTER")) want = std::atoi(e);
  int ncl = 0;
  for (int cand : {16, 8, 4}) {
    if (cand > want) continue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cand);
    cfg.blockDim = dim3(kTailThreads);
    cfg.dynamicSmemBytes = sizeof(T) * kTailStage;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cand;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int num = 0;
    if (cudaOccupancyMaxActiveClusters(&num, k_tail<T>, &cfg) == cudaSuccess && num > 0) {
      ncl = cand;
      break;
    }
  }
  cudaGetLastError();
  if (!ncl) return NSAMG_OK;
  CK(cudaMalloc(&h->tail_passes, sizeof(TailPass<T>) * rec.size()));
  CK(cudaMemcpy(h->tail_passes, rec.data(), sizeof(TailPass<T>) * rec.size(), cudaMemcpyHostToDevice));
  h->tail_l0 = l0;
  h->tail_np = (int)rec.size();
  h->tail_ncl = ncl;
  return NSAMG_OK;
}

int build_tail_any(nsamg_handle* h) {
  return h->fp32 ? build_tail(h, h->lv32) : build_tail(h, h->lv);
}

int finish_graph(nsamg_handle* h) {
  if (!h->p.use_graph) {  // count the launches of one step without running it
    cudaGraph_t tmp;
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const int64_t before = g_launches;
    enqueue_step(h, cs, 0ull);
    h->launches_per_step = (int)(g_launches - before);
    CK(cudaStreamEndCapture(cs, &tmp));
    cudaGraphDestroy(tmp);
    cudaStreamDestroy(cs);
    return NSAMG_OK;
  }
  return build_graph(h);
}

// Host-side description of a batch (concatenated systems) handed to setup_impl.
struct BatchInit {
  std::vector<double> anorm;         // ||A_0||_inf per system
  std::vector<int64_t> off;          // nsys + 1 finest-level row offsets
  std::vector<int64_t> coff;         // nsys + 1 coarsest-level row offsets
  std::vector<int64_t> cblk;         // nsys offsets of each dense inverse block
  std::vector<double> cinv;          // all dense inverse blocks (row-major), empty if none
};

int setup_batch_data(nsamg_handle* h, const BatchInit& bi);
void destroy_impl(nsamg_handle* h);

int setup_impl(const nsamg_hierarchy_desc* H, const nsamg_params* pp, void* stream, nsamg_handle* h,
               const BatchInit* bi = nullptr) {
  nsamg_params p;
  nsamg_default_params(&p);
  if (pp) p = *pp;
  int rc = check_params(p);
  if (rc) return rc;
  h->p = p;
  if (!H || H->nlevels < 1 || !H->levels) return fail(NSAMG_ERR_INVALID_ARG, "empty hierarchy");
  CK(cudaGetDevice(&h->device));
  if (stream) {
    h->stream = (cudaStream_t)stream;
  } else {
    CK(cudaStreamCreate(&h->stream));  // blocking w.r.t. the legacy default stream
    h->own_stream = true;
  }
  const int nl = H->nlevels;
  // NSAMG_SETUP_TIMING=1: phase times on stderr
  static const bool timing = [] {
    const char* e = std::getenv("NSAMG_SETUP_TIMING");
    return e && e[0] == '1';
  }();
  auto t_last = std::chrono::steady_clock::now();
  auto stamp = [&](const char* what) {
    if (!timing) return;
    cudaDeviceSynchronize();
    const auto t = std::chrono::steady_clock::now();
    std::fprintf(stderr, "nsamg setup %-18s %8.1f ms\n", what, std::chrono::duration<double, std::milli>(t - t_last).count());
    t_last = t;
  };
  for (int l = 0; l < nl; ++l) {
    const nsamg_level_desc& D = H->levels[l];
    std::string nm = "level " + std::to_string(l);
    if (l < nl - 1 && (D.P.nrows != D.A.nrows || D.R.ncols != D.A.nrows || D.P.ncols != H->levels[l + 1].A.nrows ||
                       D.R.nrows != H->levels[l + 1].A.nrows))
      return fail(NSAMG_ERR_BAD_MATRIX, nm + ": P/R dimensions do not match the levels");
    if (D.ilu_L.nrows > 0) {
      if (D.ilu_form != 0 && D.ilu_form != 1) return fail(NSAMG_ERR_INVALID_ARG, nm + ": ilu_form must be 0 or 1");
      if ((D.ilu_form == 0 && !D.ilu_dinv) || D.ilu_L.nrows != D.A.nrows || D.ilu_U.nrows != D.A.nrows)
        return fail(NSAMG_ERR_BAD_MATRIX, nm + ": ILU factor dimensions");
    }
  }
  {  // every matrix validated in parallel host threads (first failure in level order reported)
    std::vector<std::function<int()>> jobs;
    for (int l = 0; l < nl; ++l) {
      const nsamg_level_desc& D = H->levels[l];
      const std::string nm = "level " + std::to_string(l);
      jobs.push_back([&D, nm] { return validate(D.A, true, true, (nm + " A").c_str()); });
      if (l < nl - 1) {
        jobs.push_back([&D, nm] { return validate(D.P, false, false, (nm + " P").c_str()); });
        jobs.push_back([&D, nm] { return validate(D.R, false, false, (nm + " R").c_str()); });
      }
      if (D.ilu_L.nrows > 0) {
        jobs.push_back([&D, nm] { return validate(D.ilu_L, true, false, (nm + " ilu_L").c_str()); });
        jobs.push_back([&D, nm] { return validate(D.ilu_U, true, false, (nm + " ilu_U").c_str()); });
      }
    }
    if ((rc = run_parallel(jobs))) return rc;
  }
  stamp("validate");
  h->fp32 = p.vcycle_fp32 == 1;
  if ((rc = build_levels<double>(H, p, h->lv, h->fp32))) return rc;
  if (h->fp32 && (rc = build_levels<float>(H, p, h->lv32, false))) return rc;
  stamp("levels");
  if (H->coarse_inv) {
    h->nc = H->levels[nl - 1].A.nrows;
    const size_t nc2 = (size_t)h->nc * h->nc;
    if (h->fp32) {
      std::vector<float> c32(H->coarse_inv, H->coarse_inv + nc2);
      CK(cudaMalloc(&h->coarse_inv32, sizeof(float) * nc2));
      CK(cudaMemcpy(h->coarse_inv32, c32.data(), sizeof(float) * nc2, cudaMemcpyHostToDevice));
    } else {
      CK(cudaMalloc(&h->coarse_inv, sizeof(double) * nc2));
      CK(cudaMemcpy(h->coarse_inv, H->coarse_inv, sizeof(double) * nc2, cudaMemcpyHostToDevice));
    }
  }
  if ((rc = alloc_workspace(h))) return rc;
  stamp("workspace");
  h->anorm_inf = norm_inf(H->levels[0].A);
  CK(cudaMemcpy(&h->st->anorm_inf, &h->anorm_inf, sizeof(double), cudaMemcpyHostToDevice));
  if (bi && (rc = setup_batch_data(h, *bi))) return rc;
  // Threads per row: fixed by the caller or tuned on the device.
  if ((rc = tune_levels(h->lv, tuning_scratch(h), h->w, p.spmv_group, p.sell_shape, h->stream))) return rc;
  if (h->fp32) {
    // FP32 scratch for tuning: the finest level's work vectors are the largest
    if ((rc = tune_levels(h->lv32, h->lv32[0].t1, h->lv32[0].t2, p.spmv_group, p.sell_shape, h->stream))) return rc;
  }
  CK(cudaStreamSynchronize(h->stream));
  stamp("tune");
  if (h->batch) {
    if (p.use_graph) {
      rc = build_graph_fn(
          h, [h](cudaStream_t s, int init, unsigned long long co, unsigned long long ci) { enqueue_bresid(h, s, init, co, ci); },
          [h](cudaStream_t s, unsigned long long ci) { enqueue_bstep(h, s, ci); }, [h](cudaStream_t s) { enqueue_bxupdate(h, s); },
          [h](cudaStream_t s) { enqueue_sknorm(h, s); });
      if (rc) return rc;
    } else {
      cudaGraph_t tmp;
      cudaStream_t cs;
      CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      const int64_t before = g_launches;
      enqueue_bstep(h, cs, 0ull);
      h->launches_per_step = (int)(g_launches - before);
      CK(cudaStreamEndCapture(cs, &tmp));
      cudaGraphDestroy(tmp);
      cudaStreamDestroy(cs);
    }
  } else {
    if ((rc = build_tail_any(h))) return rc;
    if ((rc = finish_graph(h))) return rc;
  }
  stamp("graph");
  CK(cudaGetLastError());
  return NSAMG_OK;
}

// A solver context for `parent`: shares its (read-only) matrices, coarse inverse and tuned
// kernel shapes, owns its own level work vectors, GMRES workspace, stream and graph, so several
// solves on one hierarchy can run concurrently.
template <typename T>
int clone_level_vectors(const std::vector<Level<T>>& src, std::vector<Level<T>>& dst) {
  int rc;
  dst = src;
  for (auto& L : dst) {
    L.b = L.x = L.r = L.t1 = L.t2 = L.t3 = nullptr;
    if (!L.dinv) continue;  // matrix-only level (FP64 operator of an FP32 handle)
    T** vecs[] = {&L.b, &L.x, &L.r, &L.t1, &L.t2, &L.t3};
    for (T** v : vecs)
      if ((rc = alloc_vec(v, L.n))) return rc;
  }
  return NSAMG_OK;
}

// Device bytes of the per-context level vectors (six per level, in the V-cycle's precision):
// what clone_context adds to a context's workspace, and what the server reserves for it.
size_t level_vector_bytes(const nsamg_handle* h) {
  size_t v = 0;
  for (auto& L : h->lv) v += L.dinv ? 6 * sizeof(double) * (size_t)L.n : 0;
  for (auto& L : h->lv32) v += 6 * sizeof(float) * (size_t)L.n;
  return v;
}

int clone_context(nsamg_handle* parent, nsamg_handle** out) {
  int rc;
  *out = nullptr;
  if (parent->batch) return fail(NSAMG_ERR_INVALID_ARG, "batch handles cannot be served");
  nsamg_handle* h = new nsamg_handle();
  h->device = parent->device;
  h->p = parent->p;
  h->fp32 = parent->fp32;
  h->shared_mats = true;
  h->coarse_inv = parent->coarse_inv;
  h->coarse_inv32 = parent->coarse_inv32;
  h->nc = parent->nc;
  auto bail = [&](int code) {
    std::string keep = g_err;
    destroy_impl(h);
    g_err = keep;
    return code;
  };
  if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(fail(NSAMG_ERR_CUDA, "stream"));
  h->own_stream = true;
  if ((rc = clone_level_vectors(parent->lv, h->lv))) return bail(rc);
  if ((rc = clone_level_vectors(parent->lv32, h->lv32))) return bail(rc);
  if ((rc = alloc_workspace(h))) return bail(rc);
  h->anorm_inf = parent->anorm_inf;
  if (cudaMemcpy(&h->st->anorm_inf, &h->anorm_inf, sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(fail(NSAMG_ERR_CUDA, "state"));
  h->ctx_bytes += level_vector_bytes(h);
  if ((rc = build_tail_any(h))) return bail(rc);
  if ((rc = finish_graph(h))) return bail(rc);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return bail(fail(NSAMG_ERR_CUDA, "sync"));
  *out = h;
  return NSAMG_OK;
}

template <typename T>
int upload_raw(const std::vector<T>& hv, T** d) {
  CK(cudaMalloc(d, sizeof(T) * std::max<size_t>(hv.size(), 1)));
  if (!hv.empty()) CK(cudaMemcpy(*d, hv.data(), sizeof(T) * hv.size(), cudaMemcpyHostToDevice));
  return NSAMG_OK;
}

int setup_batch_data(nsamg_handle* h, const BatchInit& bi) {
  int rc;
  BatchData* B = new BatchData();
  h->batch = B;
  B->nsys = (int)bi.off.size() - 1;
  B->off = bi.off;
  if ((rc = upload_raw(bi.off, &B->d_off))) return rc;
  int64_t maxpart = 0;
  for (int k = 0; k < 4; ++k) {
    std::vector<int> bs(B->nsys + 1, 0);
    for (int sI = 0; sI < B->nsys; ++sI) {
      const int64_t n = bi.off[sI + 1] - bi.off[sI];
      bs[sI + 1] = bs[sI] + (int)std::max<int64_t>(1, (n + B->rpb[k] - 1) / B->rpb[k]);
    }
    B->nblocks[k] = bs[B->nsys];
    if ((rc = upload_raw(bs, &B->d_bstart[k]))) return rc;
    const int64_t per = (k == BatchData::kGram) ? 2 * (kMaxM + 1) : 3;
    maxpart = std::max<int64_t>(maxpart, per * B->nblocks[k]);
  }
  CK(cudaMalloc(&B->partials, sizeof(double) * maxpart));
  CK(cudaMalloc(&B->d_sticket, sizeof(unsigned) * 4 * B->nsys));
  CK(cudaMemset(B->d_sticket, 0, sizeof(unsigned) * 4 * B->nsys));
  CK(cudaMalloc(&B->d_gticket, sizeof(unsigned) * 4));
  CK(cudaMemset(B->d_gticket, 0, sizeof(unsigned) * 4));
  CK(cudaMalloc(&B->d_st, sizeof(GState) * B->nsys));
  CK(cudaMemset(B->d_st, 0, sizeof(GState) * B->nsys));
  for (int sI = 0; sI < B->nsys && sI < (int)bi.anorm.size(); ++sI)
    CK(cudaMemcpy(&B->d_st[sI].anorm_inf, &bi.anorm[sI], sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMallocHost(&B->h_st, sizeof(GState) * B->nsys));
  CK(cudaMalloc(&B->d_ctl, sizeof(BatchCtl)));
  CK(cudaMemset(B->d_ctl, 0, sizeof(BatchCtl)));
  CK(cudaMallocHost(&B->h_ctl, sizeof(BatchCtl)));
  if (!bi.cinv.empty()) {
    B->ncrows = (int)bi.coff.back();
    std::vector<int> rs(B->ncrows);
    for (int sI = 0; sI < B->nsys; ++sI)
      for (int64_t r = bi.coff[sI]; r < bi.coff[sI + 1]; ++r) rs[r] = sI;
    if ((rc = upload_raw(rs, &B->d_row_sys))) return rc;
    if ((rc = upload_raw(bi.coff, &B->d_coff))) return rc;
    if ((rc = upload_raw(bi.cblk, &B->d_cblk))) return rc;
    if (h->fp32) {
      std::vector<float> c32(bi.cinv.begin(), bi.cinv.end());
      if ((rc = upload_raw(c32, &B->d_cinv32))) return rc;
    } else {
      if ((rc = upload_raw(bi.cinv, &B->d_cinv))) return rc;
    }
  }
  return NSAMG_OK;
}

void destroy_batch(BatchData* B) {
  if (!B) return;
  cudaFree(B->d_off);
  for (int k = 0; k < 4; ++k) cudaFree(B->d_bstart[k]);
  cudaFree(B->partials);
  cudaFree(B->d_sticket);
  cudaFree(B->d_gticket);
  cudaFree(B->d_st);
  if (B->h_st) cudaFreeHost(B->h_st);
  cudaFree(B->d_ctl);
  if (B->h_ctl) cudaFreeHost(B->h_ctl);
  cudaFree(B->d_row_sys);
  cudaFree(B->d_coff);
  cudaFree(B->d_cblk);
  cudaFree(B->d_cinv);
  cudaFree(B->d_cinv32);
  delete B;
}

// Concatenate equal-depth hierarchies into one block-diagonal hierarchy (host), keeping the
// arrays alive in `store`.
struct ConcatStore {  // deques: references to earlier arrays stay valid while more are added
  std::deque<std::vector<int>> ints;
  std::deque<std::vector<double>> dbls;
  std::vector<nsamg_level_desc> levels;
};

nsamg_csr concat_csr(const std::vector<const nsamg_csr*>& parts, ConcatStore& store) {
  int64_t nr = 0, nc = 0, nnz = 0;
  for (auto* c : parts) {
    nr += c->nrows;
    nc += c->ncols;
    nnz += c->nnz;
  }
  store.ints.emplace_back();
  std::vector<int>& rp = store.ints.back();
  store.ints.emplace_back();
  std::vector<int>& ci = store.ints.back();
  store.dbls.emplace_back();
  std::vector<double>& v = store.dbls.back();
  rp.reserve(nr + 1);
  ci.reserve(nnz);
  v.reserve(nnz);
  rp.push_back(0);
  int64_t roff = 0, coff = 0;
  for (auto* c : parts) {
    for (int i = 0; i < c->nrows; ++i) {
      for (int64_t q = c->rowptr[i]; q < c->rowptr[i + 1]; ++q) {
        ci.push_back((int)(c->col[q] + coff));
        v.push_back(c->val[q]);
      }
      rp.push_back((int)ci.size());
    }
    roff += c->nrows;
    coff += c->ncols;
  }
  nsamg_csr out{};
  out.nrows = (int32_t)nr;
  out.ncols = (int32_t)nc;
  out.nnz = nnz;
  out.rowptr = rp.data();
  out.col = ci.data();
  out.val = v.data();
  return out;
}

int solve_batch_impl(nsamg_handle* h, const double* d_b, double* d_x, double rtol, int maxit, nsamg_stats* stats) {
  if (!h || !h->batch || !d_b || !d_x) return fail(NSAMG_ERR_INVALID_ARG, "null argument or not a batch handle");
  if (!(rtol > 0.0) || maxit < 0) return fail(NSAMG_ERR_INVALID_ARG, "rtol must be > 0 and maxit >= 0");
  CK(cudaSetDevice(h->device));
  BatchData* B = h->batch;
  cudaStream_t s = h->stream;
  BatchCtl* c = B->h_ctl;
  std::memset(c, 0, sizeof(BatchCtl));
  c->b = d_b;
  c->x = d_x;
  c->rtol = rtol;
  c->maxit = maxit;
  c->m = h->m;
  c->t_exact = h->p.t_exact;
  c->stop_nrbe = h->p.stop_nrbe;
  CK(cudaMemcpyAsync(B->d_ctl, c, sizeof(BatchCtl), cudaMemcpyHostToDevice, s));
  if (h->exec) {
    CK(cudaGraphLaunch(h->exec, s));
  } else {
    enqueue_bresid(h, s, 1, 0, 0);
    for (int cycle = 0; cycle <= maxit + 1; ++cycle) {
      CK(cudaMemcpyAsync(c, B->d_ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (c->running == 0) break;
      for (int i = 0; i < h->m; ++i) {
        const int gi_before = i;
        enqueue_bstep(h, s, 0);
        CK(cudaMemcpyAsync(c, B->d_ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (c->active == 0 || c->gi == gi_before) break;  // all stopped, or the step did not advance
      }
      enqueue_bxupdate(h, s);
      enqueue_bresid(h, s, 0, 0, 0);
    }
    enqueue_sknorm(h, s);
  }
  CK(cudaMemcpyAsync(B->h_st, B->d_st, sizeof(GState) * B->nsys, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  int worst = NSAMG_OK;
  for (int sI = 0; sI < B->nsys; ++sI) {
    const GState& g = B->h_st[sI];
    int status = g.status;
    if (status == 0 && !g.converged) status = NSAMG_NOT_CONVERGED;
    if (stats) {
      stats[sI].iters = g.iters;
      stats[sI].restarts = std::max(0, g.cycles - 1);
      stats[sI].converged = g.converged;
      stats[sI].status = status;
      stats[sI].relres_true = g.relres_true;
      stats[sI].relres_implicit = g.relres_implicit;
      stats[sI].nrbe = g.nrbe;
      stats[sI].orth_loss = g.orth_loss;
      stats[sI].sk_norm = g.sk_norm;
      stats[sI].bnorm = g.bnorm;
    }
    if (status < 0) worst = status;
    else if (status == NSAMG_NOT_CONVERGED && worst == NSAMG_OK) worst = NSAMG_NOT_CONVERGED;
  }
  if (worst < 0) return fail(worst, "a system of the batch failed (see its stats)");
  return worst;
}

void destroy_impl(nsamg_handle* h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  destroy_batch(h->batch);
  h->batch = nullptr;
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->tail_passes) cudaFree(h->tail_passes);
  if (h->tail_ctr) cudaFree(h->tail_ctr);
  if (h->graph) cudaGraphDestroy(h->graph);
  if (h->shared_mats) {
    release_level_vectors(h->lv);
    release_level_vectors(h->lv32);
  } else {
    release_levels(h->lv);
    release_levels(h->lv32);
    cudaFree(h->coarse_inv);
    cudaFree(h->coarse_inv32);
  }
  cudaFree(h->V);
  cudaFree(h->Vs);
  cudaFree(h->vin);
  cudaFree(h->Z);
  cudaFree(h->Z32);
  cudaFree(h->w);
  cudaFree(h->st);
  if (h->h_st) cudaFreeHost(h->h_st);
  cudaFree(h->scr.partials);
  cudaFree(h->scr.ticket);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
}

int nlev(nsamg_handle* h) { return h->fp32 ? (int)h->lv32.size() : (int)h->lv.size(); }

int level_ok(nsamg_handle* h, int level) {
  if (!h) return fail(NSAMG_ERR_INVALID_ARG, "null handle");
  if (level < 0 || level >= nlev(h)) return fail(NSAMG_ERR_INVALID_ARG, "level out of range");
  return NSAMG_OK;
}

void to32(nsamg_handle* h, const double* a, float* b, int64_t n) {
  launch_k(k_cast<double, float>, blocks_for(n), kThreads, h->stream, n, cref(a), vref(b), nullptr);
}

void to64(nsamg_handle* h, const float* a, double* b, int64_t n) {
  launch_k(k_cast<float, double>, blocks_for(n), kThreads, h->stream, n, cref(a), vref(b), nullptr);
}

// Standalone scratch for nsamg_gram / nsamg_update (one per device, allocated on first use).
std::mutex g_scr_mu;
std::vector<Scratch> g_scr;

// Per-device scratch of the standalone Gram / update entry points: the Gram family uses the
// first kStandaloneGramPartials doubles and ticket 0, the update family the rest and ticket 1.
constexpr int64_t kStandaloneGramPartials = 512 * 2 * (kMaxM + 1);

int standalone_scratch(Scratch* out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_scr_mu);
  if ((int)g_scr.size() <= dev) g_scr.resize(dev + 1, Scratch{nullptr, nullptr});
  if (!g_scr[dev].partials) {
    int sms = 148;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t cap = kStandaloneGramPartials + 8 * (int64_t)sms;
    CK(cudaMalloc(&g_scr[dev].partials, sizeof(double) * cap));
    CK(cudaMalloc(&g_scr[dev].ticket, sizeof(unsigned) * 4));
    CK(cudaMemset(g_scr[dev].ticket, 0, sizeof(unsigned) * 4));
  }
  *out = g_scr[dev];
  return NSAMG_OK;
}

// ------------------------------------------------------------------------------------------
// Allocation-free Gram: its scratch lives in a fixed file-scope device array instead of memory
// from cudaMalloc. Layout: bytes [0, 256) hold the last-block ticket, the block partials start
// at byte 256. Every device that loads this library holds the array until the process exits.
// ------------------------------------------------------------------------------------------
constexpr int kNoAllocBlocks = 512;  // most blocks the array has room for
constexpr size_t kNoAllocBytes = 256 + sizeof(double) * (size_t)kNoAllocBlocks * 2 * (kMaxM + 1);
static __device__ __align__(256) unsigned char g_gram_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
std::vector<void*> g_noalloc_addr;  // device address of g_gram_scratch, per device (set-up once)

// Looks up the device address of the array for the current device. In host code the array's
// name is only a host-side stand-in, so kernels must be given this address instead.
int noalloc_scratch(Scratch* out, int* blocks) {
  int dev = 0, sms = 148;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if ((int)g_noalloc_addr.size() <= dev) g_noalloc_addr.resize(dev + 1, nullptr);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      CK(cudaGetSymbolAddress(&p, g_gram_scratch));
      g_noalloc_addr[dev] = p;
    }
    base = g_noalloc_addr[dev];
  }
  out->ticket = (unsigned*)base;
  out->partials = (double*)((unsigned char*)base + 256);
  *blocks = std::min(kDfGramBlocksPerSM * sms, kNoAllocBlocks);
  return NSAMG_OK;
}

// h_out (optional): host buffer that receives x, copied in stream order right after the solve,
// before the state read-back, so the host waits once.
int solve_impl(nsamg_handle* h, const double* d_b, double* d_x, double rtol, int maxit, nsamg_stats* stats,
               double* h_out = nullptr) {
  if (!h || !d_b || !d_x) return fail(NSAMG_ERR_INVALID_ARG, "null argument");
  if (h->batch) return fail(NSAMG_ERR_INVALID_ARG, "batch handle: use nsamg_batch_solve");
  if (!(rtol > 0.0) || maxit < 0) return fail(NSAMG_ERR_INVALID_ARG, "rtol must be > 0 and maxit >= 0");
  CK(cudaSetDevice(h->device));
  cudaStream_t s = h->stream;
  GState* hs = h->h_st;
  hs->b = d_b;
  hs->x = d_x;
  hs->rtol = rtol;
  hs->maxit = maxit;
  hs->m = h->m;
  hs->t_exact = h->p.t_exact;
  hs->stop_nrbe = h->p.stop_nrbe;
  CK(cudaMemcpyAsync(h->st, hs, offsetof(GState, i), cudaMemcpyHostToDevice, s));
  if (h->exec) {
    CK(cudaGraphLaunch(h->exec, s));
  } else {
    enqueue_resid(h, s, 1, 0, 0);
    for (int cycle = 0; cycle <= maxit + 1; ++cycle) {
      CK(cudaMemcpyAsync(hs, h->st, sizeof(GState), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (hs->done) break;
      for (int i = 0; i < h->m; ++i) {
        enqueue_step(h, s, 0);
        CK(cudaMemcpyAsync(&hs->stop, &h->st->stop, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (hs->stop) break;
      }
      enqueue_xupdate(h, s);
      enqueue_resid(h, s, 0, 0, 0);
    }
    enqueue_sknorm(h, s);
  }
  if (h_out) CK(cudaMemcpyAsync(h_out, d_x, sizeof(double) * h->n, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hs, h->st, sizeof(GState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  int status = hs->status;
  if (status == 0 && !hs->converged) status = NSAMG_NOT_CONVERGED;
  if (stats) {
    stats->iters = hs->iters;
    stats->restarts = std::max(0, hs->cycles - 1);
    stats->converged = hs->converged;
    stats->status = status;
    stats->relres_true = hs->relres_true;
    stats->relres_implicit = hs->relres_implicit;
    stats->nrbe = hs->nrbe;
    stats->orth_loss = hs->orth_loss;
    stats->sk_norm = hs->sk_norm;
    stats->bnorm = hs->bnorm;
  }
  if (status < 0) return fail(status, status == NSAMG_ERR_NONFINITE ? "non-finite value in the iteration" : "solve failed");
  return status;
}

// Per-level operations. FP64 handles run the FP64 kernels on the caller's arrays; FP32-V-cycle
// handles round the inputs to FP32 in the level's work vectors, run the FP32 kernels and widen
// the result back to FP64.
template <typename T>
int level_op(nsamg_handle* h, std::vector<Level<T>>& lv, int which, int level, int backward, int x_is_zero,
             const T* in1, const T* in2, T* out) {
  Level<T>& L = lv[level];
  Ctx c{h->stream, nullptr};
  switch (which) {
    case 0: {  // spmv: out = A in1
      auto op = op_mat(L.A, cref(in1));
      op.out = vref(out);
      launch_row(op, L.A.G, h->stream);
      break;
    }
    case 1: {  // residual: out = in1 - A in2
      auto op = op_mat(L.A, cref(in2));
      op.base = cref(in1);
      op.neg = 1;
      op.out = vref(out);
      launch_row(op, L.A.G, h->stream);
      break;
    }
    case 2:  // smooth: out (= x) <- sweep(b = in1, x = out)
      smooth(h, L, cref(in1), vref(out), backward != 0, x_is_zero != 0, 1, c);
      break;
    case 3: {  // restrict: out = R in1
      auto op = op_mat(L.R, cref(in1));
      op.out = vref(out);
      launch_row(op, L.R.G, h->stream);
      break;
    }
    case 4: {  // prolong: out += P in1
      auto op = op_mat(L.P, cref(in1));
      op.add = cref((const T*)out);
      op.out = vref(out);
      launch_row(op, L.P.G, h->stream);
      break;
    }
    case 5:  // coarse solve: out = A_L^-1 in1
      coarse_solve(h, L, cref(in1), vref(out), c);
      break;
  }
  return NSAMG_OK;
}

int level_dispatch(nsamg_handle* h, int which, int level, int backward, int x_is_zero, const double* in1,
                   const double* in2, double* out) {
  CK(cudaSetDevice(h->device));
  if (!h->fp32) {
    level_op<double>(h, h->lv, which, level, backward, x_is_zero, in1, in2, out);
  } else {
    auto& lv = h->lv32;
    Level<float>& L = lv[level];
    const int nl = (int)lv.size();
    // staging: input 1 / input 2 / output in FP32 work vectors of the right sizes
    float *a = L.b, *b2 = L.x, *o = L.x;
    int na = L.n, no = L.n;
    if (which == 0) { a = L.x; o = L.b; }
    if (which == 1) { a = L.b; b2 = L.x; o = L.r; }
    if (which == 2) { a = L.b; o = L.x; }
    if (which == 3) { a = L.r; o = lv[level + 1].b; no = lv[level + 1].n; }
    if (which == 4) { a = lv[level + 1].x; na = lv[level + 1].n; o = L.x; }
    if (which == 5) { a = L.b; o = L.x; }
    (void)nl;
    to32(h, in1, a, na);
    if (which == 1) to32(h, in2, b2, L.n);
    if (which == 2 || which == 4) to32(h, out, o, no);
    level_op<float>(h, lv, which, level, backward, x_is_zero, a, b2, o);
    to64(h, o, out, no);
  }
  CK(cudaGetLastError());
  return NSAMG_OK;
}

}  // namespace

// ==========================================================================================
// C ABI
// ------------------------------------------------------------------------------------------
// FMA issue-rate probe (measurement only): every thread runs kProbeChains independent chains
// a <- a * b + c for `iters` rounds and stores their sum, so no chain can be removed. FMAs per
// launch = blocks * threads * kProbeChains * iters.
// ------------------------------------------------------------------------------------------
constexpr int kProbeChains = 8;
constexpr int kProbeThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int64_t iters, T b, T c, T* sink) {
  T a[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = (T)(threadIdx.x + k);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = fma(a[k], b, c);
  }
  T t = (T)0;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) t += a[k];
  sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = t;
}

// ==========================================================================================
extern "C" {

void nsamg_default_params(nsamg_params* p) {
  if (!p) return;
  p->smoother = NSAMG_SMOOTHER_POLY_GS;
  p->neumann_terms = 2;
  p->ilu_terms_L = 3;
  p->ilu_terms_U = 3;
  p->pre_sweeps = 1;
  p->post_sweeps = 1;
  p->coarse_sweeps = 4;
  p->restart = 30;
  p->vcycle_fp32 = 0;
  p->t_exact = 0;
  p->use_graph = 1;
  p->spmv_group = 0;
  p->sell_shape = 0;
  p->fuse_tail = 0;
  p->krylov_fp64 = 0;
  p->stop_nrbe = 0;
  p->ranks = 1;
}

int nsamg_setup_hierarchy(const nsamg_hierarchy_desc* H, const nsamg_params* p, void* cuda_stream, nsamg_handle** out) {
  if (!out) return fail(NSAMG_ERR_INVALID_ARG, "null output handle pointer");
  *out = nullptr;
  nsamg_handle* h = new nsamg_handle();
  const int rc = setup_impl(H, p, cuda_stream, h);
  if (rc != NSAMG_OK) {
    std::string keep = g_err;
    destroy_impl(h);
    g_err = keep;
    return rc;
  }
  *out = h;
  return NSAMG_OK;
}

int nsamg_solve(nsamg_handle* h, const double* d_b, double* d_x, double rtol, int maxit, nsamg_stats* st) {
  return solve_impl(h, d_b, d_x, rtol, maxit, st);
}

int nsamg_solve_host(nsamg_handle* h, const double* h_b, double* h_x, double rtol, int maxit, nsamg_stats* st) {
  if (!h || !h_b || !h_x) return fail(NSAMG_ERR_INVALID_ARG, "null argument");
  CK(cudaSetDevice(h->device));
  const size_t bytes = sizeof(double) * h->n;
  double *db = nullptr, *dx = nullptr;
  CK(cudaMallocAsync(&db, bytes, h->stream));
  CK(cudaMallocAsync(&dx, bytes, h->stream));
  CK(cudaMemcpyAsync(db, h_b, bytes, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(dx, h_x, bytes, cudaMemcpyHostToDevice, h->stream));
  // x comes back in the same stream pass as the solve state (one host wait)
  int rc = solve_impl(h, db, dx, rtol, maxit, st, h_x);
  cudaFreeAsync(db, h->stream);
  cudaFreeAsync(dx, h->stream);
  CK(cudaStreamSynchronize(h->stream));
  return rc;
}

int nsamg_apply_vcycle(nsamg_handle* h, const double* d_r, double* d_z) {
  if (!h || !d_r || !d_z) return fail(NSAMG_ERR_INVALID_ARG, "null argument");
  CK(cudaSetDevice(h->device));
  Ctx c{h->stream, nullptr};
  if (!h->fp32) {
    vcycle(h, h->lv, 0, cref(d_r), vref(d_z), c);
  } else {
    Level<float>& L0 = h->lv32[0];
    to32(h, d_r, L0.b, L0.n);
    vcycle(h, h->lv32, 0, cref((const float*)L0.b), vref(L0.x), c);
    to64(h, L0.x, d_z, L0.n);
  }
  CK(cudaGetLastError());
  return NSAMG_OK;
}

int nsamg_num_levels(nsamg_handle* h) { return h ? nlev(h) : fail(NSAMG_ERR_INVALID_ARG, "null handle"); }

int nsamg_level_size(nsamg_handle* h, int level) {
  int rc = level_ok(h, level);
  return rc ? rc : (h->fp32 ? h->lv32[level].n : h->lv[level].n);
}

int nsamg_launches_per_step(nsamg_handle* h) {
  return h ? h->launches_per_step : fail(NSAMG_ERR_INVALID_ARG, "null handle");
}

int nsamg_level_group(nsamg_handle* h, int level) {
  int rc = level_ok(h, level);
  if (rc) return rc;
  if (h->fp32) return h->lv32[level].A.use_sell ? 0 : h->lv32[level].A.G;
  return h->lv[level].A.use_sell ? 0 : h->lv[level].A.G;
}

int nsamg_level_spmv(nsamg_handle* h, int level, const double* d_x, double* d_y) {
  int rc = level_ok(h, level);
  if (rc) return rc;
  if (!d_x || !d_y) return fail(NSAMG_ERR_INVALID_ARG, "null vector");
  return level_dispatch(h, 0, level, 0, 0, d_x, nullptr, d_y);
}

int nsamg_level_residual(nsamg_handle* h, int level, const double* d_b, const double* d_x, double* d_r) {
  int rc = level_ok(h, level);
  if (rc) return rc;
  if (!d_b || !d_x || !d_r) return fail(NSAMG_ERR_INVALID_ARG, "null vector");
  return level_dispatch(h, 1, level, 0, 0, d_b, d_x, d_r);
}

int nsamg_level_smooth(nsamg_handle* h, int level, int backward, int x_is_zero, const double* d_b, double* d_x) {
  int rc = level_ok(h, level);
  if (rc) return rc;
  if (!d_b || !d_x) return fail(NSAMG_ERR_INVALID_ARG, "null vector");
  return level_dispatch(h, 2, level, backward, x_is_zero, d_b, nullptr, d_x);
}

int nsamg_level_restrict(nsamg_handle* h, int level, const double* d_r, double* d_y) {
  int rc = level_ok(h, level);
  if (rc) return rc;
  if (level >= nlev(h) - 1) return fail(NSAMG_ERR_INVALID_ARG, "coarsest level has no restriction");
  if (!d_r || !d_y) return fail(NSAMG_ERR_INVALID_ARG, "null vector");
  return level_dispatch(h, 3, level, 0, 0, d_r, nullptr, d_y);
}

int nsamg_level_prolong(nsamg_handle* h, int level, const double* d_e, double* d_x) {
  int rc = level_ok(h, level);
  if (rc) return rc;
  if (level >= nlev(h) - 1) return fail(NSAMG_ERR_INVALID_ARG, "coarsest level has no prolongation");
  if (!d_e || !d_x) return fail(NSAMG_ERR_INVALID_ARG, "null vector");
  return level_dispatch(h, 4, level, 0, 0, d_e, nullptr, d_x);
}

int nsamg_coarse_solve(nsamg_handle* h, const double* d_b, double* d_z) {
  if (!h || !d_b || !d_z) return fail(NSAMG_ERR_INVALID_ARG, "null argument");
  return level_dispatch(h, 5, nlev(h) - 1, 0, 0, d_b, nullptr, d_z);
}

namespace {
int gram_standalone(int64_t n, int i, const double* d_V, int64_t ldv, const double* d_w, double* d_out, void* stream,
                    bool fp64) {
  if (n <= 0 || i < 0 || i >= kMaxM || !d_V || !d_w || !d_out || ldv < n) return fail(NSAMG_ERR_INVALID_ARG, "bad gram arguments");
  Scratch scr;
  int rc = standalone_scratch(&scr);
  if (rc) return rc;
  int dev = 0, sms = 148;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  GramArgs ga{};
  ga.n = n;
  ga.V = d_V;
  ga.ldv = ldv;
  ga.w = d_w;
  ga.st = nullptr;
  ga.i_standalone = i;
  ga.out = d_out;
  ga.scr = scr;
  if (fp64) launch_k(k_gram, 2 * sms, kGramThreads, (cudaStream_t)stream, ga);
  else if (gram_tma_aligned(d_V, ldv, d_w)) {
    CK(gram_tma_prepare());
    launch_k_smem(k_gram_tma<true>, kDfGramBlocksPerSM * sms, kGramTmaThreads, kGramTmaSmem, (cudaStream_t)stream, ga);
  } else
    launch_k(k_gram_df<true>, kDfGramBlocksPerSM * sms, kGramThreads, (cudaStream_t)stream, ga);
  CK(cudaGetLastError());
  return NSAMG_OK;
}

int update_standalone(int64_t n, int i, double* d_V, int64_t ldv, const double* d_w, double beta, const double* d_h,
                      double* d_sumsq, void* stream, bool fp64) {
  if (n <= 0 || i < 0 || i >= kMaxM || !d_V || !d_w || !d_h || !d_sumsq || ldv < n || !(beta != 0.0))
    return fail(NSAMG_ERR_INVALID_ARG, "bad update arguments");
  Scratch scr;
  int rc = standalone_scratch(&scr);
  if (rc) return rc;
  int dev = 0, sms = 148;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  UpdateArgs ua{};
  ua.n = n;
  ua.V = d_V;
  ua.ldv = ldv;
  ua.w = d_w;
  ua.st = nullptr;
  ua.i_standalone = i;
  ua.invbeta_standalone = 1.0 / beta;
  ua.h_standalone = d_h;
  ua.sumsq_out = d_sumsq;
  ua.scr.partials = scr.partials + kStandaloneGramPartials;
  ua.scr.ticket = scr.ticket + 1;
  if (fp64) launch_k(k_update, 8 * sms, kRedThreads, (cudaStream_t)stream, ua);
  else if (gram_tma_aligned(d_V, ldv, d_w)) {
    CK(gram_tma_prepare());
    launch_k_smem(k_update_tma<true>, sms, kGramTmaThreads, kGramTmaSmem, (cudaStream_t)stream, ua);
  } else
    launch_k(k_update_df<true>, kDfUpdateBlocksPerSM * sms, kRedThreads, (cudaStream_t)stream, ua);
  CK(cudaGetLastError());
  return NSAMG_OK;
}
}  // namespace

int nsamg_gram(int64_t n, int i, const double* d_V, int64_t ldv, const double* d_w, double* d_out, void* stream) {
  return gram_standalone(n, i, d_V, ldv, d_w, d_out, stream, false);
}

int nsamg_gram_fp64(int64_t n, int i, const double* d_V, int64_t ldv, const double* d_w, double* d_out, void* stream) {
  return gram_standalone(n, i, d_V, ldv, d_w, d_out, stream, true);
}

// The split-basis kernels need 16-byte aligned columns and w (the solve allocates them so), and
// room for the last row pair.
static bool split_aligned(const void* Vs, int64_t lds, const void* w, int64_t n) {
  return ((reinterpret_cast<uintptr_t>(Vs) | reinterpret_cast<uintptr_t>(w)) & 15u) == 0 && (lds & 1) == 0 &&
         lds >= n + (n & 1);
}

int nsamg_split_basis(int64_t n, int ncols, const double* d_V, int64_t ldv, void* d_Vs, int64_t lds, void* stream) {
  if (n <= 0 || ncols < 1 || !d_V || !d_Vs || ldv < n || lds < n)
    return fail(NSAMG_ERR_INVALID_ARG, "bad split-basis arguments");
  if (!split_aligned(d_Vs, lds, d_Vs, n))
    return fail(NSAMG_ERR_INVALID_ARG, "split basis: d_Vs must be 16-byte aligned, lds even and >= n rounded up to even");
  int dev = 0, sms = 148;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  launch_k(k_split_cols, 8 * sms, kRedThreads, (cudaStream_t)stream, n, ncols, d_V, ldv, (float2*)d_Vs, lds);
  CK(cudaGetLastError());
  return NSAMG_OK;
}

int nsamg_gram_split(int64_t n, int i, const void* d_Vs, int64_t lds, const double* d_w, double* d_out, void* stream) {
  if (n <= 0 || i < 0 || i >= kMaxM || !d_Vs || !d_w || !d_out || lds < n)
    return fail(NSAMG_ERR_INVALID_ARG, "bad gram arguments");
  if (!split_aligned(d_Vs, lds, d_w, n))
    return fail(NSAMG_ERR_INVALID_ARG, "split basis: d_Vs, d_w must be 16-byte aligned, lds even and >= n rounded up to even");
  Scratch scr;
  int rc = standalone_scratch(&scr);
  if (rc) return rc;
  int dev = 0, sms = 148;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CK(gram_tma_prepare());
  GramArgs ga{};
  ga.n = n;
  ga.Vs = (const float2*)d_Vs;
  ga.ldv = lds;
  ga.w = d_w;
  ga.st = nullptr;
  ga.i_standalone = i;
  ga.out = d_out;
  ga.scr = scr;
  launch_k_smem(k_gram_s, kDfGramBlocksPerSM * sms, kGramTmaThreads, kGramSSmem, (cudaStream_t)stream, ga);
  CK(cudaGetLastError());
  return NSAMG_OK;
}

int nsamg_update_split(int64_t n, int i, void* d_Vs, int64_t lds, const double* d_w, double beta_i, const double* d_c,
                       double* d_vin, double* d_sumsq, void* stream) {
  if (n <= 0 || i < 0 || i >= kMaxM || !d_Vs || !d_w || !d_c || !d_sumsq || lds < n || !(beta_i != 0.0))
    return fail(NSAMG_ERR_INVALID_ARG, "bad update arguments");
  if (!split_aligned(d_Vs, lds, d_w, n))
    return fail(NSAMG_ERR_INVALID_ARG, "split basis: d_Vs, d_w must be 16-byte aligned, lds even and >= n rounded up to even");
  Scratch scr;
  int rc = standalone_scratch(&scr);
  if (rc) return rc;
  int dev = 0, sms = 148;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CK(gram_tma_prepare());
  UpdateArgs ua{};
  ua.n = n;
  ua.Vs = (float2*)d_Vs;
  ua.ldv = lds;
  ua.w = d_w;
  ua.st = nullptr;
  ua.i_standalone = i;
  ua.invbeta_standalone = 1.0 / beta_i;
  ua.coef_standalone = d_c;
  ua.vin = d_vin;
  ua.sumsq_out = d_sumsq;
  ua.scr.partials = scr.partials + kStandaloneGramPartials;
  ua.scr.ticket = scr.ticket + 1;
  launch_k_smem(k_update_s, sms, kGramTmaThreads, kGramTmaSmem, (cudaStream_t)stream, ua);
  CK(cudaGetLastError());
  return NSAMG_OK;
}

int nsamg_gram_noalloc(int64_t n, int i, const double* d_V, int64_t ldv, const double* d_w, double* d_out,
                       void* stream) {
  if (i < 0 || i >= kMaxM)
    return fail(NSAMG_ERR_INVALID_ARG, "nsamg_gram_noalloc: i = " + std::to_string(i) +
                                           " is beyond the fixed scratch, which holds columns 0..63 (i <= 63)");
  if (n <= 0 || !d_V || !d_w || !d_out || ldv < n) return fail(NSAMG_ERR_INVALID_ARG, "bad gram arguments");
  Scratch scr;
  int blocks = 0;
  int rc = noalloc_scratch(&scr, &blocks);
  if (rc) return rc;
  // The ticket must start at zero; clear it on every call (a plain memset, no allocation).
  CK(cudaMemsetAsync(scr.ticket, 0, sizeof(unsigned), (cudaStream_t)stream));
  GramArgs ga{};
  ga.n = n;
  ga.V = d_V;
  ga.ldv = ldv;
  ga.w = d_w;
  ga.st = nullptr;
  ga.i_standalone = i;
  ga.out = d_out;
  ga.scr = scr;
  if (gram_tma_aligned(d_V, ldv, d_w)) {
    CK(gram_tma_prepare());
    launch_k_smem(k_gram_tma<true>, blocks, kGramTmaThreads, kGramTmaSmem, (cudaStream_t)stream, ga);
  } else
    launch_k(k_gram_df<true>, blocks, kGramThreads, (cudaStream_t)stream, ga);
  CK(cudaGetLastError());
  return NSAMG_OK;
}

int nsamg_update(int64_t n, int i, double* d_V, int64_t ldv, const double* d_w, double beta, const double* d_h,
                 double* d_sumsq, void* stream) {
  return update_standalone(n, i, d_V, ldv, d_w, beta, d_h, d_sumsq, stream, false);
}

int nsamg_update_fp64(int64_t n, int i, double* d_V, int64_t ldv, const double* d_w, double beta, const double* d_h,
                      double* d_sumsq, void* stream) {
  return update_standalone(n, i, d_V, ldv, d_w, beta, d_h, d_sumsq, stream, true);
}

int nsamg_batch_setup(const nsamg_hierarchy_desc* hs, int count, const nsamg_params* p, void* cuda_stream,
                      nsamg_handle** out) {
  if (!out) return fail(NSAMG_ERR_INVALID_ARG, "null output handle pointer");
  *out = nullptr;
  if (!hs || count < 1) return fail(NSAMG_ERR_INVALID_ARG, "empty batch");
  if (p && p->ranks != 1) return fail(NSAMG_ERR_INVALID_ARG, "batch: ranks must be 1 (one block per system)");
  const int nl = hs[0].nlevels;
  int with_inv = 0;
  for (int sI = 0; sI < count; ++sI) {
    if (hs[sI].nlevels != nl || nl < 1 || !hs[sI].levels)
      return fail(NSAMG_ERR_INVALID_ARG, "batch: every system needs the same number of levels");
    with_inv += hs[sI].coarse_inv ? 1 : 0;
  }
  if (with_inv != 0 && with_inv != count)
    return fail(NSAMG_ERR_INVALID_ARG, "batch: give a coarse inverse for every system or for none");
  ConcatStore store;
  store.levels.resize(nl);
  BatchInit bi;
  bi.off.push_back(0);
  bi.coff.push_back(0);
  for (int sI = 0; sI < count; ++sI) {
    bi.anorm.push_back(norm_inf(hs[sI].levels[0].A));
    bi.off.push_back(bi.off.back() + hs[sI].levels[0].A.nrows);
    const int nc = hs[sI].levels[nl - 1].A.nrows;
    bi.coff.push_back(bi.coff.back() + nc);
    if (with_inv) {
      bi.cblk.push_back((int64_t)bi.cinv.size());
      bi.cinv.insert(bi.cinv.end(), hs[sI].coarse_inv, hs[sI].coarse_inv + (size_t)nc * nc);
    }
  }
  if (bi.off.back() > INT32_MAX) return fail(NSAMG_ERR_INVALID_ARG, "batch too large for int32 indices");
  for (int l = 0; l < nl; ++l) {
    std::vector<const nsamg_csr*> A, P, R, iL, iU;
    bool has_ilu = true;
    for (int sI = 0; sI < count; ++sI) {
      const nsamg_level_desc& D = hs[sI].levels[l];
      A.push_back(&D.A);
      if (l < nl - 1) {
        P.push_back(&D.P);
        R.push_back(&D.R);
      }
      has_ilu = has_ilu && D.ilu_L.nrows > 0 && D.ilu_form == hs[0].levels[l].ilu_form &&
                (D.ilu_form == 1 || D.ilu_dinv);
      iL.push_back(&D.ilu_L);
      iU.push_back(&D.ilu_U);
    }
    nsamg_level_desc& O = store.levels[l];
    O = nsamg_level_desc{};
    O.A = concat_csr(A, store);
    if (l < nl - 1) {
      O.P = concat_csr(P, store);
      O.R = concat_csr(R, store);
    }
    if (has_ilu) {
      O.ilu_L = concat_csr(iL, store);
      O.ilu_U = concat_csr(iU, store);
      O.ilu_form = hs[0].levels[l].ilu_form;
      auto cat = [&](const double* const* ptrs, double dflt) {
        store.dbls.emplace_back();
        auto& d = store.dbls.back();
        for (int sI = 0; sI < count; ++sI) {
          const int nr = hs[sI].levels[l].A.nrows;
          if (ptrs[sI]) d.insert(d.end(), ptrs[sI], ptrs[sI] + nr);
          else d.insert(d.end(), nr, dflt);
        }
        return d.data();
      };
      std::vector<const double*> pd(count), pr(count), pc(count);
      for (int sI = 0; sI < count; ++sI) {
        pd[sI] = hs[sI].levels[l].ilu_dinv;
        pr[sI] = hs[sI].levels[l].ilu_dr;
        pc[sI] = hs[sI].levels[l].ilu_dc;
      }
      if (O.ilu_form == 0) O.ilu_dinv = cat(pd.data(), 1.0);
      else {
        O.ilu_dr = cat(pr.data(), 1.0);
        O.ilu_dc = cat(pc.data(), 1.0);
      }
    }
  }
  nsamg_hierarchy_desc H{};
  H.nlevels = nl;
  H.levels = store.levels.data();
  H.coarse_inv = nullptr;
  nsamg_handle* h = new nsamg_handle();
  const int rc = setup_impl(&H, p, cuda_stream, h, &bi);
  if (rc != NSAMG_OK) {
    std::string keep = g_err;
    destroy_impl(h);
    g_err = keep;
    return rc;
  }
  *out = h;
  return NSAMG_OK;
}

int nsamg_batch_solve(nsamg_handle* h, const double* d_b, double* d_x, double rtol, int maxit, nsamg_stats* stats) {
  return solve_batch_impl(h, d_b, d_x, rtol, maxit, stats);
}

int nsamg_batch_count(nsamg_handle* h) {
  if (!h || !h->batch) return fail(NSAMG_ERR_INVALID_ARG, "not a batch handle");
  return h->batch->nsys;
}

int nsamg_batch_offsets(nsamg_handle* h, int64_t* out) {
  if (!h || !h->batch || !out) return fail(NSAMG_ERR_INVALID_ARG, "not a batch handle");
  std::copy(h->batch->off.begin(), h->batch->off.end(), out);
  return NSAMG_OK;
}

int nsamg_sknorm(const double* d_L, int ld, int k, double* d_out, void* stream) {
  if (!d_L || !d_out || k < 1 || k > NSAMG_MAX_RESTART || ld < k) return fail(NSAMG_ERR_INVALID_ARG, "nsamg_sknorm: bad arguments");
  ++g_launches;
  launch_k(k_sknorm_matrix, 1, kSkThreads, (cudaStream_t)stream, d_L, ld, k, d_out);
  CK(cudaGetLastError());
  return NSAMG_OK;
}

int nsamg_fma_probe(int fp64, int64_t iters, int blocks, void* d_sink, void* stream, double* fma_per_launch) {
  if ((fp64 != 0 && fp64 != 1) || iters < 1 || blocks < 1 || !d_sink)
    return fail(NSAMG_ERR_INVALID_ARG, "nsamg_fma_probe: bad arguments");
  if (fp64)
    k_fma_probe<double><<<blocks, kProbeThreads, 0, (cudaStream_t)stream>>>(iters, 0.999999, 1e-7, (double*)d_sink);
  else
    k_fma_probe<float><<<blocks, kProbeThreads, 0, (cudaStream_t)stream>>>(iters, 0.999999f, 1e-7f, (float*)d_sink);
  CK(cudaGetLastError());
  if (fma_per_launch) *fma_per_launch = (double)blocks * kProbeThreads * kProbeChains * (double)iters;
  return NSAMG_OK;
}

int nsamg_grid_barrier_test(int rounds, int missing, unsigned spin_limit, int* passed, int* status) {
  if (rounds < 1 || missing < 0 || spin_limit < 1 || !passed || !status)
    return fail(NSAMG_ERR_INVALID_ARG, "nsamg_grid_barrier_test: bad arguments");
  int dev = 0, sms = 0, coop = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return fail(NSAMG_ERR_CUDA, "nsamg_grid_barrier_test: no cooperative launch on this device");
  unsigned long long* ctr = nullptr;
  int* d = nullptr;
  CK(cudaMalloc(&ctr, sizeof(unsigned long long)));
  if (cudaMalloc(&d, 2 * sizeof(int)) != cudaSuccess) {
    cudaFree(ctr);
    return fail(NSAMG_ERR_CUDA, "nsamg_grid_barrier_test: allocation failed");
  }
  cudaMemset(ctr, 0, sizeof(unsigned long long));
  cudaMemset(d, 0, 2 * sizeof(int));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sms);
  cfg.blockDim = dim3(256);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_grid_barrier_test, ctr, rounds, missing, spin_limit, d, d + 1);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int hv[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(hv, d, sizeof(hv), cudaMemcpyDeviceToHost);
  cudaFree(ctr);
  cudaFree(d);
  if (e != cudaSuccess) return fail(NSAMG_ERR_CUDA, cudaGetErrorString(e));
  *passed = hv[0];
  *status = hv[1];
  return NSAMG_OK;
}

int nsamg_context_create(nsamg_handle* parent, nsamg_handle** out) {
  if (out) *out = nullptr;
  if (!parent || !out) return fail(NSAMG_ERR_INVALID_ARG, "nsamg_context_create: null argument");
  if (parent->batch) return fail(NSAMG_ERR_INVALID_ARG, "nsamg_context_create: batch handle");
  if (parent->shared_mats)
    return fail(NSAMG_ERR_INVALID_ARG, "nsamg_context_create: pass the handle that owns the matrices");
  CK(cudaSetDevice(parent->device));
  return clone_context(parent, out);
}

void nsamg_destroy(nsamg_handle* h) { destroy_impl(h); }

const char* nsamg_status_str(int s) {
  switch (s) {
    case NSAMG_OK: return "ok";
    case NSAMG_NOT_CONVERGED: return "not converged";
    case NSAMG_PENDING: return "pending";
    case NSAMG_ERR_INVALID_ARG: return "invalid argument";
    case NSAMG_ERR_BAD_MATRIX: return "bad matrix";
    case NSAMG_ERR_OOM: return "out of device memory";
    case NSAMG_ERR_CUDA: return "CUDA error";
    case NSAMG_ERR_TIMEOUT: return "device wait timed out";
    case NSAMG_ERR_NONFINITE: return "non-finite value";
    case NSAMG_ERR_ADMISSION: return "admission rejected";
    default: return "unknown status";
  }
}

const char* nsamg_last_error(void) { return g_err.c_str(); }

}  // extern "C"

// ==========================================================================================
// Request server: continuous batching of solves on resident hierarchies.
//
// Requests (hierarchy handle, b, x, rtol, maxit) queue in arrival order. A worker thread admits
// the head of the queue as soon as a slot is free and a solver context for its hierarchy fits in
// the device-memory budget (idle contexts are reused; idle contexts of other hierarchies are
// evicted when the budget requires), writes the request into the context's device state and
// launches the context's solve graph on the context's own stream. Solves of different contexts
// overlap on the device. Completion is signalled by a host function enqueued after the graph.
// ==========================================================================================
struct ServerReq {
  uint64_t ticket = 0;
  nsamg_handle* hier = nullptr;
  const double* b = nullptr;
  double* x = nullptr;
  double rtol = 1e-8;
  int maxit = 1000;
  double t_submit = 0, t_start = 0, t_done = 0;
  int state = 0;  // 0 queued, 1 running, 2 done, 3 cancelled, 4 rejected
  int status = NSAMG_PENDING;
  nsamg_stats stats{};
  nsamg_handle* ctx = nullptr;
  cudaEvent_t ready = nullptr;  // recorded on the caller's stream at submit: inputs are ready
};

struct ServerCtx {
  nsamg_handle* ctx = nullptr;
  nsamg_handle* hier = nullptr;
  bool busy = false;
  uint64_t last_use = 0;
};

struct nsamg_server {
  int device = 0;
  size_t budget = 0;
  int max_slots = 1;
  size_t used = 0;
  int running = 0;
  uint64_t next_ticket = 1;
  uint64_t use_clock = 0;
  std::mutex mu;                   // queue, requests, contexts, accounting (never held in CUDA calls)
  std::condition_variable cv;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, ServerReq> reqs;
  std::vector<ServerCtx> ctxs;
  std::mutex fin_mu;               // only guards `finished`; taken by the stream callbacks
  std::vector<uint64_t> finished;  // tickets whose graphs completed, not yet processed
  std::thread worker;
  bool stop = false;
  std::chrono::steady_clock::time_point t0;
  std::string last_error;
  double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

namespace {

struct DoneMsg {
  nsamg_server* srv;
  uint64_t ticket;
};

// Stream callback after a request's graph and state read-back: it only appends the ticket under
// a lock that no thread holds across a CUDA call, so it can never wait on CUDA work.
void CUDART_CB on_done(void* p) {
  DoneMsg* m = (DoneMsg*)p;
  {
    std::lock_guard<std::mutex> lk(m->srv->fin_mu);
    m->srv->finished.push_back(m->ticket);
  }
  m->srv->cv.notify_all();
  delete m;
}

// Finish requests whose graphs completed (called with `mu` held).
void server_collect(nsamg_server* S) {
  std::vector<uint64_t> done;
  {
    std::lock_guard<std::mutex> lk(S->fin_mu);
    done.swap(S->finished);
  }
  for (uint64_t t : done) {
    auto it = S->reqs.find(t);
    if (it == S->reqs.end()) continue;
    ServerReq& r = it->second;
    nsamg_handle* h = r.ctx;
    const GState* g = h->h_st;
    int status = g->status;
    if (status == 0 && !g->converged) status = NSAMG_NOT_CONVERGED;
    r.stats.iters = g->iters;
    r.stats.restarts = std::max(0, g->cycles - 1);
    r.stats.converged = g->converged;
    r.stats.status = status;
    r.stats.relres_true = g->relres_true;
    r.stats.relres_implicit = g->relres_implicit;
    r.stats.nrbe = g->nrbe;
    r.stats.orth_loss = g->orth_loss;
    r.stats.sk_norm = g->sk_norm;
    r.stats.bnorm = g->bnorm;
    r.status = status;
    r.state = 2;
    r.t_done = S->now();
    for (auto& c : S->ctxs)
      if (c.ctx == h) c.busy = false;
    S->running -= 1;
  }
}

// Bytes a new context of `hier` will hold: its workspace (the parent's, same parameters) plus its
// level vectors, by the same formula clone_context uses.
size_t context_need(nsamg_handle* hier) { return hier->ctx_bytes + level_vector_bytes(hier); }

void finish_request(nsamg_server* S, ServerReq& r, int state, int status) {
  r.state = state;
  r.status = status;
  r.stats.status = status;
  r.t_done = S->now();
}

// One admission step for the head of the queue. Called with `lk` held; CUDA work (freeing
// evicted contexts, creating a context, launching) runs with the lock released. Returns true
// if the queue head changed (started, rejected or dropped), false if it has to wait.
bool server_try_start(nsamg_server* S, std::unique_lock<std::mutex>& lk) {
  if (S->queue.empty() || S->running >= S->max_slots) return false;
  const uint64_t t = S->queue.front();
  auto found = S->reqs.find(t);
  if (found == S->reqs.end() || found->second.state != 0) {  // cancelled (and maybe already polled)
    S->queue.pop_front();
    return true;
  }
  ServerReq* r = &found->second;
  nsamg_handle* hier = r->hier;
  int slot = -1;
  for (int k = 0; k < (int)S->ctxs.size(); ++k)
    if (!S->ctxs[k].busy && S->ctxs[k].hier == hier) {
      slot = k;
      break;
    }
  if (slot < 0) {
    const size_t need = context_need(hier);
    if (need > S->budget) {  // can never fit: reject
      finish_request(S, *r, 4, NSAMG_ERR_ADMISSION);
      S->queue.pop_front();
      S->cv.notify_all();
      return true;
    }
    std::vector<nsamg_handle*> victims;
    while (S->used + need > S->budget) {  // evict least recently used idle contexts
      int v = -1;
      for (int k = 0; k < (int)S->ctxs.size(); ++k)
        if (!S->ctxs[k].busy && (v < 0 || S->ctxs[k].last_use < S->ctxs[v].last_use)) v = k;
      if (v < 0) break;
      victims.push_back(S->ctxs[v].ctx);
      S->used -= S->ctxs[v].ctx->ctx_bytes;
      S->ctxs.erase(S->ctxs.begin() + v);
    }
    if (S->used + need > S->budget) {
      if (!victims.empty()) {
        lk.unlock();
        for (nsamg_handle* v : victims) destroy_impl(v);
        lk.lock();
      }
      return false;  // wait for running solves to finish
    }
    S->used += need;  // reserve while the context is built outside the lock
    S->queue.pop_front();  // the request is being admitted: no longer cancellable
    r->state = 1;
    lk.unlock();
    for (nsamg_handle* v : victims) destroy_impl(v);
    nsamg_handle* c = nullptr;
    const int rc = clone_context(hier, &c);
    const std::string err = rc ? g_err : std::string();
    lk.lock();
    r = &S->reqs.find(t)->second;  // a request in state 1 is never released, so it is still there
    if (rc != NSAMG_OK) {
      S->used -= need;
      S->last_error = err;
      finish_request(S, *r, 4, rc);
      S->cv.notify_all();
      return true;
    }
    // the reservation becomes the context's own size (equal by construction; recorded as the
    // context's so that eviction subtracts exactly what was added)
    S->used += c->ctx_bytes;
    S->used -= need;
    S->ctxs.push_back(ServerCtx{c, hier, false, 0});
    slot = (int)S->ctxs.size() - 1;
  } else {
    S->queue.pop_front();
  }
  // start: bookkeeping under the lock, launches outside it
  ServerCtx& sc = S->ctxs[slot];
  nsamg_handle* h = sc.ctx;
  sc.busy = true;
  sc.last_use = ++S->use_clock;
  r->ctx = h;
  r->state = 1;
  r->t_start = S->now();
  S->running += 1;
  GState* hs = h->h_st;
  hs->b = r->b;
  hs->x = r->x;
  hs->rtol = r->rtol;
  hs->maxit = r->maxit;
  hs->m = h->m;
  hs->t_exact = h->p.t_exact;
  hs->stop_nrbe = h->p.stop_nrbe;
  cudaEvent_t ready = r->ready;
  lk.unlock();
  cudaStream_t st = h->stream;
  const bool ok = (!ready || cudaStreamWaitEvent(st, ready, 0) == cudaSuccess) &&
                  cudaMemcpyAsync(h->st, hs, offsetof(GState, i), cudaMemcpyHostToDevice, st) == cudaSuccess &&
                  cudaGraphLaunch(h->exec, st) == cudaSuccess &&
                  cudaMemcpyAsync(hs, h->st, sizeof(GState), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                  cudaLaunchHostFunc(st, on_done, new DoneMsg{S, t}) == cudaSuccess;
  const std::string err = ok ? std::string() : std::string(cudaGetErrorString(cudaGetLastError()));
  lk.lock();
  if (!ok) {
    ServerReq& rr = S->reqs.find(t)->second;  // a running request is not released before it finishes
    finish_request(S, rr, 2, NSAMG_ERR_CUDA);
    for (auto& c : S->ctxs)
      if (c.ctx == h) c.busy = false;
    S->running -= 1;
    S->last_error = err;
    S->cv.notify_all();
  }
  return true;
}

void server_loop(nsamg_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    server_collect(S);
    bool progressed = false;
    while (server_try_start(S, lk)) {
      progressed = true;
      server_collect(S);
    }
    if (S->stop && S->queue.empty() && S->running == 0) break;
    if (!progressed) S->cv.wait_for(lk, std::chrono::milliseconds(2));
  }
}

}  // namespace

extern "C" {

int nsamg_server_create(size_t hbm_budget_bytes, int max_slots, nsamg_server** out) {
  if (!out) return fail(NSAMG_ERR_INVALID_ARG, "null output pointer");
  *out = nullptr;
  if (max_slots < 1) return fail(NSAMG_ERR_INVALID_ARG, "max_slots must be >= 1");
  nsamg_server* S = new nsamg_server();
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return fail(NSAMG_ERR_CUDA, "no current device");
  }
  S->budget = hbm_budget_bytes;
  S->max_slots = max_slots;
  S->t0 = std::chrono::steady_clock::now();
  S->worker = std::thread(server_loop, S);
  *out = S;
  return NSAMG_OK;
}

int nsamg_server_submit(nsamg_server* S, nsamg_handle* h, const double* d_b, double* d_x, double rtol, int maxit,
                        void* ready_stream, uint64_t* ticket) {
  if (!S || !h || !d_b || !d_x || !ticket) return fail(NSAMG_ERR_INVALID_ARG, "null argument");
  if (h->batch || h->shared_mats) return fail(NSAMG_ERR_INVALID_ARG, "serve hierarchy handles from nsamg_setup_hierarchy");
  if (!h->p.use_graph) return fail(NSAMG_ERR_INVALID_ARG, "served hierarchies need use_graph = 1");
  if (!(rtol > 0.0) || maxit < 0) return fail(NSAMG_ERR_INVALID_ARG, "rtol must be > 0 and maxit >= 0");
  cudaEvent_t ev = nullptr;
  CK(cudaSetDevice(S->device));
  CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  CK(cudaEventRecord(ev, (cudaStream_t)ready_stream));
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
      cudaEventDestroy(ev);
      return fail(NSAMG_ERR_INVALID_ARG, "server is shutting down");
    }
    ServerReq r;
    r.ticket = S->next_ticket++;
    r.hier = h;
    r.b = d_b;
    r.x = d_x;
    r.rtol = rtol;
    r.maxit = maxit;
    r.t_submit = S->now();
    r.ready = ev;
    *ticket = r.ticket;
    S->reqs[r.ticket] = r;
    S->queue.push_back(r.ticket);
  }
  S->cv.notify_all();
  return NSAMG_OK;
}

int nsamg_server_poll(nsamg_server* S, uint64_t ticket, nsamg_stats* st, double* times) {
  if (!S) return fail(NSAMG_ERR_INVALID_ARG, "null server");
  cudaEvent_t ev = nullptr;
  int status;
  {
  std::lock_guard<std::mutex> lk(S->mu);
  server_collect(S);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return fail(NSAMG_ERR_INVALID_ARG, "unknown ticket");
  ServerReq& r = it->second;
  if (r.state < 2) return NSAMG_PENDING;
  if (st) *st = r.stats;
  if (times) {
    times[0] = r.t_submit;
    times[1] = r.t_start;
    times[2] = r.t_done;
  }
  status = r.status;
  ev = r.ready;
  S->reqs.erase(it);
  }
  if (ev) cudaEventDestroy(ev);
  if (status < 0) return fail(status, status == NSAMG_ERR_ADMISSION ? "request rejected by admission (too large for the budget)"
                                                                   : "request failed: " + S->last_error);
  return status;
}

int nsamg_server_wait(nsamg_server* S, uint64_t ticket, nsamg_stats* st, double* times) {
  if (!S) return fail(NSAMG_ERR_INVALID_ARG, "null server");
  {
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(NSAMG_ERR_INVALID_ARG, "unknown ticket");
    while (true) {
      server_collect(S);
      auto jt = S->reqs.find(ticket);
      if (jt == S->reqs.end() || jt->second.state >= 2) break;
      S->cv.wait_for(lk, std::chrono::milliseconds(2));
    }
  }
  return nsamg_server_poll(S, ticket, st, times);
}

int nsamg_server_cancel(nsamg_server* S, uint64_t ticket) {
  if (!S) return fail(NSAMG_ERR_INVALID_ARG, "null server");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return fail(NSAMG_ERR_INVALID_ARG, "unknown ticket");
  if (it->second.state != 0) return fail(NSAMG_ERR_INVALID_ARG, "request already started or finished");
  for (auto q = S->queue.begin(); q != S->queue.end(); ++q)
    if (*q == ticket) {
      S->queue.erase(q);
      break;
    }
  it->second.state = 3;
  it->second.status = NSAMG_ERR_INVALID_ARG;
  it->second.stats.status = NSAMG_ERR_INVALID_ARG;
  it->second.t_done = S->now();
  return NSAMG_OK;
}

int nsamg_server_info(nsamg_server* S, int64_t* out4) {
  if (!S || !out4) return fail(NSAMG_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  out4[0] = (int64_t)S->used;
  out4[1] = (int64_t)S->ctxs.size();
  out4[2] = S->running;
  out4[3] = (int64_t)S->queue.size();
  return NSAMG_OK;
}

void nsamg_server_destroy(nsamg_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    for (uint64_t t : S->queue) {  // drop queued requests
      auto it = S->reqs.find(t);
      if (it != S->reqs.end()) it->second.state = 3;
    }
    S->queue.clear();
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  cudaSetDevice(S->device);
  for (auto& c : S->ctxs) destroy_impl(c.ctx);
  for (auto& kv : S->reqs)
    if (kv.second.ready) cudaEventDestroy(kv.second.ready);
  delete S;
}

}  // extern "C"

#include "setup.cuh"
