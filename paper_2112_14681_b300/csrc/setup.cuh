// Ruge-Stuben setup on the GPU (Sec. 5.1; the paper's conclusions name moving the setup to the
// GPU, including ILU(0) by fixed-point iteration, as the next step). Every step runs in the
// kernels below; the host only sizes allocations from device-computed totals.
//
//   strength      S_i = { j != i : m(a_ij) >= theta max_{k != i} m(a_ik) }, m = |.| or -(.)
//   PMIS          weights lambda_i = |S^T_i| + u_i (u_i from one SplitMix64 step per point),
//                 rounds of local maxima over S_i u S^T_i among undecided points; undecided
//                 points that strongly depend on a new C-point become F; F-points left without a
//                 strong C-neighbour are promoted to C (all at once: see k_promote_cand)
//   BAMG-direct   w_ij = -(a_ij + beta_i / n_{C_i^s}) / (a_ii + sum_{k weak} a_ik)  (eq. bamgdir)
//   MM-ext        W = -[(D_FF + D_gamma)^-1 (A^s_FF + D_beta)] [D_beta^-1 A^s_FC], one SpGEMM
//   Galerkin      R = P^T, A_c = R (A P) by a row-wise k-way merge SpGEMM whose sums run in the
//                 order of the left operand's row (the order of a sequential row-by-row product)
//   ILU(0)        fixed-point sweeps on the pattern of A, then the row-scaled LDU form
//   coarse        dense Gauss-Jordan inverse with partial pivoting
//
// Included once by engine.cu, after its error helpers.

namespace gsetup {

constexpr int kSetupThreads = 256;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kNoCol = 0x7fffffff;

inline int nblocks(int64_t threads, int per_block = kSetupThreads) {
  return (int)std::max<int64_t>(1, (threads + per_block - 1) / per_block);
}
inline int nblocks_warp_rows(int64_t rows) { return nblocks(rows * 32); }

// ---- device memory owned by the setup (freed in the destructor) ----------------------------
struct DMem {
  std::vector<void*> ptrs;
  template <typename T>
  int alloc(T** p, int64_t count) {
    *p = nullptr;
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (size_t)std::max<int64_t>(count, 1));
    if (e != cudaSuccess) return cuda_fail(e, "setup cudaMalloc");
    ptrs.push_back((void*)*p);
    return NSAMG_OK;
  }
  void release(void* p) {
    for (auto& q : ptrs)
      if (q == p) {
        cudaFree(q);
        q = nullptr;
      }
  }
  ~DMem() {
    for (void* p : ptrs)
      if (p) cudaFree(p);
  }
};

#define SK(call)                  \
  do {                            \
    int rc_ = (call);             \
    if (rc_ != NSAMG_OK) return rc_; \
  } while (0)

// ---- exclusive scan: out[0] = 0, out[i + 1] = in[0] + ... + in[i] ---------------------------
constexpr int kScanPer = 4;
constexpr int kScanTile = kSetupThreads * kScanPer;

template <typename T>
__device__ T block_excl_scan(T v, T* total) {
  __shared__ T warp_tot[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T x = v;
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    T t = lane < nw ? warp_tot[lane] : T(0);
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(kFull, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) warp_tot[lane] = t;  // inclusive warp totals
  }
  __syncthreads();
  const T before = (w > 0 ? warp_tot[w - 1] : T(0)) + x - v;
  *total = warp_tot[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

template <typename T>
__global__ void k_tile_sum(const T* __restrict__ in, int64_t n, T* __restrict__ tsum) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  T s = 0;
  for (int k = 0; k < kScanPer; ++k)
    if (base + k < n) s += in[base + k];
  T tot;
  block_excl_scan<T>(s, &tot);
  if (threadIdx.x == 0) tsum[blockIdx.x] = tot;
}

template <typename T>
__global__ void k_tile_scan(const T* __restrict__ in, int64_t n, const T* __restrict__ tile_off, T* __restrict__ out) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  T v[kScanPer];
  T s = 0;
  for (int k = 0; k < kScanPer; ++k) {
    v[k] = (base + k < n) ? in[base + k] : T(0);
    s += v[k];
  }
  T tot;
  T run = block_excl_scan<T>(s, &tot) + (tile_off ? tile_off[blockIdx.x] : T(0));
  for (int k = 0; k < kScanPer; ++k) {
    run += v[k];
    if (base + k < n) out[base + k + 1] = run;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
}

template <typename T>
int scan_excl(const T* in, T* out, int64_t n, cudaStream_t s) {
  if (n <= 0) {
    CK(cudaMemsetAsync(out, 0, sizeof(T), s));
    return NSAMG_OK;
  }
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 1) {
    k_tile_scan<T><<<1, kSetupThreads, 0, s>>>(in, n, nullptr, out);
    CK(cudaGetLastError());
    return NSAMG_OK;
  }
  T *tsum = nullptr, *toff = nullptr;
  CK(cudaMallocAsync((void**)&tsum, sizeof(T) * tiles, s));
  CK(cudaMallocAsync((void**)&toff, sizeof(T) * (tiles + 1), s));
  k_tile_sum<T><<<(unsigned)tiles, kSetupThreads, 0, s>>>(in, n, tsum);
  int rc = scan_excl<T>(tsum, toff, tiles, s);
  if (rc == NSAMG_OK) k_tile_scan<T><<<(unsigned)tiles, kSetupThreads, 0, s>>>(in, n, toff, out);
  cudaFreeAsync(tsum, s);
  cudaFreeAsync(toff, s);
  if (rc != NSAMG_OK) return rc;
  CK(cudaGetLastError());
  return NSAMG_OK;
}

template <typename T>
int read_scalar(const T* d, T* h, cudaStream_t s) {
  CK(cudaMemcpyAsync(h, d, sizeof(T), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return NSAMG_OK;
}

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
  return v;
}
__device__ __forceinline__ int64_t warp_sum64(int64_t v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// ---- small utility kernels ------------------------------------------------------------------
__global__ void k_cast_i32_i64(const int* __restrict__ in, int64_t n, int64_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}
__global__ void k_narrow_i64_i32(const int64_t* __restrict__ in, int64_t n, int* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int)in[i];
}
__global__ void k_row_index(int n, const int* __restrict__ rp, int* __restrict__ row) {
  const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= n) return;
  for (int p = rp[i] + lane; p < rp[i + 1]; p += 32) row[p] = i;
}
__global__ void k_diag_pos(int n, const int* __restrict__ rp, const int* __restrict__ ci, int* __restrict__ dpos) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int d = -1;
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (ci[p] == i) d = p;
  dpos[i] = d;
}

// ---- strength of connection -----------------------------------------------------------------
__global__ void k_strength(int n, const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ v,
                           double theta, int neg_mode, unsigned char* __restrict__ s) {
  const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= n) return;
  const int b = rp[i], e = rp[i + 1];
  double mx = 0.0;
  for (int p = b + lane; p < e; p += 32)
    if (ci[p] != i) mx = fmax(mx, neg_mode ? -v[p] : fabs(v[p]));
  mx = warp_max(mx);
  const double thr = theta * mx;
  for (int p = b + lane; p < e; p += 32) {
    const double m = neg_mode ? -v[p] : fabs(v[p]);
    s[p] = (mx > 0.0 && ci[p] != i && v[p] != 0.0 && m >= thr) ? 1 : 0;
  }
}

// column counts of the flagged entries (integer atomics: order-free)
__global__ void k_count_cols(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                             const unsigned char* __restrict__ flag, int* __restrict__ cnt) {
  const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= n) return;
  for (int p = rp[i] + lane; p < rp[i + 1]; p += 32)
    if (!flag || flag[p]) atomicAdd(&cnt[ci[p]], 1);
}

// transpose fill: entry (i, j) goes to row j of the transpose at a cursor slot; the order inside
// a row is fixed afterwards by k_sort_rows where it matters
__global__ void k_transpose_fill(int n, const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ v,
                                 const unsigned char* __restrict__ flag, int* __restrict__ cursor, int* __restrict__ tci,
                                 double* __restrict__ tv) {
  const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= n) return;
  for (int p = rp[i] + lane; p < rp[i + 1]; p += 32) {
    if (flag && !flag[p]) continue;
    const int q = atomicAdd(&cursor[ci[p]], 1);
    tci[q] = i;
    if (tv) tv[q] = v[p];
  }
}

// insertion sort of each row by column (rows of a transpose are short)
__global__ void k_sort_rows(int n, const int* __restrict__ rp, int* __restrict__ ci, double* __restrict__ v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = rp[i], e = rp[i + 1];
  for (int p = b + 1; p < e; ++p) {
    const int c = ci[p];
    const double x = v ? v[p] : 0.0;
    int q = p - 1;
    while (q >= b && ci[q] > c) {
      ci[q + 1] = ci[q];
      if (v) v[q + 1] = v[q];
      --q;
    }
    ci[q + 1] = c;
    if (v) v[q + 1] = x;
  }
}

// ---- PMIS -----------------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood 2014): advance the state by the golden gamma, then mix.
__device__ __forceinline__ uint64_t splitmix64_step(uint64_t state) {
  uint64_t z = state + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

enum : unsigned char { ST_UNDEC = 0, ST_C = 1, ST_F = 2 };

__global__ void k_pmis_init(int n, const int* __restrict__ strp, uint64_t seed, double* __restrict__ lam,
                            unsigned char* __restrict__ st) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int infl = strp[i + 1] - strp[i];
  const uint64_t out = splitmix64_step(seed ^ (0xA24BAED4963EE407ull * (uint64_t)(i + 1)));
  lam[i] = (double)infl + (double)(out >> 11) * 0x1.0p-53;
  st[i] = infl == 0 ? ST_F : ST_UNDEC;
}

// An undecided point is selected when no undecided point of S_i u S^T_i outranks it in
// (lambda, index). The selection is written to `mark`; states are read only.
__global__ void k_pmis_select(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                              const unsigned char* __restrict__ s, const int* __restrict__ strp,
                              const int* __restrict__ stci, const double* __restrict__ lam,
                              const unsigned char* __restrict__ st, unsigned char* __restrict__ mark,
                              int* __restrict__ undecided) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool und = false;
  if (i < n) {
    und = st[i] == ST_UNDEC;
    unsigned char sel = 0;
    if (und) {
      const double li = lam[i];
      bool is_max = true;
      for (int p = rp[i]; p < rp[i + 1] && is_max; ++p) {
        if (!s[p]) continue;
        const int j = ci[p];
        if (st[j] == ST_UNDEC && (lam[j] > li || (lam[j] == li && j > i))) is_max = false;
      }
      for (int q = strp[i]; q < strp[i + 1] && is_max; ++q) {
        const int j = stci[q];
        if (j != i && st[j] == ST_UNDEC && (lam[j] > li || (lam[j] == li && j > i))) is_max = false;
      }
      sel = is_max ? 1 : 0;
    }
    mark[i] = sel;
  }
  const unsigned b = __ballot_sync(kFull, und);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(undecided, __popc(b));
}

__global__ void k_pmis_apply(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                             const unsigned char* __restrict__ s, const unsigned char* __restrict__ mark,
                             unsigned char* __restrict__ st) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (mark[i]) {
    st[i] = ST_C;
    return;
  }
  if (st[i] != ST_UNDEC) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (s[p] && mark[ci[p]]) {
      st[i] = ST_F;
      return;
    }
}

// F-points without a strong C-neighbour are promoted to C. Such a point influences no other
// point (a point that influences someone is F only because it depends on a C-point), so no
// promotion can give another candidate a C-neighbour: promoting them all at once equals
// promoting them one by one in index order.
__global__ void k_promote_cand(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                               const unsigned char* __restrict__ s, const unsigned char* __restrict__ st,
                               unsigned char* __restrict__ cand) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned char c = 0;
  if (st[i] == ST_F) {
    c = 1;
    for (int p = rp[i]; p < rp[i + 1]; ++p)
      if (s[p] && st[ci[p]] == ST_C) {
        c = 0;
        break;
      }
  }
  cand[i] = c;
}

__global__ void k_is_c(int n, const unsigned char* __restrict__ st, const unsigned char* __restrict__ cand,
                       int* __restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = (st[i] == ST_C || cand[i]) ? 1 : 0;
}

__global__ void k_cf_number(int n, const int* __restrict__ flag, const int* __restrict__ off, int* __restrict__ cf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) cf[i] = flag[i] ? off[i] : -1;
}

// ---- BAMG-direct interpolation --------------------------------------------------------------
__global__ void k_interp_count(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                               const unsigned char* __restrict__ s, const int* __restrict__ cf, int* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (cf[i] >= 0) {
    cnt[i] = 1;
    return;
  }
  int c = 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (s[p] && cf[ci[p]] >= 0) ++c;
  cnt[i] = c;
}

__global__ void k_interp_fill(int n, const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ v,
                              const unsigned char* __restrict__ s, const int* __restrict__ cf, const int* __restrict__ prp,
                              int* __restrict__ pci, double* __restrict__ pv, int* __restrict__ bad_row) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int o = prp[i];
  if (cf[i] >= 0) {
    pci[o] = cf[i];
    pv[o] = 1.0;
    return;
  }
  double aii = 0.0, weak = 0.0, beta = 0.0;
  int nc = 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    const int j = ci[p];
    if (j == i) aii += v[p];
    else if (!s[p]) weak += v[p];
    else if (cf[j] >= 0) ++nc;
    else beta += v[p];
  }
  const double den = aii + weak;
  if (den == 0.0 || nc == 0) {
    atomicMin(bad_row, i);
    return;
  }
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    const int j = ci[p];
    if (j == i || !s[p] || cf[j] < 0) continue;
    pci[o] = cf[j];
    pv[o] = -(v[p] + beta / (double)nc) / den;
    ++o;
  }
}

// ---- MM-ext interpolation ------------------------------------------------------------------
// W = -[(D_FF + D_gamma)^-1 (A^s_FF + D_beta)] [D_beta^-1 A^s_FC] = -M1 M2, rows numbered over the
// F-points (fidx). M1 row: the strong F-couplings and the diagonal beta_i, scaled by
// 1 / (a_ii + gamma_i); M2 row: the strong C-couplings scaled by 1 / beta_i (0 when beta_i = 0).
__global__ void k_flag_f(int n, const int* __restrict__ cf, int* __restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = cf[i] < 0 ? 1 : 0;
}

__global__ void k_mmext_count(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                              const unsigned char* __restrict__ s, const int* __restrict__ cf, const int* __restrict__ fidx,
                              int* __restrict__ c1, int* __restrict__ c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || cf[i] >= 0) return;
  int nf = 1, nc = 0;  // M1 keeps the diagonal entry beta_i
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    const int j = ci[p];
    if (j == i || !s[p]) continue;
    if (cf[j] >= 0) ++nc;
    else ++nf;
  }
  c1[fidx[i]] = nf;
  c2[fidx[i]] = nc;
}

__global__ void k_mmext_fill(int n, const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ v,
                             const unsigned char* __restrict__ s, const int* __restrict__ cf, const int* __restrict__ fidx,
                             const int* __restrict__ m1rp, int* __restrict__ m1ci, double* __restrict__ m1v,
                             const int* __restrict__ m2rp, int* __restrict__ m2ci, double* __restrict__ m2v,
                             int* __restrict__ bad_row) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || cf[i] >= 0) return;
  double aii = 0.0, gamma = 0.0, beta = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    const int j = ci[p];
    if (j == i) aii += v[p];
    else if (!s[p]) gamma += v[p];
    else if (cf[j] >= 0) beta += v[p];
  }
  const double den = aii + gamma;
  if (den == 0.0) {
    atomicMin(bad_row, i);
    return;
  }
  const double sc = 1.0 / den;
  const double ib = beta != 0.0 ? 1.0 / beta : 0.0;
  const int fi = fidx[i];
  int o1 = m1rp[fi], o2 = m2rp[fi];
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    const int j = ci[p];
    if (j == i) {
      m1ci[o1] = fi;
      m1v[o1++] = __dmul_rn(sc, beta);
      continue;
    }
    if (!s[p]) continue;
    if (cf[j] >= 0) {
      m2ci[o2] = cf[j];
      m2v[o2++] = __dmul_rn(ib, v[p]);
    } else {
      m1ci[o1] = fidx[j];
      m1v[o1++] = __dmul_rn(sc, v[p]);
    }
  }
}

__global__ void k_mmext_pcount(int n, const int* __restrict__ cf, const int* __restrict__ fidx, const int* __restrict__ wrp,
                               int* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  cnt[i] = cf[i] >= 0 ? 1 : wrp[fidx[i] + 1] - wrp[fidx[i]];
}

__global__ void k_mmext_pfill(int n, const int* __restrict__ cf, const int* __restrict__ fidx, const int* __restrict__ wrp,
                              const int* __restrict__ wci, const double* __restrict__ wv, const int* __restrict__ prp,
                              int* __restrict__ pci, double* __restrict__ pv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int o = prp[i];
  if (cf[i] >= 0) {
    pci[o] = cf[i];
    pv[o] = 1.0;
    return;
  }
  const int fi = fidx[i];
  for (int q = wrp[fi]; q < wrp[fi + 1]; ++q, ++o) {
    pci[o] = wci[q];
    pv[o] = -wv[q];
  }
}

// ---- SpGEMM C = A B (row-wise k-way merge) -------------------------------------------------
// Upper bound of the products of each row of C: sum over the row of A of nnz(B_k).
__global__ void k_spgemm_ub(int m, const int* __restrict__ arp, const int* __restrict__ aci, const int* __restrict__ brp,
                            int64_t* __restrict__ ub) {
  const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= m) return;
  int64_t c = 0;
  for (int p = arp[i] + lane; p < arp[i + 1]; p += 32) c += brp[aci[p] + 1] - brp[aci[p]];
  c = warp_sum64(c);
  if (lane == 0) ub[i] = c;
}

// One warp per row of C. List q of the row is row k_q of B scaled by a_{i k_q}; lists are taken
// in the order of A's row. Each step emits the smallest pending column; its value is the
// product of the first list holding it, then += the products of the later lists in list order
// (the order of a sequential row-by-row product). Products and sums are rounded separately.
// Rows with more than 32 lists keep their cursors and heads in cur/hd (one slot per entry of A).
__global__ void k_spgemm_merge(int m, const int* __restrict__ arp, const int* __restrict__ aci,
                               const double* __restrict__ av, const int* __restrict__ brp, const int* __restrict__ bci,
                               const double* __restrict__ bv, const int64_t* __restrict__ off, int* __restrict__ tci,
                               double* __restrict__ tv, int64_t* __restrict__ cnt, int* __restrict__ cur,
                               int* __restrict__ hd) {
  const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= m) return;
  const int a0 = arp[i], nl = arp[i + 1] - a0;
  int64_t o = off[i];
  if (nl <= 32) {
    int pos = 0, end = 0, head = kNoCol;
    double a = 0.0;
    if (lane < nl) {
      const int k = aci[a0 + lane];
      a = av[a0 + lane];
      pos = brp[k];
      end = brp[k + 1];
      head = pos < end ? bci[pos] : kNoCol;
    }
    while (true) {
      const int mn = (int)__reduce_min_sync(kFull, (unsigned)head);
      if (mn == kNoCol) break;
      const bool has = head == mn;
      const double prod = has ? __dmul_rn(a, bv[pos]) : 0.0;
      unsigned msk = __ballot_sync(kFull, has);
      int l = __ffs(msk) - 1;
      double acc = __shfl_sync(kFull, prod, l);
      msk &= msk - 1;
      while (msk) {
        l = __ffs(msk) - 1;
        acc = __dadd_rn(acc, __shfl_sync(kFull, prod, l));
        msk &= msk - 1;
      }
      if (lane == 0) {
        tci[o] = mn;
        tv[o] = acc;
      }
      ++o;
      if (has) {
        ++pos;
        head = pos < end ? bci[pos] : kNoCol;
      }
    }
  } else {
    const int T = (nl + 31) / 32;
    for (int t = 0; t < T; ++t) {
      const int q = lane + 32 * t;
      if (q < nl) {
        const int k = aci[a0 + q];
        const int pos = brp[k];
        cur[a0 + q] = pos;
        hd[a0 + q] = pos < brp[k + 1] ? bci[pos] : kNoCol;
      }
    }
    __syncwarp();
    while (true) {
      int lmin = kNoCol;
      for (int t = 0; t < T; ++t) {
        const int q = lane + 32 * t;
        if (q < nl) lmin = min(lmin, hd[a0 + q]);
      }
      const int mn = (int)__reduce_min_sync(kFull, (unsigned)lmin);
      if (mn == kNoCol) break;
      double acc = 0.0;
      bool started = false;
      for (int t = 0; t < T; ++t) {
        const int q = lane + 32 * t;
        const bool has = q < nl && hd[a0 + q] == mn;
        double prod = 0.0;
        if (has) prod = __dmul_rn(av[a0 + q], bv[cur[a0 + q]]);
        unsigned msk = __ballot_sync(kFull, has);
        while (msk) {
          const int l = __ffs(msk) - 1;
          const double x = __shfl_sync(kFull, prod, l);
          acc = started ? __dadd_rn(acc, x) : x;
          started = true;
          msk &= msk - 1;
        }
        if (has) {
          const int k = aci[a0 + q];
          const int np = cur[a0 + q] + 1;
          cur[a0 + q] = np;
          hd[a0 + q] = np < brp[k + 1] ? bci[np] : kNoCol;
        }
      }
      __syncwarp();
      if (lane == 0) {
        tci[o] = mn;
        tv[o] = acc;
      }
      ++o;
    }
  }
  if (lane == 0) cnt[i] = o - off[i];
}

__global__ void k_spgemm_compact(int m, const int64_t* __restrict__ off, const int64_t* __restrict__ crp64,
                                 const int* __restrict__ tci, const double* __restrict__ tv, int* __restrict__ cci,
                                 double* __restrict__ cv) {
  const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= m) return;
  const int64_t src = off[i], dst = crp64[i], len = crp64[i + 1] - crp64[i];
  for (int64_t k = lane; k < len; k += 32) {
    cci[dst + k] = tci[src + k];
    cv[dst + k] = tv[src + k];
  }
}

// ---- ILU(0) by fixed-point sweeps -----------------------------------------------------------
// For entry e = (i, j): the pairs (position of l_ik, position of u_kj), k < min(i, j), with both
// positions on the pattern; counted, then filled in the order of row i.
__device__ __forceinline__ int find_col(const int* __restrict__ ci, int b, int e, int j) {
  while (b < e) {
    const int mid = (b + e) >> 1;
    if (ci[mid] < j) b = mid + 1;
    else e = mid;
  }
  return b;
}

__global__ void k_ilu_pairs(int64_t nnz, const int* __restrict__ row, const int* __restrict__ rp, const int* __restrict__ ci,
                            const int64_t* __restrict__ pstart, int64_t* __restrict__ cnt, int64_t* __restrict__ pik,
                            int64_t* __restrict__ pkj) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = row[e], j = ci[e];
    const int kmax = min(i, j);
    int64_t c = 0, w = pstart ? pstart[e] : 0;
    for (int r = rp[i]; r < rp[i + 1] && ci[r] < kmax; ++r) {
      const int k = ci[r];
      const int f = find_col(ci, rp[k], rp[k + 1], j);
      if (f < rp[k + 1] && ci[f] == j) {
        if (pstart) {
          pik[w] = r;
          pkj[w] = f;
          ++w;
        }
        ++c;
      }
    }
    if (!pstart) cnt[e] = c;
  }
}

__global__ void k_ilu_init(int64_t nnz, const int* __restrict__ row, const int* __restrict__ ci, const double* __restrict__ a,
                           const int* __restrict__ dpos, double* __restrict__ x, int64_t* __restrict__ dpos64) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = row[e], j = ci[e];
    x[e] = (j < i) ? a[e] / a[dpos[j]] : a[e];
    if (i == j) dpos64[i] = e;
  }
}

// One Jacobi-style sweep: reads `old`, writes `nw`; the exact ILU(0) factors are its fixed point.
//   i > j:  l_ij = (a_ij - sum l_ik u_kj) / u_jj        i <= j:  u_ij = a_ij - sum l_ik u_kj
__global__ void k_ilu_fp_sweep(int64_t nnz, const int* __restrict__ row, const int* __restrict__ col,
                               const double* __restrict__ a, const int64_t* __restrict__ pstart,
                               const int64_t* __restrict__ pik, const int64_t* __restrict__ pkj,
                               const int64_t* __restrict__ dpos, const double* __restrict__ old, double* __restrict__ nw) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    double s = a[e];
    for (int64_t q = pstart[e]; q < pstart[e + 1]; ++q) s = fma(-old[pik[q]], old[pkj[q]], s);
    const int i = row[e], j = col[e];
    nw[e] = (i > j) ? s / old[dpos[j]] : s;
  }
}

// Split the combined factors into L_s (strictly lower), U_s = diag(U)^-1 (strict upper of U) and
// dinv = 1 / u_ii; lrp/urp are the scanned per-row counts.
__global__ void k_ilu_split(int n, const int* __restrict__ rp, const int* __restrict__ ci, const int* __restrict__ dpos,
                            const double* __restrict__ lu, const int* __restrict__ lrp, const int* __restrict__ urp,
                            int* __restrict__ lci, double* __restrict__ lv, int* __restrict__ uci, double* __restrict__ uv,
                            double* __restrict__ dinv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int d = dpos[i];
  const double di = 1.0 / lu[d];
  dinv[i] = di;
  int o = lrp[i];
  for (int p = rp[i]; p < d; ++p, ++o) {
    lci[o] = ci[p];
    lv[o] = lu[p];
  }
  o = urp[i];
  for (int p = d + 1; p < rp[i + 1]; ++p, ++o) {
    uci[o] = ci[p];
    uv[o] = __dmul_rn(di, lu[p]);
  }
}

__global__ void k_lower_upper_counts(int n, const int* __restrict__ rp, const int* __restrict__ dpos, int* __restrict__ lc,
                                     int* __restrict__ uc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  lc[i] = dpos[i] - rp[i];
  uc[i] = rp[i + 1] - dpos[i] - 1;
}

// ---- dense inverse of the coarsest operator (Gauss-Jordan, partial pivoting) ----------------
// M is n x 2n row-major: [A | I] on entry, [I | A^-1] on exit.
__global__ void k_dense_from_csr(int n, const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ v,
                                 double* __restrict__ M) {
  const int i = blockIdx.x;
  if (i >= n) return;
  for (int j = threadIdx.x; j < 2 * n; j += blockDim.x) M[(int64_t)i * 2 * n + j] = (j - n == i) ? 1.0 : 0.0;
  __syncthreads();
  for (int p = rp[i] + threadIdx.x; p < rp[i + 1]; p += blockDim.x) M[(int64_t)i * 2 * n + ci[p]] = v[p];
}

// Pivot of column c: the largest |M[r][c]| over r >= c (smallest r on ties); the rows are
// swapped, the pivot row is scaled to a unit pivot and column c is saved for the elimination.
__global__ void k_gj_pivot(int n, int c, double* __restrict__ M, double* __restrict__ colc, int* __restrict__ singular) {
  __shared__ double bv[kSetupThreads];
  __shared__ int br[kSetupThreads];
  const int t = threadIdx.x;
  const int64_t w = 2 * (int64_t)n;
  double best = -1.0;
  int brow = n;
  for (int r = c + t; r < n; r += blockDim.x) {
    const double a = fabs(M[r * w + c]);
    if (a > best) {
      best = a;
      brow = r;
    }
  }
  bv[t] = best;
  br[t] = brow;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (t < h && (bv[t + h] > bv[t] || (bv[t + h] == bv[t] && br[t + h] < br[t]))) {
      bv[t] = bv[t + h];
      br[t] = br[t + h];
    }
    __syncthreads();
  }
  const int pr = br[0];
  if (bv[0] <= 0.0 || pr >= n) {
    if (t == 0) *singular = 1;
    return;
  }
  if (pr != c)
    for (int64_t j = t; j < w; j += blockDim.x) {
      const double x = M[(int64_t)c * w + j];
      M[(int64_t)c * w + j] = M[(int64_t)pr * w + j];
      M[(int64_t)pr * w + j] = x;
    }
  __syncthreads();
  const double inv = 1.0 / M[(int64_t)c * w + c];
  __syncthreads();
  for (int64_t j = t; j < w; j += blockDim.x) M[(int64_t)c * w + j] *= inv;
  __syncthreads();
  for (int r = t; r < n; r += blockDim.x) colc[r] = M[(int64_t)r * w + c];
}

__global__ void k_gj_eliminate(int n, int c, double* __restrict__ M, const double* __restrict__ colc,
                               const int* __restrict__ singular) {
  if (*singular) return;
  const int r = blockIdx.y;
  if (r == c) return;
  const double f = colc[r];
  if (f == 0.0) return;
  const int64_t w = 2 * (int64_t)n;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < w; j += (int64_t)gridDim.x * blockDim.x)
    M[r * w + j] -= f * M[(int64_t)c * w + j];
}

__global__ void k_gj_extract(int n, const double* __restrict__ M, double* __restrict__ inv) {
  const int i = blockIdx.x;
  for (int j = threadIdx.x; j < n; j += blockDim.x) inv[(int64_t)i * n + j] = M[(int64_t)i * 2 * n + n + j];
}

// ==============================================================================================
// Host orchestration
// ==============================================================================================
struct GCsr {
  int n = 0, m = 0;
  int64_t nnz = 0;
  int *rp = nullptr, *ci = nullptr;
  double* v = nullptr;
};

struct GLevel {
  GCsr A, P, R, L, U;
  unsigned char* s = nullptr;  // strength flags (one per entry of A)
  int* cf = nullptr;           // coarse index or -1
  int nc = 0;
  double* dinv = nullptr;
  bool has_ilu = false;
};

// Device copy of a host CSR.
int upload_csr(DMem& mem, const nsamg_csr& h, GCsr& d, cudaStream_t s) {
  d.n = h.nrows;
  d.m = h.ncols;
  d.nnz = h.nnz;
  SK(mem.alloc(&d.rp, d.n + 1));
  SK(mem.alloc(&d.ci, d.nnz));
  SK(mem.alloc(&d.v, d.nnz));
  CK(cudaMemcpyAsync(d.rp, h.rowptr, sizeof(int) * (d.n + 1), cudaMemcpyHostToDevice, s));
  if (d.nnz) {
    CK(cudaMemcpyAsync(d.ci, h.col, sizeof(int) * d.nnz, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d.v, h.val, sizeof(double) * d.nnz, cudaMemcpyHostToDevice, s));
  }
  return NSAMG_OK;
}

// Row pointers from int counts: rp = exclusive scan (int64 on the device, checked against int32).
int rowptr_from_counts(DMem& mem, const int* cnt, int n, int** rp, int64_t* total, cudaStream_t s) {
  int64_t *c64 = nullptr, *r64 = nullptr;
  CK(cudaMallocAsync((void**)&c64, sizeof(int64_t) * std::max(n, 1), s));
  CK(cudaMallocAsync((void**)&r64, sizeof(int64_t) * (n + 1), s));
  k_cast_i32_i64<<<nblocks(n), kSetupThreads, 0, s>>>(cnt, n, c64);
  int rc = scan_excl<int64_t>(c64, r64, n, s);
  if (rc == NSAMG_OK) rc = read_scalar(r64 + n, total, s);
  if (rc == NSAMG_OK && *total > INT32_MAX) rc = fail(NSAMG_ERR_BAD_MATRIX, "setup: more than 2^31 - 1 entries in one matrix");
  if (rc == NSAMG_OK) rc = mem.alloc(rp, n + 1);
  if (rc == NSAMG_OK) k_narrow_i64_i32<<<nblocks(n + 1), kSetupThreads, 0, s>>>(r64, n + 1, *rp);
  cudaFreeAsync(c64, s);
  cudaFreeAsync(r64, s);
  if (rc != NSAMG_OK) return rc;
  CK(cudaGetLastError());
  return NSAMG_OK;
}

// Transpose (pattern of the flagged entries, or all entries with values) with sorted rows.
int transpose(DMem& mem, const GCsr& A, const unsigned char* flag, bool values, GCsr& T, cudaStream_t s) {
  int* cnt = nullptr;
  CK(cudaMallocAsync((void**)&cnt, sizeof(int) * std::max(A.m, 1), s));
  CK(cudaMemsetAsync(cnt, 0, sizeof(int) * std::max(A.m, 1), s));
  k_count_cols<<<nblocks_warp_rows(A.n), kSetupThreads, 0, s>>>(A.n, A.rp, A.ci, flag, cnt);
  T.n = A.m;
  T.m = A.n;
  int rc = rowptr_from_counts(mem, cnt, A.m, &T.rp, &T.nnz, s);
  if (rc == NSAMG_OK) rc = mem.alloc(&T.ci, T.nnz);
  if (rc == NSAMG_OK && values) rc = mem.alloc(&T.v, T.nnz);
  if (rc == NSAMG_OK) {
    CK(cudaMemcpyAsync(cnt, T.rp, sizeof(int) * std::max(A.m, 1), cudaMemcpyDeviceToDevice, s));
    k_transpose_fill<<<nblocks_warp_rows(A.n), kSetupThreads, 0, s>>>(A.n, A.rp, A.ci, A.v, flag, cnt, T.ci,
                                                                     values ? T.v : nullptr);
    if (values) k_sort_rows<<<nblocks(T.n), kSetupThreads, 0, s>>>(T.n, T.rp, T.ci, T.v);
  }
  cudaFreeAsync(cnt, s);
  if (rc != NSAMG_OK) return rc;
  CK(cudaGetLastError());
  return NSAMG_OK;
}

// C = A B.
int spgemm(DMem& mem, const GCsr& A, const GCsr& B, GCsr& C, cudaStream_t s) {
  const int m = A.n;
  int64_t *ub = nullptr, *off = nullptr, *cnt = nullptr, *crp64 = nullptr;
  int *tci = nullptr, *cur = nullptr, *hd = nullptr;
  double* tv = nullptr;
  int rc = NSAMG_OK;
  int64_t total = 0;
  auto done = [&]() {
    cudaFreeAsync(ub, s);
    cudaFreeAsync(off, s);
    cudaFreeAsync(cnt, s);
    cudaFreeAsync(crp64, s);
    cudaFreeAsync(tci, s);
    cudaFreeAsync(tv, s);
    cudaFreeAsync(cur, s);
    cudaFreeAsync(hd, s);
  };
#define SG(call)                                  \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) {                      \
      done();                                     \
      return cuda_fail(e_, "setup SpGEMM");       \
    }                                             \
  } while (0)
  SG(cudaMallocAsync((void**)&ub, sizeof(int64_t) * std::max(m, 1), s));
  SG(cudaMallocAsync((void**)&off, sizeof(int64_t) * (m + 1), s));
  SG(cudaMallocAsync((void**)&cnt, sizeof(int64_t) * std::max(m, 1), s));
  SG(cudaMallocAsync((void**)&crp64, sizeof(int64_t) * (m + 1), s));
  SG(cudaMallocAsync((void**)&cur, sizeof(int) * std::max<int64_t>(A.nnz, 1), s));
  SG(cudaMallocAsync((void**)&hd, sizeof(int) * std::max<int64_t>(A.nnz, 1), s));
  k_spgemm_ub<<<nblocks_warp_rows(m), kSetupThreads, 0, s>>>(m, A.rp, A.ci, B.rp, ub);
  rc = scan_excl<int64_t>(ub, off, m, s);
  if (rc == NSAMG_OK) rc = read_scalar(off + m, &total, s);
  if (rc != NSAMG_OK) {
    done();
    return rc;
  }
  SG(cudaMallocAsync((void**)&tci, sizeof(int) * std::max<int64_t>(total, 1), s));
  SG(cudaMallocAsync((void**)&tv, sizeof(double) * std::max<int64_t>(total, 1), s));
  k_spgemm_merge<<<nblocks_warp_rows(m), kSetupThreads, 0, s>>>(m, A.rp, A.ci, A.v, B.rp, B.ci, B.v, off, tci, tv, cnt,
                                                                cur, hd);
  rc = scan_excl<int64_t>(cnt, crp64, m, s);
  C.n = m;
  C.m = B.m;
  if (rc == NSAMG_OK) rc = read_scalar(crp64 + m, &C.nnz, s);
  if (rc == NSAMG_OK && C.nnz > INT32_MAX) rc = fail(NSAMG_ERR_BAD_MATRIX, "setup: Galerkin product exceeds 2^31 - 1 entries");
  if (rc == NSAMG_OK) rc = mem.alloc(&C.rp, m + 1);
  if (rc == NSAMG_OK) rc = mem.alloc(&C.ci, C.nnz);
  if (rc == NSAMG_OK) rc = mem.alloc(&C.v, C.nnz);
  if (rc == NSAMG_OK) {
    k_narrow_i64_i32<<<nblocks(m + 1), kSetupThreads, 0, s>>>(crp64, m + 1, C.rp);
    k_spgemm_compact<<<nblocks_warp_rows(m), kSetupThreads, 0, s>>>(m, off, crp64, tci, tv, C.ci, C.v);
  }
  done();
#undef SG
  if (rc != NSAMG_OK) return rc;
  CK(cudaGetLastError());
  return NSAMG_OK;
}

// MM-ext prolongation of level L (needs L.s, L.cf, L.nc).
int interpolate_mmext(DMem& mem, GLevel& L, cudaStream_t s) {
  const GCsr& A = L.A;
  const int n = A.n;
  DMem tmp;
  int *flag = nullptr, *fidx = nullptr, *c1 = nullptr, *c2 = nullptr, *bad = nullptr, *cnt = nullptr;
  SK(tmp.alloc(&flag, n));
  SK(tmp.alloc(&fidx, n + 1));
  SK(tmp.alloc(&bad, 1));
  SK(tmp.alloc(&cnt, n));
  k_flag_f<<<nblocks(n), kSetupThreads, 0, s>>>(n, L.cf, flag);
  SK(scan_excl<int>(flag, fidx, n, s));
  int nF = 0;
  SK(read_scalar(fidx + n, &nF, s));
  GCsr M1, M2, W;
  M1.n = M1.m = nF;
  M2.n = nF;
  M2.m = L.nc;
  SK(tmp.alloc(&c1, nF));
  SK(tmp.alloc(&c2, nF));
  k_mmext_count<<<nblocks(n), kSetupThreads, 0, s>>>(n, A.rp, A.ci, L.s, L.cf, fidx, c1, c2);
  SK(rowptr_from_counts(tmp, c1, nF, &M1.rp, &M1.nnz, s));
  SK(rowptr_from_counts(tmp, c2, nF, &M2.rp, &M2.nnz, s));
  SK(tmp.alloc(&M1.ci, M1.nnz));
  SK(tmp.alloc(&M1.v, M1.nnz));
  SK(tmp.alloc(&M2.ci, M2.nnz));
  SK(tmp.alloc(&M2.v, M2.nnz));
  const int big = INT32_MAX;
  CK(cudaMemcpyAsync(bad, &big, sizeof(int), cudaMemcpyHostToDevice, s));
  k_mmext_fill<<<nblocks(n), kSetupThreads, 0, s>>>(n, A.rp, A.ci, A.v, L.s, L.cf, fidx, M1.rp, M1.ci, M1.v, M2.rp, M2.ci,
                                                     M2.v, bad);
  int hbad = 0;
  SK(read_scalar(bad, &hbad, s));
  if (hbad != INT32_MAX)
    return fail(NSAMG_ERR_BAD_MATRIX, "setup: MM-ext interpolation undefined in row " + std::to_string(hbad) +
                                          " (a_ii + gamma_i = 0)");
  SK(spgemm(tmp, M1, M2, W, s));
  k_mmext_pcount<<<nblocks(n), kSetupThreads, 0, s>>>(n, L.cf, fidx, W.rp, cnt);
  L.P.n = n;
  L.P.m = L.nc;
  SK(rowptr_from_counts(mem, cnt, n, &L.P.rp, &L.P.nnz, s));
  SK(mem.alloc(&L.P.ci, L.P.nnz));
  SK(mem.alloc(&L.P.v, L.P.nnz));
  k_mmext_pfill<<<nblocks(n), kSetupThreads, 0, s>>>(n, L.cf, fidx, W.rp, W.ci, W.v, L.P.rp, L.P.ci, L.P.v);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return NSAMG_OK;
}

// Strength flags, PMIS splitting (cf, nc) of level A.
int coarsen(DMem& mem, GLevel& L, double theta, int neg_mode, uint64_t seed, cudaStream_t s, int* rounds_out) {
  const GCsr& A = L.A;
  const int n = A.n;
  SK(mem.alloc(&L.s, A.nnz));
  SK(mem.alloc(&L.cf, n));
  k_strength<<<nblocks_warp_rows(n), kSetupThreads, 0, s>>>(n, A.rp, A.ci, A.v, theta, neg_mode, L.s);
  DMem tmp;
  GCsr ST;
  SK(transpose(tmp, A, L.s, false, ST, s));
  double* lam = nullptr;
  unsigned char *st = nullptr, *mark = nullptr;
  int *und = nullptr, *flag = nullptr, *off = nullptr, *h_und = nullptr;
  SK(tmp.alloc(&lam, n));
  SK(tmp.alloc(&st, n));
  SK(tmp.alloc(&mark, n));
  SK(tmp.alloc(&und, 1));
  SK(tmp.alloc(&flag, n));
  SK(tmp.alloc(&off, n + 1));
  k_pmis_init<<<nblocks(n), kSetupThreads, 0, s>>>(n, ST.rp, seed, lam, st);
  CK(cudaMallocHost((void**)&h_und, sizeof(int)));
  int rounds = 0, rc = NSAMG_OK;
  const int64_t max_rounds = 10 * (int64_t)n + 10;  // every round decides at least one point
  for (; rounds < max_rounds; ++rounds) {
    cudaMemsetAsync(und, 0, sizeof(int), s);
    k_pmis_select<<<nblocks(n), kSetupThreads, 0, s>>>(n, A.rp, A.ci, L.s, ST.rp, ST.ci, lam, st, mark, und);
    k_pmis_apply<<<nblocks(n), kSetupThreads, 0, s>>>(n, A.rp, A.ci, L.s, mark, st);
    cudaError_t e = cudaMemcpyAsync(h_und, und, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "setup PMIS round");
      break;
    }
    if (*h_und == 0) break;
  }
  cudaFreeHost(h_und);
  if (rc != NSAMG_OK) return rc;
  if (rounds_out) *rounds_out = rounds;
  // promotion of F-points without a strong C-neighbour
  k_promote_cand<<<nblocks(n), kSetupThreads, 0, s>>>(n, A.rp, A.ci, L.s, st, mark);
  k_is_c<<<nblocks(n), kSetupThreads, 0, s>>>(n, st, mark, flag);
  SK(scan_excl<int>(flag, off, n, s));
  k_cf_number<<<nblocks(n), kSetupThreads, 0, s>>>(n, flag, off, L.cf);
  SK(read_scalar(off + n, &L.nc, s));
  CK(cudaGetLastError());
  return NSAMG_OK;
}

int interpolate(DMem& mem, GLevel& L, cudaStream_t s) {
  const GCsr& A = L.A;
  const int n = A.n;
  DMem tmp;
  int *cnt = nullptr, *bad = nullptr;
  SK(tmp.alloc(&cnt, n));
  SK(tmp.alloc(&bad, 1));
  k_interp_count<<<nblocks(n), kSetupThreads, 0, s>>>(n, A.rp, A.ci, L.s, L.cf, cnt);
  L.P.n = n;
  L.P.m = L.nc;
  SK(rowptr_from_counts(mem, cnt, n, &L.P.rp, &L.P.nnz, s));
  SK(mem.alloc(&L.P.ci, L.P.nnz));
  SK(mem.alloc(&L.P.v, L.P.nnz));
  const int big = INT32_MAX;
  CK(cudaMemcpyAsync(bad, &big, sizeof(int), cudaMemcpyHostToDevice, s));
  k_interp_fill<<<nblocks(n), kSetupThreads, 0, s>>>(n, A.rp, A.ci, A.v, L.s, L.cf, L.P.rp, L.P.ci, L.P.v, bad);
  int hbad = 0;
  SK(read_scalar(bad, &hbad, s));
  if (hbad != INT32_MAX)
    return fail(NSAMG_ERR_BAD_MATRIX, "setup: interpolation undefined in row " + std::to_string(hbad) +
                                          " (no strong C-neighbour or zero denominator)");
  CK(cudaGetLastError());
  return NSAMG_OK;
}

// ILU(0) pair lists of A on the device; returns the arrays the sweep kernel reads.
struct IluPairs {
  int* row = nullptr;
  int* dpos = nullptr;
  int64_t *pstart = nullptr, *pik = nullptr, *pkj = nullptr, *dpos64 = nullptr;
  int64_t npairs = 0;
};

int ilu_pairs(DMem& mem, const GCsr& A, IluPairs& P, cudaStream_t s) {
  const int n = A.n;
  SK(mem.alloc(&P.row, A.nnz));
  SK(mem.alloc(&P.dpos, n));
  SK(mem.alloc(&P.dpos64, n));
  SK(mem.alloc(&P.pstart, A.nnz + 1));
  int64_t* cnt = nullptr;
  SK(mem.alloc(&cnt, A.nnz));
  k_row_index<<<nblocks_warp_rows(n), kSetupThreads, 0, s>>>(n, A.rp, P.row);
  k_diag_pos<<<nblocks(n), kSetupThreads, 0, s>>>(n, A.rp, A.ci, P.dpos);
  const int nb = std::min(nblocks(A.nnz), 148 * 16);
  k_ilu_pairs<<<nb, kSetupThreads, 0, s>>>(A.nnz, P.row, A.rp, A.ci, nullptr, cnt, nullptr, nullptr);
  SK(scan_excl<int64_t>(cnt, P.pstart, A.nnz, s));
  SK(read_scalar(P.pstart + A.nnz, &P.npairs, s));
  mem.release(cnt);
  SK(mem.alloc(&P.pik, P.npairs));
  SK(mem.alloc(&P.pkj, P.npairs));
  k_ilu_pairs<<<nb, kSetupThreads, 0, s>>>(A.nnz, P.row, A.rp, A.ci, P.pstart, nullptr, P.pik, P.pkj);
  CK(cudaGetLastError());
  return NSAMG_OK;
}

// Fixed-point ILU(0): the combined factors (L_s below, U on and above the diagonal) in `lu`.
int ilu_fixed_point(DMem& mem, const GCsr& A, const IluPairs& P, int sweeps, double** lu, cudaStream_t s) {
  double *x = nullptr, *y = nullptr;
  SK(mem.alloc(&x, A.nnz));
  SK(mem.alloc(&y, A.nnz));
  const int nb = std::min(nblocks(A.nnz), 148 * 16);
  k_ilu_init<<<nb, kSetupThreads, 0, s>>>(A.nnz, P.row, A.ci, A.v, P.dpos, x, P.dpos64);
  for (int it = 0; it < sweeps; ++it) {
    k_ilu_fp_sweep<<<nb, kSetupThreads, 0, s>>>(A.nnz, P.row, A.ci, A.v, P.pstart, P.pik, P.pkj, P.dpos64, x, y);
    std::swap(x, y);
  }
  CK(cudaGetLastError());
  mem.release(y);
  *lu = x;
  return NSAMG_OK;
}

int ilu_level(DMem& mem, GLevel& L, int sweeps, cudaStream_t s) {
  const GCsr& A = L.A;
  const int n = A.n;
  DMem tmp;
  IluPairs P;
  SK(ilu_pairs(tmp, A, P, s));
  double* lu = nullptr;
  SK(ilu_fixed_point(tmp, A, P, sweeps, &lu, s));
  int *lc = nullptr, *uc = nullptr;
  SK(tmp.alloc(&lc, n));
  SK(tmp.alloc(&uc, n));
  k_lower_upper_counts<<<nblocks(n), kSetupThreads, 0, s>>>(n, A.rp, P.dpos, lc, uc);
  L.L.n = L.L.m = L.U.n = L.U.m = n;
  SK(rowptr_from_counts(mem, lc, n, &L.L.rp, &L.L.nnz, s));
  SK(rowptr_from_counts(mem, uc, n, &L.U.rp, &L.U.nnz, s));
  SK(mem.alloc(&L.L.ci, L.L.nnz));
  SK(mem.alloc(&L.L.v, L.L.nnz));
  SK(mem.alloc(&L.U.ci, L.U.nnz));
  SK(mem.alloc(&L.U.v, L.U.nnz));
  SK(mem.alloc(&L.dinv, n));
  k_ilu_split<<<nblocks(n), kSetupThreads, 0, s>>>(n, A.rp, A.ci, P.dpos, lu, L.L.rp, L.U.rp, L.L.ci, L.L.v, L.U.ci, L.U.v,
                                                    L.dinv);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  L.has_ilu = true;
  return NSAMG_OK;
}

int coarse_inverse(DMem& mem, const GCsr& A, double** inv, cudaStream_t s) {
  const int n = A.n;
  DMem tmp;
  double *M = nullptr, *colc = nullptr;
  int* sing = nullptr;
  SK(tmp.alloc(&M, 2 * (int64_t)n * n));
  SK(tmp.alloc(&colc, n));
  SK(tmp.alloc(&sing, 1));
  SK(mem.alloc(inv, (int64_t)n * n));
  CK(cudaMemsetAsync(sing, 0, sizeof(int), s));
  k_dense_from_csr<<<n, kSetupThreads, 0, s>>>(n, A.rp, A.ci, A.v, M);
  const dim3 eg((unsigned)std::max(1, std::min(8, (2 * n + kSetupThreads - 1) / kSetupThreads)), (unsigned)n);
  for (int c = 0; c < n; ++c) {
    k_gj_pivot<<<1, kSetupThreads, 0, s>>>(n, c, M, colc, sing);
    k_gj_eliminate<<<eg, kSetupThreads, 0, s>>>(n, c, M, colc, sing);
  }
  k_gj_extract<<<n, kSetupThreads, 0, s>>>(n, M, *inv);
  int hs = 0;
  SK(read_scalar(sing, &hs, s));
  if (hs) return fail(NSAMG_ERR_BAD_MATRIX, "setup: coarsest operator is singular");
  CK(cudaGetLastError());
  return NSAMG_OK;
}

}  // namespace gsetup

// Page-locked host array (export mirrors: device-to-host copies at full link speed, and the
// solver setup uploads from it at the same speed).
template <typename T>
struct PinnedArray {
  T* p = nullptr;
  size_t n = 0;
  PinnedArray() = default;
  PinnedArray(const PinnedArray&) = delete;
  PinnedArray& operator=(const PinnedArray&) = delete;
  PinnedArray(PinnedArray&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr, o.n = 0; }
  PinnedArray& operator=(PinnedArray&& o) noexcept {
    std::swap(p, o.p);
    std::swap(n, o.n);
    return *this;
  }
  ~PinnedArray() {
    if (p) cudaFreeHost(p);
  }
  cudaError_t resize(size_t k) {
    if (k <= n && p) return cudaSuccess;
    if (p) cudaFreeHost(p);
    p = nullptr;
    n = 0;
    cudaError_t e = cudaMallocHost((void**)&p, sizeof(T) * std::max<size_t>(k, 1));
    if (e == cudaSuccess) n = k;
    return e;
  }
  T* data() const { return p; }
};

// The hierarchy built on the device, with host mirrors filled on export.
struct nsamg_amg {
  gsetup::DMem mem;
  std::vector<gsetup::GLevel> levels;
  double* coarse_inv = nullptr;  // device, n_L^2, or null
  std::vector<int> pmis_rounds;
  // host mirrors (export)
  struct HostCsr {
    PinnedArray<int> rp, ci;
    PinnedArray<double> v;
    int n = 0, m = 0;
  };
  struct HostLevel {
    HostCsr A, P, R, L, U;
    PinnedArray<double> dinv;
  };
  std::vector<HostLevel> host;
  PinnedArray<double> host_cinv;
  std::vector<nsamg_level_desc> descs;
};

namespace gsetup {

int download_csr(const GCsr& d, nsamg_amg::HostCsr& h, cudaStream_t s) {
  h.n = d.n;
  h.m = d.m;
  CK(h.rp.resize(d.n + 1));
  CK(h.ci.resize(std::max<int64_t>(d.nnz, 1)));
  CK(h.v.resize(std::max<int64_t>(d.nnz, 1)));
  if (d.rp) CK(cudaMemcpyAsync(h.rp.data(), d.rp, sizeof(int) * (d.n + 1), cudaMemcpyDeviceToHost, s));
  if (d.nnz) {
    CK(cudaMemcpyAsync(h.ci.data(), d.ci, sizeof(int) * d.nnz, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h.v.data(), d.v, sizeof(double) * d.nnz, cudaMemcpyDeviceToHost, s));
  }
  return NSAMG_OK;
}

nsamg_csr host_view(const nsamg_amg::HostCsr& h, int64_t nnz) {
  nsamg_csr c;
  c.nrows = h.n;
  c.ncols = h.m;
  c.nnz = nnz;
  c.rowptr = h.n ? h.rp.data() : nullptr;
  c.col = h.ci.data();
  c.val = h.v.data();
  return c;
}

int build(const nsamg_csr& A0, const nsamg_amg_options& o, nsamg_amg* g, cudaStream_t s) {
  g->levels.emplace_back();
  SK(upload_csr(g->mem, A0, g->levels[0].A, s));
  while ((int)g->levels.size() < o.max_levels && g->levels.back().A.n > o.coarse_max) {
    const int l = (int)g->levels.size() - 1;
    GLevel& L = g->levels[l];
    int rounds = 0;
    SK(coarsen(g->mem, L, o.theta, o.strength_mode, o.seed + 7919ull * (uint64_t)(l + 1), s, &rounds));
    g->pmis_rounds.push_back(rounds);
    if (L.nc == 0 || (double)L.nc >= 0.9 * L.A.n) break;
    SK(o.interp == 1 ? interpolate_mmext(g->mem, L, s) : interpolate(g->mem, L, s));
    SK(transpose(g->mem, L.P, nullptr, true, L.R, s));
    DMem tmp;
    GCsr AP, Ac;
    SK(spgemm(tmp, L.A, L.P, AP, s));
    SK(spgemm(g->mem, L.R, AP, Ac, s));
    CK(cudaStreamSynchronize(s));
    g->levels.emplace_back();
    g->levels.back().A = Ac;
  }
  const int nl = (int)g->levels.size();
  for (int l = 0; l < nl - 1 && l < 64; ++l)
    if ((o.ilu_levels >> l) & 1ull) SK(ilu_level(g->mem, g->levels[l], o.ilu_sweeps, s));
  if (g->levels.back().A.n <= o.direct_max) SK(coarse_inverse(g->mem, g->levels.back().A, &g->coarse_inv, s));
  CK(cudaStreamSynchronize(s));
  return NSAMG_OK;
}

}  // namespace gsetup

// ==============================================================================================
// Solver handle straight from the device hierarchy (no host round trip): the per-level arrays the
// solve phase needs (D^-1, the l1 diagonal, the pre-scaled triangles, the plain SELL copies of
// near-uniform matrices, ILU(0) factors, transfers, coarse inverse) are formed by kernels from the
// GPU-built operators, with the same arithmetic as the host path. Matrices that are not near-
// uniform get no SELL copy here (the host path's sorted SELL-32-sigma layout is not built).
// ==============================================================================================
namespace gsetup {

// D^-1, the l1 row sums' inverses and max_i sum_j |a_ij| (flags[0], as the bits of a non-negative
// double, which order like the values); flags[1] gets bit 0 for a row with a missing or zero
// diagonal and bit 1 for a non-finite entry.
__global__ void k_diag_l1(int n, const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ v,
                          double* __restrict__ dinv, double* __restrict__ dl1, unsigned long long* __restrict__ flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = 0.0, s1 = 0.0;
  unsigned long long bad = 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    if (ci[p] == i) a = v[p];
    s1 += fabs(v[p]);
    if (!isfinite(v[p])) bad |= 2ull;
  }
  if (a == 0.0) bad |= 1ull;
  dinv[i] = 1.0 / a;
  dl1[i] = 1.0 / s1;
  if (isfinite(s1)) atomicMax(&flags[0], (unsigned long long)__double_as_longlong(s1));
  if (bad) atomicOr(&flags[1], bad);
}

__global__ void k_tri_count(int n, const int* __restrict__ rp, const int* __restrict__ ci, int lower, int* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) c += lower ? (ci[p] < i) : (ci[p] > i);
  cnt[i] = c;
}

// strictly lower (or upper) part, rows scaled by rs and columns by cs (each optional)
__global__ void k_tri_fill(int n, const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ v,
                           int lower, const double* __restrict__ rs, const double* __restrict__ cs, const int* __restrict__ trp,
                           int* __restrict__ tci, double* __restrict__ tv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int o = trp[i];
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    const int c = ci[p];
    if (lower ? c < i : c > i) {
      double x = v[p];
      if (rs) x *= rs[i];
      if (cs) x *= cs[c];
      tci[o] = c;
      tv[o] = x;
      ++o;
    }
  }
}

__global__ void k_chunk_slots(int n, int nch, const int* __restrict__ rp, int64_t* __restrict__ slots) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nch) return;
  int w = 0;
  for (int i = c * 32; i < min(n, c * 32 + 32); ++i) w = max(w, rp[i + 1] - rp[i]);
  slots[c] = 32 * (int64_t)w;
}

__global__ void k_max_slots(int nch, const int64_t* __restrict__ slots, unsigned long long* __restrict__ mx) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nch) atomicMax(mx, (unsigned long long)slots[c]);
}

__global__ void k_set_slots(int nch, int64_t v, int64_t* __restrict__ slots) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nch) slots[c] = v;
}

template <typename T>
__global__ void k_plain_fill(int n, int m, int nch, const int* __restrict__ rp, const int* __restrict__ ci,
                             const T* __restrict__ v, const int64_t* __restrict__ cptr, int* __restrict__ scol,
                             T* __restrict__ sval) {
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= nch * 32) return;
  const int c = pos >> 5, l = pos & 31, row = pos;
  const int w = (int)((cptr[c + 1] - cptr[c]) >> 5);
  const int len = row < n ? rp[row + 1] - rp[row] : 0;
  const int b = row < n ? rp[row] : 0;
  const int pad_col = len > 0 ? ci[b + len - 1] : min(row, m - 1);
  for (int j = 0; j < w; ++j) {
    const int64_t q = cptr[c] + (int64_t)j * 32 + l;
    scol[q] = j < len ? ci[b + j] : pad_col;
    sval[q] = j < len ? v[b + j] : T(0);
  }
}

template <typename TB, typename TA>
__global__ void k_convert(int64_t n, const TA* __restrict__ a, TB* __restrict__ b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = nsamg::convert<TB>(a[i]);
}

// Device CSR (FP64 values) -> DCSR<T> of the solve phase: copy or round the values, plain SELL
// copy when natural-order chunks pad by <= kPlainPad, default threads per row.
template <typename T>
int dev_upload(const GCsr& sc, DCSR<T>& d, cudaStream_t s) {
  d.n = sc.n;
  d.m = sc.m;
  d.nnz = sc.nnz;
  const int64_t cap = std::max<int64_t>(sc.nnz, 1);
  CK(cudaMalloc(&d.rp, sizeof(int) * (sc.n + 1)));
  CK(cudaMalloc(&d.ci, sizeof(int) * cap));
  CK(cudaMalloc(&d.v, sizeof(T) * cap));
  CK(cudaMemcpyAsync(d.rp, sc.rp, sizeof(int) * (sc.n + 1), cudaMemcpyDeviceToDevice, s));
  if (sc.nnz) {
    CK(cudaMemcpyAsync(d.ci, sc.ci, sizeof(int) * sc.nnz, cudaMemcpyDeviceToDevice, s));
    if constexpr (sizeof(T) == sizeof(double)) {
      CK(cudaMemcpyAsync(d.v, sc.v, sizeof(double) * sc.nnz, cudaMemcpyDeviceToDevice, s));
    } else {
      k_convert<T, double><<<nblocks(sc.nnz), kSetupThreads, 0, s>>>(sc.nnz, sc.v, d.v);
    }
  }
  d.G = default_group(sc.n, sc.nnz);
  if (sc.n >= kSellMinRows && sc.nnz > 0) {
    const int nch = (sc.n + 31) / 32;
    int64_t *slots = nullptr, *cptr = nullptr;
    CK(cudaMallocAsync((void**)&slots, sizeof(int64_t) * nch, s));
    CK(cudaMalloc(&cptr, sizeof(int64_t) * (nch + 1)));
    unsigned long long* mx = nullptr;
    CK(cudaMallocAsync((void**)&mx, sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s));
    k_chunk_slots<<<nblocks(nch), kSetupThreads, 0, s>>>(sc.n, nch, sc.rp, slots);
    k_max_slots<<<nblocks(nch), kSetupThreads, 0, s>>>(nch, slots, mx);
    unsigned long long max_slots = 0;
    int rc = read_scalar(mx, &max_slots, s);
    cudaFreeAsync(mx, s);
    // uniform chunk width (the widest chunk's) when that pads by at most kPlainPad, as on the host
    const int wmax = (int)(max_slots / 32);
    const bool uniform = 32.0 * wmax * nch <= kPlainPad * (double)sc.nnz;
    if (rc == NSAMG_OK && uniform) k_set_slots<<<nblocks(nch), kSetupThreads, 0, s>>>(nch, 32 * (int64_t)wmax, slots);
    if (rc == NSAMG_OK) rc = scan_excl<int64_t>(slots, cptr, nch, s);
    int64_t total = 0;
    if (rc == NSAMG_OK) rc = read_scalar(cptr + nch, &total, s);
    cudaFreeAsync(slots, s);
    if (rc != NSAMG_OK) {
      cudaFree(cptr);
      return rc;
    }
    if ((double)total <= kPlainPad * (double)sc.nnz) {
      d.s_width = uniform ? wmax : 0;
      d.s_cptr = cptr;
      CK(cudaMalloc(&d.s_col, sizeof(int) * std::max<int64_t>(total, 1)));
      CK(cudaMalloc(&d.s_val, sizeof(T) * std::max<int64_t>(total, 1)));
      k_plain_fill<T><<<nblocks((int64_t)nch * 32), kSetupThreads, 0, s>>>(sc.n, sc.m, nch, d.rp, d.ci, d.v, d.s_cptr,
                                                                           d.s_col, d.s_val);
      d.nchunks = nch;
      d.sell_k = 1;
    } else {
      cudaFree(cptr);
    }
  }
  CK(cudaGetLastError());
  return NSAMG_OK;
}

template <typename T>
int dev_vec(const double* src, int64_t n, T** d, cudaStream_t s) {
  CK(cudaMalloc(d, sizeof(T) * std::max<int64_t>(n, 1)));
  if constexpr (sizeof(T) == sizeof(double)) {
    CK(cudaMemcpyAsync(*d, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  } else {
    k_convert<T, double><<<nblocks(n), kSetupThreads, 0, s>>>(n, src, *d);
  }
  return NSAMG_OK;
}

// The triangle of A (strict lower / upper), rows scaled by rs, columns by cs, as DCSR<T>.
template <typename T>
int dev_tri(const GCsr& A, bool lower, const double* rs, const double* cs, DCSR<T>& d, cudaStream_t s) {
  DMem tmp;
  int* cnt = nullptr;
  SK(tmp.alloc(&cnt, A.n));
  k_tri_count<<<nblocks(A.n), kSetupThreads, 0, s>>>(A.n, A.rp, A.ci, lower ? 1 : 0, cnt);
  GCsr T0;
  T0.n = T0.m = A.n;
  SK(rowptr_from_counts(tmp, cnt, A.n, &T0.rp, &T0.nnz, s));
  SK(tmp.alloc(&T0.ci, T0.nnz));
  SK(tmp.alloc(&T0.v, T0.nnz));
  k_tri_fill<<<nblocks(A.n), kSetupThreads, 0, s>>>(A.n, A.rp, A.ci, A.v, lower ? 1 : 0, rs, cs, T0.rp, T0.ci, T0.v);
  SK(dev_upload<T>(T0, d, s));
  CK(cudaStreamSynchronize(s));
  return NSAMG_OK;
}

template <typename T>
int dev_build_levels(nsamg_amg* g, const nsamg_params& p, std::vector<Level<T>>& lvs, bool only_A0, double* anorm,
                     cudaStream_t s) {
  const int nl = only_A0 ? 1 : (int)g->levels.size();
  lvs.resize(nl);
  for (int l = 0; l < nl; ++l) {
    const GLevel& G = g->levels[l];
    Level<T>& L = lvs[l];
    L.n = G.A.n;
    SK(dev_upload<T>(G.A, L.A, s));
    if (only_A0) break;
    DMem tmp;
    double *dinv = nullptr, *dl1 = nullptr;
    unsigned long long* flags = nullptr;
    SK(tmp.alloc(&dinv, L.n));
    SK(tmp.alloc(&dl1, L.n));
    SK(tmp.alloc(&flags, 2));
    CK(cudaMemsetAsync(flags, 0, 2 * sizeof(unsigned long long), s));
    k_diag_l1<<<nblocks(L.n), kSetupThreads, 0, s>>>(L.n, G.A.rp, G.A.ci, G.A.v, dinv, dl1, flags);
    unsigned long long hf[2] = {0, 0};
    CK(cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hf[1] & 2ull) return fail(NSAMG_ERR_BAD_MATRIX, "level " + std::to_string(l) + " A: non-finite value");
    if (hf[1] & 1ull) return fail(NSAMG_ERR_BAD_MATRIX, "level " + std::to_string(l) + " A: missing or zero diagonal");
    if (l == 0 && anorm) std::memcpy(anorm, &hf[0], sizeof(double));
    SK(dev_vec<T>(dinv, L.n, &L.dinv, s));
    SK(dev_vec<T>(dl1, L.n, &L.dl1inv, s));
    SK(dev_tri<T>(G.A, true, dinv, dinv, L.L2, s));
    SK(dev_tri<T>(G.A, false, dinv, dinv, L.U2, s));
    SK(dev_tri<T>(G.A, true, dinv, nullptr, L.L1, s));
    SK(dev_tri<T>(G.A, false, dinv, nullptr, L.U1, s));
    if (l < (int)g->levels.size() - 1 && G.P.rp) {
      SK(dev_upload<T>(G.P, L.P, s));
      SK(dev_upload<T>(G.R, L.R, s));
    }
    const bool want_ilu = (p.smoother == NSAMG_SMOOTHER_ILU0) || (p.smoother == NSAMG_SMOOTHER_HYBRID_ILU0 && l == 0);
    if (want_ilu && G.has_ilu) {
      SK(dev_upload<T>(G.L, L.iL, s));
      SK(dev_upload<T>(G.U, L.iU, s));
      SK(dev_vec<T>(G.dinv, L.n, &L.idinv, s));
      L.ilu = true;
    }
    L.kind = (p.smoother == NSAMG_SMOOTHER_JACOBI_L1) ? 'j' : (L.ilu ? 'i' : 'p');
    T** vecs[] = {&L.b, &L.x, &L.r, &L.t1, &L.t2, &L.t3};
    for (T** v : vecs) SK(alloc_vec(v, L.n));
    CK(cudaStreamSynchronize(s));
  }
  return NSAMG_OK;
}

int dev_setup_impl(nsamg_amg* g, const nsamg_params* pp, void* stream, nsamg_handle* h) {
  nsamg_params p;
  nsamg_default_params(&p);
  if (pp) p = *pp;
  int rc = check_params(p);
  if (rc) return rc;
  if (p.ranks != 1)
    return fail(NSAMG_ERR_INVALID_ARG, "nsamg_amg_setup_solver: ranks > 1 needs a host hierarchy (block-diagonal ILU factors)");
  h->p = p;
  CK(cudaGetDevice(&h->device));
  if (stream) {
    h->stream = (cudaStream_t)stream;
  } else {
    CK(cudaStreamCreate(&h->stream));
    h->own_stream = true;
  }
  cudaStream_t s = h->stream;
  h->fp32 = p.vcycle_fp32 == 1;
  double anorm = 0.0;
  SK(dev_build_levels<double>(g, p, h->lv, h->fp32, h->fp32 ? nullptr : &anorm, s));
  if (h->fp32) SK(dev_build_levels<float>(g, p, h->lv32, false, &anorm, s));
  if (g->coarse_inv) {
    h->nc = g->levels.back().A.n;
    const int64_t nc2 = (int64_t)h->nc * h->nc;
    if (h->fp32) SK(dev_vec<float>(g->coarse_inv, nc2, &h->coarse_inv32, s));
    else SK(dev_vec<double>(g->coarse_inv, nc2, &h->coarse_inv, s));
  }
  SK(alloc_workspace(h));
  h->anorm_inf = anorm;
  CK(cudaMemcpy(&h->st->anorm_inf, &h->anorm_inf, sizeof(double), cudaMemcpyHostToDevice));
  SK(tune_levels(h->lv, tuning_scratch(h), h->w, p.spmv_group, p.sell_shape, s));
  if (h->fp32) SK(tune_levels(h->lv32, h->lv32[0].t1, h->lv32[0].t2, p.spmv_group, p.sell_shape, s));
  CK(cudaStreamSynchronize(s));
  SK(build_tail_any(h));
  SK(finish_graph(h));
  CK(cudaGetLastError());
  return NSAMG_OK;
}

}  // namespace gsetup

extern "C" {

void nsamg_amg_default_options(nsamg_amg_options* o) {
  if (!o) return;
  o->theta = 0.25;
  o->strength_mode = 0;
  o->max_levels = 25;
  o->coarse_max = 512;
  o->direct_max = 512;
  o->seed = 0;
  o->ilu_levels = 1;
  o->ilu_sweeps = 3;
  o->interp = 0;
}

int nsamg_amg_build(const nsamg_csr* A, const nsamg_amg_options* opt, void* cuda_stream, nsamg_amg** out) {
  if (out) *out = nullptr;
  if (!A || !opt || !out) return fail(NSAMG_ERR_INVALID_ARG, "nsamg_amg_build: null argument");
  if (!(opt->theta >= 0.0 && opt->theta <= 1.0) || opt->max_levels < 1 || opt->coarse_max < 1 || opt->direct_max < 0 ||
      opt->direct_max > 8192 || opt->ilu_sweeps < 0 || (opt->strength_mode != 0 && opt->strength_mode != 1) ||
      (opt->interp != 0 && opt->interp != 1))
    return fail(NSAMG_ERR_INVALID_ARG, "nsamg_amg_build: option out of range");
  int rc = validate(*A, true, true, "amg A");
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  nsamg_amg* g = new (std::nothrow) nsamg_amg();
  if (!g) return fail(NSAMG_ERR_OOM, "nsamg_amg_build: host allocation");
  rc = gsetup::build(*A, *opt, g, s);
  if (rc != NSAMG_OK) {
    std::string keep = g_err;
    cudaStreamSynchronize(s);
    delete g;
    g_err = keep;
    return rc;
  }
  *out = g;
  return NSAMG_OK;
}

int nsamg_amg_num_levels(const nsamg_amg* g) { return g ? (int)g->levels.size() : 0; }

int nsamg_amg_level_info(const nsamg_amg* g, int l, int32_t* n, int64_t* nnz, int32_t* nc, int32_t* pmis_rounds) {
  if (!g || l < 0 || l >= (int)g->levels.size()) return fail(NSAMG_ERR_INVALID_ARG, "nsamg_amg_level_info: bad level");
  const auto& L = g->levels[l];
  if (n) *n = L.A.n;
  if (nnz) *nnz = L.A.nnz;
  if (nc) *nc = L.cf ? L.nc : 0;
  if (pmis_rounds) *pmis_rounds = l < (int)g->pmis_rounds.size() ? g->pmis_rounds[l] : 0;
  return NSAMG_OK;
}

int nsamg_amg_level_splitting(const nsamg_amg* g, int l, int32_t* cf, uint8_t* strong) {
  if (!g || l < 0 || l >= (int)g->levels.size()) return fail(NSAMG_ERR_INVALID_ARG, "nsamg_amg_level_splitting: bad level");
  const auto& L = g->levels[l];
  if (!L.cf || !L.s) return fail(NSAMG_ERR_INVALID_ARG, "nsamg_amg_level_splitting: level was not coarsened");
  if (cf) CK(cudaMemcpy(cf, L.cf, sizeof(int) * L.A.n, cudaMemcpyDeviceToHost));
  if (strong && L.A.nnz) CK(cudaMemcpy(strong, L.s, L.A.nnz, cudaMemcpyDeviceToHost));
  return NSAMG_OK;
}

int nsamg_amg_export(nsamg_amg* g, nsamg_hierarchy_desc* out) {
  if (!g || !out) return fail(NSAMG_ERR_INVALID_ARG, "nsamg_amg_export: null argument");
  cudaStream_t s = 0;
  const int nl = (int)g->levels.size();
  g->host.clear();
  g->host.resize(nl);
  g->descs.assign(nl, {});
  for (int l = 0; l < nl; ++l) {
    const auto& L = g->levels[l];
    auto& H = g->host[l];
    int rc = gsetup::download_csr(L.A, H.A, s);
    if (!rc && L.P.rp) rc = gsetup::download_csr(L.P, H.P, s);
    if (!rc && L.R.rp) rc = gsetup::download_csr(L.R, H.R, s);
    if (!rc && L.has_ilu) {
      rc = gsetup::download_csr(L.L, H.L, s);
      if (!rc) rc = gsetup::download_csr(L.U, H.U, s);
      if (!rc) {
        cudaError_t e = H.dinv.resize(L.A.n);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(H.dinv.data(), L.dinv, sizeof(double) * L.A.n, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) rc = cuda_fail(e, "nsamg_amg_export");
      }
    }
    if (rc) return rc;
  }
  if (g->coarse_inv) {
    const int64_t nc = g->levels.back().A.n;
    CK(g->host_cinv.resize(nc * nc));
    CK(cudaMemcpyAsync(g->host_cinv.data(), g->coarse_inv, sizeof(double) * nc * nc, cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  for (int l = 0; l < nl; ++l) {
    const auto& L = g->levels[l];
    auto& H = g->host[l];
    nsamg_level_desc& d = g->descs[l];
    std::memset(&d, 0, sizeof(d));
    d.A = gsetup::host_view(H.A, L.A.nnz);
    if (L.P.rp) {
      d.P = gsetup::host_view(H.P, L.P.nnz);
      d.R = gsetup::host_view(H.R, L.R.nnz);
    }
    if (L.has_ilu) {
      d.ilu_L = gsetup::host_view(H.L, L.L.nnz);
      d.ilu_U = gsetup::host_view(H.U, L.U.nnz);
      d.ilu_dinv = H.dinv.data();
      d.ilu_form = 0;
    }
  }
  out->nlevels = nl;
  out->levels = g->descs.data();
  out->coarse_inv = g->coarse_inv ? g->host_cinv.data() : nullptr;
  return NSAMG_OK;
}

int nsamg_amg_setup_solver(nsamg_amg* g, const nsamg_params* p, void* cuda_stream, nsamg_handle** out) {
  if (out) *out = nullptr;
  if (!g || !p || !out) return fail(NSAMG_ERR_INVALID_ARG, "nsamg_amg_setup_solver: null argument");
  nsamg_handle* h = new nsamg_handle();
  const int rc = gsetup::dev_setup_impl(g, p, cuda_stream, h);
  if (rc != NSAMG_OK) {
    std::string keep = g_err;
    destroy_impl(h);
    g_err = keep;
    return rc;
  }
  *out = h;
  return NSAMG_OK;
}

void nsamg_amg_destroy(nsamg_amg* g) {
  if (!g) return;
  cudaDeviceSynchronize();
  delete g;
}

int nsamg_ilu0_fixed_point(const nsamg_csr* A, int sweeps, double* lu_out, void* stream) {
  if (!A || !lu_out || sweeps < 0) return fail(NSAMG_ERR_INVALID_ARG, "bad arguments");
  int rc = validate(*A, true, true, "ilu0 A");
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  gsetup::DMem mem;
  gsetup::GCsr dA;
  gsetup::IluPairs P;
  double* lu = nullptr;
  rc = gsetup::upload_csr(mem, *A, dA, s);
  if (!rc) rc = gsetup::ilu_pairs(mem, dA, P, s);
  if (!rc) rc = gsetup::ilu_fixed_point(mem, dA, P, sweeps, &lu, s);
  if (!rc) {
    cudaError_t e = cudaMemcpyAsync(lu_out, lu, sizeof(double) * A->nnz, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "nsamg_ilu0_fixed_point");
  }
  if (rc) cudaStreamSynchronize(s);
  return rc;
}

}  // extern "C"
