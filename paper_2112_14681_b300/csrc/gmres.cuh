// One-reduce MGS-GMRES device kernels (Algorithm 1 with the truncated projection T = I - L).
//
//   k_gram     step 6: a = [V_i, vt]^T vt, s = [V_i, vt]^T w in one pass, then (last block)
//              steps 7-11: beta = sqrt(a_i), new L row a/beta, r scaled (1/beta, 1/beta^2),
//              h = (I - L) r  (or (I + L)^-1 r), Hessenberg column.
//   k_update   steps 8 and 12: v_i = vt/beta in place, vt_{i+1} = w/beta - V h, plus
//              ||vt_{i+1}||^2 in the same pass; the last block closes column i (H_{i+1,i}),
//              applies the Givens rotations (steps 13-14) and decides whether to stop.
//   k_xupdate  x += sum_j z_j y_j / beta_j (end of a cycle; Z stores unnormalised M^-1 vt_j).
//   k_resid    true residual r = b - A x into V[:,0] with ||r||^2 and ||b||^2, then (last block)
//              the restart / stop decision (eq. relres).
// All reductions: per-block partials in global scratch, the last block to arrive (atomic
// ticket) sums them in fixed block order, so results are bitwise repeatable.
#pragma once
#include "kernels.cuh"

namespace nsamg {

constexpr int kGramThreads = 512;
constexpr int kGramWarps = kGramThreads / 32;
constexpr int kGramSlots = (kMaxM + kGramWarps - 1) / kGramWarps;  // columns per warp
constexpr int kGramTile = 1024;
constexpr int kRedThreads = 256;

struct Scratch {
  double* partials;   // >= blocks * 2 * (kMaxM + 1)
  unsigned* ticket;   // one counter per kernel kind (zero between launches)
};

// Sets the CUDA graph loop condition when running inside a graph (handle != 0).
__device__ __forceinline__ void set_cond(unsigned long long handle, int v) {
  if (handle) cudaGraphSetConditional((cudaGraphConditionalHandle)handle, (unsigned)v);
}

__device__ __forceinline__ bool last_block(unsigned* ticket) {
  __shared__ bool is_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    is_last = (t == gridDim.x - 1);
    if (is_last) *ticket = 0u;  // reset for the next launch (all other blocks already arrived)
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// Fixed-order reduction of nv values over nb block partials (layout partials[b * stride + v])
// into red[v]; called by every thread of the last block.
__device__ inline void reduce_partials(const double* partials, int nb, int stride, int nv, double* red) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int v = warp; v < nv; v += nw) {
    double s = 0.0;
    for (int b = lane; b < nb; b += 32) s += __ldcg(partials + (int64_t)b * stride + v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[v] = s;
  }
  __syncthreads();
}

// ------------------------------------------------------------------------------------------
// Gram: columns 0..i of V (column i is vt), against vt and w.
// standalone: i is given (nsamg_gram); otherwise read from the state and finalised.
// ------------------------------------------------------------------------------------------
struct GramArgs {
  int64_t n;
  const double* V;
  int64_t ldv;
  const double* w;
  GState* st;          // null for the standalone kernel
  int i_standalone;
  double* out;         // standalone: 2(i+1) results
  Scratch scr;
};

__global__ void __launch_bounds__(kGramThreads) k_gram(GramArgs a) {
  pdl_enter();
  __shared__ double s_vt[kGramTile];
  __shared__ double s_w[kGramTile];
  __shared__ double red[2 * (kMaxM + 1)];
  GState* st = a.st;
  if (st && st->stop) return;
  const int i = st ? st->i : a.i_standalone;
  const int ncol = i + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // Warps form C column groups x R row groups (C * R = 16) so that all warps (and all four SM
  // sub-partitions' FP64 units) stay busy whatever the number of columns.
  const int C = ncol <= 1 ? 1 : ncol <= 2 ? 2 : ncol <= 4 ? 4 : ncol <= 8 ? 8 : 16;
  const int R = kGramWarps / C;
  const int cg = warp % C, rg = warp / C;
  const int64_t chunk = ((a.n + gridDim.x - 1) / gridDim.x + kGramTile - 1) / kGramTile * kGramTile;
  const int64_t r0 = (int64_t)blockIdx.x * chunk;
  const int64_t r1 = min(a.n, r0 + chunk);
  const double* vt = a.V + (int64_t)i * a.ldv;
  double acc_a[kGramSlots], acc_s[kGramSlots];
#pragma unroll
  for (int s = 0; s < kGramSlots; ++s) acc_a[s] = acc_s[s] = 0.0;
  for (int64_t t0 = r0; t0 < r1; t0 += kGramTile) {
    const int tn = (int)((r1 - t0) < (int64_t)kGramTile ? (r1 - t0) : (int64_t)kGramTile);
    __syncthreads();
    for (int r = threadIdx.x; r < tn; r += kGramThreads) {
      s_vt[r] = __ldcs(vt + t0 + r);
      s_w[r] = __ldcs(a.w + t0 + r);
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < kGramSlots; ++s) {
      const int j = cg + s * C;
      if (j > i) break;
      if (j < i) {
        const double* vj = a.V + (int64_t)j * a.ldv + t0;
#pragma unroll 2
        for (int r = lane + 32 * rg; r < tn; r += 32 * R) {
          const double x = __ldcs(vj + r);
          acc_a[s] = fma(x, s_vt[r], acc_a[s]);
          acc_s[s] = fma(x, s_w[r], acc_s[s]);
        }
      } else {
        for (int r = lane + 32 * rg; r < tn; r += 32 * R) {
          const double x = s_vt[r];
          acc_a[s] = fma(x, x, acc_a[s]);
          acc_s[s] = fma(x, s_w[r], acc_s[s]);
        }
      }
    }
  }
  const int stride = 2 * (kMaxM + 1);
  __shared__ double s_part[kGramWarps][2 * (kMaxM + 1)];
#pragma unroll
  for (int s = 0; s < kGramSlots; ++s) {
    const int j = cg + s * C;
    if (j > i) break;
    double va = acc_a[s], vs = acc_s[s];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      va += __shfl_xor_sync(0xffffffffu, va, o);
      vs += __shfl_xor_sync(0xffffffffu, vs, o);
    }
    if (lane == 0) {
      s_part[rg][j] = va;
      s_part[rg][kMaxM + 1 + j] = vs;
    }
  }
  __syncthreads();
  for (int v = threadIdx.x; v < 2 * ncol; v += blockDim.x) {
    const int col = v < ncol ? v : (kMaxM + 1) + (v - ncol);
    double sum = 0.0;
    for (int g = 0; g < R; ++g) sum += s_part[g][col];
    a.scr.partials[(int64_t)blockIdx.x * stride + col] = sum;
  }
  if (!last_block(a.scr.ticket)) return;
  // red[0..i] = a, red[kMaxM+1 .. kMaxM+1+i] = s
  {
    const int wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int v = wp; v < 2 * ncol; v += nw) {
      const int col = v < ncol ? v : (kMaxM + 1) + (v - ncol);
      double sum = 0.0;
      for (int b = lane; b < (int)gridDim.x; b += 32) sum += __ldcg(a.scr.partials + (int64_t)b * stride + col);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (lane == 0) red[col] = sum;
    }
    __syncthreads();
  }
  if (!st) {
    for (int v = threadIdx.x; v < ncol; v += blockDim.x) {
      a.out[v] = red[v];
      a.out[ncol + v] = red[kMaxM + 1 + v];
    }
    return;
  }
  // ---- finalise (steps 7-11) ----
  __shared__ double s_r[kMaxM + 1];
  __shared__ double s_beta;
  constexpr int LD = kMaxM + 1;
  if (threadIdx.x == 0) {
    const double aii = red[i];
    const double beta = sqrt(aii);
    s_beta = beta;
    if (!(beta > 0.0) || !isfinite(beta)) {
      // beta = 0 cannot occur here (a zero vector closes the previous column first);
      // a non-finite value aborts the solve.
      st->status = isfinite(beta) ? 0 : -6;
      st->stop = 1;
      st->done = 1;
    }
    st->beta[i] = beta;
    st->invbeta[i] = 1.0 / beta;
    if (i == 0) st->g[0] = beta;
  }
  __syncthreads();
  if (st->stop) return;
  const double invb = 1.0 / s_beta;
  for (int j = threadIdx.x; j <= i; j += blockDim.x) {
    if (j < i) {
      st->L[i * LD + j] = red[j] * invb;
      s_r[j] = red[kMaxM + 1 + j] * invb;
    } else {
      s_r[j] = red[kMaxM + 1 + j] * invb * invb;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // loss of orthogonality of the cycle so far (Sec. 3): ||I - V^T V||_F ~ sqrt(2)||L||_F
    double l2 = (i == 0) ? 0.0 : st->lsum;
    for (int j = 0; j < i; ++j) l2 = fma(st->L[i * LD + j], st->L[i * LD + j], l2);
    st->lsum = l2;
    st->orth_loss = sqrt(2.0 * l2);
  }
  if (!st->t_exact) {
    // h = (I - L) r: row q of L times r, one thread per row.
    for (int q = threadIdx.x; q <= i; q += blockDim.x) {
      double acc = s_r[q];
      for (int j = 0; j < q; ++j) acc = fma(-st->L[q * LD + j], s_r[j], acc);
      st->h[q] = acc;
      st->R[i * LD + q] = acc;
    }
  } else if (threadIdx.x < 32) {
    // h = (I + L)^-1 r by forward substitution, one warp, dot products across lanes.
    for (int q = 0; q <= i; ++q) {
      double acc = 0.0;
      for (int j = lane; j < q; j += 32) acc = fma(st->L[q * LD + j], st->h[j], acc);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) {
        const double hq = s_r[q] - acc;
        st->h[q] = hq;
        st->R[i * LD + q] = hq;
      }
      __syncwarp();
    }
  }
}

// ------------------------------------------------------------------------------------------
// Update: v_i = vt / beta (in place), vt_{i+1} = w / beta - sum_{j<=i} h_j v_j, ||vt_{i+1}||^2.
// ------------------------------------------------------------------------------------------
struct UpdateArgs {
  int64_t n;
  double* V;
  int64_t ldv;
  const double* w;
  GState* st;
  unsigned long long cond_inner;  // graph conditional handle (0 outside graphs)
  // standalone
  int i_standalone;
  double invbeta_standalone;
  const double* h_standalone;
  double* sumsq_out;
  Scratch scr;
  float* v32;  // if set: FP32 copy of vt_{i+1} (the next V-cycle's input when it runs in FP32)
};

__global__ void __launch_bounds__(kRedThreads) k_update(UpdateArgs a) {
  pdl_enter();
  __shared__ double s_h[kMaxM + 1];
  __shared__ double s_red[kRedThreads / 32];
  GState* st = a.st;
  if (st && st->stop) {  // stopped earlier in this step (error in the Gram): end the inner loop
    if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(a.cond_inner, 0);
    return;
  }
  const int i = st ? st->i : a.i_standalone;
  const double invb = st ? st->invbeta[i] : a.invbeta_standalone;
  for (int j = threadIdx.x; j <= i; j += blockDim.x) s_h[j] = st ? st->h[j] : a.h_standalone[j];
  __syncthreads();
  double* vi = a.V + (int64_t)i * a.ldv;
  double* vn = a.V + (int64_t)(i + 1) * a.ldv;
  const double hi = s_h[i];
  double ss = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.n; r += (int64_t)gridDim.x * blockDim.x) {
    const double v = __ldcs(vi + r) * invb;
    vi[r] = v;
    double acc = fma(-hi, v, __ldcs(a.w + r) * invb);
#pragma unroll 8
    for (int j = 0; j < i; ++j) acc = fma(-s_h[j], __ldcs(a.V + (int64_t)j * a.ldv + r), acc);
    vn[r] = acc;
    if (a.v32) a.v32[r] = narrow_f64(acc);
    ss = fma(acc, acc, ss);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
    a.scr.partials[blockIdx.x] = t;
  }
  if (!last_block(a.scr.ticket)) return;
  __shared__ double s_tot;
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) s += __ldcg(a.scr.partials + b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) s_tot = s;
  }
  __syncthreads();
  if (!st) {
    if (threadIdx.x == 0) *a.sumsq_out = s_tot;
    return;
  }
  // ---- close column i: H_{i+1,i} = ||vt_{i+1}||, Givens (steps 13-14), stop decision ----
  __shared__ int s_stop, s_k;
  constexpr int LD = kMaxM + 1;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    double* col = st->R + i * LD;
    const double hsub = sqrt(s_tot);
    for (int q = 0; q < i; ++q) {
      const double t = st->cs[q] * col[q] + st->sn[q] * col[q + 1];
      col[q + 1] = -st->sn[q] * col[q] + st->cs[q] * col[q + 1];
      col[q] = t;
    }
    double c = 1.0, s = 0.0;
    const double aa = col[i];
    if (hsub != 0.0) {
      const double rho = hypot(aa, hsub);
      c = aa / rho;
      s = hsub / rho;
      col[i] = rho;
    }
    st->cs[i] = c;
    st->sn[i] = s;
    st->g[i + 1] = -s * st->g[i];
    st->g[i] = c * st->g[i];
    st->iters += 1;
    const int k = i + 1;
    st->k = k;
    const double res = fabs(st->g[i + 1]);
    const double scale = st->bnorm > 0.0 ? st->bnorm : 1.0;
    st->relres_implicit = res / scale;
    const bool finite = isfinite(res) && isfinite(hsub) && isfinite(col[i]);
    int stop = (!finite) || res <= st->rtol * scale || hsub == 0.0 || k >= st->m || st->iters >= st->maxit;
    if (!finite) st->status = -6;
    if (!stop) st->beta[i + 1] = hsub;  // provisional; the next Gram recomputes it
    s_stop = stop;
    s_k = k;
    st->stop = stop;
    if (!stop) st->i = i + 1;
  }
  __syncthreads();
  if (s_stop) {
    // Back substitution R y = g (k x k upper triangular), coefficients y_j / beta_j.
    if (threadIdx.x < 32) {
      const int k = s_k;
      for (int q = k - 1; q >= 0; --q) {
        double acc = 0.0;
        for (int j = q + 1 + lane; j < k; j += 32) acc = fma(st->R[j * LD + q], st->coef[j], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) st->coef[q] = (st->g[q] - acc) / st->R[q * LD + q];
        __syncwarp();
      }
      __syncwarp();
      for (int q = lane; q < k; q += 32) st->coef[q] *= st->invbeta[q];
    }
  }
  if (threadIdx.x == 0) set_cond(a.cond_inner, s_stop ? 0 : 1);
}

// ------------------------------------------------------------------------------------------
// x += sum_{j<k} coef_j Z[:, j]   (x-update at the end of a cycle, Algorithm 1 last step)
// ------------------------------------------------------------------------------------------
template <typename TZ>
__global__ void __launch_bounds__(kRedThreads) k_xupdate(int64_t n, const TZ* Z, int64_t ldz, GState* st) {
  pdl_enter();
  __shared__ double s_c[kMaxM];
  if (st->done && st->status < 0) return;
  const int k = st->k;
  for (int j = threadIdx.x; j < k; j += blockDim.x) s_c[j] = st->coef[j];
  __syncthreads();
  double* x = st->x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    double acc = x[r];
    for (int j = 0; j < k; ++j) acc = fma(s_c[j], convert<double>(__ldcs(Z + (int64_t)j * ldz + r)), acc);
    x[r] = acc;
  }
}

// Block-wide fixed-order sum of one double per thread (blockDim.x == kRedThreads).
__device__ inline double block_sum(double v, double* s_tmp) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) s_tmp[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kRedThreads / 32; ++w) t += s_tmp[w];
  return t;  // valid in thread 0
}

// ------------------------------------------------------------------------------------------
// True residual and restart control: r = b - A x -> V[:, 0], ||r||^2, ||b||^2.
// init = 1 for the first call of a solve (sets ||b||).
// ------------------------------------------------------------------------------------------
struct ResidArgs {
  int n;
  const int* rp;
  const int* ci;
  const double* v;
  double* r;           // V[:, 0]
  float* r32;          // if set: FP32 copy of r (the first V-cycle input of a cycle in FP32)
  GState* st;
  int init;
  unsigned long long cond_outer, cond_inner;
  Scratch scr;
};

template <int G>
__global__ void __launch_bounds__(kRedThreads) k_resid(ResidArgs a) {
  pdl_enter();
  __shared__ double s_tmp[kRedThreads / 32];
  GState* st = a.st;
  const int was_done = a.init ? 0 : st->done;  // an error earlier in the cycle already ended the solve
  const double* b = st->b;
  const double* x = st->x;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int row = (int)(gid / G);
  const int lane = (int)(gid & (G - 1));
  double rr = 0.0, bb = 0.0, xx = 0.0;
  if (row < a.n) {
    double acc = 0.0;
    const int rb = __ldg(a.rp + row), re = __ldg(a.rp + row + 1);
    for (int p = rb + lane; p < re; p += G) acc = fma(__ldg(a.v + p), x[__ldg(a.ci + p)], acc);
    if constexpr (G > 1) {
      const unsigned seg = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(seg, acc, o, G);
    }
    if (lane == 0) {
      const double bi = b[row];
      const double ri = bi - acc;
      const double xi = x[row];
      a.r[row] = ri;
      if (a.r32) a.r32[row] = narrow_f64(ri);
      rr = ri * ri;
      bb = bi * bi;
      xx = xi * xi;
    }
  }
  const double tr = block_sum(rr, s_tmp);
  const double tb = block_sum(bb, s_tmp);
  const double tx = block_sum(xx, s_tmp);
  if (threadIdx.x == 0) {
    a.scr.partials[3 * (int64_t)blockIdx.x] = tr;
    a.scr.partials[3 * (int64_t)blockIdx.x + 1] = tb;
    a.scr.partials[3 * (int64_t)blockIdx.x + 2] = tx;
  }
  if (!last_block(a.scr.ticket)) return;
  double pr = 0.0, pb = 0.0, px = 0.0;
  for (int bI = threadIdx.x; bI < (int)gridDim.x; bI += blockDim.x) {
    pr += __ldcg(a.scr.partials + 3 * (int64_t)bI);
    pb += __ldcg(a.scr.partials + 3 * (int64_t)bI + 1);
    px += __ldcg(a.scr.partials + 3 * (int64_t)bI + 2);
  }
  const double R2 = block_sum(pr, s_tmp);
  const double B2 = block_sum(pb, s_tmp);
  const double X2 = block_sum(px, s_tmp);
  if (threadIdx.x == 0) {
    if (a.init) {
      st->bnorm = sqrt(B2);
      st->iters = 0;
      st->cycles = 0;
      st->status = 0;
      st->done = 0;
      st->relres_implicit = 1.0;
    }
    // relative residual (eq. relres); for b = 0 the absolute residual is used instead
    const double scale = st->bnorm > 0.0 ? st->bnorm : 1.0;
    const double relres = sqrt(R2) / scale;
    st->relres_true = relres;
    // norm-wise relative backward error (Sec. 3): ||r|| / (||b|| + ||A||_inf ||x||)
    const double den = st->bnorm + st->anorm_inf * sqrt(X2);
    st->nrbe = den > 0.0 ? sqrt(R2) / den : 0.0;
    const bool finite = isfinite(R2) && isfinite(st->bnorm);
    const bool conv = finite && relres <= st->rtol;
    const bool err = !finite || st->status < 0;
    // A cycle that added no Arnoldi column cannot make progress: stop (bounds the outer loop).
    const bool no_progress = !a.init && st->k == 0;
    const bool stop_all = was_done || no_progress || conv || err || st->iters >= st->maxit || st->cycles > st->maxit;
    st->converged = conv ? 1 : 0;
    if (!finite) st->status = -6;
    else if (!err) st->status = conv ? 0 : 1;
    st->done = stop_all ? 1 : 0;
    if (a.init) st->klast = 0;
    else if (st->k > 0) st->klast = st->k;
    st->i = 0;
    st->k = 0;
    st->stop = stop_all ? 1 : 0;
    if (!stop_all) st->cycles += 1;
    set_cond(a.cond_outer, stop_all ? 0 : 1);
    set_cond(a.cond_inner, stop_all ? 0 : 1);
  }
}

// ------------------------------------------------------------------------------------------
// ||S_k||_2 of the last cycle, S_k = (I + U_k)^-1 U_k with U_k = L_k^T the strictly upper part of
// V_k^T V_k (Sec. 3: the basis has lost linear independence exactly when ||S_k||_2 = 1).
// One block: column c of S by back substitution (thread c), then power iteration on S^T S with
// the Rayleigh quotient ||S x||^2 (||x|| = 1), stopped when it changes by <= 1e-15 relative or
// after kSkIters iterations. Fixed-order sums: the result is deterministic.
// ------------------------------------------------------------------------------------------
constexpr int kSkThreads = 64;
constexpr int kSkIters = 300;

__device__ double sk_norm_block(const double* __restrict__ L, int ld, int k) {
  __shared__ double S[kMaxM][kMaxM + 1];
  __shared__ double x[kMaxM], y[kMaxM];
  __shared__ double s_val, s_prev;
  __shared__ int s_stop;
  const int t = threadIdx.x;
  if (k <= 1) return 0.0;
  if (t < k) {
    const int c = t;
    for (int r = c; r < k; ++r) S[r][c] = 0.0;
    for (int r = c - 1; r >= 0; --r) {
      double acc = L[c * ld + r];  // U[r][c]
      for (int j = r + 1; j < c; ++j) acc = fma(-L[j * ld + r], S[j][c], acc);
      S[r][c] = acc;
    }
    x[c] = 1.0 + 0.5 * (double)((c * 37) % 64) / 64.0;  // fixed start with no special direction
  }
  if (t == 0) {
    s_prev = -1.0;
    s_stop = 0;
  }
  __syncthreads();
  if (t == 0) {
    double q = 0.0;
    for (int c = 0; c < k; ++c) q = fma(x[c], x[c], q);
    s_val = 1.0 / sqrt(q);
  }
  __syncthreads();
  if (t < k) x[t] *= s_val;
  __syncthreads();
  double lam = 0.0;
  for (int it = 0; it < kSkIters; ++it) {
    if (t < k) {  // y = S x (S strictly upper: columns > r)
      double acc = 0.0;
      for (int c = t + 1; c < k; ++c) acc = fma(S[t][c], x[c], acc);
      y[t] = acc;
    }
    __syncthreads();
    if (t == 0) {
      double q = 0.0;
      for (int r = 0; r < k; ++r) q = fma(y[r], y[r], q);
      s_val = q;  // Rayleigh quotient of S^T S
    }
    __syncthreads();
    lam = s_val;
    if (t < k) {  // x <- S^T y (rows < c)
      double acc = 0.0;
      for (int r = 0; r < t; ++r) acc = fma(S[r][t], y[r], acc);
      x[t] = acc;
    }
    __syncthreads();
    if (t == 0) {
      double q = 0.0;
      for (int c = 0; c < k; ++c) q = fma(x[c], x[c], q);
      const bool done = q == 0.0 || fabs(lam - s_prev) <= 1e-15 * lam;
      s_prev = lam;
      s_stop = done ? 1 : 0;
      s_val = q > 0.0 ? 1.0 / sqrt(q) : 0.0;
    }
    __syncthreads();
    if (s_stop) break;
    if (t < k) x[t] *= s_val;
    __syncthreads();
  }
  return sqrt(lam);
}

__global__ void k_sknorm_states(GState* __restrict__ states) {
  pdl_enter();
  GState* st = states + blockIdx.x;
  const double v = sk_norm_block(st->L, kMaxM + 1, min(st->klast, kMaxM));
  if (threadIdx.x == 0) st->sk_norm = v;
}

__global__ void k_sknorm_matrix(const double* __restrict__ L, int ld, int k, double* __restrict__ out) {
  pdl_enter();
  const double v = sk_norm_block(L, ld, k);
  if (threadIdx.x == 0) *out = v;
}

}  // namespace nsamg
