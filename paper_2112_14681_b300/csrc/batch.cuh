// Batched one-reduce GMRES over many independent systems (block-diagonal batching).
//
// All systems' levels are concatenated into block-diagonal matrices, so every V-cycle and SpMV
// kernel covers every system in one launch. The Krylov steps run in lock step (one step index
// for the batch); each system keeps its own GState (beta, L, Hessenberg/Givens, convergence)
// and stops on its own. Reductions are segmented: each block works on rows of one system, the
// last block of a system (per-system ticket) finalises that system in fixed block order, and
// the last block of the launch (global ticket) updates the batch loop control.
#pragma once
#include "gmres.cuh"

namespace nsamg {

struct BatchCtl {
  const double* b;  // concatenated right-hand sides (all systems)
  double* x;        // concatenated solutions
  double rtol;
  int maxit;
  int m;
  int t_exact;
  int gi;           // current Arnoldi step of the batch
  int active;       // systems still stepping in this cycle
  int running;      // systems not finished
  int cycles;
  int stop_nrbe;    // 1: stop on the backward error instead of the relative residual
  int pad;
};

struct BatchArgs {
  int nsys;
  const int64_t* off;   // nsys + 1 row offsets
  const int* bstart;    // nsys + 1 block offsets for this kernel's rows-per-block
  int64_t rpb;          // rows per block
  GState* st;           // nsys states
  BatchCtl* ctl;
  double* V;
  int64_t ldv;
  const double* w;
  double* partials;     // per block
  unsigned* sticket;    // per system
  unsigned* gticket;    // one
  unsigned long long cond_outer, cond_inner;
};

__device__ __forceinline__ int find_system(const int* bstart, int nsys, int b) {
  int lo = 0, hi = nsys;  // bstart[lo] <= b < bstart[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (bstart[mid] <= b) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Per-system last-block detection; returns true in the block that finished system s last.
__device__ __forceinline__ bool last_of_system(unsigned* tk, int nb) {
  __shared__ bool is_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(tk, 1u);
    is_last = (t == (unsigned)nb - 1u);
    if (is_last) *tk = 0u;
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// ------------------------------------------------------------------------------------------
// Gram for every active system (Algorithm 1 steps 6-11 per system), in double-FP32 like the
// single-system kernels (the FP64 pipe would bound it at ~0.25 of HBM): per tile, vt and w are
// split once into shared memory; warps form C column groups x 16/C row groups over columns
// 0..i (column i is vt itself, taken from the staged split); each column entry is split on the
// fly and multiplied by TwoProduct + TwoSum (Dot2) into (sum, error) pairs; a warp reduce-scatter
// combines them, FP64 takes over for the block and system sums (fixed order). A block whose vt
// or w leaves the double-FP32 window recomputes its rows in FP64.
// ------------------------------------------------------------------------------------------
// Columns per warp of k_bgram: few enough that two blocks fit an SM (64 registers a thread).
constexpr int kBGramSlots = 4;

__global__ void __launch_bounds__(kGramThreads, 2) k_bgram(BatchArgs a) {
  pdl_enter();
  __shared__ float4 s_sp[kDfTile];  // per row of the tile: (vt_hi, vt_lo, w_hi, w_lo)
  __shared__ double red[2 * (kMaxM + 1)];
  __shared__ double s_part[kGramWarps][2 * (kMaxM + 1)];
  __shared__ unsigned s_max;
  __shared__ int s_sys;
  if (threadIdx.x == 0) {
    s_sys = find_system(a.bstart, a.nsys, blockIdx.x);
    s_max = 0u;
  }
  __syncthreads();
  const int sys = s_sys;
  GState* st = a.st + sys;
  const bool active = !st->stop;
  const int i = a.ctl->gi;
  const int ncol = i + 1;
  const int nb = a.bstart[sys + 1] - a.bstart[sys];
  const int stride = 2 * (kMaxM + 1);
  if (active) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int C = df_groups(ncol, kBGramSlots);
    const int R = kGramWarps / C;
    const int S = (ncol + C - 1) / C;
    const int cg = warp % C, rg = warp / C;
    const int rows_w = kDfTile / R;
    const int64_t r0 = a.off[sys] + (int64_t)(blockIdx.x - a.bstart[sys]) * a.rpb;
    const int64_t r1 = min(a.off[sys + 1], r0 + a.rpb);
    const double* vt = a.V + (int64_t)i * a.ldv;
    float sa[kBGramSlots], ca[kBGramSlots], sw[kBGramSlots], cw[kBGramSlots];
#pragma unroll
    for (int q = 0; q < kBGramSlots; ++q) sa[q] = ca[q] = sw[q] = cw[q] = 0.f;
    unsigned mx = 0u;
    for (int64_t t0 = r0; t0 < r1; t0 += kDfTile) {
      const int tn = (int)((r1 - t0) < (int64_t)kDfTile ? (r1 - t0) : (int64_t)kDfTile);
      __syncthreads();
      for (int r = threadIdx.x; r < kDfTile; r += kGramThreads) {
        float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < tn) {
          const double x = __ldcs(vt + t0 + r), y = __ldcs(a.w + t0 + r);
          mx = max(mx, max(abs_hiword(x), abs_hiword(y)));
          split_df(x, q.x, q.y);
          split_df(y, q.z, q.w);
        }
        s_sp[r] = q;
      }
      __syncthreads();
      for (int k = 0; k < rows_w; k += 32) {
        const int r = rg * rows_w + k + lane;
        if (r >= tn) break;
        const float4 q = s_sp[r];
        double xv[kBGramSlots];
#pragma unroll
        for (int sl = 0; sl < kBGramSlots; ++sl) {
          const int j = cg + sl * C;
          xv[sl] = (sl < S && j < i) ? __ldcs(a.V + (int64_t)j * a.ldv + t0 + r) : 0.0;
        }
#pragma unroll
        for (int sl = 0; sl < kBGramSlots; ++sl) {
          const int j = cg + sl * C;
          if (sl < S && j <= i) {
            float xh = q.x, xl = q.y;  // column i: vt, already split
            if (j < i) split_df(xv[sl], xh, xl);
            dot2_step(sa[sl], ca[sl], xh, xl, q.x, q.y);
            dot2_step(sw[sl], cw[sl], xh, xl, q.z, q.w);
          }
        }
      }
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) atomicMax(&s_max, mx);
    __syncthreads();
    if (df_window(s_max)) {
      float as[16], ac[16];
#pragma unroll
      for (int sl = 0; sl < kDfSlots; ++sl) {
        as[2 * sl] = sl < kBGramSlots ? sa[sl < kBGramSlots ? sl : 0] : 0.f;
        ac[2 * sl] = sl < kBGramSlots ? ca[sl < kBGramSlots ? sl : 0] : 0.f;
        as[2 * sl + 1] = sl < kBGramSlots ? sw[sl < kBGramSlots ? sl : 0] : 0.f;
        ac[2 * sl + 1] = sl < kBGramSlots ? cw[sl < kBGramSlots ? sl : 0] : 0.f;
      }
      df_warp_reduce16(as, ac);
      const int qd = lane >> 1, sl = qd >> 1, j = cg + sl * C;
      if ((lane & 1) == 0 && sl < S && j <= i)
        s_part[rg][(qd & 1) ? (kMaxM + 1 + j) : j] = widen_normal(as[0]) + widen_normal(ac[0]);
    } else {  // FP64 recomputation of this block's rows (vt or w outside the double-FP32 window)
#pragma unroll 1
      for (int sl = 0; sl < S; ++sl) {
        const int j = cg + sl * C;
        double fa = 0.0, fw = 0.0;
        if (j <= i) {
          const double* vj = a.V + (int64_t)j * a.ldv;
          for (int64_t t0 = r0; t0 < r1; t0 += kDfTile)
            for (int r = rg * rows_w + lane; r < (rg + 1) * rows_w && t0 + r < r1; r += 32) {
              const double x = vj[t0 + r];
              fa = fma(x, vt[t0 + r], fa);
              fw = fma(x, a.w[t0 + r], fw);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          fa += __shfl_xor_sync(0xffffffffu, fa, o);
          fw += __shfl_xor_sync(0xffffffffu, fw, o);
        }
        if (lane == 0 && j <= i) {
          s_part[rg][j] = fa;
          s_part[rg][kMaxM + 1 + j] = fw;
        }
      }
    }
    __syncthreads();
    for (int v = threadIdx.x; v < 2 * ncol; v += blockDim.x) {
      const int col = v < ncol ? v : (kMaxM + 1) + (v - ncol);
      double sum = 0.0;
      for (int g = 0; g < R; ++g) sum += s_part[g][col];
      a.partials[(int64_t)blockIdx.x * stride + col] = sum;
    }
  }
  if (!last_of_system(a.sticket + sys, nb)) return;
  if (!active) return;
  const int lane = threadIdx.x & 31;
  {
    const int wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int b0 = a.bstart[sys];
    for (int v = wp; v < 2 * ncol; v += nw) {
      const int col = v < ncol ? v : (kMaxM + 1) + (v - ncol);
      double sum = 0.0;
      for (int b = lane; b < nb; b += 32) sum += __ldcg(a.partials + (int64_t)(b0 + b) * stride + col);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (lane == 0) red[col] = sum;
    }
    __syncthreads();
  }
  __shared__ double s_r[kMaxM + 1];
  __shared__ double s_beta;
  constexpr int LD = kMaxM + 1;
  if (threadIdx.x == 0) {
    const double beta = sqrt(red[i]);
    s_beta = beta;
    if (!(beta > 0.0) || !isfinite(beta)) {
      st->status = isfinite(beta) ? 0 : -6;
      st->stop = 1;
      st->done = 1;
      atomicSub(&a.ctl->active, 1);
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
  if (!a.ctl->t_exact) {
    for (int q = threadIdx.x; q <= i; q += blockDim.x) {
      double acc = s_r[q];
      for (int j = 0; j < q; ++j) acc = fma(-st->L[q * LD + j], s_r[j], acc);
      st->h[q] = acc;
      st->R[i * LD + q] = acc;
    }
  } else if (threadIdx.x < 32) {
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
// Update + Givens per active system; the last block of the launch advances the batch step. The
// new vector vt_{i+1} = w / beta_i - sum_j h_j v_j is formed in double-FP32 (w / beta_i and
// v_i = vt_i / beta_i by one FP64 multiply each, every entry split on the fly, the -h_j split
// once per block; four (sum, error) pairs) and stored as FP64; rows whose w / beta_i, and every
// row when the coefficients, leave the double-FP32 window are computed in FP64.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kRedThreads) k_bupdate(BatchArgs a) {
  pdl_enter();
  __shared__ double s_h[kMaxM + 1];
  __shared__ float2 s_hs[kMaxM + 1];  // -h_j split
  __shared__ unsigned s_cmax;
  __shared__ double s_red[kRedThreads / 32];
  __shared__ int s_sys;
  if (threadIdx.x == 0) s_sys = find_system(a.bstart, a.nsys, blockIdx.x);
  __syncthreads();
  const int sys = s_sys;
  GState* st = a.st + sys;
  const bool active = !st->stop;
  const int i = a.ctl->gi;
  const int nb = a.bstart[sys + 1] - a.bstart[sys];
  const int lane = threadIdx.x & 31;
  if (active) {
    const double invb = st->invbeta[i];
    if (threadIdx.x == 0) s_cmax = 0u;
    __syncthreads();
    for (int j = threadIdx.x; j <= i; j += blockDim.x) {
      s_h[j] = st->h[j];
      s_hs[j] = split2(-st->h[j]);
      atomicMax(&s_cmax, abs_hiword(st->h[j]));
    }
    __syncthreads();
    const bool cok = df_window(s_cmax);
    double* vi = a.V + (int64_t)i * a.ldv;
    double* vn = a.V + (int64_t)(i + 1) * a.ldv;
    const int64_t r0 = a.off[sys] + (int64_t)(blockIdx.x - a.bstart[sys]) * a.rpb;
    const int64_t r1 = min(a.off[sys + 1], r0 + a.rpb);
    double ss = 0.0;
    float qs = 0.f, qc = 0.f;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
      const double v = __ldcs(vi + r) * invb;
      vi[r] = v;
      const double wb = __ldcs(a.w + r) * invb;
      double acc;
      if (cok && df_window(abs_hiword(wb))) {
        // w / beta_i - sum_j h_j v_j in four (sum, error) pairs, columns four at a time
        float ps[4] = {0.f, 0.f, 0.f, 0.f}, pc[4] = {0.f, 0.f, 0.f, 0.f};
        split_df(wb, ps[0], pc[0]);
        for (int j0 = 0; j0 < i; j0 += 4) {
          double x[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) x[k] = j0 + k < i ? __ldcs(a.V + (int64_t)(j0 + k) * a.ldv + r) : 0.0;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            float xh, xl;
            split_df(x[k], xh, xl);
            const float2 hh = j0 + k < i ? s_hs[j0 + k] : make_float2(0.f, 0.f);
            dot2_step(ps[k], pc[k], hh.x, hh.y, xh, xl);
          }
        }
        {  // column i: v_i = vt_i / beta_i
          float xh, xl;
          split_df(v, xh, xl);
          dot2_step(ps[1], pc[1], s_hs[i].x, s_hs[i].y, xh, xl);
        }
        df_add(ps[0], pc[0], ps[1], pc[1]);
        df_add(ps[2], pc[2], ps[3], pc[3]);
        df_add(ps[0], pc[0], ps[2], pc[2]);
        const float tt = __fadd_rn(ps[0], pc[0]);
        const float z = __fsub_rn(tt, ps[0]);
        const float e = __fadd_rn(__fsub_rn(ps[0], __fsub_rn(tt, z)), __fsub_rn(pc[0], z));
        acc = widen_normal(tt) + widen_normal(e);
        dot2_step(qs, qc, tt, e, tt, e);
      } else {  // outside the double-FP32 window: FP64
        acc = fma(-s_h[i], v, wb);
        for (int j = 0; j < i; ++j) acc = fma(-s_h[j], __ldcs(a.V + (int64_t)j * a.ldv + r), acc);
        ss = fma(acc, acc, ss);
      }
      vn[r] = acc;
    }
    // block sum of the squares: double-FP32 part per warp, FP64 part
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float rs = __shfl_xor_sync(0xffffffffu, qs, o), rc = __shfl_xor_sync(0xffffffffu, qc, o);
      if (lane & o) {
        df_add(rs, rc, qs, qc);
        qs = rs;
        qc = rc;
      } else {
        df_add(qs, qc, rs, rc);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    ss += widen_normal(qs) + widen_normal(qc);  // every lane holds the warp's double-FP32 total
    if (lane == 0) s_red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
      a.partials[blockIdx.x] = t;
    }
  }
  if (last_of_system(a.sticket + sys, nb) && active) {
    __shared__ double s_tot;
    __shared__ int s_stop, s_k;
    constexpr int LD = kMaxM + 1;
    if (threadIdx.x < 32) {
      double sum = 0.0;
      const int b0 = a.bstart[sys];
      for (int b = lane; b < nb; b += 32) sum += __ldcg(a.partials + b0 + b);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (lane == 0) s_tot = sum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double* col = st->R + i * LD;
      const double hsub = sqrt(s_tot);
      for (int q = 0; q < i; ++q) {
        const double t = st->cs[q] * col[q] + st->sn[q] * col[q + 1];
        col[q + 1] = -st->sn[q] * col[q] + st->cs[q] * col[q + 1];
        col[q] = t;
      }
      double c = 1.0, s = 0.0;
      if (hsub != 0.0) {
        const double rho = hypot(col[i], hsub);
        c = col[i] / rho;
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
      const double den = a.ctl->stop_nrbe ? st->bnorm + st->anorm_inf * st->xnorm : scale;
      const bool finite = isfinite(res) && isfinite(hsub) && isfinite(col[i]);
      const int stop = (!finite) || res <= a.ctl->rtol * (den > 0.0 ? den : 1.0) || hsub == 0.0 || k >= a.ctl->m ||
                       st->iters >= a.ctl->maxit;
      if (!finite) st->status = -6;
      st->stop = stop;
      s_stop = stop;
      s_k = k;
      if (stop) atomicSub(&a.ctl->active, 1);
    }
    __syncthreads();
    if (s_stop && threadIdx.x < 32) {
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
  // batch step control: the last block of the launch
  if (!last_block(a.gticket)) return;
  if (threadIdx.x == 0) {
    BatchCtl* c = a.ctl;
    const int more = (c->active > 0) && (c->gi + 1 < c->m);
    if (more) c->gi += 1;
    set_cond(a.cond_inner, more);
  }
}

// x += sum_j coef_j Z[:, j] for each system over its rows (k_s columns of its last cycle).
template <typename TZ>
__global__ void __launch_bounds__(kRedThreads) k_bxupdate(BatchArgs a, const TZ* Z, int64_t ldz) {
  pdl_enter();
  __shared__ double s_c[kMaxM];
  __shared__ int s_sys;
  if (threadIdx.x == 0) s_sys = find_system(a.bstart, a.nsys, blockIdx.x);
  __syncthreads();
  const int sys = s_sys;
  GState* st = a.st + sys;
  if (st->done && st->status < 0) return;
  const int k = st->k;
  for (int j = threadIdx.x; j < k; j += blockDim.x) s_c[j] = st->coef[j];
  __syncthreads();
  double* x = a.ctl->x;
  const int64_t r0 = a.off[sys] + (int64_t)(blockIdx.x - a.bstart[sys]) * a.rpb;
  const int64_t r1 = min(a.off[sys + 1], r0 + a.rpb);
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    double acc = x[r];
    for (int j = 0; j < k; ++j) acc = fma(s_c[j], convert<double>(__ldcs(Z + (int64_t)j * ldz + r)), acc);
    x[r] = acc;
  }
}

// True residual r = b - A x of every system into V[:, 0], per-system restart decision, and
// (last block of the launch) the batch loop conditions. A is the block-diagonal finest level.
struct BResidArgs {
  BatchArgs ba;
  const int* rp;
  const int* ci;
  const double* v;
  int init;
};

__global__ void __launch_bounds__(kRedThreads) k_bresid(BResidArgs ra) {
  pdl_enter();
  BatchArgs& a = ra.ba;
  __shared__ double s_tmp[kRedThreads / 32];
  __shared__ int s_sys;
  if (threadIdx.x == 0) s_sys = find_system(a.bstart, a.nsys, blockIdx.x);
  __syncthreads();
  const int sys = s_sys;
  GState* st = a.st + sys;
  const int nb = a.bstart[sys + 1] - a.bstart[sys];
  const int was_done = ra.init ? 0 : st->done;
  const double* b = a.ctl->b;
  const double* x = a.ctl->x;
  const int64_t r0 = a.off[sys] + (int64_t)(blockIdx.x - a.bstart[sys]) * a.rpb;
  const int64_t r1 = min(a.off[sys + 1], r0 + a.rpb);
  double rr = 0.0, bb = 0.0, xx = 0.0;
  for (int64_t row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    double acc = 0.0;
    const int rb = __ldg(ra.rp + row), re = __ldg(ra.rp + row + 1);
    for (int p = rb; p < re; ++p) acc = fma(__ldg(ra.v + p), x[__ldg(ra.ci + p)], acc);
    const double bi = b[row];
    const double ri = bi - acc;
    const double xi = x[row];
    a.V[row] = ri;
    rr = fma(ri, ri, rr);
    bb = fma(bi, bi, bb);
    xx = fma(xi, xi, xx);
  }
  const double tr = block_sum(rr, s_tmp);
  const double tb = block_sum(bb, s_tmp);
  const double tx = block_sum(xx, s_tmp);
  if (threadIdx.x == 0) {
    a.partials[3 * (int64_t)blockIdx.x] = tr;
    a.partials[3 * (int64_t)blockIdx.x + 1] = tb;
    a.partials[3 * (int64_t)blockIdx.x + 2] = tx;
  }
  if (last_of_system(a.sticket + sys, nb)) {
    double pr = 0.0, pb = 0.0, px = 0.0;
    const int b0 = a.bstart[sys];
    for (int q = threadIdx.x; q < nb; q += blockDim.x) {
      pr += __ldcg(a.partials + 3 * (int64_t)(b0 + q));
      pb += __ldcg(a.partials + 3 * (int64_t)(b0 + q) + 1);
      px += __ldcg(a.partials + 3 * (int64_t)(b0 + q) + 2);
    }
    const double R2 = block_sum(pr, s_tmp);
    const double B2 = block_sum(pb, s_tmp);
    const double X2 = block_sum(px, s_tmp);
    if (threadIdx.x == 0) {
      if (ra.init) {
        st->bnorm = sqrt(B2);
        st->iters = 0;
        st->cycles = 0;
        st->status = 0;
        st->done = 0;
        st->relres_implicit = 1.0;
      }
      if (!was_done) {
        const double scale = st->bnorm > 0.0 ? st->bnorm : 1.0;
        const double relres = sqrt(R2) / scale;
        st->relres_true = relres;
        const double den = st->bnorm + st->anorm_inf * sqrt(X2);
        st->nrbe = den > 0.0 ? sqrt(R2) / den : 0.0;
        st->xnorm = sqrt(X2);
        const bool finite = isfinite(R2) && isfinite(st->bnorm);
        const bool conv = finite && (a.ctl->stop_nrbe ? st->nrbe <= a.ctl->rtol : relres <= a.ctl->rtol);
        const bool err = !finite || st->status < 0;
        const bool no_progress = !ra.init && st->k == 0;
        const bool fin = no_progress || conv || err || st->iters >= a.ctl->maxit || st->cycles > a.ctl->maxit;
        st->converged = conv ? 1 : 0;
        if (!finite) st->status = -6;
        else if (!err) st->status = conv ? 0 : 1;
        st->done = fin ? 1 : 0;
        if (!fin) st->cycles += 1;
      }
      if (ra.init) st->klast = 0;
      else if (st->k > 0) st->klast = st->k;
      st->i = 0;
      st->k = 0;
      st->stop = st->done;
    }
  }
  if (!last_block(a.gticket)) return;
  if (threadIdx.x == 0) {
    BatchCtl* c = a.ctl;
    int running = 0;
    for (int s = 0; s < a.nsys; ++s) running += a.st[s].done ? 0 : 1;
    c->running = running;
    c->active = running;
    c->gi = 0;
    c->cycles += running ? 1 : 0;
    set_cond(a.cond_outer, running > 0 && c->cycles <= c->maxit + 1);
    set_cond(a.cond_inner, running > 0);
  }
}

// Dense coarse solves of every system: z_rows(s) = C_s b_rows(s); one warp per coarse row.
template <typename TC, typename T>
__global__ void k_bdense_gemv(int nrows, const int* row_sys, const int64_t* coff, const int64_t* cblk,
                              const TC* __restrict__ C, VRef<const T> bref, VRef<T> zref, const int* skip) {
  pdl_enter();
  if (skip && *skip) return;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nrows) return;
  const int s = row_sys[warp];
  const int64_t o = coff[s];
  const int nc = (int)(coff[s + 1] - o);
  const int lr = warp - (int)o;
  const T* b = bref.get() + o;
  const TC* Cr = C + cblk[s] + (int64_t)lr * nc;
  T acc = T(0);
  for (int j = lane; j < nc; j += 32) acc = fma((T)Cr[j], b[j], acc);
#pragma unroll
  for (int q = 16; q > 0; q >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, q);
  if (lane == 0) zref.get()[warp] = acc;
}

}  // namespace nsamg
