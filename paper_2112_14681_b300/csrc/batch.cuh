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
  // split basis (krylov_fp64 = 0): column j = vt_j as row-pair (hi, lo) groups over the
  // concatenated rows, leading dimension ldv; the next V-cycle input in FP64 (vin) or FP32 (v32)
  float2* Vs;
  double* vin;
  float* v32;
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

// Last block of a system in a batched Gram: fixed-order sum of the system's block partials, then
// steps 7-11 of Algorithm 1 on its state. split: columns j < i hold vt_j = beta_j v_j (their
// products are scaled by 1 / beta_j) and column 0 is r / r0_scale.
__device__ void bgram_tail(const BatchArgs& a, GState* st, int sys, int i, int nb, bool split) {
  __shared__ double red[2 * (kMaxM + 1)];
  const int ncol = i + 1;
  const int stride = 2 * (kMaxM + 1);
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
  if (split) {
    for (int j = threadIdx.x; j < i; j += blockDim.x) {
      red[j] *= st->invbeta[j];
      red[kMaxM + 1 + j] *= st->invbeta[j];
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
    if (i == 0) st->g[0] = split ? beta * st->r0_scale : beta;
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
  bgram_tail(a, st, sys, i, nb, false);
}

// End of a batched update: the last block of each active system sums its block partials of
// ||vt_{i+1}||^2 (fixed order), applies the Givens rotations and the stop test (and, on stop,
// solves for the coefficients); the last block of the launch advances the batch step.
__device__ void bupdate_tail(const BatchArgs& a, GState* st, int sys, bool active, int i, int nb) {
  const int lane = threadIdx.x & 31;
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
  bupdate_tail(a, st, sys, active, i, nb);
}

// ------------------------------------------------------------------------------------------
// Split basis for batches (krylov_fp64 = 0): the single-system layout over the concatenated
// rows (column j = vt_j unnormalised as row-pair (hi, lo) groups, column 0 scaled to unit order
// per system), so the batched Gram and update read FP32 operands with no per-read split and run
// on packed FP32x2 instructions. A system's rows need not start or end on a pair boundary: the
// pairs inside a block's rows run packed, and a block's odd first or last row (its group's other
// lane belongs to the neighbouring system) is handled on its own, read and written lane by lane
// (rp_get / rp_set), so two systems never write the same 4-byte word.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void group_f2(float4 v, f2_t& hi, f2_t& lo) {
  hi = f2_pack(v.x, v.y);
  lo = f2_pack(v.z, v.w);
}

// Columns per warp of k_bgram_s (packed (sum, error) accumulators: 8 registers a column)
constexpr int kBGramSSlots = 4;

// One warp's products over the block's rows [r0, r1): its NS columns cg + sl C (only the last
// slot can pass column i; its discarded products then read column i) against column i (vt_i)
// and w (FP64, split here), one row pair a lane (two pairs in flight), then the lone first / last
// row; the two lanes of each accumulator are added at the end.
template <int NS>
__device__ __forceinline__ void bgram_s_rows(const BatchArgs& a, int nv, int C, int cg, int rg, int R, int64_t r0,
                                             int64_t r1, float (&sa)[kBGramSSlots], float (&ca)[kBGramSSlots],
                                             float (&sw)[kBGramSSlots], float (&cw)[kBGramSSlots], unsigned& mx) {
  const int lane = threadIdx.x & 31;
  f2_t s_a[NS], c_a[NS], s_w[NS], c_w[NS];
  const float4* col[NS];
#pragma unroll
  for (int sl = 0; sl < NS; ++sl) {
    s_a[sl] = c_a[sl] = s_w[sl] = c_w[sl] = 0ull;
    col[sl] = reinterpret_cast<const float4*>(a.Vs + (int64_t)min(cg + sl * C, nv - 1) * a.ldv);
  }
  const float4* colv = reinterpret_cast<const float4*>(a.Vs + (int64_t)(nv - 1) * a.ldv);
  const double2* w2 = reinterpret_cast<const double2*>(a.w);
  const f2_t m1 = f2_pack(-1.f, -1.f);
  const int64_t g1 = r1 >> 1;
#pragma unroll 2
  for (int64_t g = ((r0 + 1) >> 1) + rg * 32 + lane; g < g1; g += 32 * R) {
    f2_t qh, ql;
    group_f2(__ldg(colv + g), qh, ql);
    const double2 wv = __ldg(w2 + g);
    float4 x[NS];
#pragma unroll
    for (int sl = 0; sl < NS; ++sl) x[sl] = __ldcs(col[sl] + g);
    mx = max(mx, max(abs_hiword(wv.x), abs_hiword(wv.y)));
    float wh0, wl0, wh1, wl1;
    split_df(wv.x, wh0, wl0);
    split_df(wv.y, wh1, wl1);
    const f2_t wh = f2_pack(wh0, wh1), wl = f2_pack(wl0, wl1);
    const f2_t nqh = f2_mul(qh, m1), nwh = f2_mul(wh, m1);
#pragma unroll
    for (int sl = 0; sl < NS; ++sl) {
      f2_t xh, xl;
      group_f2(x[sl], xh, xl);
      dot2_step2(s_a[sl], c_a[sl], xh, xl, qh, ql, nqh);
      dot2_step2(s_w[sl], c_w[sl], xh, xl, wh, wl, nwh);
    }
  }
  // lone rows: lane 0 of the first row group takes an odd first row, lane 1 an odd last row
  if (rg == 0 && lane < 2) {
    const int64_t row = lane == 0 ? r0 : r1 - 1;
    const bool lone = row >= r0 && row < r1 && (lane == 0 ? (r0 & 1) : (r1 & 1)) != 0;
    if (lone) {
      const float2* vcol = a.Vs + (int64_t)(nv - 1) * a.ldv;
      const float2 q = rp_get(vcol, row);
      const double xw = a.w[row];
      mx = max(mx, abs_hiword(xw));
      float q2, q3;
      split_df(xw, q2, q3);
      const f2_t qh = f2_pack(q.x, 0.f), ql = f2_pack(q.y, 0.f), nqh = f2_pack(-q.x, 0.f);
      const f2_t wh = f2_pack(q2, 0.f), wl = f2_pack(q3, 0.f), nwh = f2_pack(-q2, 0.f);
#pragma unroll
      for (int sl = 0; sl < NS; ++sl) {
        const float2 x = rp_get(a.Vs + (int64_t)min(cg + sl * C, nv - 1) * a.ldv, row);
        const f2_t xh = f2_pack(x.x, 0.f), xl = f2_pack(x.y, 0.f);
        dot2_step2(s_a[sl], c_a[sl], xh, xl, qh, ql, nqh);
        dot2_step2(s_w[sl], c_w[sl], xh, xl, wh, wl, nwh);
      }
    }
  }
#pragma unroll
  for (int sl = 0; sl < NS; ++sl) {  // lane sums: even rows + odd rows
    float s0, s1, c0, c1;
    f2_unpack(s_a[sl], s0, s1);
    f2_unpack(c_a[sl], c0, c1);
    df_add(s0, c0, s1, c1);
    sa[sl] = s0;
    ca[sl] = c0;
    f2_unpack(s_w[sl], s0, s1);
    f2_unpack(c_w[sl], c0, c1);
    df_add(s0, c0, s1, c1);
    sw[sl] = s0;
    cw[sl] = c0;
  }
}

// Batched Gram on the split basis (Algorithm 1 steps 6-11 per active system): per block the
// products a_j = vt_j . vt_i and s_j = vt_j . w (j <= i) over its rows of one system in
// double-FP32, FP64 for the block and system sums (fixed order); the system's last block scales
// a_j, s_j (j < i) by 1 / beta_j and finalises. A block whose w leaves the double-FP32 window
// recomputes its rows in FP64 from the stored pairs.
__global__ void __launch_bounds__(kGramThreads, 1) k_bgram_s(BatchArgs a) {
  pdl_enter();
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
  const int nv = i + 1;
  const int nb = a.bstart[sys + 1] - a.bstart[sys];
  const int stride = 2 * (kMaxM + 1);
  if (active) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int C = df_groups(nv, kBGramSSlots);
    const int R = kGramWarps / C;
    const int S = (nv + C - 1) / C;
    const int cg = warp % C, rg = warp / C;
    const int64_t r0 = a.off[sys] + (int64_t)(blockIdx.x - a.bstart[sys]) * a.rpb;
    const int64_t r1 = min(a.off[sys + 1], r0 + a.rpb);
    float sa[kBGramSSlots], ca[kBGramSSlots], sw[kBGramSSlots], cw[kBGramSSlots];
#pragma unroll
    for (int q = 0; q < kBGramSSlots; ++q) sa[q] = ca[q] = sw[q] = cw[q] = 0.f;
    unsigned mx = 0u;
    switch (S) {
      case 1: bgram_s_rows<1>(a, nv, C, cg, rg, R, r0, r1, sa, ca, sw, cw, mx); break;
      case 2: bgram_s_rows<2>(a, nv, C, cg, rg, R, r0, r1, sa, ca, sw, cw, mx); break;
      case 3: bgram_s_rows<3>(a, nv, C, cg, rg, R, r0, r1, sa, ca, sw, cw, mx); break;
      default: bgram_s_rows<4>(a, nv, C, cg, rg, R, r0, r1, sa, ca, sw, cw, mx); break;
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) atomicMax(&s_max, mx);
    __syncthreads();
    if (df_window(s_max)) {
      float as[16], ac[16];
#pragma unroll
      for (int sl = 0; sl < kDfSlots; ++sl) {
        as[2 * sl] = sl < kBGramSSlots ? sa[sl < kBGramSSlots ? sl : 0] : 0.f;
        ac[2 * sl] = sl < kBGramSSlots ? ca[sl < kBGramSSlots ? sl : 0] : 0.f;
        as[2 * sl + 1] = sl < kBGramSSlots ? sw[sl < kBGramSSlots ? sl : 0] : 0.f;
        ac[2 * sl + 1] = sl < kBGramSSlots ? cw[sl < kBGramSSlots ? sl : 0] : 0.f;
      }
      df_warp_reduce16(as, ac);
      const int qd = lane >> 1, sl = qd >> 1, j = cg + sl * C;
      if ((lane & 1) == 0 && sl < S && j < nv)
        s_part[rg][(qd & 1) ? (kMaxM + 1 + j) : j] = widen_normal(as[0]) + widen_normal(ac[0]);
    } else {  // FP64 recomputation of this block's rows from the stored pairs (w outside the window)
      const float2* vi = a.Vs + (int64_t)i * a.ldv;
#pragma unroll 1
      for (int sl = 0; sl < S; ++sl) {
        const int j = cg + sl * C;
        double fa = 0.0, fw = 0.0;
        if (j < nv) {
          const float2* vj = a.Vs + (int64_t)j * a.ldv;
          for (int64_t r = r0 + rg * 32 + lane; r < r1; r += 32 * R) {
            const double x = join2(rp_get(vj, r));
            fa = fma(x, join2(rp_get(vi, r)), fa);
            fw = fma(x, a.w[r], fw);
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          fa += __shfl_xor_sync(0xffffffffu, fa, o);
          fw += __shfl_xor_sync(0xffffffffu, fw, o);
        }
        if (lane == 0 && j < nv) {
          s_part[rg][j] = fa;
          s_part[rg][kMaxM + 1 + j] = fw;
        }
      }
    }
    __syncthreads();
    for (int v = threadIdx.x; v < 2 * nv; v += blockDim.x) {
      const int col = v < nv ? v : (kMaxM + 1) + (v - nv);
      double sum = 0.0;
      for (int g = 0; g < R; ++g) sum += s_part[g][col];
      a.partials[(int64_t)blockIdx.x * stride + col] = sum;
    }
  }
  if (!last_of_system(a.sticket + sys, nb)) return;
  if (!active) return;
  bgram_tail(a, st, sys, i, nb, true);
}

// NW basis columns j0 .. j0 + NW - 1 (j0 a multiple of 4) of one row pair into the pair
// accumulators (1 + j) mod 4 (accumulator 0 starts with w / beta_i); coefficient records
// cf[j] hold the split of -h_j / beta_j in both lanes.
template <int NW>
__device__ __forceinline__ void bupd_cols(const float2* __restrict__ Vs, int64_t ldv, int64_t g, int j0,
                                          const UpdCoef* cf, f2_t (&ps)[4], f2_t (&pc)[4]) {
  float4 x[NW];
#pragma unroll
  for (int k = 0; k < NW; ++k) x[k] = __ldcs(reinterpret_cast<const float4*>(Vs + (int64_t)(j0 + k) * ldv) + g);
#pragma unroll
  for (int k = 0; k < NW; ++k) {
    const float4 hl = cf[j0 + k].hl, nh = cf[j0 + k].nh;
    f2_t xh, xl;
    group_f2(x[k], xh, xl);
    dot2_step2(ps[(1 + k) & 3], pc[(1 + k) & 3], xh, xl, f2_pack(hl.x, hl.y), f2_pack(hl.z, hl.w), f2_pack(nh.x, nh.y));
  }
}

// FP64 recomputation of one row of the batched split update (outside the double-FP32 window, or
// a block's lone first / last row): stored into its own lane of column i + 1 and the next
// V-cycle input.
__device__ __forceinline__ void bupd_row_fp64(const BatchArgs& a, const double* __restrict__ s_c, int i, int64_t row,
                                              double wb, float2* vnext, double& q64) {
  double acc = wb;
  for (int j = 0; j <= i; ++j) acc = fma(-s_c[j], join2(rp_get(a.Vs + (int64_t)j * a.ldv, row)), acc);
  rp_set(vnext, row, split2(acc));
  if (a.v32) a.v32[row] = narrow_f64(acc);
  else a.vin[row] = acc;
  q64 = fma(acc, acc, q64);
}

// Batched update on the split basis (Algorithm 1 step 12 per active system):
//   vt_{i+1} = w / beta_i - sum_{j<=i} (h_j / beta_j) vt_j
// one thread per row pair, w / beta_i formed in FP64 and split, the sum in four packed
// (sum, error) pairs, stored as a normalised row-pair group in column i + 1 and, for the next
// V-cycle, in FP64 (vin) or FP32 (v32, the high part); ||vt_{i+1}||^2 in double-FP32 per thread,
// FP64 across blocks; then the per-system Givens step and stop test.
__global__ void __launch_bounds__(kRedThreads) k_bupdate_s(BatchArgs a) {
  pdl_enter();
  __shared__ double s_c[kMaxM + 1];    // h_j / beta_j
  __shared__ UpdCoef s_cf[kMaxM + 1];  // -h_j / beta_j split, in both lanes
  __shared__ unsigned s_cmax;
  __shared__ double s_red[kRedThreads / 32];
  __shared__ int s_sys;
  if (threadIdx.x == 0) {
    s_sys = find_system(a.bstart, a.nsys, blockIdx.x);
    s_cmax = 0u;
  }
  __syncthreads();
  const int sys = s_sys;
  GState* st = a.st + sys;
  const bool active = !st->stop;
  const int i = a.ctl->gi;
  const int nb = a.bstart[sys + 1] - a.bstart[sys];
  const int lane = threadIdx.x & 31;
  if (active) {
    const double invb = st->invbeta[i];
    for (int j = threadIdx.x; j <= i; j += blockDim.x) {
      const double cj = st->h[j] * st->invbeta[j];
      s_c[j] = cj;
      const float2 h = split2(-cj);
      s_cf[j].hl = make_float4(h.x, h.x, h.y, h.y);
      s_cf[j].nh = make_float4(-h.x, -h.x, 0.f, 0.f);
      atomicMax(&s_cmax, abs_hiword(cj));
    }
    __syncthreads();
    const bool cok = df_window(s_cmax);
    float2* vnext = a.Vs + (int64_t)(i + 1) * a.ldv;
    const int64_t r0 = a.off[sys] + (int64_t)(blockIdx.x - a.bstart[sys]) * a.rpb;
    const int64_t r1 = min(a.off[sys + 1], r0 + a.rpb);
    const int64_t g1 = r1 >> 1;
    const int nfull = (i + 1) & ~3;
    const f2_t m1 = f2_pack(-1.f, -1.f);
    f2_t qs2 = 0ull, qc2 = 0ull;
    double q64 = 0.0;
    for (int64_t g = ((r0 + 1) >> 1) + threadIdx.x; g < g1; g += blockDim.x) {
      const int64_t row = 2 * g;
      const double2 wv = __ldcs(reinterpret_cast<const double2*>(a.w) + g);
      const double wb0 = wv.x * invb, wb1 = wv.y * invb;
      if (cok && df_window(abs_hiword(wb0)) && df_window(abs_hiword(wb1))) {
        f2_t ps[4] = {0ull, 0ull, 0ull, 0ull}, pc[4] = {0ull, 0ull, 0ull, 0ull};
        float h0, l0, h1, l1;
        split_df(wb0, h0, l0);
        split_df(wb1, h1, l1);
        ps[0] = f2_pack(h0, h1);
        pc[0] = f2_pack(l0, l1);
#pragma unroll 2
        for (int j0 = 0; j0 < nfull; j0 += 4) bupd_cols<4>(a.Vs, a.ldv, g, j0, s_cf, ps, pc);
        switch (i + 1 - nfull) {
          case 1: bupd_cols<1>(a.Vs, a.ldv, g, nfull, s_cf, ps, pc); break;
          case 2: bupd_cols<2>(a.Vs, a.ldv, g, nfull, s_cf, ps, pc); break;
          case 3: bupd_cols<3>(a.Vs, a.ldv, g, nfull, s_cf, ps, pc); break;
          default: break;
        }
        df_add2(ps[0], pc[0], ps[1], pc[1]);
        df_add2(ps[2], pc[2], ps[3], pc[3]);
        df_add2(ps[0], pc[0], ps[2], pc[2]);
        const f2_t tt = f2_add(ps[0], pc[0]);  // normalised pairs (TwoSum)
        const f2_t z = f2_sub(tt, ps[0]);
        const f2_t e = f2_add(f2_sub(ps[0], f2_sub(tt, z)), f2_sub(pc[0], z));
        asm volatile("st.global.v2.b64 [%0], {%1, %2};" ::"l"(vnext + row), "l"(tt), "l"(e) : "memory");
        float t0f, t1f, e0f, e1f;
        f2_unpack(tt, t0f, t1f);
        f2_unpack(e, e0f, e1f);
        if (a.v32) {
          a.v32[row] = t0f;
          a.v32[row + 1] = t1f;
        } else {
          reinterpret_cast<double2*>(a.vin)[g] =
              make_double2(widen_normal(t0f) + widen_normal(e0f), widen_normal(t1f) + widen_normal(e1f));
        }
        dot2_step2(qs2, qc2, tt, e, tt, e, f2_mul(tt, m1));
      } else {
        bupd_row_fp64(a, s_c, i, row, wb0, vnext, q64);
        bupd_row_fp64(a, s_c, i, row + 1, wb1, vnext, q64);
      }
    }
    if (threadIdx.x < 2) {  // lone rows: thread 0 an odd first row, thread 1 an odd last row
      const int64_t row = threadIdx.x == 0 ? r0 : r1 - 1;
      if (row >= r0 && row < r1 && (threadIdx.x == 0 ? (r0 & 1) : (r1 & 1)) != 0)
        bupd_row_fp64(a, s_c, i, row, a.w[row] * invb, vnext, q64);
    }
    float qs, qc;
    {
      float s0, s1, c0, c1;
      f2_unpack(qs2, s0, s1);
      f2_unpack(qc2, c0, c1);
      df_add(s0, c0, s1, c1);
      qs = s0;
      qc = c0;
    }
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
    double ss = q64;
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
  bupdate_tail(a, st, sys, active, i, nb);
}

// Column 0 of a cycle for every running system (k_col0 per system): r <- r / 2^e with ||r|| =
// f 2^e, f in [0.5, 1) (exact), column 0 = split(r) row by row, r0_scale = 2^e, and the FP32
// copy for an FP32 V-cycle. r is the residual k_bresid wrote into vin.
__global__ void __launch_bounds__(kRedThreads) k_bcol0(BatchArgs a) {
  pdl_enter();
  __shared__ int s_sys;
  if (threadIdx.x == 0) s_sys = find_system(a.bstart, a.nsys, blockIdx.x);
  __syncthreads();
  const int sys = s_sys;
  GState* st = a.st + sys;
  if (st->stop) return;
  const double rn = st->rnorm;
  int e = 0;
  if (rn > 0.0 && isfinite(rn)) frexp(rn, &e);
  const double sc = ldexp(1.0, -e);
  if (blockIdx.x == a.bstart[sys] && threadIdx.x == 0) st->r0_scale = ldexp(1.0, e);
  const int64_t r0 = a.off[sys] + (int64_t)(blockIdx.x - a.bstart[sys]) * a.rpb;
  const int64_t r1 = min(a.off[sys + 1], r0 + a.rpb);
  for (int64_t row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    const double x = a.vin[row] * sc;
    a.vin[row] = x;
    rp_set(a.Vs, row, split2(x));
    if (a.v32) a.v32[row] = narrow_f64(x);
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
      st->rnorm = sqrt(R2);
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
