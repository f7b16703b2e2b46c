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
constexpr int kDfGramBlocksPerSM = 1;    // k_gram_df: 512 threads, up to 128 registers each
constexpr int kDfUpdateBlocksPerSM = 4;  // k_update_df: 256 threads

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
// Double-FP32 arithmetic for the one-reduce kernels.
//
// B300 issues FP64 FMAs at ~1/80 of its FP32 rate, so an FP64 Gram (2(i+1) products per row)
// and update (i+1) would be bound by the FP64 pipe, not by HBM. These kernels keep every vector
// in FP64 in memory but form the i-dependent products from two FP32 parts per FP64 value:
//   split_df:  x = hi + lo + d, hi the first 24 significant bits of x, lo the next 23, |d| <=
//              2^-46 |x|, formed by integer operations on the bit pattern (no FP64 instruction);
//   products:  TwoProduct in its FMA form, p + e = hi_a * hi_b exactly, plus the cross terms;
//   sums:      TwoSum (Knuth) into a running (sum, error) pair: the Dot2 scheme of Ogita, Rump
//              and Oishi (SIAM J. Sci. Comput. 26, 2005); each pair absorbs at most a few dozen
//              terms before pairs are combined.
// The result of a dot product is accurate to ~2^-45 of sum |a_k b_k| instead of FP64's
// n 2^-53 bound. Every operation below is an explicit _rn intrinsic, so the compiler can
// neither contract nor reassociate the error-free transformations.
// Validity window: a split is exact for 2^-103 <= |x| < 2^128 and gives (0, 0) below; the
// kernels check the magnitudes they meet and recompute in FP64 where data leave
// [2^-50, 2^60] (products must neither overflow nor lose the low part to underflow).
// ------------------------------------------------------------------------------------------
constexpr unsigned kDfTiny = (1023u - 103u) << 20;  // |x| < 2^-103 splits to (0, 0)
constexpr unsigned kDfLow = (1023u - 50u) << 20;    // window: 2^-50 <= max |x| ...
constexpr unsigned kDfHigh = (1023u + 60u) << 20;   // ... < 2^60 (or all zero)

__device__ __forceinline__ unsigned abs_hiword(double x) { return (unsigned)__double2hiint(x) & 0x7fffffffu; }

// Largest |x| seen (as the high word of |x|) lies in the double-FP32 window (or is zero).
__device__ __forceinline__ bool df_window(unsigned maxhw) {
  return maxhw == 0u || (maxhw >= kDfLow && maxhw < kDfHigh);
}

__device__ __forceinline__ void split_df(double x, float& hi, float& lo) {
  const unsigned lw = (unsigned)__double2loint(x), hw = (unsigned)__double2hiint(x);
  const unsigned sgn = hw & 0x80000000u;
  const bool tiny = (hw & 0x7fffffffu) < kDfTiny;
  // (hw:lw) << 3 puts the low 9 exponent bits and 23 mantissa bits in one word; subtracting 384
  // from the 9-bit field maps every exponent of the binary32 normal range (1023 - 126 .. 1023 +
  // 127) to its binary32 biased value (bit 31 stays clear).
  unsigned t = __funnelshift_l(lw, hw, 3) - 0xC0000000u;
  t = tiny ? 0u : t;
  hi = __uint_as_float(t | sgn);
  // lo: the next 23 bits (lw bits 28..6) as a binary32 number whose unit is 2^-23 ulp(hi):
  // (2^e_lo + m 2^(e_lo - 23)) - 2^e_lo with e_lo = e_hi - 23, exact.
  int eb = (int)(t & 0x7f800000u) - (23 << 23);
  eb = max(eb, 0);
  const unsigned ebs = (unsigned)eb | sgn;
  lo = __fsub_rn(__uint_as_float(((lw >> 6) & (tiny ? 0u : 0x7fffffu)) | ebs), __uint_as_float(ebs));
}

// (s, c) += (ah + al)(bh + bl): TwoProduct of the high parts, cross terms into the error, TwoSum.
__device__ __forceinline__ void dot2_step(float& s, float& c, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

// (s, c) += (s2, c2)
__device__ __forceinline__ void df_add(float& s, float& c, float s2, float c2) {
  const float t = __fadd_rn(s, s2);
  const float z = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(s2, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(c2, err));
}

// binary32 -> binary64 by integer operations for normal numbers and zero (subnormal inputs,
// |f| < 2^-126, give 0).
__device__ __forceinline__ double widen_normal(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned a = u & 0x7fffffffu;
  const unsigned hw = a < 0x00800000u ? 0u : (((a >> 3) + (896u << 20)) | (u & 0x80000000u));
  const unsigned lw = a < 0x00800000u ? 0u : (u << 29);
  return __hiloint2double((int)hw, (int)lw);
}

// Warp reduce-scatter of 16 (sum, error) pairs acc[q] (recursive halving, fixed order): on return
// lanes 2q and 2q + 1 hold the warp total of pair q in acc[0].
__device__ __forceinline__ void df_warp_reduce16(float (&as)[16], float (&ac)[16]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int lev = 0; lev < 4; ++lev) {
    const int o = 16 >> lev, half = 8 >> lev;
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const float ss = upper ? as[k] : as[k + half], sc = upper ? ac[k] : ac[k + half];
      float ks = upper ? as[k + half] : as[k], kc = upper ? ac[k + half] : ac[k];
      float rs = __shfl_xor_sync(0xffffffffu, ss, o), rc = __shfl_xor_sync(0xffffffffu, sc, o);
      // fixed order: the lower lane's value first
      if (upper) { df_add(rs, rc, ks, kc); ks = rs; kc = rc; } else { df_add(ks, kc, rs, rc); }
      as[k] = ks;
      ac[k] = kc;
    }
  }
  float rs = __shfl_xor_sync(0xffffffffu, as[0], 1), rc = __shfl_xor_sync(0xffffffffu, ac[0], 1);
  if (lane & 1) { float s0 = rs, c0 = rc; df_add(s0, c0, as[0], ac[0]); as[0] = s0; ac[0] = c0; }
  else df_add(as[0], ac[0], rs, rc);
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
  const float2* Vs;    // split basis (k_gram_s): column j = vt_j as (hi, lo) pairs, leading dimension ldv
};

// Last block of a Gram launch: fixed-order sum of the block partials (layout: column j of a at
// j, of s at kMaxM + 1 + j), then either the 2(i+1) results (standalone) or steps 7-11 of
// Algorithm 1 on the solver state.
__device__ void gram_tail(const GramArgs& a, int i) {
  __shared__ double red[2 * (kMaxM + 1)];
  GState* st = a.st;
  const int ncol = i + 1;
  const int lane = threadIdx.x & 31;
  const int stride = 2 * (kMaxM + 1);
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
  if (a.Vs) {  // split basis: column j < i holds vt_j = beta_j v_j
    for (int j = threadIdx.x; j < i; j += blockDim.x) {
      red[j] *= st->invbeta[j];
      red[kMaxM + 1 + j] *= st->invbeta[j];
    }
    __syncthreads();
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
      if (st->status != NSAMG_ERR_TIMEOUT) st->status = isfinite(beta) ? 0 : -6;
      st->stop = 1;
      st->done = 1;
    }
    st->beta[i] = beta;
    st->invbeta[i] = 1.0 / beta;
    if (i == 0) st->g[0] = a.Vs ? beta * st->r0_scale : beta;  // split basis: column 0 is r / r0_scale
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


__global__ void __launch_bounds__(kGramThreads) k_gram(GramArgs a) {
  pdl_enter();
  __shared__ double s_vt[kGramTile];
  __shared__ double s_w[kGramTile];
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
  gram_tail(a, i);
}


// ------------------------------------------------------------------------------------------
// Gram in double-FP32 (the solve's default): the i products of each row with the normalised
// columns v_0..v_{i-1} use split_df / dot2_step; column i (vt . vt, vt . w) stays FP64 (two FMAs
// per row). Per tile, vt and w are split once into shared memory; warps form C column groups x
// 16/C row groups, each warp owning at most kDfSlots columns (C chosen for the best balance).
// Each thread keeps 2 x kDfSlots (sum, error) pairs over its rows of the block's chunk; a warp
// reduce-scatter combines them, then FP64 takes over for the block and grid sums (same partial
// layout and last-block finalise as k_gram). A block whose vt, w (and, with CHECK_V, V) maxima
// leave the double-FP32 window recomputes its chunk in FP64; the choice depends only on the
// data, so results stay bitwise repeatable.
// ------------------------------------------------------------------------------------------
constexpr int kDfSlots = 8;
constexpr int kDfTile = 1024;

// Column groups C (a power of two <= 16): the smallest C * ceil(nv / C) (the busiest warp's
// share) with at most kDfSlots columns per warp; ties go to the smaller C, i.e. more columns per
// warp, over which each row's fixed work (loading and splitting vt and w) is spread.
__device__ __forceinline__ int df_groups(int nv, int max_slots = kDfSlots) {
  int best = 16, cost = 16 * ((nv + 15) / 16);
#pragma unroll
  for (int c = 8; c >= 1; c >>= 1) {
    const int sl = (nv + c - 1) / c;
    if (sl <= max_slots && c * sl <= cost) {
      best = c;
      cost = c * sl;
    }
  }
  return best;
}

template <bool CHECK_V>
__global__ void __launch_bounds__(kGramThreads, 1) k_gram_df(GramArgs a) {
  pdl_enter();
  __shared__ float4 s_sp[kDfTile];  // per row of the tile: (vt_hi, vt_lo, w_hi, w_lo)
  __shared__ double s_part[kGramWarps][2 * (kMaxM + 1)];
  __shared__ double s_col[2][kGramThreads];
  __shared__ unsigned s_max[2];
  GState* st = a.st;
  if (st && st->stop) return;
  const int i = st ? st->i : a.i_standalone;
  const int nv = i;  // normalised columns 0..i-1
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int C = df_groups(nv > 0 ? nv : 1);
  const int R = kGramWarps / C;
  const int S = (nv + C - 1) / C;
  const int cg = warp % C, rg = warp / C;
  const int rows_w = kDfTile / R;
  const int64_t chunk = ((a.n + gridDim.x - 1) / gridDim.x + kDfTile - 1) / kDfTile * kDfTile;
  const int64_t r0 = (int64_t)blockIdx.x * chunk;
  const int64_t r1 = min(a.n, r0 + chunk);
  const double* vt = a.V + (int64_t)i * a.ldv;
  if (threadIdx.x < 2) s_max[threadIdx.x] = 0u;
  __syncthreads();
  float sa[kDfSlots], ca[kDfSlots], sw[kDfSlots], cw[kDfSlots];
#pragma unroll
  for (int s = 0; s < kDfSlots; ++s) sa[s] = ca[s] = sw[s] = cw[s] = 0.f;
  double aii = 0.0, aiw = 0.0;
  unsigned mx = 0u, mv = 0u;
  for (int64_t t0 = r0; t0 < r1; t0 += kDfTile) {
    const int tn = (int)((r1 - t0) < (int64_t)kDfTile ? (r1 - t0) : (int64_t)kDfTile);
    __syncthreads();
    for (int r = threadIdx.x; r < kDfTile; r += kGramThreads) {
      float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < tn) {
        const double x = __ldcs(vt + t0 + r), y = __ldcs(a.w + t0 + r);
        aii = fma(x, x, aii);
        aiw = fma(x, y, aiw);
        mx = max(mx, max(abs_hiword(x), abs_hiword(y)));
        split_df(x, q.x, q.y);
        split_df(y, q.z, q.w);
      }
      s_sp[r] = q;
    }
    __syncthreads();
    if (S > 0) {
      for (int k = 0; k < rows_w; k += 32) {
        const int r = rg * rows_w + k + lane;
        if (r >= tn) break;
        const float4 q = s_sp[r];
        double xv[kDfSlots];
#pragma unroll
        for (int s = 0; s < kDfSlots; ++s) {
          const int j = cg + s * C;
          xv[s] = (s < S && j < nv) ? __ldcs(a.V + (int64_t)j * a.ldv + t0 + r) : 0.0;
        }
#pragma unroll
        for (int s = 0; s < kDfSlots; ++s) {
          if (s < S) {
            if (CHECK_V) mv = max(mv, abs_hiword(xv[s]));
            float xh, xl;
            split_df(xv[s], xh, xl);
            dot2_step(sa[s], ca[s], xh, xl, q.x, q.y);
            dot2_step(sw[s], cw[s], xh, xl, q.z, q.w);
          }
        }
      }
    }
  }
  // window test on the block maxima (vt and w always; V columns when they may be unnormalised)
  mx = __reduce_max_sync(0xffffffffu, mx);
  mv = __reduce_max_sync(0xffffffffu, mv);
  if (lane == 0) {
    atomicMax(&s_max[0], mx);
    atomicMax(&s_max[1], mv);
  }
  s_col[0][threadIdx.x] = aii;
  s_col[1][threadIdx.x] = aiw;
  __syncthreads();
  const bool fp64 = !df_window(s_max[0]) || (CHECK_V && !df_window(s_max[1]));
  if (!fp64) {
    float as[16], ac[16];
#pragma unroll
    for (int s = 0; s < kDfSlots; ++s) {
      as[2 * s] = sa[s];
      ac[2 * s] = ca[s];
      as[2 * s + 1] = sw[s];
      ac[2 * s + 1] = cw[s];
    }
    df_warp_reduce16(as, ac);
    const int q = lane >> 1, s = q >> 1, j = cg + s * C;
    if ((lane & 1) == 0 && s < S && j < nv)
      s_part[rg][(q & 1) ? (kMaxM + 1 + j) : j] = widen_normal(as[0]) + widen_normal(ac[0]);
  } else {
    // FP64 recomputation of this block's chunk (data outside the double-FP32 window)
#pragma unroll 1
    for (int s = 0; s < S; ++s) {
      const int j = cg + s * C;
      double fa = 0.0, fw = 0.0;
      if (j < nv) {
        const double* vj = a.V + (int64_t)j * a.ldv;
        for (int64_t t0 = r0; t0 < r1; t0 += kDfTile) {
          for (int r = rg * rows_w + lane; r < (rg + 1) * rows_w && t0 + r < r1; r += 32) {
            const double x = vj[t0 + r];
            fa = fma(x, vt[t0 + r], fa);
            fw = fma(x, a.w[t0 + r], fw);
          }
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
  // column i (vt): fixed-order sum of the 512 per-thread FP64 partials by two warps
  if (warp < 2) {
    double v = 0.0;
    for (int t = lane; t < kGramThreads; t += 32) v += s_col[warp][t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_part[0][warp ? (kMaxM + 1 + i) : i] = v;
  }
  __syncthreads();
  const int stride = 2 * (kMaxM + 1);
  for (int v = threadIdx.x; v < 2 * (i + 1); v += blockDim.x) {
    const int col = v <= i ? v : (kMaxM + 1) + (v - i - 1);
    const int j = v <= i ? v : v - i - 1;
    double sum = 0.0;
    if (j == i) sum = s_part[0][col];
    else
      for (int g = 0; g < R; ++g) sum += s_part[g][col];  // the R row-group warps of j's column group
    a.scr.partials[(int64_t)blockIdx.x * stride + col] = sum;
  }
  if (!last_block(a.scr.ticket)) return;
  gram_tail(a, i);
}


// ------------------------------------------------------------------------------------------
// Asynchronous bulk copies (global -> shared, the TMA engine's 1D form) and mbarriers.
// Every wait is bounded: after kSpinLimit polls it reports failure instead of spinning on.
// ------------------------------------------------------------------------------------------
constexpr int kSpinLimit = 1 << 15;         // polls of a wait before it gives up
constexpr unsigned kSuspendNs = 100000u;    // each poll may suspend the thread up to 100 us

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// The thread sleeps in the poll until the phase completes or kSuspendNs pass, instead of
// spinning on issue slots the consumers need.
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0u;
}
// true once the phase with the given parity has completed; false after kSpinLimit polls
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  for (int k = 0; k < kSpinLimit; ++k)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// bytes (a multiple of 16) from 16-byte aligned global src to 16-byte aligned shared dst;
// completion is counted on the mbarrier's transaction count
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// ------------------------------------------------------------------------------------------
// Gram in double-FP32 with a bulk-copy pipeline (the solve's kernel when every column start is
// 16-byte aligned). One block per SM: 16 consumer warps (the C x R column/row groups of
// k_gram_df) and one producer warp whose lane 0 streams each tile (rows [t0, t0 + T) of the i
// columns, vt and w) into a ring of kGramTmaStages shared-memory stages with cp.async.bulk, one
// full/empty mbarrier pair per stage. The consumers split vt and w per row themselves (no block
// barrier between tiles), read V from the stage, and release it with one arrive per warp. A
// ragged odd last row is read from global memory. Same partial layout, window test, FP64
// fallback and last-block finalise as k_gram_df. A wait that gives up (it cannot, unless the
// copy engine stalls) makes the block's partials NaN and, in a solve, sets NSAMG_ERR_TIMEOUT.
// ------------------------------------------------------------------------------------------
constexpr int kGramTmaConsumers = 16;
constexpr int kGramTmaThreads = 32 * (kGramTmaConsumers + 1);
constexpr int kRingBytes = 192 * 1024;  // stage area of a ring (all its stages)
constexpr int kGramTmaStages = 3;
constexpr int kGramTmaStageBytes = kRingBytes / kGramTmaStages;
constexpr int kGramTmaSmem = kRingBytes + 2 * 3 * 8;  // stages + full/empty barriers (up to 3 stages)

// Rows per tile: the largest multiple of 32 R for which a stage (i columns + vt + w) fits,
// at most 2048 (for i <= 64 this is always at least 32 R).
__device__ __forceinline__ int tma_tile_rows(int i, int R) {
  const int per = kGramTmaStageBytes / (8 * (i + 2));
  const int t = per / (32 * R) * (32 * R);
  return t < 2048 ? t : 2048;
}

// One stage ring: NST buffers of BYTES / NST bytes followed by the full and empty mbarriers.
// Item k uses stage k % NST in round k / NST.
template <int NST, int BYTES = kRingBytes>
struct RingT {
  static constexpr int kStages = NST;
  static constexpr int kStageBytes = BYTES / NST;
  static_assert(kStageBytes % 16 == 0, "bulk copies need 16-byte aligned stages");
  double* stage;
  unsigned full0, empty0;
  __device__ __forceinline__ double* buf(int k) const { return stage + (int64_t)(k % NST) * (kStageBytes / 8); }
  __device__ __forceinline__ unsigned full(int k) const { return full0 + 8u * (unsigned)(k % NST); }
  __device__ __forceinline__ unsigned empty(int k) const { return empty0 + 8u * (unsigned)(k % NST); }
  __device__ __forceinline__ unsigned round(int k) const { return (unsigned)(k / NST) & 1u; }
};
using Ring = RingT<kGramTmaStages>;

template <int NST, int BYTES = kRingBytes>
__device__ __forceinline__ RingT<NST, BYTES> ring_init_t(unsigned char* dsm) {
  RingT<NST, BYTES> g;
  g.stage = reinterpret_cast<double*>(dsm);
  g.full0 = smem_u32(dsm + BYTES);
  g.empty0 = g.full0 + 8u * NST;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(g.full0 + 8u * s, 1u);
      mbar_init(g.empty0 + 8u * s, (unsigned)kGramTmaConsumers);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  return g;
}
__device__ __forceinline__ Ring ring_init(unsigned char* dsm) { return ring_init_t<kGramTmaStages>(dsm); }

// Producer (one warp): for every item k < nitems, lane 0 waits until the item's stage is free
// and arms its full barrier with the item's byte count, then the 32 lanes issue the item's
// segments in parallel (segment q by lane q mod 32). seg(k, q, &src, &dst_off) describes segment q
// of item k (nseg(k) of them), each rows(k) doubles (rounded down to even) long. Returns false
// (in every lane) if a wait gave up; before returning, lane 0 waits (bounded) for the copies
// still in flight.
template <class RG, typename NSeg, typename Rows, typename Seg>
__device__ bool ring_produce(const RG& g, int nitems, NSeg nseg, Rows rows, Seg seg, volatile int* abort) {
  const int lane = threadIdx.x & 31;
  int issued = 0;
  bool ok = true;
  for (int k = 0; k < nitems; ++k) {
    int go = 1;
    if (lane == 0) go = mbar_wait(g.empty(k), g.round(k) ^ 1u) ? 1 : 0;
    go = __shfl_sync(0xffffffffu, go, 0);
    if (!go) {
      ok = false;
      break;
    }
    if (*abort) break;
    const int te = rows(k) & ~1;
    const int ns = nseg(k);
    if (lane == 0) {
      if (te > 0) mbar_expect_tx(g.full(k), 8u * (unsigned)te * (unsigned)ns);
      else mbar_arrive(g.full(k));  // nothing to copy (a one-row tile): the consumers read global memory
    }
    __syncwarp();
    if (te > 0) {
      double* dst = g.buf(k);
      for (int q = lane; q < ns; q += 32) {
        const double* src;
        int off;
        seg(k, q, &src, &off);
        bulk_g2s(smem_u32(dst + off), src, 8u * (unsigned)te, g.full(k));
      }
    }
    issued = k + 1;
  }
  if (lane == 0)
    for (int k = (issued > RG::kStages ? issued - RG::kStages : 0); k < issued; ++k)
      if (!mbar_wait(g.full(k), g.round(k))) ok = false;
  return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

// The same with one thread issuing every copy (k_gram_tma's producer).
template <class RG, typename NSeg, typename Rows, typename Seg>
__device__ bool ring_produce_lane0(const RG& g, int nitems, NSeg nseg, Rows rows, Seg seg, volatile int* abort) {
  int issued = 0;
  bool ok = true;
  for (int k = 0; k < nitems; ++k) {
    if (!mbar_wait(g.empty(k), g.round(k) ^ 1u)) {
      ok = false;
      break;
    }
    if (*abort) break;
    const int te = rows(k) & ~1;
    if (te > 0) {
      const int ns = nseg(k);
      const unsigned bytes = 8u * (unsigned)te;
      mbar_expect_tx(g.full(k), bytes * (unsigned)ns);
      double* dst = g.buf(k);
      for (int q = 0; q < ns; ++q) {
        const double* src;
        int off;
        seg(k, q, &src, &off);
        bulk_g2s(smem_u32(dst + off), src, bytes, g.full(k));
      }
    } else {
      mbar_arrive(g.full(k));  // nothing to copy (a one-row tile): the consumers read global memory
    }
    issued = k + 1;
  }
  for (int k = (issued > RG::kStages ? issued - RG::kStages : 0); k < issued; ++k)
    if (!mbar_wait(g.full(k), g.round(k))) ok = false;
  return ok;
}

// Consumer warp: wait for item k (every lane polls, so that no branch on the lane index leaves
// the warp split for the tile's work); false if the wait gave up in any lane.
template <class RG>
__device__ __forceinline__ bool ring_acquire(const RG& g, int k) {
  const bool ok = mbar_wait(g.full(k), g.round(k));
  return __all_sync(0xffffffffu, ok);
}
// One arrive per warp on the stage's empty barrier, by lane 0 through a predicate (no branch).
template <class RG>
__device__ __forceinline__ void ring_release(const RG& g, int k) {
  __syncwarp();
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.eq.u32 p, %1, 0;\n\t@p mbarrier.arrive.shared::cta.b64 _, [%0];\n\t}" ::"r"(
          g.empty(k)),
      "r"(threadIdx.x & 31)
      : "memory");
}

// Gram consumer work on one staged tile: rows [rb, re) (all in shared memory, stride 32 over the
// warp) times the warp's NS columns cg + s C, and (column group 0) the FP64 vt . vt, vt . w.
template <int NS, bool CHECK_V>
__device__ __forceinline__ void gram_rows(const double* __restrict__ sb, int T, int nv, int C, int cg, int rb, int re,
                                          float (&sa)[kDfSlots], float (&ca)[kDfSlots], float (&sw)[kDfSlots],
                                          float (&cw)[kDfSlots], double& aii, double& aiw, unsigned& mx,
                                          unsigned& mv) {
  const int lane = threadIdx.x & 31;
  for (int r = rb + lane; r < re; r += 32) {
    const double xt = sb[nv * T + r], xw = sb[(nv + 1) * T + r];
    if (cg == 0) {
      aii = fma(xt, xt, aii);
      aiw = fma(xt, xw, aiw);
      mx = max(mx, max(abs_hiword(xt), abs_hiword(xw)));
    }
    if constexpr (NS > 0) {
      float q0, q1, q2, q3;
      split_df(xt, q0, q1);
      split_df(xw, q2, q3);
      double xv[NS];
#pragma unroll
      for (int sl = 0; sl < NS; ++sl) {
        // only the last slot can pass the last column; its (discarded) products then read column nv - 1
        const int j = (sl == NS - 1) ? min(cg + sl * C, nv - 1) : cg + sl * C;
        xv[sl] = sb[j * T + r];
      }
#pragma unroll
      for (int sl = 0; sl < NS; ++sl) {
        if (CHECK_V) mv = max(mv, abs_hiword(xv[sl]));
        float xh, xl;
        split_df(xv[sl], xh, xl);
        dot2_step(sa[sl], ca[sl], xh, xl, q0, q1);
        dot2_step(sw[sl], cw[sl], xh, xl, q2, q3);
      }
    }
  }
}

// The same for one row read from global memory (the odd last row of a chunk), any slot count.
template <bool CHECK_V>
__device__ __forceinline__ void gram_row_global(const GramArgs& a, const double* vt, int64_t row, int nv, int S,
                                                int C, int cg, float (&sa)[kDfSlots], float (&ca)[kDfSlots],
                                                float (&sw)[kDfSlots], float (&cw)[kDfSlots], double& aii,
                                                double& aiw, unsigned& mx, unsigned& mv) {
  const double xt = vt[row], xw = a.w[row];
  if (cg == 0) {
    aii = fma(xt, xt, aii);
    aiw = fma(xt, xw, aiw);
    mx = max(mx, max(abs_hiword(xt), abs_hiword(xw)));
  }
  float q0, q1, q2, q3;
  split_df(xt, q0, q1);
  split_df(xw, q2, q3);
#pragma unroll
  for (int sl = 0; sl < kDfSlots; ++sl) {
    const int j = cg + sl * C;
    if (sl < S && j < nv) {
      const double x = a.V[(int64_t)j * a.ldv + row];
      if (CHECK_V) mv = max(mv, abs_hiword(x));
      float xh, xl;
      split_df(x, xh, xl);
      dot2_step(sa[sl], ca[sl], xh, xl, q0, q1);
      dot2_step(sw[sl], cw[sl], xh, xl, q2, q3);
    }
  }
}

template <bool CHECK_V>
__global__ void __launch_bounds__(kGramTmaThreads, 1) k_gram_tma(GramArgs a) {
  pdl_enter();
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ double s_part[kGramWarps][2 * (kMaxM + 1)];
  __shared__ unsigned s_max[2];
  __shared__ volatile int s_abort;
  GState* st = a.st;
  if (st && st->stop) return;
  const int i = st ? st->i : a.i_standalone;
  const int nv = i;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int C = df_groups(nv > 0 ? nv : 1);
  const int R = kGramWarps / C;
  const int S = (nv + C - 1) / C;
  const int T = tma_tile_rows(i, R);
  const int rows_w = T / R;
  const int64_t chunk = ((a.n + gridDim.x - 1) / gridDim.x + T - 1) / T * T;
  const int64_t r0 = (int64_t)blockIdx.x * chunk;
  const int64_t r1 = min(a.n, r0 + chunk);
  const int ntiles = r1 > r0 ? (int)((r1 - r0 + T - 1) / T) : 0;
  const double* vt = a.V + (int64_t)i * a.ldv;
  const Ring g = ring_init(dsm);
  if (threadIdx.x == 0) {
    s_max[0] = s_max[1] = 0u;
    s_abort = 0;
  }
  __syncthreads();
  float sa[kDfSlots], ca[kDfSlots], sw[kDfSlots], cw[kDfSlots];
#pragma unroll
  for (int s = 0; s < kDfSlots; ++s) sa[s] = ca[s] = sw[s] = cw[s] = 0.f;
  double aii = 0.0, aiw = 0.0;
  unsigned mx = 0u, mv = 0u;
  const int cg = warp % C, rg = warp / C;
  auto tile_rows = [&](int k) -> int {
    const int64_t t0 = r0 + (int64_t)k * T;
    return (int)((r1 - t0) < (int64_t)T ? (r1 - t0) : (int64_t)T);
  };
  if (warp == kGramTmaConsumers) {
    if (lane == 0) {  // producer (one thread): per tile the i columns, vt and w
      const bool ok = ring_produce_lane0(
          g, ntiles, [&](int) { return nv + 2; }, tile_rows,
          [&](int k, int q, const double** src, int* off) {
            const int64_t t0 = r0 + (int64_t)k * T;
            *src = (q < nv ? a.V + (int64_t)q * a.ldv : (q == nv ? vt : a.w)) + t0;
            *off = q * T;
          },
          &s_abort);
      if (!ok && lane == 0) s_abort = 1;
    }
  } else {
    for (int k = 0; k < ntiles; ++k) {
      if (!ring_acquire(g, k)) {
        s_abort = 1;
        break;
      }
      const int tn = tile_rows(k), te = tn & ~1;
      const double* sb = g.buf(k);
      const int rb = rg * rows_w, re = min((rg + 1) * rows_w, te);
      switch (S) {
#define NSAMG_GRAM_ROWS(NS)                                                                            \
  case NS:                                                                                             \
    gram_rows<NS, CHECK_V>(sb, T, nv, C, cg, rb, re, sa, ca, sw, cw, aii, aiw, mx, mv);                \
    break;
        NSAMG_GRAM_ROWS(0)
        NSAMG_GRAM_ROWS(1)
        NSAMG_GRAM_ROWS(2)
        NSAMG_GRAM_ROWS(3)
        NSAMG_GRAM_ROWS(4)
        NSAMG_GRAM_ROWS(5)
        NSAMG_GRAM_ROWS(6)
        NSAMG_GRAM_ROWS(7)
        NSAMG_GRAM_ROWS(8)
#undef NSAMG_GRAM_ROWS
        default: break;
      }
      if (te < tn && te >= rg * rows_w && te < (rg + 1) * rows_w && lane == 0)  // the odd last row
        gram_row_global<CHECK_V>(a, vt, r0 + (int64_t)k * T + te, nv, S, C, cg, sa, ca, sw, cw, aii, aiw, mx, mv);
      ring_release(g, k);
    }
  }
  // ---- block epilogue (as k_gram_df) ----
  if (warp < kGramTmaConsumers) {
    mx = __reduce_max_sync(0xffffffffu, mx);
    mv = __reduce_max_sync(0xffffffffu, mv);
    if (lane == 0) {
      atomicMax(&s_max[0], mx);
      atomicMax(&s_max[1], mv);
    }
  }
  __syncthreads();
  const bool abort = s_abort != 0;
  const bool fp64 = !abort && (!df_window(s_max[0]) || (CHECK_V && !df_window(s_max[1])));
  if (warp < kGramTmaConsumers) {
    if (!fp64) {
      float as[16], ac[16];
#pragma unroll
      for (int s = 0; s < kDfSlots; ++s) {
        as[2 * s] = sa[s];
        ac[2 * s] = ca[s];
        as[2 * s + 1] = sw[s];
        ac[2 * s + 1] = cw[s];
      }
      df_warp_reduce16(as, ac);
      const int qd = lane >> 1, sl = qd >> 1, j = cg + sl * C;
      if ((lane & 1) == 0 && sl < S && j < nv)
        s_part[rg][(qd & 1) ? (kMaxM + 1 + j) : j] = widen_normal(as[0]) + widen_normal(ac[0]);
    } else {
      // FP64 recomputation of this block's chunk (data outside the double-FP32 window)
#pragma unroll 1
      for (int sl = 0; sl < S; ++sl) {
        const int j = cg + sl * C;
        double fa = 0.0, fw = 0.0;
        if (j < nv) {
          const double* vj = a.V + (int64_t)j * a.ldv;
          for (int64_t t0 = r0; t0 < r1; t0 += T)
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
        if (lane == 0 && j < nv) {
          s_part[rg][j] = fa;
          s_part[rg][kMaxM + 1 + j] = fw;
        }
      }
    }
    if (cg == 0) {  // column i: the R row-group warps of column group 0 hold its FP64 partials
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        aii += __shfl_xor_sync(0xffffffffu, aii, o);
        aiw += __shfl_xor_sync(0xffffffffu, aiw, o);
      }
      if (lane == 0) {
        s_part[rg][i] = aii;
        s_part[rg][kMaxM + 1 + i] = aiw;
      }
    }
  }
  __syncthreads();
  const int stride = 2 * (kMaxM + 1);
  for (int v = threadIdx.x; v < 2 * (i + 1); v += blockDim.x) {
    const int col = v <= i ? v : (kMaxM + 1) + (v - i - 1);
    double sum = 0.0;
    for (int g2 = 0; g2 < R; ++g2) sum += s_part[g2][col];
    a.scr.partials[(int64_t)blockIdx.x * stride + col] = abort ? __longlong_as_double(0x7ff8000000000000ll) : sum;
  }
  if (abort && threadIdx.x == 0 && st) st->status = NSAMG_ERR_TIMEOUT;
  if (!last_block(a.scr.ticket)) return;
  gram_tail(a, i);
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
  // split basis (k_update_s): column j = vt_j as (hi, lo) pairs; vt_{i+1} is written to column i+1
  // and, if vin is set, as FP64 to vin (the next V-cycle's input when it runs in FP64).
  // Standalone: coef_standalone[j] = h_j / beta_j (j <= i), the coefficients of the stored vt_j.
  float2* Vs;
  double* vin;
  const double* coef_standalone;
};

// Last block of an update launch: fixed-order sum of the block partials of ||vt_{i+1}||^2, then
// (standalone) the sum, or (in a solve) H_{i+1,i}, the Givens rotations and the stop decision.
__device__ void update_tail(const UpdateArgs& a, int i) {
  GState* st = a.st;
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
    // backward-error stop (Sec. 3): the denominator uses ||x|| at the start of the cycle, the
    // only norm of x known before the x-update; the true-residual test then decides exactly
    const double den = st->stop_nrbe ? st->bnorm + st->anorm_inf * st->xnorm : scale;
    const bool finite = isfinite(res) && isfinite(hsub) && isfinite(col[i]);
    int stop = (!finite) || res <= st->rtol * (den > 0.0 ? den : 1.0) || hsub == 0.0 || k >= st->m ||
               st->iters >= st->maxit;
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
  update_tail(a, i);
}


// ------------------------------------------------------------------------------------------
// Update in double-FP32 (the solve's default). Per row: v_i = vt/beta and w/beta are formed in
// FP64 (one multiply each; v_i is stored as before), then vt_{i+1} = w/beta - sum_{j<=i} h_j v_j
// accumulates from split(w/beta) in four (sum, error) pairs (columns 4q + k in pair k, so the
// dependency chains are short), combined in a fixed order and stored as the FP64 value
// sum + error (one FP64 add). ||vt_{i+1}||^2 accumulates per thread in double-FP32 and is
// summed in FP64 across blocks (fixed order). Rows whose w/beta, v_i (or, with CHECK_V, V
// entries) leave the double-FP32 window, and every row when the h_j do, are computed in FP64.
// ------------------------------------------------------------------------------------------
template <bool CHECK_V>
__global__ void __launch_bounds__(kRedThreads) k_update_df(UpdateArgs a) {
  pdl_enter();
  __shared__ double s_h[kMaxM + 1];
  __shared__ float2 s_hs[kMaxM + 1];  // -h_j as (hi, lo)
  __shared__ double s_red[kRedThreads / 32];
  __shared__ unsigned s_hmax;
  GState* st = a.st;
  if (st && st->stop) {  // stopped earlier in this step (error in the Gram): end the inner loop
    if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(a.cond_inner, 0);
    return;
  }
  const int i = st ? st->i : a.i_standalone;
  const double invb = st ? st->invbeta[i] : a.invbeta_standalone;
  if (threadIdx.x == 0) s_hmax = 0u;
  __syncthreads();
  for (int j = threadIdx.x; j <= i; j += blockDim.x) {
    const double hj = st ? st->h[j] : a.h_standalone[j];
    s_h[j] = hj;
    float hh, hl;
    split_df(-hj, hh, hl);
    s_hs[j] = make_float2(hh, hl);
    atomicMax(&s_hmax, abs_hiword(hj));
  }
  __syncthreads();
  const bool hok = df_window(s_hmax);
  double* vi = a.V + (int64_t)i * a.ldv;
  double* vn = a.V + (int64_t)(i + 1) * a.ldv;
  float qs = 0.f, qc = 0.f;  // sum of squares of the double-FP32 rows
  double q64 = 0.0;          // ... of the FP64 rows
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.n; r += (int64_t)gridDim.x * blockDim.x) {
    const double v = __ldcs(vi + r) * invb;
    vi[r] = v;
    const double wb = __ldcs(a.w + r) * invb;
    bool ok = hok && df_window(max(abs_hiword(v), abs_hiword(wb)));
    double acc = 0.0;
    if (ok) {
      // four independent (sum, error) pairs over the columns j = 4q + k (short dependency
      // chains), combined in a fixed order at the end
      float s0, c0, vh, vl;
      split_df(wb, s0, c0);
      split_df(v, vh, vl);
      float s1 = 0.f, c1 = 0.f, s2 = 0.f, c2 = 0.f, s3 = 0.f, c3 = 0.f;
      {
        const float2 hs = s_hs[i];
        dot2_step(s1, c1, hs.x, hs.y, vh, vl);
      }
      unsigned mvr = 0u;
      const double* col = a.V + r;
      int j = 0;
#pragma unroll 2
      for (; j + 4 <= i; j += 4) {
        double x[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) x[k] = __ldcs(col + (int64_t)(j + k) * a.ldv);
        float xh[4], xl[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (CHECK_V) mvr = max(mvr, abs_hiword(x[k]));
          split_df(x[k], xh[k], xl[k]);
        }
        const float2 h0 = s_hs[j], h1 = s_hs[j + 1], h2 = s_hs[j + 2], h3 = s_hs[j + 3];
        dot2_step(s0, c0, h0.x, h0.y, xh[0], xl[0]);
        dot2_step(s1, c1, h1.x, h1.y, xh[1], xl[1]);
        dot2_step(s2, c2, h2.x, h2.y, xh[2], xl[2]);
        dot2_step(s3, c3, h3.x, h3.y, xh[3], xl[3]);
      }
      for (; j < i; ++j) {
        const double x = __ldcs(col + (int64_t)j * a.ldv);
        if (CHECK_V) mvr = max(mvr, abs_hiword(x));
        float xh, xl;
        split_df(x, xh, xl);
        const float2 hs = s_hs[j];
        dot2_step(s2, c2, hs.x, hs.y, xh, xl);
      }
      df_add(s0, c0, s1, c1);
      df_add(s2, c2, s3, c3);
      df_add(s0, c0, s2, c2);
      if (CHECK_V && !df_window(mvr)) {
        ok = false;
      } else {
        acc = widen_normal(s0) + widen_normal(c0);
        // (t, e): the pair renormalised (TwoSum), the operands of its square
        const float t = __fadd_rn(s0, c0);
        const float z = __fsub_rn(t, s0);
        const float e = __fadd_rn(__fsub_rn(s0, __fsub_rn(t, z)), __fsub_rn(c0, z));
        if (a.v32) a.v32[r] = t;
        dot2_step(qs, qc, t, e, t, e);
      }
    }
    if (!ok) {
      acc = fma(-s_h[i], v, wb);
      for (int j = 0; j < i; ++j) acc = fma(-s_h[j], __ldcs(a.V + (int64_t)j * a.ldv + r), acc);
      if (a.v32) a.v32[r] = narrow_f64(acc);
      q64 = fma(acc, acc, q64);
    }
    vn[r] = acc;
  }
  // block sum of the squares: double-FP32 part reduced per warp, FP64 part only if a row needed it
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
  double wsum = widen_normal(qs) + widen_normal(qc);
  if (__syncthreads_or(q64 != 0.0)) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q64 += __shfl_xor_sync(0xffffffffu, q64, o);
    wsum += q64;
  }
  if (lane == 0) s_red[warp] = wsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
    a.scr.partials[blockIdx.x] = t;
  }
  if (!last_block(a.scr.ticket)) return;
  update_tail(a, i);
}


// ------------------------------------------------------------------------------------------
// Update in double-FP32 with the bulk-copy pipeline (the solve's kernel when every column start
// is 16-byte aligned). One block per SM; each consumer thread owns one row of a 512-row tile.
// The producer streams the tile's columns in chunks of kUpdChunk (vt and w first, then
// V_0 .. V_{i-1}) through the stage ring; per row, v_i = vt/beta and w/beta are formed in FP64
// (v_i is stored), and vt_{i+1} = w/beta - sum_j h_j v_j accumulates in four (sum, error) pairs
// (column j in pair j mod 4) across the chunks, then is stored as the FP64 value sum + error.
// Rows whose values leave the double-FP32 window (or, with CHECK_V, whose V entries do) are
// recomputed in FP64 from global memory; the odd last row of a chunk is read from global memory.
// ||vt_{i+1}||^2 and the last-block work as in k_update_df.
// ------------------------------------------------------------------------------------------
constexpr int kUpdTile = 32 * kGramTmaConsumers;                    // one row per consumer thread
constexpr int kUpdChunk = kGramTmaStageBytes / (8 * kUpdTile);      // columns per stage (16)

struct UpdRow {
  float s[4], c[4];  // four (sum, error) pairs
  double v, wb;      // v_i and w / beta of the row
  unsigned mvr;      // largest |V entry| of the row (high word)
  bool ok;           // the row stays in double-FP32
};

// columns [cb, ce) of the row's sequence (0: vt, 1: w, 2 + j: V_j); x(c) gives the value
template <bool CHECK_V, typename X>
__device__ __forceinline__ void upd_columns(UpdRow& u, int cb, int ce, double invb, const float2* __restrict__ s_hs,
                                            int i, X x) {
  int c = cb;
  if (c == 0) {
    u.v = x(0) * invb;
    u.wb = x(1) * invb;
    u.ok = u.ok && df_window(max(abs_hiword(u.v), abs_hiword(u.wb)));
    float vh, vl;
    split_df(u.wb, u.s[0], u.c[0]);
    split_df(u.v, vh, vl);
    const float2 hs = s_hs[i];
    dot2_step(u.s[1], u.c[1], hs.x, hs.y, vh, vl);
    c = 2;
  }
  // columns c .. ce - 1 are V_{c-2}; the k-th column of the chunk goes to pair k mod 4 (a fixed
  // assignment, so the row's sum is split the same way every time)
#pragma unroll
  for (int k = 0; k < kUpdChunk; ++k) {
    const int cc = c + k;
    if (cc < ce) {
      const double xv = x(cc);
      if (CHECK_V) u.mvr = max(u.mvr, abs_hiword(xv));
      float xh, xl;
      split_df(xv, xh, xl);
      const float2 hs = s_hs[cc - 2];
      dot2_step(u.s[k & 3], u.c[k & 3], hs.x, hs.y, xh, xl);
    }
  }
}

template <bool CHECK_V>
__global__ void __launch_bounds__(kGramTmaThreads, 1) k_update_tma(UpdateArgs a) {
  pdl_enter();
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ double s_h[kMaxM + 1];
  __shared__ float2 s_hs[kMaxM + 1];  // -h_j as (hi, lo)
  __shared__ double s_red[kGramTmaConsumers];
  __shared__ unsigned s_hmax;
  __shared__ volatile int s_abort;
  GState* st = a.st;
  if (st && st->stop) {  // stopped earlier in this step (error in the Gram): end the inner loop
    if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(a.cond_inner, 0);
    return;
  }
  const int i = st ? st->i : a.i_standalone;
  const double invb = st ? st->invbeta[i] : a.invbeta_standalone;
  const Ring g = ring_init(dsm);
  if (threadIdx.x == 0) {
    s_hmax = 0u;
    s_abort = 0;
  }
  __syncthreads();
  for (int j = threadIdx.x; j <= i; j += blockDim.x) {
    const double hj = st ? st->h[j] : a.h_standalone[j];
    s_h[j] = hj;
    float hh, hl;
    split_df(-hj, hh, hl);
    s_hs[j] = make_float2(hh, hl);
    atomicMax(&s_hmax, abs_hiword(hj));
  }
  __syncthreads();
  const bool hok = df_window(s_hmax);
  double* vi = a.V + (int64_t)i * a.ldv;
  double* vn = a.V + (int64_t)(i + 1) * a.ldv;
  const double* vtc = vi;
  const int ncols = i + 2, nchunks = (ncols + kUpdChunk - 1) / kUpdChunk;
  const int64_t chunk = ((a.n + gridDim.x - 1) / gridDim.x + kUpdTile - 1) / kUpdTile * kUpdTile;
  const int64_t r0 = (int64_t)blockIdx.x * chunk;
  const int64_t r1 = min(a.n, r0 + chunk);
  const int ntiles = r1 > r0 ? (int)((r1 - r0 + kUpdTile - 1) / kUpdTile) : 0;
  const int nitems = ntiles * nchunks;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto tile_rows = [&](int kt) -> int {
    const int64_t t0 = r0 + (int64_t)kt * kUpdTile;
    return (int)((r1 - t0) < (int64_t)kUpdTile ? (r1 - t0) : (int64_t)kUpdTile);
  };
  auto col_ptr = [&](int c) -> const double* {
    return c == 0 ? vtc : (c == 1 ? a.w : a.V + (int64_t)(c - 2) * a.ldv);
  };
  float qs = 0.f, qc = 0.f;  // sum of squares of the double-FP32 rows
  double q64 = 0.0;          // ... of the FP64 rows
  if (warp == kGramTmaConsumers) {
    {  // producer warp
      const bool ok = ring_produce(
          g, nitems, [&](int k) { const int cb = (k % nchunks) * kUpdChunk; return min(ncols, cb + kUpdChunk) - cb; },
          [&](int k) { return tile_rows(k / nchunks); },
          [&](int k, int q, const double** src, int* off) {
            const int c = (k % nchunks) * kUpdChunk + q;
            *src = col_ptr(c) + r0 + (int64_t)(k / nchunks) * kUpdTile;
            *off = q * kUpdTile;
          },
          &s_abort);
      if (!ok && lane == 0) s_abort = 1;
    }
  } else {
    const int t = threadIdx.x;  // the row of each tile this thread owns
    for (int kt = 0; kt < ntiles; ++kt) {
      const int tn = tile_rows(kt), te = tn & ~1;
      const int64_t row = r0 + (int64_t)kt * kUpdTile + t;
      UpdRow u;
#pragma unroll
      for (int p = 0; p < 4; ++p) u.s[p] = u.c[p] = 0.f;
      u.v = u.wb = 0.0;
      u.mvr = 0u;
      u.ok = hok;
      bool aborted = false;
      for (int kc = 0; kc < nchunks; ++kc) {
        const int k = kt * nchunks + kc;
        if (!ring_acquire(g, k)) {
          aborted = true;
          break;
        }
        const int cb = kc * kUpdChunk, ce = min(ncols, cb + kUpdChunk);
        const double* sb = g.buf(k);
        if (t < te)
          upd_columns<CHECK_V>(u, cb, ce, invb, s_hs, i, [&](int c) { return sb[(c - cb) * kUpdTile + t]; });
        else if (t < tn)
          upd_columns<CHECK_V>(u, cb, ce, invb, s_hs, i, [&](int c) { return col_ptr(c)[row]; });
        ring_release(g, k);
      }
      if (aborted) {
        s_abort = 1;
        break;
      }
      if (t < tn) {
        vi[row] = u.v;
        double acc = 0.0;
        bool ok = u.ok && (!CHECK_V || df_window(u.mvr));
        if (ok) {
          float s0 = u.s[0], c0 = u.c[0], s2 = u.s[2], c2 = u.c[2];
          df_add(s0, c0, u.s[1], u.c[1]);
          df_add(s2, c2, u.s[3], u.c[3]);
          df_add(s0, c0, s2, c2);
          acc = widen_normal(s0) + widen_normal(c0);
          const float tt = __fadd_rn(s0, c0);
          const float z = __fsub_rn(tt, s0);
          const float e = __fadd_rn(__fsub_rn(s0, __fsub_rn(tt, z)), __fsub_rn(c0, z));
          if (a.v32) a.v32[row] = tt;
          dot2_step(qs, qc, tt, e, tt, e);
        } else {
          acc = fma(-s_h[i], u.v, u.wb);
          for (int j = 0; j < i; ++j) acc = fma(-s_h[j], a.V[(int64_t)j * a.ldv + row], acc);
          if (a.v32) a.v32[row] = narrow_f64(acc);
          q64 = fma(acc, acc, q64);
        }
        vn[row] = acc;
      }
    }
  }
  // block sum of the squares (consumers): double-FP32 part per warp, FP64 part only if a row needed it
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
  double wsum = widen_normal(qs) + widen_normal(qc);
  if (__syncthreads_or(q64 != 0.0)) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q64 += __shfl_xor_sync(0xffffffffu, q64, o);
    wsum += q64;
  }
  if (lane == 0 && warp < kGramTmaConsumers) s_red[warp] = wsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < kGramTmaConsumers; ++w) tot += s_red[w];
    a.scr.partials[blockIdx.x] = s_abort ? __longlong_as_double(0x7ff8000000000000ll) : tot;
    if (s_abort && st) st->status = NSAMG_ERR_TIMEOUT;
  }
  if (!last_block(a.scr.ticket)) return;
  update_tail(a, i);
}


// ------------------------------------------------------------------------------------------
// Split basis (the solve's layout when krylov_fp64 = 0). Column j of the Krylov basis holds vt_j,
// the unnormalised vector of step j, as (hi, lo) float pairs (split_df; 8 bytes per entry, as in
// FP64), so the Gram and update read FP32 operands with no per-read split. The normalisation
// v_j = vt_j / beta_j is folded into the coefficients. Column 0 is the true residual scaled by an
// exact power of two to unit order (k_col0) so that every stored vector lies well inside the FP32
// range (later columns inherit unit order from the normalised Arnoldi process); the scale goes
// into g_0, the right-hand side of the least-squares problem.
//
// Row-pair layout: rows 2g and 2g + 1 of a column share the 16-byte group g, stored as
// (hi_2g, hi_2g+1, lo_2g, lo_2g+1). One 16-byte load then gives the hi parts and the lo parts of
// two rows as the two lanes of packed FP32 pairs (below), which the Gram and update feed straight
// into packed instructions, one row per lane. A column's bytes for rows [2g0, 2g1) are contiguous
// as in a plain layout. When n is odd, the second lane of the last group (row n) is zero.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float2 split2(double x) {
  float h, l;
  split_df(x, h, l);
  return make_float2(h, l);
}

// FP64 value of a stored pair (widened by integer operations, one FP64 add)
__device__ __forceinline__ double join2(float2 p) { return widen_normal(p.x) + widen_normal(p.y); }

// (hi, lo) of row r of a row-pair column
__device__ __forceinline__ float2 rp_get(const float2* col, int64_t r) {
  const float* f = reinterpret_cast<const float*>(col) + 4 * (r >> 1) + (r & 1);
  return make_float2(f[0], f[2]);
}
__device__ __forceinline__ void rp_set(float2* col, int64_t r, float2 v) {
  float* f = reinterpret_cast<float*>(col) + 4 * (r >> 1) + (r & 1);
  f[0] = v.x;
  f[2] = v.y;
}
// the group of rows (2g, 2g + 1) from their pairs
__device__ __forceinline__ float4 rp_group(float2 a, float2 b) { return make_float4(a.x, b.x, a.y, b.y); }

struct Col0Args {
  int64_t n;
  double* r;      // the FP64 residual (k_resid's output); scaled in place
  float* r32;     // if set: FP32 copy of the scaled residual (FP32 V-cycle input)
  float2* col;    // basis column 0 (row-pair layout)
  GState* st;
};

// Column 0 of a cycle: s = 2^-e with ||r|| = f 2^e, f in [0.5, 1); r <- s r (exact), column 0 =
// split(r), r0_scale = 2^e. One thread per row pair.
__global__ void __launch_bounds__(kRedThreads) k_col0(Col0Args a) {
  pdl_enter();
  GState* st = a.st;
  if (st->stop) return;
  const double rn = st->rnorm;
  int e = 0;
  if (rn > 0.0 && isfinite(rn)) frexp(rn, &e);
  const double sc = ldexp(1.0, -e);
  if (blockIdx.x == 0 && threadIdx.x == 0) st->r0_scale = ldexp(1.0, e);
  float4* col = reinterpret_cast<float4*>(a.col);
  const int64_t ng = (a.n + 1) >> 1;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = 2 * g;
    const bool two = r + 1 < a.n;
    const double x0 = a.r[r] * sc;
    const double x1 = two ? a.r[r + 1] * sc : 0.0;
    a.r[r] = x0;
    if (two) a.r[r + 1] = x1;
    col[g] = rp_group(split2(x0), split2(x1));
    if (a.r32) {
      a.r32[r] = narrow_f64(x0);
      if (two) a.r32[r + 1] = narrow_f64(x1);
    }
  }
}

// Standalone conversion of FP64 columns into split row-pair columns (column j of V -> column j of
// Vs; the second lane of the last group is zero when n is odd).
__global__ void __launch_bounds__(kRedThreads) k_split_cols(int64_t n, int ncols, const double* __restrict__ V,
                                                            int64_t ldv, float2* __restrict__ Vs, int64_t lds) {
  pdl_enter();
  const int64_t ng = (n + 1) >> 1;
  for (int j = 0; j < ncols; ++j) {
    const double* v = V + (int64_t)j * ldv;
    float4* col = reinterpret_cast<float4*>(Vs + (int64_t)j * lds);
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
      const int64_t r = 2 * g;
      col[g] = rp_group(split2(v[r]), split2(r + 1 < n ? v[r + 1] : 0.0));
    }
  }
}

// Packed FP32 pairs (the f32x2 instructions of sm_100 and later): one instruction applies the
// operation, correctly rounded, to both 32-bit lanes of a 64-bit register pair, so each lane's
// result is bitwise that of the scalar instruction. Low lane = first argument of f2_pack.
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t f2_pack(float lo, float hi) {
  f2_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(f2_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b) {
  f2_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b) {
  f2_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b) {
  f2_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
  f2_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// 16-byte shared-memory loads: a row-pair group as two packed pairs (hi lanes, lo lanes), and two
// FP64 values
__device__ __forceinline__ void lds_group(unsigned addr, f2_t& hi, f2_t& lo) {
  asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(hi), "=l"(lo) : "r"(addr));
}
__device__ __forceinline__ void lds_d2(unsigned addr, double& x0, double& x1) {
  asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(x0), "=d"(x1) : "r"(addr));
}

// dot2_step in both lanes: (s, c) += (xh + xl)(bh + bl), with nbh = -bh. The product is formed
// negated (exact), which turns TwoSum's p terms into subtractions; every lane's sequence of
// rounded operations is that of dot2_step, so the results are bitwise the same.
__device__ __forceinline__ void dot2_step2(f2_t& s, f2_t& c, f2_t xh, f2_t xl, f2_t bh, f2_t bl, f2_t nbh) {
  const f2_t np = f2_mul(xh, nbh);  // -p
  f2_t e = f2_fma(xh, bh, np);       // xh bh - p, exact
  e = f2_fma(xh, bl, e);
  e = f2_fma(xl, bh, e);
  const f2_t t = f2_sub(s, np);  // s + p
  const f2_t z = f2_sub(t, s);
  const f2_t err = f2_sub(f2_sub(s, f2_sub(t, z)), f2_add(np, z));  // (s - (t - z)) + (p - z)
  s = t;
  c = f2_add(c, f2_add(err, e));
}

// df_add in both lanes: (s, c) += (s2, c2)
__device__ __forceinline__ void df_add2(f2_t& s, f2_t& c, f2_t s2, f2_t c2) {
  const f2_t t = f2_add(s, s2);
  const f2_t z = f2_sub(t, s);
  const f2_t err = f2_add(f2_sub(s, f2_sub(t, z)), f2_sub(s2, z));
  s = t;
  c = f2_add(c, f2_add(c2, err));
}

// Columns per warp in k_gram_s: its packed (sum, error) accumulators take 8 registers a column,
// and a 17-warp block leaves at most 96 registers a thread; fewer columns a warp also give each
// warp more row pairs of a tile (measured best at 4).
constexpr int kGramSSlots = 4;

// Consumer warp of k_gram_s: every tile of the block's chunk, row pairs dealt to the R row-group
// warps in groups of 32 pairs (round robin), times the warp's NS columns cg + sl C (only the last
// slot can pass the last column; its discarded products then read column nv - 1), against column
// i (the stage's column nv - 1) and w (FP64 at stage column nv, split here). Each thread works on
// a row pair with packed instructions, one row per lane, and keeps (sum, error) pairs per lane;
// the two lanes are added at the end. The tile loop sits inside the slot-count specialisation so
// the accumulators keep their registers from tile to tile. Returns false if a wait gave up.
template <int NS, class RG>
__device__ __forceinline__ bool gram_consume_s(const RG& g, const float2* __restrict__ Vs, const double* __restrict__ w,
                                               int64_t ldv, int nv, int T, int C, int cg, int rg, int R, int64_t r0,
                                               int64_t r1, int ntiles, float (&sa)[kGramSSlots],
                                               float (&ca)[kGramSSlots], float (&sw)[kGramSSlots],
                                               float (&cw)[kGramSSlots], unsigned& mx) {
  const int lane = threadIdx.x & 31;
  f2_t s_a[NS], c_a[NS], s_w[NS], c_w[NS];
  unsigned offb[NS];  // byte offset of each slot's column in a stage
#pragma unroll
  for (int sl = 0; sl < NS; ++sl) {
    s_a[sl] = c_a[sl] = s_w[sl] = c_w[sl] = 0ull;
    offb[sl] = 8u * (unsigned)(min(cg + sl * C, nv - 1) * T);
  }
  const unsigned offv = 8u * (unsigned)((nv - 1) * T), offw = 8u * (unsigned)(nv * T);
  const f2_t m1 = f2_pack(-1.f, -1.f);
  const int step = 32 * R;
  bool ok = true;
  int64_t t0 = r0;
  for (int k = 0; k < ntiles; ++k, t0 += T) {
    if (!ring_acquire(g, k)) {
      ok = false;
      break;
    }
    const int tn = (int)min((int64_t)T, r1 - t0), te = tn & ~1;
    const unsigned base = smem_u32(g.buf(k));
    for (int pr = rg * 32 + lane; pr < (te >> 1); pr += step) {
      const unsigned rb = base + 16u * (unsigned)pr;
      f2_t qh, ql;
      lds_group(rb + offv, qh, ql);
      double w0, w1;
      lds_d2(rb + offw, w0, w1);
      mx = max(mx, max(abs_hiword(w0), abs_hiword(w1)));
      float wh0, wl0, wh1, wl1;
      split_df(w0, wh0, wl0);
      split_df(w1, wh1, wl1);
      const f2_t wh = f2_pack(wh0, wh1), wl = f2_pack(wl0, wl1);
      const f2_t nqh = f2_mul(qh, m1), nwh = f2_mul(wh, m1);
      f2_t xh[NS], xl[NS];
#pragma unroll
      for (int sl = 0; sl < NS; ++sl) lds_group(rb + offb[sl], xh[sl], xl[sl]);
#pragma unroll
      for (int sl = 0; sl < NS; ++sl) {
        dot2_step2(s_a[sl], c_a[sl], xh[sl], xl[sl], qh, ql, nqh);
        dot2_step2(s_w[sl], c_w[sl], xh[sl], xl[sl], wh, wl, nwh);
      }
    }
    if (te < tn && ((te >> 1) >> 5) % R == rg && lane == 0) {  // the odd last row (its pair group's warp)
      const int64_t row = t0 + te;
      const float2 q = rp_get(Vs + (int64_t)(nv - 1) * ldv, row);
      const double xw = w[row];
      mx = max(mx, abs_hiword(xw));
      float q2, q3;
      split_df(xw, q2, q3);
      const f2_t qh = f2_pack(q.x, 0.f), ql = f2_pack(q.y, 0.f), nqh = f2_pack(-q.x, 0.f);
      const f2_t wh = f2_pack(q2, 0.f), wl = f2_pack(q3, 0.f), nwh = f2_pack(-q2, 0.f);
#pragma unroll
      for (int sl = 0; sl < NS; ++sl) {
        const float2 x = rp_get(Vs + (int64_t)min(cg + sl * C, nv - 1) * ldv, row);
        const f2_t xh = f2_pack(x.x, 0.f), xl = f2_pack(x.y, 0.f);
        dot2_step2(s_a[sl], c_a[sl], xh, xl, qh, ql, nqh);
        dot2_step2(s_w[sl], c_w[sl], xh, xl, wh, wl, nwh);
      }
    }
    ring_release(g, k);
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
  return ok;
}

// The streaming part of k_gram_s with an NST-stage ring: tiles of T rows (the largest multiple of
// 32 for which a stage holds columns 0..i and w, at most 2048), the block's row range [r0, r1),
// the producer warp and the consumer warps' products. Few columns stream best through three
// stages; many columns (short tiles) through two larger ones.
constexpr int kGramTwoStageCols = 30;
// The Gram's ring: nearly all of the block's shared memory (divisible into 16-byte aligned stages
// for 2, 3 and 4 stages); kGramStagesSmall stages below kGramTwoStageCols columns.
constexpr int kGramRingBytes = 227328;
constexpr int kGramSSmem = kGramRingBytes + 2 * 4 * 8;
static_assert(kGramRingBytes >= kGramWarps * 2 * (kMaxM + 1) * 8, "the partials fit in the ring");
constexpr int kGramStagesSmall = 3;

template <int NST>
__device__ __forceinline__ void gram_s_stream(const GramArgs& a, unsigned char* dsm, int nv, int C, int cg, int rg,
                                              int R, int S, int& T_out, int64_t& r0_out, int64_t& r1_out,
                                              float (&sa)[kGramSSlots], float (&ca)[kGramSSlots],
                                              float (&sw)[kGramSSlots], float (&cw)[kGramSSlots], unsigned& mx,
                                              unsigned* s_max,
                                              volatile int* s_abort) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  using RG = RingT<NST, kGramRingBytes>;
  const int T = min(2048, RG::kStageBytes / (8 * (nv + 1)) / 32 * 32);
  const int64_t chunk = ((a.n + gridDim.x - 1) / gridDim.x + T - 1) / T * T;
  const int64_t r0 = (int64_t)blockIdx.x * chunk;
  const int64_t r1 = min(a.n, r0 + chunk);
  T_out = T;
  r0_out = r0;
  r1_out = r1;
  const int ntiles = r1 > r0 ? (int)((r1 - r0 + T - 1) / T) : 0;
  const float2* Vs = a.Vs;
  const RG g = ring_init_t<NST, kGramRingBytes>(dsm);
  if (threadIdx.x == 0) {
    *s_max = 0u;
    *s_abort = 0;
  }
  __syncthreads();
  auto tile_rows = [&](int k) -> int {
    const int64_t t0 = r0 + (int64_t)k * T;
    return (int)((r1 - t0) < (int64_t)T ? (r1 - t0) : (int64_t)T);
  };
  if (warp == kGramTmaConsumers) {
    {  // producer warp: per tile the columns 0..i and w
      const bool ok = ring_produce(
          g, ntiles, [&](int) { return nv + 1; }, tile_rows,
          [&](int k, int q, const double** src, int* off) {
            const int64_t t0 = r0 + (int64_t)k * T;
            *src = q < nv ? reinterpret_cast<const double*>(Vs + (int64_t)q * a.ldv + t0) : a.w + t0;
            *off = q * T;
          },
          s_abort);
      if (!ok && lane == 0) *s_abort = 1;
    }
  } else {
    bool ok = true;
    switch (S) {
#define NSAMG_GRAM_CONSUME_S(NS)                                                                         \
  case NS:                                                                                               \
    ok = gram_consume_s<NS>(g, Vs, a.w, a.ldv, nv, T, C, cg, rg, R, r0, r1, ntiles, sa, ca, sw, cw, mx); \
    break;
      NSAMG_GRAM_CONSUME_S(1)
      NSAMG_GRAM_CONSUME_S(2)
      NSAMG_GRAM_CONSUME_S(3)
      NSAMG_GRAM_CONSUME_S(4)
#undef NSAMG_GRAM_CONSUME_S
      default: break;
    }
    if (!ok) *s_abort = 1;
  }
}

// Gram on the split basis with the bulk-copy ring: a_j = vt_j . vt_i and s_j = vt_j . w for
// j = 0..i, all in double-FP32 (column i included), per block and then in FP64 across blocks
// (fixed order); the finalise scales a_j, s_j (j < i) by 1 / beta_j. Each tile: columns 0..i of
// the basis and w. A block whose w leaves the double-FP32 window recomputes its chunk in FP64
// from the stored pairs. Aligned operands required (the solve allocates them so).
__global__ void __launch_bounds__(kGramTmaThreads, 1) k_gram_s(GramArgs a) {
  pdl_enter();
  extern __shared__ __align__(128) unsigned char dsm[];
  // the per-warp partials reuse the ring's stage memory once the stream has drained
  double (*s_part)[2 * (kMaxM + 1)] = reinterpret_cast<double (*)[2 * (kMaxM + 1)]>(dsm);
  __shared__ unsigned s_max;
  __shared__ volatile int s_abort;
  GState* st = a.st;
  if (st && st->stop) return;
  const int i = st ? st->i : a.i_standalone;
  const int nv = i + 1;  // columns 0..i
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int C = df_groups(nv, kGramSSlots);
  const int R = kGramWarps / C;
  const int S = (nv + C - 1) / C;
  float sa[kGramSSlots], ca[kGramSSlots], sw[kGramSSlots], cw[kGramSSlots];
#pragma unroll
  for (int sl = 0; sl < kGramSSlots; ++sl) sa[sl] = ca[sl] = sw[sl] = cw[sl] = 0.f;
  unsigned mx = 0u;
  const int cg = warp % C, rg = warp / C;
  int T;
  int64_t r0, r1;
  const float2* Vs = a.Vs;
  if (nv < kGramTwoStageCols)
    gram_s_stream<kGramStagesSmall>(a, dsm, nv, C, cg, rg, R, S, T, r0, r1, sa, ca, sw, cw, mx, &s_max, &s_abort);
  else
    gram_s_stream<2>(a, dsm, nv, C, cg, rg, R, S, T, r0, r1, sa, ca, sw, cw, mx, &s_max, &s_abort);
  if (warp < kGramTmaConsumers) {
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) atomicMax(&s_max, mx);
  }
  __syncthreads();
  const bool abort = s_abort != 0;
  const bool fp64 = !abort && !df_window(s_max);
  if (warp < kGramTmaConsumers) {
    if (!fp64) {
      float as[16], ac[16];
#pragma unroll
      for (int sl = 0; sl < kDfSlots; ++sl) {
        as[2 * sl] = sl < kGramSSlots ? sa[sl < kGramSSlots ? sl : 0] : 0.f;
        ac[2 * sl] = sl < kGramSSlots ? ca[sl < kGramSSlots ? sl : 0] : 0.f;
        as[2 * sl + 1] = sl < kGramSSlots ? sw[sl < kGramSSlots ? sl : 0] : 0.f;
        ac[2 * sl + 1] = sl < kGramSSlots ? cw[sl < kGramSSlots ? sl : 0] : 0.f;
      }
      df_warp_reduce16(as, ac);
      const int qd = lane >> 1, sl = qd >> 1, j = cg + sl * C;
      if ((lane & 1) == 0 && sl < S && j < nv)
        s_part[rg][(qd & 1) ? (kMaxM + 1 + j) : j] = widen_normal(as[0]) + widen_normal(ac[0]);
    } else {
      // FP64 recomputation of this block's chunk from the stored pairs (w outside the window)
      const float2* vi = Vs + (int64_t)i * a.ldv;
#pragma unroll 1
      for (int sl = 0; sl < S; ++sl) {
        const int j = cg + sl * C;
        double fa = 0.0, fw = 0.0;
        if (j < nv) {
          const float2* vj = Vs + (int64_t)j * a.ldv;
          for (int64_t t0 = r0; t0 < r1; t0 += T)
            for (int r = rg * 32 + lane; r < T && t0 + r < r1; r += 32 * R) {
              const double x = join2(rp_get(vj, t0 + r));
              fa = fma(x, join2(rp_get(vi, t0 + r)), fa);
              fw = fma(x, a.w[t0 + r], fw);
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
  }
  __syncthreads();
  const int stride = 2 * (kMaxM + 1);
  for (int v = threadIdx.x; v < 2 * (i + 1); v += blockDim.x) {
    const int col = v <= i ? v : (kMaxM + 1) + (v - i - 1);
    double sum = 0.0;
    for (int g2 = 0; g2 < R; ++g2) sum += s_part[g2][col];
    a.scr.partials[(int64_t)blockIdx.x * stride + col] = abort ? __longlong_as_double(0x7ff8000000000000ll) : sum;
  }
  if (abort && threadIdx.x == 0 && st) st->status = NSAMG_ERR_TIMEOUT;
  if (!last_block(a.scr.ticket)) return;
  gram_tail(a, i);
}

// ------------------------------------------------------------------------------------------
// Update on the split basis with the bulk-copy ring (one consumer thread per row pair of a
// 1024-row tile, columns streamed through three 64 KB stages in chunks of kUpdSChunk: w first,
// then vt_0 .. vt_i):
//   vt_{i+1} = w / beta_i - sum_{j<=i} (h_j / beta_j) vt_j,
// w / beta_i formed in FP64 (one multiply a row) and split, the sum in four (sum, error) pairs
// of packed instructions (one row per lane); the result is stored as a normalised row-pair group
// in column i+1 and, for the next V-cycle, as FP64 in vin or rounded to FP32 in v32.
// ||vt_{i+1}||^2 in double-FP32 per thread, FP64 across blocks. Row pairs in which w / beta_i
// leaves the double-FP32 window, and every row when the coefficients do, are computed in FP64
// from the stored pairs, as is the odd last row of an odd n.
// ------------------------------------------------------------------------------------------
constexpr int kUpdPairs = 32 * kGramTmaConsumers;                   // row pairs per tile (one per consumer)
constexpr int kUpdSTile = 2 * kUpdPairs;                            // rows per tile (1024)
constexpr int kUpdSStages = 3;                                      // three 64 KB stages
constexpr int kUpdSChunk = RingT<kUpdSStages>::kStageBytes / (8 * kUpdSTile);  // columns per stage (8)
constexpr unsigned kUpdColBytes = 8u * kUpdSTile;                   // bytes of one column in a stage
static_assert(kUpdSChunk == 8, "k_update_s dispatches chunk widths 1..8");

// Coefficient of basis column j in shared memory: the split (h, l) of -h_j / beta_j as the pairs
// (h, h), (l, l) and (-h, -h), each value in both lanes.
struct __align__(16) UpdCoef {
  float4 hl;  // (h, h, l, l)
  float4 nh;  // (-h, -h, 0, 0)
};

__device__ __forceinline__ f2_t lds_pair(unsigned addr) {
  f2_t v;
  asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(addr));
  return v;
}

// NW staged columns of a chunk for one row pair: column k at byte k * kUpdColBytes from addr,
// coefficient record cf + k, into pair accumulator (K0 + k) mod 4 (the global column's index
// mod 4, with column 0 = w).
template <int NW, int K0>
__device__ __forceinline__ void upd_cols_s(unsigned addr, unsigned cf, f2_t (&ps)[4], f2_t (&pc)[4]) {
  f2_t xh[NW], xl[NW];
#pragma unroll
  for (int k = 0; k < NW; ++k) lds_group(addr + (unsigned)k * kUpdColBytes, xh[k], xl[k]);
#pragma unroll
  for (int k = 0; k < NW; ++k) {
    f2_t hh, hl;
    lds_group(cf + 32u * k, hh, hl);
    const f2_t nh = lds_pair(cf + 32u * k + 16u);
    dot2_step2(ps[(K0 + k) & 3], pc[(K0 + k) & 3], xh[k], xl[k], hh, hl, nh);
  }
}

// FP64 recomputation of one row (outside the double-FP32 window, or the odd last row)
__device__ __forceinline__ double upd_row_fp64(const UpdateArgs& a, const double* __restrict__ s_c, int i, int64_t row,
                                               double wb, float2* vnext, double& q64) {
  double acc = wb;
  for (int j = 0; j <= i; ++j) acc = fma(-s_c[j], join2(rp_get(a.Vs + (int64_t)j * a.ldv, row)), acc);
  rp_set(vnext, row, split2(acc));
  if (a.v32) a.v32[row] = narrow_f64(acc);
  if (a.vin) a.vin[row] = acc;
  q64 = fma(acc, acc, q64);
  return acc;
}

__global__ void __launch_bounds__(kGramTmaThreads, 1) k_update_s(UpdateArgs a) {
  pdl_enter();
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ double s_c[kMaxM + 1];    // h_j / beta_j
  __shared__ UpdCoef s_cf[kMaxM + 1];  // -h_j / beta_j split, in both lanes
  __shared__ double s_red[kGramTmaConsumers];
  __shared__ unsigned s_cmax;
  __shared__ volatile int s_abort;
  GState* st = a.st;
  if (st && st->stop) {  // stopped earlier in this step (error in the Gram): end the inner loop
    if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(a.cond_inner, 0);
    return;
  }
  const int i = st ? st->i : a.i_standalone;
  const double invb = st ? st->invbeta[i] : a.invbeta_standalone;
  const RingT<kUpdSStages> g = ring_init_t<kUpdSStages>(dsm);
  if (threadIdx.x == 0) {
    s_cmax = 0u;
    s_abort = 0;
  }
  __syncthreads();
  for (int j = threadIdx.x; j <= i; j += blockDim.x) {
    const double cj = st ? st->h[j] * st->invbeta[j] : a.coef_standalone[j];
    s_c[j] = cj;
    const float2 h = split2(-cj);
    s_cf[j].hl = make_float4(h.x, h.x, h.y, h.y);
    s_cf[j].nh = make_float4(-h.x, -h.x, 0.f, 0.f);
    atomicMax(&s_cmax, abs_hiword(cj));
  }
  __syncthreads();
  const bool cok = df_window(s_cmax);
  const float2* Vs = a.Vs;
  float2* vnext = a.Vs + (int64_t)(i + 1) * a.ldv;
  const int ncols = i + 2, nchunks = (ncols + kUpdSChunk - 1) / kUpdSChunk;  // column 0: w, 1 + j: vt_j
  const int64_t chunk = ((a.n + gridDim.x - 1) / gridDim.x + kUpdSTile - 1) / kUpdSTile * kUpdSTile;
  const int64_t r0 = (int64_t)blockIdx.x * chunk;
  const int64_t r1 = min(a.n, r0 + chunk);
  const int ntiles = r1 > r0 ? (int)((r1 - r0 + kUpdSTile - 1) / kUpdSTile) : 0;
  const int nitems = ntiles * nchunks;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto tile_rows = [&](int kt) -> int {
    const int64_t t0 = r0 + (int64_t)kt * kUpdSTile;
    return (int)((r1 - t0) < (int64_t)kUpdSTile ? (r1 - t0) : (int64_t)kUpdSTile);
  };
  auto col_ptr = [&](int c) -> const double* {
    return c == 0 ? a.w : reinterpret_cast<const double*>(Vs + (int64_t)(c - 1) * a.ldv);
  };
  const bool vin16 = a.vin && (reinterpret_cast<uintptr_t>(a.vin) & 15u) == 0;
  f2_t qs2 = 0ull, qc2 = 0ull;
  double q64 = 0.0;
  if (warp == kGramTmaConsumers) {
    {  // producer warp
      const bool ok = ring_produce(
          g, nitems, [&](int k) { const int cb = (k % nchunks) * kUpdSChunk; return min(ncols, cb + kUpdSChunk) - cb; },
          [&](int k) { return tile_rows(k / nchunks); },
          [&](int k, int q, const double** src, int* off) {
            const int c = (k % nchunks) * kUpdSChunk + q;
            *src = col_ptr(c) + r0 + (int64_t)(k / nchunks) * kUpdSTile;
            *off = q * kUpdSTile;
          },
          &s_abort);
      if (!ok && lane == 0) s_abort = 1;
    }
  } else {
    const int t = threadIdx.x;
    const unsigned cf0 = smem_u32(s_cf);
    const f2_t m1 = f2_pack(-1.f, -1.f);
    bool aborted = false;
    for (int kt = 0; kt < ntiles && !aborted; ++kt) {
      const int tn = tile_rows(kt), te = tn & ~1;
      const int64_t row = r0 + (int64_t)kt * kUpdSTile + 2 * t;  // this thread's rows: row, row + 1
      const bool staged = 2 * t < te;
      f2_t ps[4] = {0ull, 0ull, 0ull, 0ull}, pc[4] = {0ull, 0ull, 0ull, 0ull};
      double wb0 = 0.0, wb1 = 0.0;
      for (int kc = 0; kc < nchunks; ++kc) {
        const int k = kt * nchunks + kc;
        if (!ring_acquire(g, k)) {
          aborted = true;
          break;
        }
        if (staged) {
          const int cb = kc * kUpdSChunk, ce = min(ncols, cb + kUpdSChunk);
          const unsigned addr = smem_u32(g.buf(k)) + 16u * (unsigned)t;
          if (kc == 0) {  // column 0 is w
            double w0, w1;
            lds_d2(addr, w0, w1);
            wb0 = w0 * invb;
            wb1 = w1 * invb;
            float h0, l0, h1, l1;
            split_df(wb0, h0, l0);
            split_df(wb1, h1, l1);
            ps[0] = f2_pack(h0, h1);
            pc[0] = f2_pack(l0, l1);
            switch (ce - 1) {
#define NSAMG_UPD_COLS0(NW) \
  case NW:                  \
    upd_cols_s<NW, 1>(addr + kUpdColBytes, cf0, ps, pc); \
    break;
              NSAMG_UPD_COLS0(1) NSAMG_UPD_COLS0(2) NSAMG_UPD_COLS0(3) NSAMG_UPD_COLS0(4)
              NSAMG_UPD_COLS0(5) NSAMG_UPD_COLS0(6) NSAMG_UPD_COLS0(7)
#undef NSAMG_UPD_COLS0
              default: break;
            }
          } else {
            const unsigned cf = cf0 + 32u * (unsigned)(cb - 1);
            switch (ce - cb) {
#define NSAMG_UPD_COLS(NW) \
  case NW:                 \
    upd_cols_s<NW, 0>(addr, cf, ps, pc); \
    break;
              NSAMG_UPD_COLS(1) NSAMG_UPD_COLS(2) NSAMG_UPD_COLS(3) NSAMG_UPD_COLS(4)
              NSAMG_UPD_COLS(5) NSAMG_UPD_COLS(6) NSAMG_UPD_COLS(7) NSAMG_UPD_COLS(8)
#undef NSAMG_UPD_COLS
              default: break;
            }
          }
        }
        ring_release(g, k);
      }
      if (aborted) break;
      if (staged) {
        if (cok && df_window(abs_hiword(wb0)) && df_window(abs_hiword(wb1))) {
          df_add2(ps[0], pc[0], ps[1], pc[1]);
          df_add2(ps[2], pc[2], ps[3], pc[3]);
          df_add2(ps[0], pc[0], ps[2], pc[2]);
          // normalised pairs (TwoSum): stored, squared and rounded for the FP32 copy
          const f2_t tt = f2_add(ps[0], pc[0]);
          const f2_t z = f2_sub(tt, ps[0]);
          const f2_t e = f2_add(f2_sub(ps[0], f2_sub(tt, z)), f2_sub(pc[0], z));
          asm volatile("st.global.v2.b64 [%0], {%1, %2};" ::"l"(vnext + row), "l"(tt), "l"(e) : "memory");
          float t0f, t1f, e0f, e1f;
          f2_unpack(tt, t0f, t1f);
          f2_unpack(e, e0f, e1f);
          const double acc0 = widen_normal(t0f) + widen_normal(e0f);
          const double acc1 = widen_normal(t1f) + widen_normal(e1f);
          if (a.v32) {
            a.v32[row] = t0f;
            a.v32[row + 1] = t1f;
          }
          if (vin16) {
            *reinterpret_cast<double2*>(a.vin + row) = make_double2(acc0, acc1);
          } else if (a.vin) {
            a.vin[row] = acc0;
            a.vin[row + 1] = acc1;
          }
          dot2_step2(qs2, qc2, tt, e, tt, e, f2_mul(tt, m1));
        } else {
          upd_row_fp64(a, s_c, i, row, wb0, vnext, q64);
          upd_row_fp64(a, s_c, i, row + 1, wb1, vnext, q64);
        }
      } else if (2 * t == te && te < tn) {  // the odd last row (n odd): FP64; its group's second lane stays 0
        upd_row_fp64(a, s_c, i, row, a.w[row] * invb, vnext, q64);
        rp_set(vnext, row + 1, make_float2(0.f, 0.f));
      }
    }
    if (aborted) s_abort = 1;
  }
  float qs, qc;
  {
    float q0, q1, c0, c1;
    f2_unpack(qs2, q0, q1);
    f2_unpack(qc2, c0, c1);
    df_add(q0, c0, q1, c1);
    qs = q0;
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
  double wsum = widen_normal(qs) + widen_normal(qc);
  if (__syncthreads_or(q64 != 0.0)) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q64 += __shfl_xor_sync(0xffffffffu, q64, o);
    wsum += q64;
  }
  if (lane == 0 && warp < kGramTmaConsumers) s_red[warp] = wsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w2 = 0; w2 < kGramTmaConsumers; ++w2) tot += s_red[w2];
    a.scr.partials[blockIdx.x] = s_abort ? __longlong_as_double(0x7ff8000000000000ll) : tot;
    if (s_abort && st) st->status = NSAMG_ERR_TIMEOUT;
  }
  if (!last_block(a.scr.ticket)) return;
  update_tail(a, i);
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
  double* r;           // V[:, 0] (FP64 basis) or the FP64 residual vector (split basis)
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
    st->xnorm = sqrt(X2);
    st->rnorm = sqrt(R2);
    const bool finite = isfinite(R2) && isfinite(st->bnorm);
    const bool conv = finite && (st->stop_nrbe ? st->nrbe <= st->rtol : relres <= st->rtol);
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
