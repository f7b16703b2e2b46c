/* Plain C client of the nsamg C ABI: builds a small 2D Poisson hierarchy by hand (two levels,
 * piecewise-constant aggregation of 2x2 blocks as P, R = P^T, Galerkin A_c = R A P, dense
 * coarse inverse), solves A x = b through nsamg_solve_host and checks the residual itself.
 * Exit code 0 on success. Build: gcc abi_smoke.c -I include -L <lib dir> -lnsamg -lm */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "nsamg.h"

#define NX 16
#define N (NX * NX)
#define NC ((NX / 2) * (NX / 2))

static int rp[N + 1], ci[5 * N];
static double va[5 * N];
static int prp[N + 1], pci[N];
static double pv[N];
static int rrp[NC + 1], rci[N];
static double rv[N];
static int crp[NC + 1], cci[NC * NC];
static double cv[NC * NC];
static double Ac[NC * NC], Cinv[NC * NC];

static int invert(double* a, double* inv, int n) { /* Gauss-Jordan with partial pivoting */
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) inv[i * n + j] = (i == j);
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(a[r * n + c]) > fabs(a[p * n + c])) p = r;
    if (a[p * n + c] == 0.0) return -1;
    for (int j = 0; j < n; ++j) {
      double t = a[c * n + j]; a[c * n + j] = a[p * n + j]; a[p * n + j] = t;
      t = inv[c * n + j]; inv[c * n + j] = inv[p * n + j]; inv[p * n + j] = t;
    }
    const double d = a[c * n + c];
    for (int j = 0; j < n; ++j) { a[c * n + j] /= d; inv[c * n + j] /= d; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = a[r * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) { a[r * n + j] -= f * a[c * n + j]; inv[r * n + j] -= f * inv[c * n + j]; }
    }
  }
  return 0;
}

int main(void) {
  int nnz = 0;
  for (int y = 0; y < NX; ++y)
    for (int x = 0; x < NX; ++x) {
      const int i = x + NX * y;
      rp[i] = nnz;
      if (y > 0) { ci[nnz] = i - NX; va[nnz++] = -1.0; }
      if (x > 0) { ci[nnz] = i - 1; va[nnz++] = -1.0; }
      ci[nnz] = i; va[nnz++] = 4.0;
      if (x < NX - 1) { ci[nnz] = i + 1; va[nnz++] = -1.0; }
      if (y < NX - 1) { ci[nnz] = i + NX; va[nnz++] = -1.0; }
    }
  rp[N] = nnz;
  /* P: each fine node maps to its 2x2 aggregate */
  for (int i = 0; i < N; ++i) {
    const int x = i % NX, y = i / NX;
    prp[i] = i;
    pci[i] = (x / 2) + (NX / 2) * (y / 2);
    pv[i] = 1.0;
  }
  prp[N] = N;
  /* R = P^T */
  int cnt[NC];
  memset(cnt, 0, sizeof(cnt));
  for (int i = 0; i < N; ++i) cnt[pci[i]]++;
  rrp[0] = 0;
  for (int c = 0; c < NC; ++c) rrp[c + 1] = rrp[c] + cnt[c];
  int fillp[NC];
  memcpy(fillp, rrp, sizeof(fillp));
  for (int i = 0; i < N; ++i) { const int c = pci[i]; rci[fillp[c]] = i; rv[fillp[c]++] = 1.0; }
  /* A_c = R A P (dense, small) */
  memset(Ac, 0, sizeof(Ac));
  for (int i = 0; i < N; ++i)
    for (int p = rp[i]; p < rp[i + 1]; ++p) Ac[pci[i] * NC + pci[ci[p]]] += va[p];
  int cn = 0;
  for (int r = 0; r < NC; ++r) {
    crp[r] = cn;
    for (int c = 0; c < NC; ++c)
      if (Ac[r * NC + c] != 0.0) { cci[cn] = c; cv[cn++] = Ac[r * NC + c]; }
  }
  crp[NC] = cn;
  double tmp[NC * NC];
  memcpy(tmp, Ac, sizeof(tmp));
  if (invert(tmp, Cinv, NC)) { fprintf(stderr, "singular coarse matrix\n"); return 2; }

  nsamg_level_desc lv[2];
  memset(lv, 0, sizeof(lv));
  lv[0].A = (nsamg_csr){N, N, nnz, rp, ci, va};
  lv[0].P = (nsamg_csr){N, NC, N, prp, pci, pv};
  lv[0].R = (nsamg_csr){NC, N, N, rrp, rci, rv};
  lv[1].A = (nsamg_csr){NC, NC, cn, crp, cci, cv};
  nsamg_hierarchy_desc H = {2, lv, Cinv};
  nsamg_params p;
  nsamg_default_params(&p);
  nsamg_handle* h = NULL;
  int rc = nsamg_setup_hierarchy(&H, &p, NULL, &h);
  if (rc != NSAMG_OK) { fprintf(stderr, "setup: %s (%s)\n", nsamg_status_str(rc), nsamg_last_error()); return 3; }
  double b[N], x[N];
  for (int i = 0; i < N; ++i) { b[i] = sin(0.1 * i) + 0.5; x[i] = 0.0; }
  nsamg_stats st;
  rc = nsamg_solve_host(h, b, x, 1e-10, 200, &st);
  if (rc != NSAMG_OK) { fprintf(stderr, "solve: %s (%s)\n", nsamg_status_str(rc), nsamg_last_error()); return 4; }
  double rn = 0.0, bn = 0.0;
  for (int i = 0; i < N; ++i) {
    double ax = 0.0;
    for (int q = rp[i]; q < rp[i + 1]; ++q) ax += va[q] * x[ci[q]];
    rn += (b[i] - ax) * (b[i] - ax);
    bn += b[i] * b[i];
  }
  const double rel = sqrt(rn / bn);
  printf("iters=%d restarts=%d relres=%.3e reported=%.3e nrbe=%.3e\n", st.iters, st.restarts, rel, st.relres_true, st.nrbe);
  /* an invalid argument is reported, not crashed on */
  if (nsamg_solve_host(h, NULL, x, 1e-8, 10, &st) != NSAMG_ERR_INVALID_ARG) return 5;
  nsamg_destroy(h);
  return (rel <= 1e-10 && st.converged) ? 0 : 6;
}
