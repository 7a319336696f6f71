/*
 * Oracle for the batched Hines solver -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, serial, obviously-correct FP64 CPU code.  It shares nothing with the
 * CUDA path (no headers, helpers or tables) and is only ever called by the
 * tests, by __graft_entry__.smoke() and by the CPU-baseline leg of bench.py.
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no FMA contraction,
 * so every product and sum is rounded exactly as written).
 *
 * Matrix convention (Section 2 of the paper): one cell is an N x N symmetric
 * matrix A with A[i][i] = d[i] and A[i][p[i]] = A[p[i]][i] = u[i] for i > 0;
 * p[0] = -1 and 0 <= p[i] < i (Hines numbering).  u[0] is ignored.
 * Listing 2 of the paper indexes the coupling by the parent in its
 * elimination sweep but by the row itself in its substitution sweep; on a tree
 * a parent compartment has several children, so only the per-child coupling
 * u[i] = A[i][p[i]] is well defined, and both sweeps use it here (the same
 * holds for Listing 1 with p[i] = i-1).
 *
 * Batches: cells are concatenated; off[c] .. off[c+1] is cell c and parent
 * indices are cell-local.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_BAD_SIZE (-1)
#define ORACLE_NOT_HINES (-2)
#define ORACLE_NOMEM (-3)

/* p[0] == -1 and 0 <= p[i] < i (the numbering Section 2 requires). */
int oracle_check_parent(int64_t n, const int32_t *p) {
  if (n < 0) return ORACLE_BAD_SIZE;
  if (n == 0) return ORACLE_OK;
  if (p[0] != -1) return ORACLE_NOT_HINES;
  for (int64_t i = 1; i < n; ++i)
    if (p[i] < 0 || (int64_t)p[i] >= i) return ORACLE_NOT_HINES;
  return ORACLE_OK;
}

/* Section 2: the tridiagonal case (Listing 1's Thomas algorithm), u[i] =
 * A[i][i-1].  Gaussian elimination from the last row up: row i is the only
 * row below row i-1 that still couples to it, so subtracting the multiple
 * l = A[i-1][i] / A[i][i] of row i from row i-1 clears that coupling and
 * changes only row i-1's diagonal and right-hand side.  What is left is lower
 * bidiagonal and is solved from the first row down.  In place: d becomes the
 * eliminated diagonal, b the solution. */
void oracle_thomas(int64_t n, double *d, const double *u, double *b) {
  if (n <= 0) return;
  for (int64_t row = n - 1; row > 0; --row) {
    const double l = u[row] / d[row];
    d[row - 1] -= l * u[row];
    b[row - 1] -= l * b[row];
  }
  for (int64_t row = 0; row < n; ++row) {
    const double known = row == 0 ? 0.0 : u[row] * b[row - 1];
    b[row] = (b[row] - known) / d[row];
  }
}

/* Section 2: the tree case (the Hines algorithm, Listing 2 with reading C1:
 * the coupling of row i to its parent is u[i] in both sweeps).  Because every
 * parent is numbered before its children, the rows can be eliminated from the
 * last to the first exactly as above, each row into its parent row p[i]
 * instead of row i-1: when row i is reached, all of its children are already
 * folded into it, and its one remaining off-diagonal entry is the coupling to
 * the parent.  The remaining system has one entry per row left of the
 * diagonal, to the parent, whose unknown is known once the rows are solved
 * from the root outwards.  In place: d becomes the eliminated diagonal, b the
 * solution x. */
int oracle_hines(int64_t n, const int32_t *p, double *d, const double *u, double *b) {
  int rc = oracle_check_parent(n, p);
  if (rc != ORACLE_OK || n == 0) return rc;
  for (int64_t row = n - 1; row > 0; --row) {
    const int64_t par = p[row];
    const double l = u[row] / d[row];
    d[par] -= l * u[row];
    b[par] -= l * b[row];
  }
  for (int64_t row = 0; row < n; ++row) {
    const double known = row == 0 ? 0.0 : u[row] * b[p[row]];
    b[row] = (b[row] - known) / d[row];
  }
  return ORACLE_OK;
}

/* y = A x for one cell (plain definition of the Hines matrix). */
void oracle_matvec(int64_t n, const int32_t *p, const double *d, const double *u, const double *x, double *y) {
  for (int64_t i = 0; i < n; ++i) y[i] = d[i] * x[i];
  for (int64_t i = 1; i < n; ++i) {
    y[i] = y[i] + u[i] * x[p[i]];
    y[p[i]] = y[p[i]] + u[i] * x[i];
  }
}

static int clamp_threads(int nthreads) { return nthreads < 1 ? 1 : nthreads; }

/* x = A^{-1} b for every cell of a batch; d and b are not modified. */
int oracle_solve_batch(int32_t n_cells, const int64_t *off, const int32_t *p, const double *d, const double *u,
                       const double *b, double *x, int nthreads) {
  int status = ORACLE_OK;
#pragma omp parallel for schedule(dynamic, 1) num_threads(clamp_threads(nthreads))
  for (int32_t c = 0; c < n_cells; ++c) {
    int64_t lo = off[c], n = off[c + 1] - off[c];
    double *dd = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!dd) {
#pragma omp atomic write
      status = ORACLE_NOMEM;
      continue;
    }
    memcpy(dd, d + lo, sizeof(double) * (size_t)n);
    memcpy(x + lo, b + lo, sizeof(double) * (size_t)n);
    int rc = oracle_hines(n, p + lo, dd, u + lo, x + lo);
    if (rc != ORACLE_OK) {
#pragma omp atomic write
      status = rc;
    }
    free(dd);
  }
  return status;
}

/* y = A x for every cell of a batch. */
void oracle_matvec_batch(int32_t n_cells, const int64_t *off, const int32_t *p, const double *d, const double *u,
                         const double *x, double *y) {
  for (int32_t c = 0; c < n_cells; ++c) {
    int64_t lo = off[c];
    oracle_matvec(off[c + 1] - lo, p + lo, d + lo, u + lo, x + lo, y + lo);
  }
}

/* Per-cell Skeel condition number cond(A, x) = || |A^{-1}| |A| |x| ||_inf / ||x||_inf.
 * With u <= 0 the matrix is an M-matrix, A^{-1} >= 0 elementwise, so the
 * numerator is one more solve with right-hand side |A| |x|. */
int oracle_skeel_batch(int32_t n_cells, const int64_t *off, const int32_t *p, const double *d, const double *u,
                       const double *x, double *cond, int nthreads) {
  int status = ORACLE_OK;
#pragma omp parallel for schedule(dynamic, 1) num_threads(clamp_threads(nthreads))
  for (int32_t c = 0; c < n_cells; ++c) {
    int64_t lo = off[c], n = off[c + 1] - off[c];
    if (n == 0) { cond[c] = 0.0; continue; }
    double *dd = (double *)malloc(sizeof(double) * (size_t)n);
    double *y = (double *)malloc(sizeof(double) * (size_t)n);
    if (!dd || !y) {
      free(dd); free(y);
#pragma omp atomic write
      status = ORACLE_NOMEM;
      continue;
    }
    const int32_t *pc = p + lo;
    const double *uc = u + lo, *xc = x + lo;
    for (int64_t i = 0; i < n; ++i) y[i] = fabs(d[lo + i]) * fabs(xc[i]);
    for (int64_t i = 1; i < n; ++i) {
      y[i] = y[i] + fabs(uc[i]) * fabs(xc[pc[i]]);
      y[pc[i]] = y[pc[i]] + fabs(uc[i]) * fabs(xc[i]);
    }
    memcpy(dd, d + lo, sizeof(double) * (size_t)n);
    oracle_hines(n, pc, dd, uc, y);
    double num = 0.0, den = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      if (fabs(y[i]) > num) num = fabs(y[i]);
      if (fabs(xc[i]) > den) den = fabs(xc[i]);
    }
    cond[c] = den > 0.0 ? num / den : 0.0;
    free(dd); free(y);
  }
  return status;
}

/*
 * Passive-cable time stepping (Section 1, the implicit-Euler finite-volume
 * system for V^{k+1}).  Per compartment: s = sigma*c_m/dt, leak conductance g
 * (current I = -g (V - E) per unit sigma), reversal E; per edge i -> p[i]:
 * axial coefficient a[i] (a[0] unused).  The system of step k is
 *   d_i = s_i (1 + theta dt g_i) + sum_{j in N(i)} a_ij
 *   b_i = s_i V_i^k + s_i dt g_i (E - (1 - theta) V_i^k)
 *   A[i][p[i]] = -a_i
 * theta = 0 evaluates the current at the old step exactly as the paper's
 * equation does; theta = 1 takes the leak at the new step (linearly implicit).
 * V is advanced in place; v_soma[k * n_cells + c] receives V^{k+1} of the
 * first compartment of cell c (nullable).
 */
static void rebuild_system(int64_t n, const int32_t *p, const double *s, const double *g, const double *a,
                           const double *V, double dt, double E, int theta, double *d, double *u, double *b) {
  for (int64_t i = 0; i < n; ++i) {
    d[i] = s[i] * (1.0 + (double)theta * dt * g[i]);
    b[i] = s[i] * V[i] + s[i] * dt * g[i] * (E - (1.0 - (double)theta) * V[i]);
    u[i] = 0.0;
  }
  for (int64_t i = 1; i < n; ++i) {
    d[i] = d[i] + a[i];
    d[p[i]] = d[p[i]] + a[i];
    u[i] = -a[i];
  }
}

int oracle_steps_batch(int32_t n_cells, const int64_t *off, const int32_t *p, const double *s, const double *g,
                       const double *a, double *V, int nsteps, double dt, double E, int theta, double *v_soma,
                       int nthreads) {
  int status = ORACLE_OK;
#pragma omp parallel for schedule(dynamic, 1) num_threads(clamp_threads(nthreads))
  for (int32_t c = 0; c < n_cells; ++c) {
    int64_t lo = off[c], n = off[c + 1] - off[c];
    if (n == 0) continue;
    int rc = oracle_check_parent(n, p + lo);
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    double *u = (double *)malloc(sizeof(double) * (size_t)n);
    if (rc != ORACLE_OK || !d || !u) {
      free(d); free(u);
#pragma omp atomic write
      status = rc != ORACLE_OK ? rc : ORACLE_NOMEM;
      continue;
    }
    double *Vc = V + lo;
    for (int k = 0; k < nsteps; ++k) {
      rebuild_system(n, p + lo, s + lo, g + lo, a + lo, Vc, dt, E, theta, d, u, Vc); /* b overwrites V */
      oracle_hines(n, p + lo, d, u, Vc);
      if (v_soma) v_soma[(int64_t)k * n_cells + c] = Vc[0];
    }
    free(d); free(u);
  }
  return status;
}

/*
 * Adjoint of the time stepper for L = sum_c sum_{k=1..K} (V_0^k(c) - target_c)^2.
 * A is symmetric, so lambda^k = A^{-1} Vbar^k is one more Hines solve, and
 *   dL/dd_i   = -lambda_i V_i          (from A V = b)
 *   dL/da_e   = -(lambda_i - lambda_p)(V_i - V_p)   for the edge e = (i, p[i])
 *   dL/db_i   =  lambda_i
 * chained through d(g), b(g, V^{k-1}) as defined in rebuild_system.  Plain
 * reverse sweep over all K stored states (no checkpointing).  Outputs per cell
 * loss[c] and per compartment grad_g, grad_a (grad_a[first of cell] = 0).
 */
int oracle_adjoint_batch(int32_t n_cells, const int64_t *off, const int32_t *p, const double *s, const double *g,
                         const double *a, const double *V0, const double *target, int nsteps, double dt, double E,
                         int theta, double *loss, double *grad_g, double *grad_a, int nthreads) {
  int status = ORACLE_OK;
#pragma omp parallel for schedule(dynamic, 1) num_threads(clamp_threads(nthreads))
  for (int32_t c = 0; c < n_cells; ++c) {
    int64_t lo = off[c], n = off[c + 1] - off[c];
    loss[c] = 0.0;
    if (n == 0) continue;
    const int32_t *pc = p + lo;
    const double *sc = s + lo, *gc = g + lo, *ac = a + lo;
    int rc = oracle_check_parent(n, pc);
    size_t states = (size_t)(nsteps + 1) * (size_t)n;
    double *Vs = (double *)malloc(sizeof(double) * states);
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    double *u = (double *)malloc(sizeof(double) * (size_t)n);
    double *vbar = (double *)malloc(sizeof(double) * (size_t)n);
    double *lam = (double *)malloc(sizeof(double) * (size_t)n);
    if (rc != ORACLE_OK || !Vs || !d || !u || !vbar || !lam) {
      free(Vs); free(d); free(u); free(vbar); free(lam);
#pragma omp atomic write
      status = rc != ORACLE_OK ? rc : ORACLE_NOMEM;
      continue;
    }
    /* forward, keeping every state */
    memcpy(Vs, V0 + lo, sizeof(double) * (size_t)n);
    for (int k = 0; k < nsteps; ++k) {
      double *Vk = Vs + (size_t)k * n, *Vn = Vs + (size_t)(k + 1) * n;
      rebuild_system(n, pc, sc, gc, ac, Vk, dt, E, theta, d, u, Vn);
      oracle_hines(n, pc, d, u, Vn);
      double e = Vn[0] - target[c];
      loss[c] = loss[c] + e * e;
    }
    for (int64_t i = 0; i < n; ++i) { grad_g[lo + i] = 0.0; grad_a[lo + i] = 0.0; vbar[i] = 0.0; }
    /* reverse sweep */
    for (int k = nsteps; k >= 1; --k) {
      const double *Vk = Vs + (size_t)k * n, *Vm = Vs + (size_t)(k - 1) * n;
      vbar[0] = vbar[0] + 2.0 * (Vk[0] - target[c]);
      rebuild_system(n, pc, sc, gc, ac, Vm, dt, E, theta, d, u, lam); /* lam gets b (unused) */
      memcpy(lam, vbar, sizeof(double) * (size_t)n);
      oracle_hines(n, pc, d, u, lam); /* lambda^k = A^{-1} Vbar^k (A symmetric) */
      for (int64_t i = 0; i < n; ++i) {
        double dLdd = -lam[i] * Vk[i];
        double dLdb = lam[i];
        grad_g[lo + i] = grad_g[lo + i] + dLdd * sc[i] * (double)theta * dt +
                         dLdb * sc[i] * dt * (E - (1.0 - (double)theta) * Vm[i]);
      }
      for (int64_t i = 1; i < n; ++i)
        grad_a[lo + i] = grad_a[lo + i] - (lam[i] - lam[pc[i]]) * (Vk[i] - Vk[pc[i]]);
      for (int64_t i = 0; i < n; ++i)
        vbar[i] = lam[i] * sc[i] * (1.0 - (1.0 - (double)theta) * dt * gc[i]);
    }
    free(Vs); free(d); free(u); free(vbar); free(lam);
  }
  return status;
}
