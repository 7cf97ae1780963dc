/*
 * kp_oracle.c -- plain, slow FP64 CPU oracle for the cross-matrix Krylov
 * projection solver (arXiv 2511.17634).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the package smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header or constant with the
 * CUDA library; the two meet only through the seeded synthetic inputs.
 *
 * Every routine is written for readability, one system at a time, in FP64,
 * in the order the paper states the method:
 *
 *   - Sec. 2.3, Eq. (6)-(9) and the coefficient listing under Eq. (11):
 *     backward-Euler / central-difference discretisation of the log-density
 *     Fokker-Planck equation (Eq. 5) with the semi-explicit (Picard-lagged)
 *     linearisation of <grad m, grad m>.  Appendix "Coefficient Definitions"
 *     repeats the same coefficients in another algebraic form.
 *   - Sec. 2.3, Eq. (12)-(15): the block-tridiagonal matrix form with the
 *     unknowns ordered y-fastest: k = i*H + j for column i (x, "east") and
 *     row j (y, "north").
 *   - Sec. 3, Phase 1: a Krylov solve of the seed system to a tolerance; the
 *     orthonormal basis V_a of K_a(A_seed, r0) is kept per timestep.  The
 *     paper names BiCGSTAB for the solve, but BiCGSTAB builds no orthonormal
 *     basis; this oracle uses restarted GMRES(m) with modified Gram-Schmidt
 *     Arnoldi (reorthogonalised) and Givens rotations (Saad, Iterative Methods, 2003, Alg. 6.9)
 *     and keeps the first cycle's Arnoldi vectors and Hessenberg matrix.
 *     orc_bicgstab is the paper's BiCGSTAB as an alternative: its key
 *     vectors, orthonormalised, form V_a, and A_proj = V_a^T A_seed V_a is
 *     then formed explicitly (orc_project_dense).
 *   - Sec. 3, Phase 2: A_proj = V^T A_seed V (equal to H_a from Arnoldi),
 *     b_proj = V^T b_i, solve A_proj alpha = b_proj, x0 = V alpha, then an
 *     iterative solve of A_i x = b_i from x0 (GMRES(m) again).
 *
 *   - End of Sec. 2.3 and Sec. 4.1: the score of each solved timestep by
 *     central differences and one explicit step of the probability-flow ODE
 *     that embeds it (orc_score, orc_embed_step).
 *
 * Storage convention: an H x W channel is a vector of N = H*W doubles with
 * index p = i*H + j, i in [0,W) the x (east-west) index and j in [0,H) the
 * y (north-south) index.  North = (i, j+1) = p+1, south = p-1, east =
 * (i+1, j) = p+H, west = p-H.  Points outside the grid are zero (zero
 * padding, Sec. 2.3), for the unknown, for the lagged m~ and for f.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_NOT_CONVERGED 1
#define ORC_ERR_ARG -1

int orc_dense_lu_solve(int n, double* A, double* b, double* x);

/* Value of a grid field at (i, j), zero outside the grid (zero padding). */
static double at(const double* f, int H, int W, int i, int j) {
  if (f == NULL || i < 0 || i >= W || j < 0 || j >= H) return 0.0;
  return f[i * H + j];
}

/*
 * Coefficients of the five-point system at every grid point, Sec. 2.3
 * (listing after Eq. 11):
 *   C_diag  = 1/dt + 2 g^2 / h^2
 *   C_north = -g^2/(2h^2) + fy/(2h) - g^2/(8h^2) (m~_{i,j+1} - m~_{i,j-1})
 *   C_south = -g^2/(2h^2) - fy/(2h) + g^2/(8h^2) (m~_{i,j+1} - m~_{i,j-1})
 *   C_east  = -g^2/(2h^2) + fx/(2h) - g^2/(8h^2) (m~_{i+1,j} - m~_{i-1,j})
 *   C_west  = -g^2/(2h^2) - fx/(2h) + g^2/(8h^2) (m~_{i+1,j} - m~_{i-1,j})
 * g2 is (g^n)^2.  fx, fy may be NULL (f = 0, as in the paper's experiments).
 * Output C has 5*N entries: C[5p+0..4] = diag, east, west, north, south.
 */
void orc_coeffs(int H, int W, double g2, double dt, double h, const double* mt,
                const double* fx, const double* fy, double* C) {
  double c = g2 / (2.0 * h * h);
  double e = g2 / (8.0 * h * h);
  for (int i = 0; i < W; ++i) {
    for (int j = 0; j < H; ++j) {
      int p = i * H + j;
      double dmx = at(mt, H, W, i + 1, j) - at(mt, H, W, i - 1, j);
      double dmy = at(mt, H, W, i, j + 1) - at(mt, H, W, i, j - 1);
      double fxp = at(fx, H, W, i, j);
      double fyp = at(fy, H, W, i, j);
      C[5 * p + 0] = 1.0 / dt + 2.0 * g2 / (h * h);
      C[5 * p + 1] = -c + fxp / (2.0 * h) - e * dmx; /* east  */
      C[5 * p + 2] = -c - fxp / (2.0 * h) + e * dmx; /* west  */
      C[5 * p + 3] = -c + fyp / (2.0 * h) - e * dmy; /* north */
      C[5 * p + 4] = -c - fyp / (2.0 * h) + e * dmy; /* south */
    }
  }
}

/*
 * Right-hand side, Sec. 2.3 (given with the coefficients after Eq. 11):
 *   b_{i,j} = m^{n-1}_{i,j}/dt - [(fx_{i+1,j} - fx_{i-1,j}) + (fy_{i,j+1} - fy_{i,j-1})]/(2h)
 */
void orc_rhs(int H, int W, double dt, double h, const double* mprev, const double* fx,
             const double* fy, double* b) {
  for (int i = 0; i < W; ++i) {
    for (int j = 0; j < H; ++j) {
      int p = i * H + j;
      double divf = (at(fx, H, W, i + 1, j) - at(fx, H, W, i - 1, j)) +
                    (at(fy, H, W, i, j + 1) - at(fy, H, W, i, j - 1));
      b[p] = mprev[p] / dt - divf / (2.0 * h);
    }
  }
}

/* y = A x with A given by its stencil coefficients (Eq. 11); out-of-grid
 * neighbours of x are zero. */
void orc_apply(int H, int W, const double* C, const double* x, double* y) {
  for (int i = 0; i < W; ++i) {
    for (int j = 0; j < H; ++j) {
      int p = i * H + j;
      y[p] = C[5 * p + 0] * x[p] + C[5 * p + 1] * at(x, H, W, i + 1, j) +
             C[5 * p + 2] * at(x, H, W, i - 1, j) + C[5 * p + 3] * at(x, H, W, i, j + 1) +
             C[5 * p + 4] * at(x, H, W, i, j - 1);
    }
  }
}

/*
 * Explicit sparse matrix in CSR form, assembled from the block structure of
 * Eq. (12)-(15): W x W blocks of size H x H; diagonal blocks M tridiagonal
 * (south below, diag, north above), off-diagonal blocks L (west, to the
 * previous column) and U (east, to the next column) diagonal, with per-row
 * values.  Columns in each row are sorted.  rowptr has N+1 entries; col and
 * val need at most 5N entries.  Returns the number of non-zeros.
 */
int orc_csr(int H, int W, const double* C, int* rowptr, int* col, double* val) {
  int nnz = 0;
  for (int blk = 0; blk < W; ++blk) {        /* block row = grid column i */
    for (int r = 0; r < H; ++r) {            /* row inside the block = j  */
      int row = blk * H + r;
      rowptr[row] = nnz;
      if (blk > 0) { col[nnz] = (blk - 1) * H + r; val[nnz] = C[5 * row + 2]; ++nnz; } /* L */
      if (r > 0) { col[nnz] = row - 1; val[nnz] = C[5 * row + 4]; ++nnz; }             /* M sub   */
      col[nnz] = row; val[nnz] = C[5 * row + 0]; ++nnz;                                 /* M diag  */
      if (r < H - 1) { col[nnz] = row + 1; val[nnz] = C[5 * row + 3]; ++nnz; }         /* M super */
      if (blk < W - 1) { col[nnz] = (blk + 1) * H + r; val[nnz] = C[5 * row + 1]; ++nnz; } /* U */
    }
  }
  rowptr[H * W] = nnz;
  return nnz;
}

void orc_csr_matvec(int n, const int* rowptr, const int* col, const double* val,
                    const double* x, double* y) {
  for (int r = 0; r < n; ++r) {
    double s = 0.0;
    for (int k = rowptr[r]; k < rowptr[r + 1]; ++k) s += val[k] * x[col[k]];
    y[r] = s;
  }
}

static double dot(int n, const double* a, const double* b) {
  double s = 0.0;
  for (int k = 0; k < n; ++k) s += a[k] * b[k];
  return s;
}

static double nrm2(int n, const double* a) { return sqrt(dot(n, a, a)); }

/* Givens rotation (c, s) with  [c s; -s c] [a; b] = [r; 0]. */
static void givens(double a, double b, double* c, double* s) {
  if (b == 0.0) { *c = 1.0; *s = 0.0; return; }
  double r = hypot(a, b);
  *c = a / r;
  *s = b / r;
}

/*
 * Restarted GMRES(m) on A x = b, A given by stencil coefficients C.
 * Arnoldi with modified Gram-Schmidt (two sweeps), Hessenberg least squares
 * by Givens rotations, restart from the true residual r = b - A x (Saad 2003, Alg. 6.9
 * and Prop. 6.9).  Stops when ||b - A x||_2 <= tol ||b||_2 (true residual,
 * recomputed at the end of every cycle) or when maxit Arnoldi steps have run.
 *
 *  x        in: initial guess, out: final iterate.
 *  info[0]  Arnoldi steps taken (matrix-vector products excluding residuals).
 *  rel_res  out: ||b - A x|| / ||b|| of the returned x.
 *  hist     optional (maxit+1 entries): the Givens residual estimate |g_{j+1}|/||b||
 *           after every Arnoldi step, preceded by the initial true relative residual.
 *  cap_a    if > 0 and capV != NULL: keep the first cycle's Arnoldi vectors
 *           v_1..v_{a'+1} (capV, column-major N x (cap_a+1)) and the unrotated
 *           Hessenberg matrix Hbar (capH, column-major (cap_a+1) x cap_a), where
 *           a' = min(cap_a, steps of the first cycle); *cap_used = a' and
 *           *cap_next = 1 if v_{a'+1} exists (no exact breakdown at step a').
 *  cap_fixed if non-zero (and capV != NULL): the basis has the fixed dimension
 *           a = min(cap_a, m) of Sec. 3 (V_a^n spans K_a(A^n, r0); Sec. 5.2 runs
 *           a = 20): the residual test does not end the first cycle before it
 *           has taken a Arnoldi steps -- only an exact breakdown or maxit does --
 *           so the kept basis is the whole a-dimensional Krylov space even when
 *           the solve converges in fewer steps.  The cycle's iterate is then the
 *           GMRES minimiser over K_a, at least as accurate as the one at the
 *           step where the test was first met.
 * Returns ORC_OK or ORC_NOT_CONVERGED.
 */
int orc_gmres(int H, int W, const double* C, const double* b, double* x, double tol, int m,
              int maxit, int* iters, double* rel_res, double* hist, int cap_a, double* capV,
              double* capH, int* cap_used, int* cap_next, int cap_fixed) {
  int N = H * W;
  double* V = (double*)calloc((size_t)N * (m + 1), sizeof(double));
  double* Hh = (double*)calloc((size_t)(m + 1) * m, sizeof(double)); /* rotated, col-major */
  double* Hraw = (double*)calloc((size_t)(m + 1) * m, sizeof(double));
  double* g = (double*)calloc((size_t)(m + 1), sizeof(double));
  double* cs = (double*)calloc((size_t)m, sizeof(double));
  double* sn = (double*)calloc((size_t)m, sizeof(double));
  double* y = (double*)calloc((size_t)m, sizeof(double));
  double* r = (double*)calloc((size_t)N, sizeof(double));
  double* w = (double*)calloc((size_t)N, sizeof(double));
#define HH(i, j) Hh[(size_t)(j) * (m + 1) + (i)]
#define HR(i, j) Hraw[(size_t)(j) * (m + 1) + (i)]
  int status = ORC_NOT_CONVERGED;
  int steps = 0, cycle = 0, nh = 0;
  double bnorm = nrm2(N, b);
  if (cap_used) *cap_used = 0;
  if (cap_next) *cap_next = 0;
  if (bnorm == 0.0) {
    for (int k = 0; k < N; ++k) x[k] = 0.0;
    *iters = 0; *rel_res = 0.0;
    if (hist) hist[0] = 0.0;
    status = ORC_OK;
    goto done;
  }
  orc_apply(H, W, C, x, r);
  for (int k = 0; k < N; ++k) r[k] = b[k] - r[k];
  double beta = nrm2(N, r);
  if (hist) hist[nh++] = beta / bnorm;
  for (;;) {
    if (beta <= tol * bnorm) { status = ORC_OK; break; }
    if (steps >= maxit) break;
    for (int k = 0; k < N; ++k) V[k] = r[k] / beta;
    memset(g, 0, sizeof(double) * (m + 1));
    g[0] = beta;
    int kdone = 0, breakdown = 0;
    for (int j = 0; j < m; ++j) {
      double* vj = V + (size_t)j * N;
      orc_apply(H, W, C, vj, w);
      ++steps;
      double wnorm0 = nrm2(N, w);
      /* Modified Gram-Schmidt, run twice.  Sec. 3 stores an orthonormal
       * basis; a single MGS sweep loses orthogonality in proportion to
       * cond(A)/||r_j|| (Paige, Rozloznik & Strakos 2006), which at 1e-10
       * residuals is ~1e-6 and would corrupt V^T b in Phase 2.  The second
       * sweep ("twice is enough", Giraud et al. 2005) keeps it at O(eps). */
      for (int i = 0; i <= j; ++i) HR(i, j) = 0.0;
      for (int sweep = 0; sweep < 2; ++sweep) {
        for (int i = 0; i <= j; ++i) {
          double* vi = V + (size_t)i * N;
          double hij = dot(N, w, vi);
          for (int k = 0; k < N; ++k) w[k] -= hij * vi[k];
          HR(i, j) += hij;
        }
      }
      for (int i = 0; i <= j; ++i) HH(i, j) = HR(i, j);
      double hn = nrm2(N, w);
      HH(j + 1, j) = hn;
      HR(j + 1, j) = hn;
      breakdown = !(hn > 1e-14 * wnorm0);           /* happy breakdown */
      if (!breakdown) {
        double* vn = V + (size_t)(j + 1) * N;
        for (int k = 0; k < N; ++k) vn[k] = w[k] / hn;
      }
      for (int i = 0; i < j; ++i) {                  /* earlier rotations */
        double t1 = HH(i, j), t2 = HH(i + 1, j);
        HH(i, j) = cs[i] * t1 + sn[i] * t2;
        HH(i + 1, j) = -sn[i] * t1 + cs[i] * t2;
      }
      givens(HH(j, j), HH(j + 1, j), &cs[j], &sn[j]);
      HH(j, j) = cs[j] * HH(j, j) + sn[j] * HH(j + 1, j);
      HH(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      if (hist) hist[nh++] = fabs(g[j + 1]) / bnorm;
      kdone = j + 1;
      /* fixed a: the first cycle of a capturing solve reaches a steps before
       * the residual test may end it */
      int short_of_a = cap_fixed && capV != NULL && cycle == 0 && cap_a > 0 && kdone < cap_a;
      if ((fabs(g[j + 1]) <= tol * bnorm && !short_of_a) || breakdown || steps >= maxit) break;
    }
    /* back substitution R y = g */
    for (int i = kdone - 1; i >= 0; --i) {
      double s = g[i];
      for (int l = i + 1; l < kdone; ++l) s -= HH(i, l) * y[l];
      y[i] = s / HH(i, i);
    }
    for (int i = 0; i < kdone; ++i) {
      double* vi = V + (size_t)i * N;
      for (int k = 0; k < N; ++k) x[k] += y[i] * vi[k];
    }
    if (cycle == 0 && cap_a > 0 && capV != NULL) {
      int a = kdone < cap_a ? kdone : cap_a;
      int nxt = (a < kdone) || !breakdown;         /* v_{a+1} was formed */
      memcpy(capV, V, sizeof(double) * (size_t)N * (a + (nxt ? 1 : 0)));
      if (capH) {
        for (int jj = 0; jj < a; ++jj)
          for (int ii = 0; ii <= a; ++ii)
            capH[(size_t)jj * (cap_a + 1) + ii] = (ii <= jj + 1) ? HR(ii, jj) : 0.0;
      }
      if (cap_used) *cap_used = a;
      if (cap_next) *cap_next = nxt;
    }
    ++cycle;
    orc_apply(H, W, C, x, r);                        /* true residual */
    for (int k = 0; k < N; ++k) r[k] = b[k] - r[k];
    beta = nrm2(N, r);
  }
  *iters = steps;
  *rel_res = beta / bnorm;
done:
  free(V); free(Hh); free(Hraw); free(g); free(cs); free(sn); free(y); free(r); free(w);
#undef HH
#undef HR
  return status;
}

/*
 * Sec. 3, Phase 1 as the paper states it: BiCGSTAB (van der Vorst 1992) on
 * A x = b, A given by stencil coefficients C.  Each iteration k forms the
 * search direction p_k, v = A p_k, the intermediate residual s_k = r_{k-1} -
 * alpha v, t = A s_k, the smoothing step omega = <t,s>/<t,t> and the residual
 * r_k = s_k - omega t; x gains alpha p_k + omega s_k.  Stops when the updated
 * residual satisfies ||r|| <= tol ||b|| (or ||s|| does, after the half step),
 * then checks the true residual b - A x and, if it is still above tol ||b||,
 * restarts from it (shadow residual reset to that residual).  A zero rho or
 * omega also ends the sweep and restarts.  At most maxit iterations.
 *
 * Basis (the paper keeps the key vectors of the iteration): during the first
 * sweep, r_0 and then s_k, r_k of every iteration, in that order, all lying in
 * the Krylov space of A and r_0 (the j-th kept vector in K_{j+1}).  Each is
 * orthogonalised against the vectors kept so far by modified Gram-Schmidt
 * run twice and kept, normalised, if what remains is above 1e-10 of its
 * norm, until cap_a vectors are kept.  capV: column-major N x cap_a;
 * *cap_used = vectors kept.
 *
 *  x        in: initial guess, out: final iterate.
 *  iters    out: BiCGSTAB iterations (two operator applications each).
 *  rel_res  out: ||b - A x|| / ||b|| of the returned x.
 * Returns ORC_OK or ORC_NOT_CONVERGED.
 */
static void keep_vector(int N, const double* u, int cap_a, double* capV, int* used, double* w) {
  if (!capV || *used >= cap_a) return;
  double n0 = nrm2(N, u);
  if (!(n0 > 0.0)) return;
  memcpy(w, u, sizeof(double) * N);
  for (int sweep = 0; sweep < 2; ++sweep)
    for (int i = 0; i < *used; ++i) {
      const double* vi = capV + (size_t)i * N;
      double h = dot(N, w, vi);
      for (int k = 0; k < N; ++k) w[k] -= h * vi[k];
    }
  double n1 = nrm2(N, w);
  if (!(n1 > 1e-10 * n0)) return;
  double* vn = capV + (size_t)(*used) * N;
  for (int k = 0; k < N; ++k) vn[k] = w[k] / n1;
  ++*used;
}

int orc_bicgstab(int H, int W, const double* C, const double* b, double* x, double tol,
                 int maxit, int* iters, double* rel_res, int cap_a, double* capV, int* cap_used) {
  int N = H * W;
  double* r = (double*)calloc((size_t)N, sizeof(double));
  double* rh = (double*)calloc((size_t)N, sizeof(double));
  double* p = (double*)calloc((size_t)N, sizeof(double));
  double* v = (double*)calloc((size_t)N, sizeof(double));
  double* sv = (double*)calloc((size_t)N, sizeof(double));
  double* t = (double*)calloc((size_t)N, sizeof(double));
  double* w = (double*)calloc((size_t)N, sizeof(double));
  int status = ORC_NOT_CONVERGED, it = 0, sweep = 0;
  int used = 0;
  double bnorm = nrm2(N, b), rn = 0.0;
  if (bnorm == 0.0) {
    for (int k = 0; k < N; ++k) x[k] = 0.0;
    status = ORC_OK;
  }
  while (status != ORC_OK) {
    orc_apply(H, W, C, x, r);                          /* true residual */
    for (int k = 0; k < N; ++k) r[k] = b[k] - r[k];
    rn = nrm2(N, r);
    if (rn <= tol * bnorm) { status = ORC_OK; break; }
    if (it >= maxit) break;
    int keep = (sweep == 0);
    if (keep) keep_vector(N, r, cap_a, capV, &used, w);
    memcpy(rh, r, sizeof(double) * N);
    memset(p, 0, sizeof(double) * N);
    memset(v, 0, sizeof(double) * N);
    double rho_old = 1.0, alpha = 1.0, omega = 1.0;
    while (it < maxit) {
      double rho = dot(N, rh, r);
      if (rho == 0.0) break;
      double beta = (rho / rho_old) * (alpha / omega);
      for (int k = 0; k < N; ++k) p[k] = r[k] + beta * (p[k] - omega * v[k]);
      orc_apply(H, W, C, p, v);
      alpha = rho / dot(N, rh, v);
      for (int k = 0; k < N; ++k) sv[k] = r[k] - alpha * v[k];
      ++it;
      if (keep) keep_vector(N, sv, cap_a, capV, &used, w);
      if (nrm2(N, sv) <= tol * bnorm) {
        for (int k = 0; k < N; ++k) x[k] += alpha * p[k];
        break;
      }
      orc_apply(H, W, C, sv, t);
      double tt = dot(N, t, t);
      omega = tt > 0.0 ? dot(N, t, sv) / tt : 0.0;
      for (int k = 0; k < N; ++k) x[k] += alpha * p[k] + omega * sv[k];
      for (int k = 0; k < N; ++k) r[k] = sv[k] - omega * t[k];
      if (keep) keep_vector(N, r, cap_a, capV, &used, w);
      if (nrm2(N, r) <= tol * bnorm || omega == 0.0) break;
      rho_old = rho;
    }
    ++sweep;
  }
  *iters = it;
  *rel_res = bnorm > 0.0 ? rn / bnorm : 0.0;
  if (cap_used) *cap_used = used;
  free(r); free(rh); free(p); free(v); free(sv); free(t); free(w);
  return status;
}

/*
 * Phase 2 of Sec. 3 for a seed basis without a Hessenberg relation (the
 * BiCGSTAB basis): A_proj = V_a^T A_seed V_a is formed explicitly (Aproj,
 * row-major a x a, as the caller built it from the seed's operator),
 *   c = V_a^T r,  A_proj alpha = c (dense LU, partial pivoting),  x0 = xinit + V_a alpha.
 * V: column-major N x a.  Returns 0, or 1 if A_proj is singular (x0 = xinit).
 */
int orc_project_dense(int N, int a, const double* V, const double* Aproj, const double* r,
                      const double* xinit, double* x0) {
  for (int k = 0; k < N; ++k) x0[k] = xinit ? xinit[k] : 0.0;
  if (a <= 0) return 0;
  double* A = (double*)malloc(sizeof(double) * a * a);
  double* c = (double*)malloc(sizeof(double) * a);
  double* alpha = (double*)malloc(sizeof(double) * a);
  memcpy(A, Aproj, sizeof(double) * a * a);
  for (int l = 0; l < a; ++l) c[l] = dot(N, V + (size_t)l * N, r);
  int rc = orc_dense_lu_solve(a, A, c, alpha);
  if (rc == 0)
    for (int i = 0; i < a; ++i)
      for (int k = 0; k < N; ++k) x0[k] += alpha[i] * V[(size_t)i * N + k];
  free(A); free(c); free(alpha);
  return rc == 0 ? 0 : 1;
}

/*
 * Seed cycling with subspace expansion (Sec. 5.2 runs it with a new seed every
 * 50 images and the subspace capped at a = 20; the paragraph the source of
 * Sec. 3 leaves commented out describes accumulating the key vectors of each
 * new seed into an increasingly rich basis).  The basis served by a new seed
 * is built from its own basis vectors Vown (a_own of them) first, then the
 * previous accumulated basis Vprev (a_prev), each vector orthogonalised by
 * modified Gram-Schmidt run twice against those kept and kept, normalised, if
 * more than 1e-10 of its norm remains, until cap_a vectors are kept; so the
 * newest seed's space is always whole and older ones fill what room is left.
 * A_proj = V^T A_seed V is then formed with the new seed's operator C
 * (row-major count x count).  V, Vown, Vprev: column-major N x (count).
 * Returns the number of vectors kept.
 */
int orc_accumulate(int H, int W, const double* C, int a_own, const double* Vown, int a_prev,
                   const double* Vprev, int cap_a, double* V, double* Aproj) {
  int N = H * W;
  int used = 0;
  double* w = (double*)malloc(sizeof(double) * N);
  for (int k = 0; k < a_own; ++k) keep_vector(N, Vown + (size_t)k * N, cap_a, V, &used, w);
  for (int k = 0; k < a_prev; ++k) keep_vector(N, Vprev + (size_t)k * N, cap_a, V, &used, w);
  double* Av = (double*)malloc(sizeof(double) * N);
  for (int k = 0; k < used; ++k) {
    orc_apply(H, W, C, V + (size_t)k * N, Av);
    for (int l = 0; l < used; ++l) Aproj[(size_t)l * used + k] = dot(N, V + (size_t)l * N, Av);
  }
  free(w); free(Av);
  return used;
}

/*
 * Phase 2 of Sec. 3: Galerkin projection of one target onto a stored seed
 * basis.  V is N x (a+1) column-major (v_{a+1} present iff has_next), Hbar
 * the unrotated (a+1) x a Hessenberg matrix of the seed's Arnoldi process
 * (leading dimension lda = cap_a + 1), so that A_seed V_a = V_{a+1} Hbar and
 * V_a^T A_seed V_a = H_a (its top a x a block).
 *   c      = V_a^T r                        (b_proj)
 *   alpha  = H_a^{-1} c                      (Givens QR of H_a)
 *   x0     = xinit + V_a alpha
 * If a pivot of the QR of H_a is below 1e-14 ||H_a||_max (H_a numerically
 * singular) and v_{a+1} exists, alpha instead minimises ||Hbar alpha - V_{a+1}^T r||.
 * r is the right-hand side (or the residual of xinit); xinit may be NULL (zero).
 * Returns 1 if the least-squares fallback was used, 0 otherwise.
 */
int orc_project(int N, int a, int lda, int has_next, const double* V, const double* Hbar,
                const double* r, const double* xinit, double* x0) {
  int used_lsq = 0;
  int rows = a + 1;
  double* R = (double*)calloc((size_t)rows * a, sizeof(double));
  double* c = (double*)calloc((size_t)rows, sizeof(double));
  double* alpha = (double*)calloc((size_t)(a > 0 ? a : 1), sizeof(double));
  double hmax = 0.0;
  for (int j = 0; j < a; ++j)
    for (int i = 0; i < a; ++i) hmax = fmax(hmax, fabs(Hbar[(size_t)j * lda + i]));
  for (int pass = 0; pass < 2; ++pass) {
    int lsq = (pass == 1);
    int nr = lsq ? a + 1 : a;                /* rows taken from Hbar */
    for (int j = 0; j < a; ++j)
      for (int i = 0; i < rows; ++i) R[(size_t)j * rows + i] = (i < nr) ? Hbar[(size_t)j * lda + i] : 0.0;
    for (int i = 0; i < nr; ++i) c[i] = dot(N, V + (size_t)i * N, r);
    /* Givens QR: zero the subdiagonal of column j against row j */
    for (int j = 0; j < a; ++j) {
      if (j + 1 >= nr) break;
      double cc, ss;
      givens(R[(size_t)j * rows + j], R[(size_t)j * rows + j + 1], &cc, &ss);
      for (int l = j; l < a; ++l) {
        double t1 = R[(size_t)l * rows + j], t2 = R[(size_t)l * rows + j + 1];
        R[(size_t)l * rows + j] = cc * t1 + ss * t2;
        R[(size_t)l * rows + j + 1] = -ss * t1 + cc * t2;
      }
      double t1 = c[j], t2 = c[j + 1];
      c[j] = cc * t1 + ss * t2;
      c[j + 1] = -ss * t1 + cc * t2;
    }
    int singular = 0;
    for (int j = 0; j < a; ++j)
      if (!(fabs(R[(size_t)j * rows + j]) > 1e-14 * hmax)) singular = 1;
    if (singular && !lsq && has_next) continue;  /* retry as least squares */
    for (int i = a - 1; i >= 0; --i) {
      double s = c[i];
      for (int l = i + 1; l < a; ++l) s -= R[(size_t)l * rows + i] * alpha[l];
      alpha[i] = (R[(size_t)i * rows + i] != 0.0) ? s / R[(size_t)i * rows + i] : 0.0;
    }
    used_lsq = lsq;
    break;
  }
  for (int k = 0; k < N; ++k) x0[k] = xinit ? xinit[k] : 0.0;
  for (int i = 0; i < a; ++i)
    for (int k = 0; k < N; ++k) x0[k] += alpha[i] * V[(size_t)i * N + k];
  free(R); free(c); free(alpha);
  return used_lsq;
}

/*
 * Dense LU with partial pivoting (Doolittle, row interchanges), solving
 * A x = b in place; A is n x n row-major and is overwritten.  Test-only
 * reference for tiny grids.  Returns 0, or -1 if a pivot is exactly zero.
 */
int orc_dense_lu_solve(int n, double* A, double* b, double* x) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int r = k + 1; r < n; ++r)
      if (fabs(A[(size_t)r * n + k]) > fabs(A[(size_t)piv * n + k])) piv = r;
    if (A[(size_t)piv * n + k] == 0.0) return -1;
    if (piv != k) {
      for (int c2 = 0; c2 < n; ++c2) {
        double t = A[(size_t)k * n + c2]; A[(size_t)k * n + c2] = A[(size_t)piv * n + c2]; A[(size_t)piv * n + c2] = t;
      }
      double t = b[k]; b[k] = b[piv]; b[piv] = t;
    }
    for (int r = k + 1; r < n; ++r) {
      double l = A[(size_t)r * n + k] / A[(size_t)k * n + k];
      A[(size_t)r * n + k] = l;
      for (int c2 = k + 1; c2 < n; ++c2) A[(size_t)r * n + c2] -= l * A[(size_t)k * n + c2];
      b[r] -= l * b[k];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int c2 = r + 1; c2 < n; ++c2) s -= A[(size_t)r * n + c2] * x[c2];
    x[r] = s / A[(size_t)r * n + r];
  }
  return 0;
}

/*
 * One timestep n of the method for a set of seed and target channels that
 * share one grid size (Sec. 2.3 and Sec. 3, both phases):
 *   seeds:   A_s(m~ = m_s^{n-1}) m_s^n = m_s^{n-1}/dt (f = 0), GMRES(m_seed)
 *            from x0 = 0 to tol_seed, keeping the first-cycle basis (a vectors);
 *            with seed_solver = 1, BiCGSTAB instead (the paper's Phase 1),
 *            keeping its key vectors (orc_bicgstab) and A_proj = V^T A_s V.
 *   targets: mode 0 (projected): x0 = V_a H_a^{-1} V_a^T b_i with the basis of
 *            seed target_seed[i] (x0 = V_a A_proj^{-1} V_a^T b_i after
 *            BiCGSTAB seeds, and after seeds with a predecessor in seed_prev,
 *            which serve the accumulated basis of orc_accumulate); mode 1
 *            (plain): x0 = 0; mode 2 (warm):
 *            x0 = m_i^{n-1}; mode 3 (exact Galerkin): x0 = V_a G^{-1} V_a^T b_i
 *            with G = V_a^T A_i V_a; mode 4 (a given initial guess, judged and
 *            projected in residual form): the guess xinit_i is kept unless the
 *            warm start m_i^{n-1} leaves a strictly smaller residual norm (the
 *            method without the guess is the guess's fallback and the residual
 *            the judge); a kept guess is projected, x0 = xinit_i + V_a H_a^{-1}
 *            V_a^T (b_i - A_i xinit_i) (the explicit A_proj after BiCGSTAB or
 *            cycled seeds), the fallback starts as mode 2 does, x0 = m_i^{n-1};
 *            mode 5 (the given guess alone): x0 = xinit_i; then GMRES(m_ref)
 *            on A_i to tol_ref.
 *            xinit ([ntgt][N], modes 4 and 5 only) is read, never written.
 * fixed_a != 0: the seed's basis has the fixed dimension a of Sec. 3 (its
 * first GMRES cycle takes min(a, m_seed) Arnoldi steps; see orc_gmres).
 * picard > 1 adds Picard iterations k = 2..picard (Sec. 2.3, m~ = m^{n,(k-1)}):
 * the coefficients are rebuilt from the latest iterate, the right-hand side
 * stays m^{n-1}/dt and GMRES starts from that iterate; the seed basis is the
 * one of the first solve.
 * mseed/mtgt hold m^{n-1} on entry and m^n on return ([count][N]).
 * seed_it/tgt_it receive Arnoldi steps, tgt_res the final relative residual,
 * tgt_status the GMRES status (0 converged).  OpenMP (if compiled in) runs
 * independent systems in parallel; each system's arithmetic is unchanged.
 */
/*
 * Sec. 3, Phase 2 without the seed-matrix shortcut: the Galerkin projection
 * with the target's own operator A_i (coefficients C) onto the seed's basis,
 *   G = V_a^T A_i V_a (a x a),  c = V_a^T r,  G alpha = c,  x0 = xinit + V_a alpha.
 * The paper replaces G by the seed's H_a = V_a^T A_seed V_a; this is the
 * exact version it approximates.  G is solved by dense LU with partial
 * pivoting.  Returns 0, or 1 if G is singular (then x0 = xinit).
 */
int orc_project_galerkin(int H, int W, const double* C, int a, const double* V, const double* r,
                         const double* xinit, double* x0) {
  int N = H * W;
  for (int k = 0; k < N; ++k) x0[k] = xinit ? xinit[k] : 0.0;
  if (a <= 0) return 0;
  double* G = (double*)malloc(sizeof(double) * a * a);
  double* c = (double*)malloc(sizeof(double) * a);
  double* alpha = (double*)malloc(sizeof(double) * a);
  double* Av = (double*)malloc(sizeof(double) * N);
  for (int k = 0; k < a; ++k) {
    orc_apply(H, W, C, V + (size_t)k * N, Av);
    for (int l = 0; l < a; ++l) G[l * a + k] = dot(N, V + (size_t)l * N, Av);   /* row-major */
  }
  for (int l = 0; l < a; ++l) c[l] = dot(N, V + (size_t)l * N, r);
  int rc = orc_dense_lu_solve(a, G, c, alpha);
  if (rc == 0)
    for (int i = 0; i < a; ++i)
      for (int k = 0; k < N; ++k) x0[k] += alpha[i] * V[(size_t)i * N + k];
  free(G); free(c); free(alpha); free(Av);
  return rc == 0 ? 0 : 1;
}

void orc_march_step(int H, int W, double dt, double h, double g2, int nseed, double* mseed,
                    int ntgt, double* mtgt, const int* target_seed, int mode, double tol_seed,
                    int m_seed, int a, double tol_ref, int m_ref, int maxit, int* seed_it,
                    int* tgt_it, double* tgt_res, int* tgt_status, double* tgt_x0res, int picard,
                    int seed_solver, const int* seed_prev, int fixed_a, const double* xinit) {
  int K = picard > 1 ? picard : 1;
  int N = H * W;
  int lda = a + 1;
  double* basis = (double*)calloc((size_t)nseed * N * (a + 1), sizeof(double));
  double* hess = (double*)calloc((size_t)nseed * (a + 1) * a, sizeof(double));
  double* aproj = (double*)calloc((size_t)nseed * (a > 0 ? a * a : 1), sizeof(double));
  int* used = (int*)calloc((size_t)(nseed > 0 ? nseed : 1), sizeof(int));
  int* nxt = (int*)calloc((size_t)(nseed > 0 ? nseed : 1), sizeof(int));
  int* dense = (int*)calloc((size_t)(nseed > 0 ? nseed : 1), sizeof(int));
  double* mprev = (double*)malloc(sizeof(double) * (size_t)(nseed > 0 ? nseed : 1) * N);
  memcpy(mprev, mseed, sizeof(double) * (size_t)nseed * N);
#pragma omp parallel for schedule(dynamic, 1)
  for (int s = 0; s < nseed; ++s) {
    double* C = (double*)malloc(sizeof(double) * 5 * N);
    double* b = (double*)malloc(sizeof(double) * N);
    double* x = (double*)calloc((size_t)N, sizeof(double));
    double* ms = mseed + (size_t)s * N;
    double rr;
    orc_coeffs(H, W, g2, dt, h, ms, NULL, NULL, C);
    orc_rhs(H, W, dt, h, ms, NULL, NULL, b);
    if (seed_solver == 1) {
      double* Vs = basis + (size_t)s * N * (a + 1);
      orc_bicgstab(H, W, C, b, x, tol_seed, maxit, &seed_it[s], &rr, a, Vs, &used[s]);
      nxt[s] = 0;
      dense[s] = 1;
      /* A_proj = V^T A_seed V (row-major used x used) */
      int u = used[s];
      double* Av = (double*)malloc(sizeof(double) * N);
      for (int k = 0; k < u; ++k) {
        orc_apply(H, W, C, Vs + (size_t)k * N, Av);
        for (int l = 0; l < u; ++l) aproj[(size_t)s * a * a + (size_t)l * u + k] = dot(N, Vs + (size_t)l * N, Av);
      }
      free(Av);
    } else {
      orc_gmres(H, W, C, b, x, tol_seed, m_seed, maxit, &seed_it[s], &rr, NULL, a,
                basis + (size_t)s * N * (a + 1), hess + (size_t)s * (a + 1) * a, &used[s], &nxt[s],
                fixed_a);
    }
    /* Picard iterations k = 2..K (Sec. 2.3): lag the nonlinear term on the
     * latest iterate, same right-hand side, warm start from that iterate */
    for (int k = 1; k < K; ++k) {
      int it = 0;
      orc_coeffs(H, W, g2, dt, h, x, NULL, NULL, C);
      orc_gmres(H, W, C, b, x, tol_seed, m_seed, maxit, &it, &rr, NULL, 0, NULL, NULL, NULL, NULL, 0);
      seed_it[s] += it;
    }
    memcpy(ms, x, sizeof(double) * N);
    free(C); free(b); free(x);
  }
  /* seed cycling: each seed with a predecessor serves the accumulated basis
   * (its own vectors, then the predecessor's accumulated ones), in seed order */
  for (int s = 0; seed_prev && s < nseed; ++s) {
    int q = seed_prev[s];
    if (q < 0 || q >= s) continue;
    double* C = (double*)malloc(sizeof(double) * 5 * N);
    double* Vn = (double*)calloc((size_t)N * (a + 1), sizeof(double));
    orc_coeffs(H, W, g2, dt, h, mprev + (size_t)s * N, NULL, NULL, C);
    int u = orc_accumulate(H, W, C, used[s], basis + (size_t)s * N * (a + 1), used[q],
                           basis + (size_t)q * N * (a + 1), a, Vn, aproj + (size_t)s * a * a);
    memcpy(basis + (size_t)s * N * (a + 1), Vn, sizeof(double) * (size_t)N * (a + 1));
    used[s] = u;
    nxt[s] = 0;
    dense[s] = 1;
    free(C); free(Vn);
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int t = 0; t < ntgt; ++t) {
    double* C = (double*)malloc(sizeof(double) * 5 * N);
    double* b = (double*)malloc(sizeof(double) * N);
    double* x = (double*)calloc((size_t)N, sizeof(double));
    double* r = (double*)malloc(sizeof(double) * N);
    double* mt = mtgt + (size_t)t * N;
    orc_coeffs(H, W, g2, dt, h, mt, NULL, NULL, C);
    orc_rhs(H, W, dt, h, mt, NULL, NULL, b);
    if (mode == 4 || mode == 5) {
      /* a given initial guess; mode 4 projects its residual (Sec. 3, Phase 2
       * applied to r = b - A x_init) */
      const double* xi = xinit + (size_t)t * N;
      if (mode == 5) {
        memcpy(x, xi, sizeof(double) * N);
      } else {
        int s = target_seed[t];
        double* rw = (double*)malloc(sizeof(double) * N);
        orc_apply(H, W, C, xi, r);
        for (int k = 0; k < N; ++k) r[k] = b[k] - r[k];
        orc_apply(H, W, C, mt, rw);                    /* the warm start m^{n-1} */
        for (int k = 0; k < N; ++k) rw[k] = b[k] - rw[k];
        if (nrm2(N, rw) < nrm2(N, r))                  /* the fallback, as in mode 2 */
          memcpy(x, mt, sizeof(double) * N);
        else if (dense[s])
          orc_project_dense(N, used[s], basis + (size_t)s * N * (a + 1), aproj + (size_t)s * a * a, r,
                            xi, x);
        else
          orc_project(N, used[s], lda, nxt[s], basis + (size_t)s * N * (a + 1),
                      hess + (size_t)s * (a + 1) * a, r, xi, x);
        free(rw);
      }
    } else if (mode == 0 && dense[target_seed[t]]) {
      int s = target_seed[t];
      orc_project_dense(N, used[s], basis + (size_t)s * N * (a + 1), aproj + (size_t)s * a * a, b,
                        NULL, x);
    } else if (mode == 0) {
      int s = target_seed[t];
      orc_project(N, used[s], lda, nxt[s], basis + (size_t)s * N * (a + 1),
                  hess + (size_t)s * (a + 1) * a, b, NULL, x);
    } else if (mode == 2) {
      memcpy(x, mt, sizeof(double) * N);
    } else if (mode == 3) {
      int s = target_seed[t];
      orc_project_galerkin(H, W, C, used[s], basis + (size_t)s * N * (a + 1), b, NULL, x);
    }
    if (tgt_x0res) {
      orc_apply(H, W, C, x, r);
      double rn = 0.0;
      for (int k = 0; k < N; ++k) rn += (b[k] - r[k]) * (b[k] - r[k]);
      tgt_x0res[t] = sqrt(rn) / nrm2(N, b);
    }
    tgt_status[t] = orc_gmres(H, W, C, b, x, tol_ref, m_ref, maxit, &tgt_it[t], &tgt_res[t],
                              NULL, 0, NULL, NULL, NULL, NULL, 0);
    for (int k = 1; k < K; ++k) {               /* Picard iterations, as for the seeds */
      int it = 0;
      orc_coeffs(H, W, g2, dt, h, x, NULL, NULL, C);
      tgt_status[t] = orc_gmres(H, W, C, b, x, tol_ref, m_ref, maxit, &it, &tgt_res[t], NULL, 0,
                                NULL, NULL, NULL, NULL, 0);
      tgt_it[t] += it;
    }
    memcpy(mt, x, sizeof(double) * N);
    free(C); free(b); free(x); free(r);
  }
  free(basis); free(hess); free(aproj); free(used); free(nxt); free(dense); free(mprev);
}


/*
 * Score of a solved timestep by central differences (end of Sec. 2.3), with
 * the zero padding of the discretisation outside the grid:
 *   sx(i,j) = (m_{i+1,j} - m_{i-1,j}) / (2h),   sy(i,j) = (m_{i,j+1} - m_{i,j-1}) / (2h).
 * The printed formula divides by 2; a central-difference derivative with grid
 * spacing h divides by 2h, which is what is used here.
 */
void orc_score(int H, int W, double h, const double* m, double* sx, double* sy) {
  for (int i = 0; i < W; ++i)
    for (int j = 0; j < H; ++j) {
      sx[i * H + j] = (at(m, H, W, i + 1, j) - at(m, H, W, i - 1, j)) / (2.0 * h);
      sy[i * H + j] = (at(m, H, W, i, j + 1) - at(m, H, W, i, j - 1)) / (2.0 * h);
    }
}

/*
 * One explicit (forward Euler) step of the probability-flow ODE of Sec. 4.1,
 * dx/dt = f - g^2/2 grad m, with f = 0:
 *   x^n = x^{n-1} + dt * (-(g^{n-1})^2 / 2) * grad m^{n-1},
 * for the two components (ex, ey) of x, in place.  g2prev = (g^{n-1})^2.
 */
void orc_embed_step(int N, double dt, double g2prev, const double* sx, const double* sy, double* ex,
                    double* ey) {
  for (int p = 0; p < N; ++p) {
    ex[p] += dt * (-0.5 * g2prev * sx[p]);
    ey[p] += dt * (-0.5 * g2prev * sy[p]);
  }
}


/* Threads of the OpenMP loops over independent systems (benchmark control;
 * no arithmetic changes). */
void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
