/*
 * Sequential (Gauss-Seidel) domain propagation with constraint marking,
 * Alg. 1 -- the paper's cpu_seq method.
 *
 * TEST INFRASTRUCTURE ONLY (see dp_oracle.c).  This file deliberately shares
 * no code with the round-synchronous oracle in dp_oracle.c: it uses the
 * bound-candidate formulas of Eq. 3a/3b as printed (minimum/maximum activity
 * plus the variable's own bound) instead of the residual form of Eq. 5, it
 * reads and writes bounds in place (a bound found for one constraint is seen
 * by the next one), and it visits only marked constraints.
 *
 * Its purpose is the limit-point cross-check of Sec. 1.1: iterated domain
 * propagation has a unique limit point, so a correct round-synchronous
 * implementation and this sequential one must reach the same bounds whenever
 * both converge (exactly on bounded pure-integer problems, and within the
 * comparison tolerance of Sec. 4.3 otherwise).
 *
 * Same readings as the round-synchronous oracle for the improvement
 * threshold, integer rounding epsilon, infinity threshold and feasibility
 * tolerance.  A "round" here is one pass over the constraint list; the
 * count includes the final pass that found no change.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static double seq_tol(double eps, double v) { return eps * fmax(1.0, fabs(v)); }

int orc_seq_propagate(int32_t m, int32_t n, const int64_t *row_ptr,
                      const int32_t *col, const double *val, const double *lb,
                      const double *ub, const uint8_t *vartype,
                      const double *lhs_in, const double *rhs_in,
                      int32_t max_rounds, double eps_int, double tau_rel,
                      double eps_feas, double inf_threshold, double *x_lo,
                      double *x_hi, int32_t *infeasible, int32_t *rounds) {
  if (m < 0 || n < 0) return -1;
  int64_t nnz = row_ptr[m];
  size_t mm = (size_t)(m > 0 ? m : 1);
  /* column-major copy of the pattern, used only for marking (Alg. 1) */
  int64_t *cptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  int32_t *crow = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  uint8_t *marked = (uint8_t *)malloc(mm);
  double *lhs = (double *)malloc(sizeof(double) * mm);
  double *rhs = (double *)malloc(sizeof(double) * mm);
  double *snap = NULL;
  int64_t maxlen = 0;
  for (int32_t i = 0; i < m; ++i)
    if (row_ptr[i + 1] - row_ptr[i] > maxlen) maxlen = row_ptr[i + 1] - row_ptr[i];
  snap = (double *)malloc(sizeof(double) * 2 * (size_t)(maxlen > 0 ? maxlen : 1));
  if (!cptr || !crow || !marked || !lhs || !rhs || !snap) {
    free(cptr); free(crow); free(marked); free(lhs); free(rhs); free(snap);
    return -4;
  }
  for (int64_t k = 0; k < nnz; ++k) cptr[col[k] + 1] += 1;
  for (int32_t j = 0; j < n; ++j) cptr[j + 1] += cptr[j];
  {
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!fill) { free(cptr); free(crow); free(marked); free(lhs); free(rhs); free(snap); return -4; }
    memcpy(fill, cptr, sizeof(int64_t) * ((size_t)n + 1));
    for (int32_t i = 0; i < m; ++i)
      for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) crow[fill[col[k]]++] = i;
    free(fill);
  }

  /* normalisation, as in the round-synchronous oracle */
  for (int32_t j = 0; j < n; ++j) {
    double l = lb[j], u = ub[j];
    if (isnan(l) || isnan(u) || l >= inf_threshold || u <= -inf_threshold) {
      free(cptr); free(crow); free(marked); free(lhs); free(rhs); free(snap);
      return isnan(l) || isnan(u) ? -3 : -1;
    }
    if (l <= -inf_threshold) l = -INFINITY;
    if (u >= inf_threshold) u = INFINITY;
    if (vartype[j]) {
      if (l > -INFINITY) l = ceil(l - eps_int);
      if (u < INFINITY) u = floor(u + eps_int);
    }
    x_lo[j] = l;
    x_hi[j] = u;
  }
  for (int32_t i = 0; i < m; ++i) {
    lhs[i] = lhs_in[i] <= -inf_threshold ? -INFINITY : lhs_in[i];
    rhs[i] = rhs_in[i] >= inf_threshold ? INFINITY : rhs_in[i];
    marked[i] = 1; /* mark all constraints */
  }

  *infeasible = 0;
  *rounds = 0;
  for (int32_t j = 0; j < n; ++j)
    if (x_lo[j] > x_hi[j] + (vartype[j] ? 0.0 : seq_tol(eps_feas, x_hi[j]))) *infeasible = 1;

  int found = 1;
  while (found && !*infeasible && *rounds < max_rounds) {
    found = 0;
    *rounds += 1;
    for (int32_t c = 0; c < m && !*infeasible; ++c) {
      if (!marked[c]) continue;
      marked[c] = 0;
      /* activities of constraint c (Eq. 2a/2b) with infinity counts; the
       * bounds used are snapshotted so that Eq. 3 adds back the very value
       * that went into the activity */
      double amin = 0.0, amax = 0.0;
      int nmin_inf = 0, nmax_inf = 0;
      int64_t b = row_ptr[c], e = row_ptr[c + 1];
      for (int64_t k = b; k < e; ++k) {
        double a = val[k];
        double lo = x_lo[col[k]], hi = x_hi[col[k]];
        double vmin = a > 0.0 ? lo : hi;
        double vmax = a > 0.0 ? hi : lo;
        snap[2 * (k - b)] = vmin;
        snap[2 * (k - b) + 1] = vmax;
        if (vmin == INFINITY || vmin == -INFINITY) nmin_inf++; else amin += a * vmin;
        if (vmax == INFINITY || vmax == -INFINITY) nmax_inf++; else amax += a * vmax;
      }
      /* Step 2 */
      if (nmin_inf == 0 && rhs[c] < INFINITY && amin > rhs[c] + seq_tol(eps_feas, rhs[c])) { *infeasible = 1; break; }
      if (nmax_inf == 0 && lhs[c] > -INFINITY && amax < lhs[c] - seq_tol(eps_feas, lhs[c])) { *infeasible = 1; break; }
      /* Step 3 for each variable of c, Eq. 3a/3b */
      for (int64_t k = b; k < e; ++k) {
        int32_t v = col[k];
        double a = val[k];
        double vmin = snap[2 * (k - b)], vmax = snap[2 * (k - b) + 1];
        int vmin_inf = (vmin == INFINITY || vmin == -INFINITY);
        int vmax_inf = (vmax == INFINITY || vmax == -INFINITY);
        /* from the right-hand side and the minimum activity */
        double c_rhs = NAN;
        if (rhs[c] < INFINITY) {
          if (nmin_inf == 0) c_rhs = (rhs[c] - amin) / a + vmin;
          else if (nmin_inf == 1 && vmin_inf) c_rhs = (rhs[c] - amin) / a;
        }
        /* from the left-hand side and the maximum activity */
        double c_lhs = NAN;
        if (lhs[c] > -INFINITY) {
          if (nmax_inf == 0) c_lhs = (lhs[c] - amax) / a + vmax;
          else if (nmax_inf == 1 && vmax_inf) c_lhs = (lhs[c] - amax) / a;
        }
        double newlo = a > 0.0 ? c_lhs : c_rhs; /* NAN = no candidate */
        double newhi = a > 0.0 ? c_rhs : c_lhs;
        if (vartype[v]) {
          if (!isnan(newlo)) newlo = ceil(newlo - eps_int);
          if (!isnan(newhi)) newhi = floor(newhi + eps_int);
        }
        if (!isnan(newlo) && fabs(newlo) >= inf_threshold) newlo = NAN;
        if (!isnan(newhi) && fabs(newhi) >= inf_threshold) newhi = NAN;
        int changed_v = 0;
        if (!isnan(newlo)) {
          double cur = x_lo[v];
          int better = cur == -INFINITY ||
                       (vartype[v] ? newlo > cur : newlo > cur + tau_rel * fmax(1.0, fabs(cur)));
          if (better) { x_lo[v] = newlo; changed_v = 1; }
        }
        if (!isnan(newhi)) {
          double cur = x_hi[v];
          int better = cur == INFINITY ||
                       (vartype[v] ? newhi < cur : newhi < cur - tau_rel * fmax(1.0, fabs(cur)));
          if (better) { x_hi[v] = newhi; changed_v = 1; }
        }
        if (changed_v) {
          found = 1;
          if (x_lo[v] > x_hi[v] + (vartype[v] ? 0.0 : seq_tol(eps_feas, x_hi[v]))) { *infeasible = 1; break; }
          /* mark all constraints that contain v */
          for (int64_t q = cptr[v]; q < cptr[v + 1]; ++q) marked[crow[q]] = 1;
        }
      }
    }
  }
  free(cptr); free(crow); free(marked); free(lhs); free(rhs); free(snap);
  return 0;
}
