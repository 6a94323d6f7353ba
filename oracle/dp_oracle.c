/*
 * Plain, single-threaded CPU oracle for round-synchronous domain propagation
 * of linear constraints  lhs <= A x <= rhs,  lb <= x <= ub  (Eq. 1).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: it exists so that tests, the smoke check and the CPU
 * baseline leg of the benchmark can check the CUDA path against a slow,
 * obviously correct restatement of the method.  It shares no code, header,
 * table or helper with the CUDA library.
 *
 * All arithmetic is IEEE binary64.  Build with -O2 -ffp-contract=off so that
 * the compiler never fuses a product and a sum on its own; every fused
 * multiply-add below is an explicit fma() call.
 *
 * What one round computes (Alg. 2, the schematic GPU-parallel algorithm, with
 * the round-synchronous reading: every row reads the bounds as they were at
 * the end of the previous round):
 *   1. per row, the minimum and maximum activity (Def. 1, Eq. 2a/2b), with
 *      infinite contributions counted apart from the finite sum (Sec. 3.4);
 *   2. per row, the infeasibility test of Step 2 (Sec. 1.1);
 *   3. per nonzero, the bound candidates of Eq. 3a/3b, written with the
 *      residual activities of Eq. 5a/5b (Sec. 3.4), integer candidates
 *      rounded (Step 3, last sentence);
 *   4. per variable, the best candidate that improves the old bound by more
 *      than the termination threshold (Sec. 1.1, last paragraph; Sec. 3.5);
 *   5. the empty-domain test that makes Steps 1-2 optional (Sec. 1.1).
 *
 * Readings of the paper where it is silent (the numbers are parameters):
 *   - improvement threshold tau_rel: a continuous lower-bound candidate c is
 *     accepted iff  L == -inf  or  c > L + tau_rel*max(1,|L|)  (upper bound
 *     mirrored); an integer candidate is accepted iff it is strictly better;
 *   - integer rounding: lower candidates ceil(c - eps_int), upper candidates
 *     floor(c + eps_int);
 *   - |value| >= inf_threshold means infinite; candidates of such magnitude
 *     are discarded;
 *   - feasibility tolerance eps_feas * max(1,|side|) for Step 2 and the
 *     crossing test (integer variables cross iff L > U);
 *   - the round count includes the final round that found no change.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_NAN (-3)
#define ORC_ERR_OOM (-4)

/* unit roundoff of binary64 */
static const double ORC_U = 1.1102230246251565e-16;

static double side_tol(double eps_feas, double side) {
  return eps_feas * fmax(1.0, fabs(side));
}

/*
 * Input normalisation applied once before round 1:
 *   |v| >= inf_threshold -> +-inf for bounds and sides;
 *   integer variables: lb = ceil(lb - eps_int), ub = floor(ub + eps_int)
 *   (Step 3 of Sec. 1.1 rounds integer bounds; we apply the same rounding to
 *   the given bounds so that every integer bound is integral from the start).
 * Rejects NaN anywhere and the contradictory infinities lb=+inf, ub=-inf,
 * lhs=+inf, rhs=-inf.
 */
int orc_normalise(int32_t m, int32_t n, double *lb, double *ub,
                  const uint8_t *vartype, double *lhs, double *rhs,
                  double eps_int, double inf_threshold) {
  for (int32_t j = 0; j < n; ++j) {
    if (isnan(lb[j]) || isnan(ub[j])) return ORC_ERR_NAN;
    if (lb[j] <= -inf_threshold) lb[j] = -INFINITY;
    if (lb[j] >= inf_threshold) return ORC_ERR_ARG;
    if (ub[j] >= inf_threshold) ub[j] = INFINITY;
    if (ub[j] <= -inf_threshold) return ORC_ERR_ARG;
    if (vartype[j]) {
      if (isfinite(lb[j])) lb[j] = ceil(lb[j] - eps_int);
      if (isfinite(ub[j])) ub[j] = floor(ub[j] + eps_int);
    }
  }
  for (int32_t i = 0; i < m; ++i) {
    if (isnan(lhs[i]) || isnan(rhs[i])) return ORC_ERR_NAN;
    if (lhs[i] <= -inf_threshold) lhs[i] = -INFINITY;
    if (lhs[i] >= inf_threshold) return ORC_ERR_ARG;
    if (rhs[i] >= inf_threshold) rhs[i] = INFINITY;
    if (rhs[i] <= -inf_threshold) return ORC_ERR_ARG;
  }
  return ORC_OK;
}

/*
 * Error-analysis side outputs of one round (all optional, pass NULL).
 * They are not part of the method.  A parity test needs them because the
 * activity sums of Eq. 2 may be summed in another order by a parallel
 * implementation: every decision that compares a rounded quantity with a
 * threshold (integer rounding, acceptance threshold, infinity threshold,
 * Step 2, the crossing test) is flagged as a "tie" when the quantity lies
 * within a rigorous bound on that reordering error of the threshold.
 *   lb_tie[j], ub_tie[j]  : 1 if a decision about this bound was a tie;
 *   lb_err[j], ub_err[j]  : bound on the reordering error of the new value
 *                           (0 when the bound did not change);
 *   inf_tie               : 1 if the infeasibility verdict was a tie.
 */
typedef struct {
  uint8_t *lb_tie, *ub_tie;
  double *lb_err, *ub_err;
  int32_t *inf_tie;
} orc_analysis;

/* distance from x to the nearest integer */
static double dist_int(double x) { return fabs(x - nearbyint(x)); }

/*
 * One propagation round (Alg. 2, loop body) from the state (L, U).
 * Writes the new state to (Lnew, Unew) -- which must not alias (L, U) --
 * and sets *changed and *infeasible.
 */
int orc_round(int32_t m, int32_t n, const int64_t *row_ptr,
              const int32_t *col, const double *val, const double *L,
              const double *U, const uint8_t *vartype, const double *lhs,
              const double *rhs, double eps_int, double tau_rel,
              double eps_feas, double inf_threshold, double *Lnew,
              double *Unew, int32_t *changed, int32_t *infeasible,
              uint8_t *lb_tie, uint8_t *ub_tie, double *lb_err,
              double *ub_err, int32_t *inf_tie) {
  orc_analysis an = {lb_tie, ub_tie, lb_err, ub_err, inf_tie};
  int analyse = (lb_tie && ub_tie && lb_err && ub_err && inf_tie);
  double *minfin = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  double *maxfin = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  int32_t *mininf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  int32_t *maxinf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  double *absmin = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  double *absmax = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  if (!minfin || !maxfin || !mininf || !maxinf || !absmin || !absmax) {
    free(minfin); free(maxfin); free(mininf); free(maxinf); free(absmin); free(absmax);
    return ORC_ERR_OOM;
  }
  *changed = 0;
  *infeasible = 0;
  if (analyse) {
    memset(an.lb_tie, 0, (size_t)n);
    memset(an.ub_tie, 0, (size_t)n);
    for (int32_t j = 0; j < n; ++j) an.lb_err[j] = an.ub_err[j] = 0.0;
    *an.inf_tie = 0;
  }

  /* --- 1. activities (Def. 1, Eq. 2a/2b) with infinity counts (Sec. 3.4) --- */
  for (int32_t i = 0; i < m; ++i) {
    double sfin_min = 0.0, sfin_max = 0.0, sabs_min = 0.0, sabs_max = 0.0;
    int32_t cinf_min = 0, cinf_max = 0;
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      int32_t j = col[k];
      double a = val[k];
      /* Def. 1: b = l if a > 0 else u for the minimum; swapped for the max */
      double bmin = (a > 0.0) ? L[j] : U[j];
      double bmax = (a > 0.0) ? U[j] : L[j];
      if (isinf(bmin)) {
        cinf_min += 1; /* contributes -inf to the minimum activity */
      } else {
        sfin_min = fma(a, bmin, sfin_min);
        sabs_min += fabs(a * bmin);
      }
      if (isinf(bmax)) {
        cinf_max += 1; /* contributes +inf to the maximum activity */
      } else {
        sfin_max = fma(a, bmax, sfin_max);
        sabs_max += fabs(a * bmax);
      }
    }
    minfin[i] = sfin_min;
    maxfin[i] = sfin_max;
    mininf[i] = cinf_min;
    maxinf[i] = cinf_max;
    absmin[i] = sabs_min;
    absmax[i] = sabs_max;

    /* --- 2. Step 2: the row cannot be satisfied --- */
    int64_t len = row_ptr[i + 1] - row_ptr[i];
    double e_min = 2.0 * (double)(len + 2) * ORC_U * sabs_min;
    double e_max = 2.0 * (double)(len + 2) * ORC_U * sabs_max;
    if (cinf_min == 0 && isfinite(rhs[i])) {
      double thr = rhs[i] + side_tol(eps_feas, rhs[i]);
      if (sfin_min > thr) *infeasible = 1;
      if (analyse && fabs(sfin_min - thr) <= e_min + 2.0 * ORC_U * fabs(thr)) *an.inf_tie = 1;
    }
    if (cinf_max == 0 && isfinite(lhs[i])) {
      double thr = lhs[i] - side_tol(eps_feas, lhs[i]);
      if (sfin_max < thr) *infeasible = 1;
      if (analyse && fabs(sfin_max - thr) <= e_max + 2.0 * ORC_U * fabs(thr)) *an.inf_tie = 1;
    }
  }

  /* --- 3./4. candidates per nonzero and their filtered application --- */
  for (int32_t j = 0; j < n; ++j) {
    Lnew[j] = L[j];
    Unew[j] = U[j];
  }
  for (int32_t i = 0; i < m; ++i) {
    int64_t len = row_ptr[i + 1] - row_ptr[i];
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      int32_t j = col[k];
      double a = val[k];
      double bmin = (a > 0.0) ? L[j] : U[j];
      double bmax = (a > 0.0) ? U[j] : L[j];

      /* residual activities, Eq. 5a/5b, with the exactly-one-infinity rule */
      double resmin, resmax;
      if (mininf[i] == 0)
        resmin = fma(-a, bmin, minfin[i]);
      else if (mininf[i] == 1 && isinf(bmin))
        resmin = minfin[i];
      else
        resmin = -INFINITY;
      if (maxinf[i] == 0)
        resmax = fma(-a, bmax, maxfin[i]);
      else if (maxinf[i] == 1 && isinf(bmax))
        resmax = maxfin[i];
      else
        resmax = INFINITY;

      /* Eq. 3a (a > 0) and Eq. 3b (a < 0) in residual form:
       *   from  a x_j <= rhs - resmin  and  a x_j >= lhs - resmax. */
      double lc = -INFINITY, uc = INFINITY;
      double lside = 0.0, uside = 0.0, lres = 0.0, ures = 0.0;
      if (a > 0.0) {
        if (isfinite(rhs[i]) && isfinite(resmin)) { uc = (rhs[i] - resmin) / a; uside = rhs[i]; ures = resmin; }
        if (isfinite(lhs[i]) && isfinite(resmax)) { lc = (lhs[i] - resmax) / a; lside = lhs[i]; lres = resmax; }
      } else {
        if (isfinite(rhs[i]) && isfinite(resmin)) { lc = (rhs[i] - resmin) / a; lside = rhs[i]; lres = resmin; }
        if (isfinite(lhs[i]) && isfinite(resmax)) { uc = (lhs[i] - resmax) / a; uside = lhs[i]; ures = resmax; }
      }

      /* bound on the reordering error of each raw candidate (analysis only):
       * the residual inherits the row sum's error, at most 2 gamma_(len+2)
       * times the absolute sum, plus the rounding of the subtraction and the
       * division, all divided by |a|. */
      double lerr = 0.0, uerr = 0.0;
      if (analyse) {
        double fa = fabs(a);
        if (isfinite(lc)) {
          double s = (a > 0.0) ? absmax[i] : absmin[i];
          double e_res = 2.0 * (double)(len + 2) * ORC_U * (s + fabs(a * bmax) + fabs(a * bmin));
          lerr = 2.0 * ((e_res + 2.0 * ORC_U * (fabs(lside) + fabs(lres))) / fa + 2.0 * ORC_U * fabs(lc));
        }
        if (isfinite(uc)) {
          double s = (a > 0.0) ? absmin[i] : absmax[i];
          double e_res = 2.0 * (double)(len + 2) * ORC_U * (s + fabs(a * bmax) + fabs(a * bmin));
          uerr = 2.0 * ((e_res + 2.0 * ORC_U * (fabs(uside) + fabs(ures))) / fa + 2.0 * ORC_U * fabs(uc));
        }
      }

      /* Step 3: integer candidates are rounded */
      if (vartype[j]) {
        if (isfinite(lc)) {
          if (analyse && dist_int(lc - eps_int) <= lerr) an.lb_tie[j] = 1;
          lc = ceil(lc - eps_int);
        }
        if (isfinite(uc)) {
          if (analyse && dist_int(uc + eps_int) <= uerr) an.ub_tie[j] = 1;
          uc = floor(uc + eps_int);
        }
      }

      /* candidates of infinite magnitude carry no information */
      if (isfinite(lc) && fabs(lc) >= inf_threshold) {
        if (analyse && fabs(fabs(lc) - inf_threshold) <= lerr) an.lb_tie[j] = 1;
        lc = -INFINITY;
      } else if (analyse && isfinite(lc) && fabs(fabs(lc) - inf_threshold) <= lerr) {
        an.lb_tie[j] = 1;
      }
      if (isfinite(uc) && fabs(uc) >= inf_threshold) {
        if (analyse && fabs(fabs(uc) - inf_threshold) <= uerr) an.ub_tie[j] = 1;
        uc = INFINITY;
      } else if (analyse && isfinite(uc) && fabs(fabs(uc) - inf_threshold) <= uerr) {
        an.ub_tie[j] = 1;
      }

      /* filtered update: only a candidate that improves the old bound by
       * more than the threshold becomes a new bound (Sec. 3.5) */
      if (isfinite(lc)) {
        int accept;
        if (L[j] == -INFINITY) {
          accept = 1;
        } else if (vartype[j]) {
          accept = lc > L[j];
        } else {
          double thr = L[j] + tau_rel * fmax(1.0, fabs(L[j]));
          accept = lc > thr;
          if (analyse && fabs(lc - thr) <= lerr + 2.0 * ORC_U * fabs(thr)) an.lb_tie[j] = 1;
        }
        if (accept) {
          if (lc > Lnew[j]) Lnew[j] = lc;
          *changed = 1;
          if (analyse && !vartype[j] && lerr > an.lb_err[j]) an.lb_err[j] = lerr;
        }
      }
      if (isfinite(uc)) {
        int accept;
        if (U[j] == INFINITY) {
          accept = 1;
        } else if (vartype[j]) {
          accept = uc < U[j];
        } else {
          double thr = U[j] - tau_rel * fmax(1.0, fabs(U[j]));
          accept = uc < thr;
          if (analyse && fabs(uc - thr) <= uerr + 2.0 * ORC_U * fabs(thr)) an.ub_tie[j] = 1;
        }
        if (accept) {
          if (uc < Unew[j]) Unew[j] = uc;
          *changed = 1;
          if (analyse && !vartype[j] && uerr > an.ub_err[j]) an.ub_err[j] = uerr;
        }
      }
    }
  }

  /* --- 5. empty domain: the new bounds cross (Sec. 1.1, Steps 1-2 remark) --- */
  for (int32_t j = 0; j < n; ++j) {
    double tol = vartype[j] ? 0.0 : side_tol(eps_feas, Unew[j]);
    if (Lnew[j] > Unew[j] + tol) *infeasible = 1;
    if (analyse && isfinite(Lnew[j]) && isfinite(Unew[j]) &&
        fabs(Lnew[j] - Unew[j] - tol) <= an.lb_err[j] + an.ub_err[j] + 2.0 * ORC_U * fabs(Unew[j]) &&
        (an.lb_err[j] > 0.0 || an.ub_err[j] > 0.0))
      *an.inf_tie = 1;
  }

  free(minfin); free(maxfin); free(mininf); free(maxinf); free(absmin); free(absmax);
  return ORC_OK;
}

/*
 * The full iteration (Alg. 2): normalise, then repeat rounds until a round
 * finds no change, finds the problem infeasible, or max_rounds rounds ran.
 * lb/ub/lhs/rhs are not modified; results go to lb_out/ub_out.
 * *rounds counts every executed round; *status is 1 when the cap was hit
 * while the last round still changed a bound, else 0.
 * If trace_lb/trace_ub are not NULL they receive the state after each round
 * (row r of a max_rounds x n array).
 */
int orc_propagate(int32_t m, int32_t n, const int64_t *row_ptr,
                  const int32_t *col, const double *val, const double *lb,
                  const double *ub, const uint8_t *vartype, const double *lhs,
                  const double *rhs, int32_t max_rounds, double eps_int,
                  double tau_rel, double eps_feas, double inf_threshold,
                  double *lb_out, double *ub_out, int32_t *infeasible,
                  int32_t *rounds, int32_t *status, double *trace_lb,
                  double *trace_ub) {
  if (m < 0 || n < 0 || max_rounds < 0) return ORC_ERR_ARG;
  size_t nn = (size_t)(n > 0 ? n : 1), mm = (size_t)(m > 0 ? m : 1);
  double *L = (double *)malloc(sizeof(double) * nn);
  double *U = (double *)malloc(sizeof(double) * nn);
  double *L2 = (double *)malloc(sizeof(double) * nn);
  double *U2 = (double *)malloc(sizeof(double) * nn);
  double *sl = (double *)malloc(sizeof(double) * mm);
  double *sr = (double *)malloc(sizeof(double) * mm);
  if (!L || !U || !L2 || !U2 || !sl || !sr) {
    free(L); free(U); free(L2); free(U2); free(sl); free(sr);
    return ORC_ERR_OOM;
  }
  memcpy(L, lb, sizeof(double) * (size_t)n);
  memcpy(U, ub, sizeof(double) * (size_t)n);
  memcpy(sl, lhs, sizeof(double) * (size_t)m);
  memcpy(sr, rhs, sizeof(double) * (size_t)m);
  int rc = orc_normalise(m, n, L, U, vartype, sl, sr, eps_int, inf_threshold);
  *infeasible = 0;
  *rounds = 0;
  *status = 0;
  int32_t changed = 0;
  for (int32_t r = 1; rc == ORC_OK && r <= max_rounds; ++r) {
    int32_t infeas = 0;
    rc = orc_round(m, n, row_ptr, col, val, L, U, vartype, sl, sr, eps_int,
                   tau_rel, eps_feas, inf_threshold, L2, U2, &changed,
                   &infeas, NULL, NULL, NULL, NULL, NULL);
    if (rc != ORC_OK) break;
    double *t = L; L = L2; L2 = t;
    t = U; U = U2; U2 = t;
    *rounds = r;
    if (trace_lb) memcpy(trace_lb + (size_t)(r - 1) * (size_t)n, L, sizeof(double) * (size_t)n);
    if (trace_ub) memcpy(trace_ub + (size_t)(r - 1) * (size_t)n, U, sizeof(double) * (size_t)n);
    if (infeas) { *infeasible = 1; break; }
    if (!changed) break;
  }
  if (rc == ORC_OK) {
    if (!*infeasible && changed && *rounds == max_rounds) *status = 1;
    memcpy(lb_out, L, sizeof(double) * (size_t)n);
    memcpy(ub_out, U, sizeof(double) * (size_t)n);
  }
  free(L); free(U); free(L2); free(U2); free(sl); free(sr);
  return rc;
}
