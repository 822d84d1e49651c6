/*
 * FP64 CPU oracle for the ridge-regularised dual of a matching LP.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this code; the library's product path
 * never calls it and shares no code with it.
 *
 * What it computes (DuaLip-GPU technical report, arXiv 2603.04621):
 *   LP (Eq. 1):            min c^T x  s.t.  A x <= b,  x in C
 *   smoothed dual (Eq. 2): g(mu) = min_{x in C} c^T x + (gamma/2)||x||_W^2 + mu^T (A x - b)
 *   Danskin gradient (Section 3.1): grad g(mu) = A x*(mu) - b,
 *                          x*(mu) = Pi_C( -(A^T mu + c) / gamma )
 *   matching structure (Section 3.2, Eqs. 3-5 and Definition 1): with one
 *   family A = [D_1 ... D_I], D_i = diag(a_i.), so (A^T mu)_ij = a_ij mu_j and
 *   (A x)_j = sum_i a_ij x_ij; with m families each source block stacks m
 *   diagonal blocks D_ki (rows k J + j); C = product over sources of
 *   {x_i >= 0, sum_j x_ij <= 1} (or the unit box).
 *   primal scaling (Section 5.1, "Primal scaling", view (i)): the ridge term
 *   becomes (gamma/2) sum w_e x_e^2 with w_e = v_e^2, v_e = |a_e| (1 where a_e = 0).
 *   Jacobi row normalisation (Section 5.1): D_j = ||A'_j||^-1 with the row norm
 *   taken in the metric of the ridge term, 1 for an empty or all-zero row.
 *
 * Everything is double precision; float inputs are widened exactly.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2

/* ---------------------------------------------------------------------- */
/* Compensated summation (Neumaier 1974, improved Kahan-Babuska).          */
typedef struct { double s, comp; } nsum_t;
static inline void nsum_add(nsum_t* a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->comp += (a->s - t) + v;
  else a->comp += (v - t) + a->s;
  a->s = t;
}
static inline double nsum_get(const nsum_t* a) { return a->s + a->comp; }

/* ---------------------------------------------------------------------- */
/* Per-source projection (Section 3.2, Eqs. 4-5; Section 3.1 for x*).
 *
 * The block problem for one source, with r_e = -(c_e + a_e mu_j) and
 * alpha_e = 1 / (gamma w_e), is
 *     min_x  sum_e [ x_e^2 / (2 alpha_e) - r_e x_e ]   s.t. x >= 0, sum_e x_e <= 1.
 * Its KKT conditions give x_e = alpha_e (r_e - tau)_+ with a multiplier
 * tau >= 0 of the sum constraint: tau = 0 when sum_e alpha_e (r_e)_+ <= 1,
 * else the unique tau > 0 with sum_e alpha_e (r_e - tau)_+ = 1.  For w = 1
 * this is the Euclidean projection of s = r / gamma onto the set.
 */
typedef struct { double r, alpha; } ra_t;
static int cmp_r_desc(const void* p, const void* q) {
  double a = ((const ra_t*)p)->r, b = ((const ra_t*)q)->r;
  return (a < b) - (a > b);
}

/* Exact threshold by sorting (Held, Wolfe and Crowder 1974; Duchi et al. 2008),
 * written for per-coordinate weights: with r sorted in decreasing order and
 * tau_k = (sum_{l<=k} alpha_l r_l - 1) / sum_{l<=k} alpha_l, the active set is
 * the longest prefix k with r_k > tau_k. */
static double tau_sort(int64_t n, const double* r, const double* alpha, ra_t* buf) {
  double s0 = 0.0;
  for (int64_t e = 0; e < n; ++e) if (r[e] > 0) s0 += alpha[e] * r[e];
  if (s0 <= 1.0) return 0.0;
  for (int64_t e = 0; e < n; ++e) { buf[e].r = r[e]; buf[e].alpha = alpha[e]; }
  qsort(buf, (size_t)n, sizeof(ra_t), cmp_r_desc);
  double sr = 0.0, sa = 0.0, tau = 0.0;
  for (int64_t k = 0; k < n; ++k) {
    double sr2 = sr + buf[k].alpha * buf[k].r, sa2 = sa + buf[k].alpha;
    double tk = (sr2 - 1.0) / sa2;
    if (buf[k].r > tk) { sr = sr2; sa = sa2; tau = tk; }
    else break;
  }
  return tau;
}

/* Exact threshold by Michelot's finite algorithm (Michelot 1986), started
 * from the set {r_e > 0}, which contains the active set whenever tau > 0:
 * repeatedly set tau to the value that makes the linear sum over the current
 * set equal to 1 and drop the members with r_e <= tau, until no member drops. */
static double tau_michelot(int64_t n, const double* r, const double* alpha, unsigned char* in) {
  double s0 = 0.0;
  for (int64_t e = 0; e < n; ++e) if (r[e] > 0) s0 += alpha[e] * r[e];
  if (s0 <= 1.0) return 0.0;
  for (int64_t e = 0; e < n; ++e) in[e] = r[e] > 0;
  double tau = 0.0;
  for (;;) {
    double sr = 0.0, sa = 0.0;
    for (int64_t e = 0; e < n; ++e) if (in[e]) { sr += alpha[e] * r[e]; sa += alpha[e]; }
    tau = (sr - 1.0) / sa;
    int changed = 0;
    for (int64_t e = 0; e < n; ++e) if (in[e] && !(r[e] > tau)) { in[e] = 0; changed = 1; }
    if (!changed) break;
  }
  return tau;
}

int oracle_project(int64_t n, const double* r, const double* alpha, int method, double* x,
                   double* tau_out) {
  if (n < 0) return OR_EINVAL;
  double tau = 0.0;
  if (n > 0) {
    if (method == 0) {
      ra_t* buf = (ra_t*)malloc(sizeof(ra_t) * (size_t)n);
      if (!buf) return OR_ENOMEM;
      tau = tau_sort(n, r, alpha, buf);
      free(buf);
    } else {
      unsigned char* in = (unsigned char*)malloc((size_t)n);
      if (!in) return OR_ENOMEM;
      tau = tau_michelot(n, r, alpha, in);
      free(in);
    }
  }
  for (int64_t e = 0; e < n; ++e) x[e] = r[e] > tau ? alpha[e] * (r[e] - tau) : 0.0;
  if (tau_out) *tau_out = tau;
  return OR_OK;
}

/* ---------------------------------------------------------------------- */
/*
 * Constraint families (Section 3.2, Definition 1): with m families every
 * edge e = (i, j) has m coefficients a_{k,e} (k = 0..m-1, stored family-major,
 * a[k E + e]) and enters the m rows (k, j) of A, numbered k J + j: the dual,
 * the gradient and b have R = m J entries.  So
 *   (A^T mu)_e = sum_k a_{k,e} mu_{k J + j},  (A x)_{k J + j} = sum_{e -> j} a_{k,e} x_e.
 * m = 1 is the single family used everywhere else.
 */
typedef struct oracle_problem {
  int64_t I, E;
  int32_t J;       /* destinations */
  int32_t m;       /* constraint families */
  int64_t R;       /* rows of A: m J */
  const int64_t* off;
  const int32_t* dst;
  const float *c, *a, *b;
  int weighted;
  int box;         /* C = [0, 1]^E (the unit-box clamp) instead of per-source simplices */
  int64_t* tix;    /* edges in destination-major order, ascending edge index */
  int64_t* toff;   /* [J+1] */
  int64_t dmax;
} oracle_problem;

void oracle_destroy(oracle_problem* p) {
  if (!p) return;
  free(p->tix);
  free(p->toff);
  free(p);
}

oracle_problem* oracle_create_multi(int64_t I, int32_t J, int32_t m, const int64_t* off,
                                    const int32_t* dst, const float* c, const float* a,
                                    const float* b, int weighted) {
  if (I < 0 || J < 0 || m < 1 || (I > 0 && !off)) return NULL;
  oracle_problem* p = (oracle_problem*)calloc(1, sizeof(oracle_problem));
  if (!p) return NULL;
  p->I = I; p->J = J; p->off = off; p->dst = dst; p->c = c; p->a = a; p->b = b;
  p->m = m;
  p->R = (int64_t)m * J;
  p->weighted = weighted;
  p->E = I > 0 ? off[I] : 0;
  for (int64_t i = 0; i < I; ++i) {
    int64_t d = off[i + 1] - off[i];
    if (d > p->dmax) p->dmax = d;
  }
  /* destination-major index by a stable counting sort */
  p->toff = (int64_t*)calloc((size_t)J + 1, sizeof(int64_t));
  p->tix = (int64_t*)malloc(sizeof(int64_t) * (size_t)(p->E > 0 ? p->E : 1));
  if (!p->toff || !p->tix) { oracle_destroy(p); return NULL; }
  for (int64_t e = 0; e < p->E; ++e) p->toff[dst[e] + 1]++;
  for (int32_t j = 0; j < J; ++j) p->toff[j + 1] += p->toff[j];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * ((size_t)J + 1));
  if (!fill) { oracle_destroy(p); return NULL; }
  memcpy(fill, p->toff, sizeof(int64_t) * ((size_t)J + 1));
  for (int64_t e = 0; e < p->E; ++e) p->tix[fill[dst[e]]++] = e;
  free(fill);
  return p;
}

oracle_problem* oracle_create(int64_t I, int32_t J, const int64_t* off, const int32_t* dst,
                              const float* c, const float* a, const float* b, int weighted) {
  return oracle_create_multi(I, J, 1, off, dst, c, a, b, weighted);
}

/* coefficient of edge e in family k */
static inline double coef(const oracle_problem* p, int k, int64_t e) {
  return (double)p->a[(int64_t)k * p->E + e];
}

/* Switch the simple constraint set to the unit box [0, 1]^E (Section 6's
 * unit-box clamp map).  The block problem then separates by edge: each x_e
 * minimises x^2 / (2 alpha_e) - r_e x over [0, 1], so x_e = min(1, alpha_e (r_e)_+). */
void oracle_set_box(oracle_problem* p, int box) { p->box = box ? 1 : 0; }

/* ridge weight of an edge with primal scaling: w_e = v_e^2 with v_e the norm of
 * the edge's column of A, sum_k a_{k,e}^2 (1 where the column is zero); 1
 * without primal scaling */
static inline double edge_w(const oracle_problem* p, int64_t e) {
  if (!p->weighted) return 1.0;
  double s = 0.0;
  for (int k = 0; k < p->m; ++k) s += coef(p, k, e) * coef(p, k, e);
  return s != 0.0 ? s : 1.0;
}

/* Jacobi row scale D_r = (sum_{e in row r} a_{k,e}^2 / w_e)^(-1/2) for row
 * r = k J + j, 1 for a zero row. */
int oracle_row_scale(const oracle_problem* p, double* D) {
  for (int k = 0; k < p->m; ++k)
    for (int32_t j = 0; j < p->J; ++j) {
      nsum_t s = {0, 0};
      for (int64_t t = p->toff[j]; t < p->toff[j + 1]; ++t) {
        int64_t e = p->tix[t];
        double av = coef(p, k, e);
        nsum_add(&s, av * av / edge_w(p, e));
      }
      double n2 = nsum_get(&s);
      D[(int64_t)k * p->J + j] = n2 > 0.0 ? 1.0 / sqrt(n2) : 1.0;
    }
  return OR_OK;
}

/* Squared spectral norm of D A W^-1/2 (D = I when NULL).  Rows of different
 * destinations share no column, so D A W^-1 A^T D is block diagonal with one
 * m x m block per destination j, M_kl = D_kj D_lj sum_{e -> j} a_{k,e} a_{l,e} / w_e;
 * the norm is the largest eigenvalue over the blocks (power iteration on each
 * positive semidefinite block; with one family the block is that one entry).
 * L = the norm / gamma bounds the Lipschitz constant of grad g (Appendix A). */
double oracle_norm2_sq(const oracle_problem* p, const double* D /* NULL = unscaled */) {
  const int m = p->m;
  double best = 0.0;
  double* M = (double*)calloc((size_t)m * m, sizeof(double));
  double* v = (double*)malloc(sizeof(double) * (size_t)m);
  double* u = (double*)malloc(sizeof(double) * (size_t)m);
  if (!M || !v || !u) { free(M); free(v); free(u); return -1.0; }
  for (int32_t j = 0; j < p->J; ++j) {
    memset(M, 0, sizeof(double) * (size_t)m * m);
    for (int64_t t = p->toff[j]; t < p->toff[j + 1]; ++t) {
      int64_t e = p->tix[t];
      double w = edge_w(p, e);
      for (int k = 0; k < m; ++k)
        for (int l = 0; l < m; ++l) M[k * m + l] += coef(p, k, e) * coef(p, l, e) / w;
    }
    if (D)
      for (int k = 0; k < m; ++k)
        for (int l = 0; l < m; ++l)
          M[k * m + l] *= D[(int64_t)k * p->J + j] * D[(int64_t)l * p->J + j];
    double lam = 0.0;
    if (m == 1) {
      lam = M[0];
    } else {
      for (int k = 0; k < m; ++k) v[k] = 1.0 + 0.1 * k;
      for (int it = 0; it < 500; ++it) {
        double nrm = 0.0;
        for (int k = 0; k < m; ++k) {
          u[k] = 0.0;
          for (int l = 0; l < m; ++l) u[k] += M[k * m + l] * v[l];
          nrm += u[k] * u[k];
        }
        nrm = sqrt(nrm);
        if (nrm == 0.0) break;
        for (int k = 0; k < m; ++k) v[k] = u[k] / nrm;
        lam = nrm;
      }
    }
    if (lam > best) best = lam;
  }
  free(M); free(v); free(u);
  return best;
}

/*
 * One evaluation of the smoothed dual at mu (original coordinates).
 * Outputs (any may be NULL): x[E], ax[J] = A x, grad[J] = A x - b and
 *   scal[0] = g(mu)                                  (Eq. 2)
 *   scal[1] = c^T x                                  (LP objective at x)
 *   scal[2] = (gamma/2) sum_e w_e x_e^2              (ridge term)
 *   scal[3] = ||(A x - b)_+||_2                      (Appendix A, Lemma 2)
 *   scal[4] = mu^T (A x - b)
 */
int oracle_eval(const oracle_problem* p, const double* mu, double gamma, int method, double* x_out,
                double* ax_out, double* grad_out, double* scal) {
  if (!(gamma > 0)) return OR_EINVAL;
  const int64_t I = p->I;
  const int32_t J = p->J;
  const int64_t R = p->R;
  double* x = x_out;
  double* xbuf = NULL;
  if (!x) {
    xbuf = (double*)malloc(sizeof(double) * (size_t)(p->E > 0 ? p->E : 1));
    if (!xbuf) return OR_ENOMEM;
    x = xbuf;
  }
  double* src_lin = (double*)calloc((size_t)(I > 0 ? I : 1), sizeof(double)); /* sum (c + a mu) x */
  double* src_cx = (double*)calloc((size_t)(I > 0 ? I : 1), sizeof(double));
  double* src_wxx = (double*)calloc((size_t)(I > 0 ? I : 1), sizeof(double));
  double* axv = (double*)malloc(sizeof(double) * (size_t)(R > 0 ? R : 1));
  int fail = !src_lin || !src_cx || !src_wxx || !axv;
  if (!fail) {
#pragma omp parallel
    {
      int64_t n = p->dmax > 0 ? p->dmax : 1;
      double* r = (double*)malloc(sizeof(double) * (size_t)n);
      double* al = (double*)malloc(sizeof(double) * (size_t)n);
      ra_t* buf = (ra_t*)malloc(sizeof(ra_t) * (size_t)n);
      unsigned char* in = (unsigned char*)malloc((size_t)n);
      if (!r || !al || !buf || !in) {
#pragma omp atomic write
        fail = 1;
      } else {
#pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < I; ++i) {
          int64_t e0 = p->off[i], d = p->off[i + 1] - e0;
          for (int64_t k = 0; k < d; ++k) {
            int64_t e = e0 + k;
            double am = 0.0;  /* (A^T mu)_e */
            for (int f = 0; f < p->m; ++f) am += coef(p, f, e) * mu[(int64_t)f * J + p->dst[e]];
            r[k] = -((double)p->c[e] + am);
            al[k] = 1.0 / (gamma * edge_w(p, e));
          }
          double tau = 0.0;
          if (!p->box) tau = method == 0 ? tau_sort(d, r, al, buf) : tau_michelot(d, r, al, in);
          nsum_t lin = {0, 0}, cx = {0, 0}, wxx = {0, 0};
          for (int64_t k = 0; k < d; ++k) {
            int64_t e = e0 + k;
            double xe = r[k] > tau ? al[k] * (r[k] - tau) : 0.0;
            if (p->box && xe > 1.0) xe = 1.0;
            x[e] = xe;
            nsum_add(&lin, -r[k] * xe);
            nsum_add(&cx, (double)p->c[e] * xe);
            nsum_add(&wxx, edge_w(p, e) * xe * xe);
          }
          src_lin[i] = nsum_get(&lin);
          src_cx[i] = nsum_get(&cx);
          src_wxx[i] = nsum_get(&wxx);
        }
      }
      free(r); free(al); free(buf); free(in);
    }
  }
  if (fail) {
    free(xbuf); free(src_lin); free(src_cx); free(src_wxx); free(axv);
    return OR_ENOMEM;
  }
  /* A x per row (family k, destination j), summed in ascending source order */
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t row = 0; row < R; ++row) {
    const int f = (int)(row / J);
    const int32_t j = (int32_t)(row % J);
    nsum_t s = {0, 0};
    for (int64_t k = p->toff[j]; k < p->toff[j + 1]; ++k) {
      int64_t e = p->tix[k];
      nsum_add(&s, coef(p, f, e) * x[e]);
    }
    axv[row] = nsum_get(&s);
  }
  nsum_t lin = {0, 0}, cx = {0, 0}, wxx = {0, 0}, mub = {0, 0}, inf = {0, 0}, comp = {0, 0};
  for (int64_t i = 0; i < I; ++i) {
    nsum_add(&lin, src_lin[i]);
    nsum_add(&cx, src_cx[i]);
    nsum_add(&wxx, src_wxx[i]);
  }
  for (int64_t row = 0; row < R; ++row) {
    double gj = axv[row] - (double)p->b[row];
    nsum_add(&mub, mu[row] * (double)p->b[row]);
    nsum_add(&comp, mu[row] * gj);
    if (gj > 0) nsum_add(&inf, gj * gj);
    if (ax_out) ax_out[row] = axv[row];
    if (grad_out) grad_out[row] = gj;
  }
  double reg = 0.5 * gamma * nsum_get(&wxx);
  if (scal) {
    scal[0] = nsum_get(&lin) + reg - nsum_get(&mub);
    scal[1] = nsum_get(&cx);
    scal[2] = reg;
    scal[3] = sqrt(nsum_get(&inf));
    scal[4] = nsum_get(&comp);
  }
  free(xbuf); free(src_lin); free(src_cx); free(src_wxx); free(axv);
  return OR_OK;
}

/* ---------------------------------------------------------------------- */
/* Dual ascent (Section 5 and Appendix B).
 *
 * The paper runs a Nesterov-accelerated gradient ascent whose step follows a
 * running estimate of the local Lipschitz constant, capped by a maximum step
 * (Appendix B), on the row-normalised dual (Section 5.1), with gamma decayed
 * on a schedule and the step cap scaled in proportion to gamma (Section 5.1,
 * "Regularization decay"; Section 7 uses halving every 25 iterations).  The
 * cited Scala source is not part of the paper, so the iteration is fixed here
 * as follows (lam, y in normalised coordinates lam' with mu = D lam'):
 *   gamma_k = max(gamma_final, gamma_0 * 2^-floor(k / halve_every))
 *   on a change of gamma (restart on): t = 1, y = lam, no secant history
 *   G_k     = D (A x*(D y_k) - b)                 (gradient in lam')
 *   eta_max = max_step * gamma_k / gamma_0
 *   eta_k   = min(eta_max, ||y_k - y_{k-1}|| / ||G_k - G_{k-1}||)  (secant estimate)
 *             or min(init_step, eta_max) right after a (re)start
 *   adaptive restart (restart_on_decrease): if g(D y_k) < g(D y_{k-1}) at the
 *             same gamma, t_k = 1 (no momentum in the next point; the secant
 *             history is kept)
 *   lam_{k+1} = max(0, y_k + eta_k G_k)
 *   t_{k+1}   = (1 + sqrt(1 + 4 t_k^2)) / 2
 *   y_{k+1}   = max(0, lam_{k+1} + ((t_k - 1) / t_{k+1}) (lam_{k+1} - lam_k))
 * Stopping (checked after every check_every-th evaluation, at the final gamma):
 *   gap_rel    = |mu^T (A x - b)| / max(1, |p|, |g|), p = c^T x + ridge term
 *   infeas_rel = ||(A x - b)_+||_2 / max(1, ||b||_2)
 * both <= their tolerances.  The returned point is the last evaluated y.
 */
typedef struct {
  double gamma0, gamma_final;
  int32_t halve_every;
  double max_step, init_step;
  int32_t max_iters;
  double tol_gap, tol_infeas;
  int32_t check_every;
  int32_t row_normalize;
  int32_t restart_on_gamma_change;
  int32_t stop_on_tol;
  int32_t restart_on_decrease;
} oracle_solve_opts;

typedef struct {
  int32_t iters;
  int32_t converged;
  double dual, primal_lin, reg, infeas, gap_rel, infeas_rel, gamma;
  int32_t restarts;  /* adaptive restarts taken */
} oracle_solve_result;

#define TRACE_W 8

static double gamma_at(const oracle_solve_opts* o, int32_t k) {
  double g = o->gamma0 * ldexp(1.0, -(k / (o->halve_every > 0 ? o->halve_every : 1)));
  if (o->halve_every <= 0) g = o->gamma0;
  return g > o->gamma_final ? g : o->gamma_final;
}

int oracle_solve(const oracle_problem* p, const oracle_solve_opts* o, double* lambda_io,
                 oracle_solve_result* res, double* trace) {
  const int32_t J = (int32_t)p->R;  /* dual entries: one per row of A */
  if (!(o->gamma0 > 0) || !(o->gamma_final > 0) || o->max_iters < 0) return OR_EINVAL;
  size_t n = (size_t)(J > 0 ? J : 1);
  double *D = malloc(n * 8), *lam = malloc(n * 8), *y = malloc(n * 8), *yp = malloc(n * 8),
         *G = malloc(n * 8), *Gp = malloc(n * 8), *mu = malloc(n * 8), *grad = malloc(n * 8),
         *lamn = malloc(n * 8);
  if (!D || !lam || !y || !yp || !G || !Gp || !mu || !grad || !lamn) {
    free(D); free(lam); free(y); free(yp); free(G); free(Gp); free(mu); free(grad); free(lamn);
    return OR_ENOMEM;
  }
  if (o->row_normalize) oracle_row_scale(p, D);
  else for (int32_t j = 0; j < J; ++j) D[j] = 1.0;
  double bnorm = 0.0;
  for (int32_t j = 0; j < J; ++j) bnorm += (double)p->b[j] * (double)p->b[j];
  bnorm = sqrt(bnorm);
  for (int32_t j = 0; j < J; ++j) {
    double v = lambda_io[j] / D[j];
    lam[j] = v > 0 ? v : 0.0;
    y[j] = lam[j];
  }
  double t = 1.0, gprev = 0.0, obj_prev = 0.0;
  int have_prev = 0, converged = 0, rc = OR_OK, restarts = 0;
  int32_t k = 0, iters = 0;
  double scal[5] = {0, 0, 0, 0, 0}, gap_rel = 0.0, inf_rel = 0.0, gk = o->gamma0;
  for (k = 0; k < o->max_iters; ++k) {
    gk = gamma_at(o, k);
    if (k > 0 && gk != gprev && o->restart_on_gamma_change) {
      t = 1.0;
      memcpy(y, lam, n * 8);
      have_prev = 0;
    }
    gprev = gk;
    for (int32_t j = 0; j < J; ++j) mu[j] = D[j] * y[j];
    rc = oracle_eval(p, mu, gk, 0, NULL, NULL, grad, scal);
    if (rc) break;
    iters = k + 1;
    for (int32_t j = 0; j < J; ++j) G[j] = D[j] * grad[j];
    double pval = scal[1] + scal[2];
    double den = fmax(1.0, fmax(fabs(pval), fabs(scal[0])));
    gap_rel = fabs(scal[4]) / den;
    inf_rel = scal[3] / fmax(1.0, bnorm);
    if (trace) {
      double* tr = trace + (size_t)k * TRACE_W;
      tr[0] = gk; tr[1] = scal[0]; tr[2] = pval; tr[3] = scal[3];
      tr[4] = gap_rel; tr[5] = inf_rel; tr[6] = 0.0; tr[7] = scal[4];
    }
    int check = o->check_every > 0 ? ((k + 1) % o->check_every == 0) : 1;
    if (o->stop_on_tol && check && gk == o->gamma_final && gap_rel <= o->tol_gap &&
        inf_rel <= o->tol_infeas) {
      converged = 1;
      break;
    }
    if (k == o->max_iters - 1) break;
    double eta_max = o->max_step * gk / o->gamma0, eta;
    if (have_prev) {
      double dy = 0.0, dg = 0.0;
      for (int32_t j = 0; j < J; ++j) {
        double u = y[j] - yp[j], v = G[j] - Gp[j];
        dy += u * u; dg += v * v;
      }
      eta = dg > 0.0 ? fmin(eta_max, sqrt(dy) / sqrt(dg)) : eta_max;
    } else {
      eta = fmin(o->init_step, eta_max);
    }
    if (trace) trace[(size_t)k * TRACE_W + 6] = eta;
    /* the dual objective fell since the last evaluation at this gamma: drop
       the momentum (the secant history stays) */
    if (o->restart_on_decrease && have_prev && scal[0] < obj_prev) {
      t = 1.0;
      restarts++;
    }
    obj_prev = scal[0];
    double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    double beta = (t - 1.0) / tn;
    for (int32_t j = 0; j < J; ++j) {
      double v = y[j] + eta * G[j];
      lamn[j] = v > 0 ? v : 0.0;
    }
    memcpy(yp, y, n * 8);
    memcpy(Gp, G, n * 8);
    for (int32_t j = 0; j < J; ++j) {
      double v = lamn[j] + beta * (lamn[j] - lam[j]);
      y[j] = v > 0 ? v : 0.0;
      lam[j] = lamn[j];
    }
    t = tn;
    have_prev = 1;
  }
  if (rc == OR_OK) {
    for (int32_t j = 0; j < J; ++j) lambda_io[j] = mu[j];
    if (res) {
      res->iters = iters; res->converged = converged;
      res->dual = scal[0]; res->primal_lin = scal[1]; res->reg = scal[2]; res->infeas = scal[3];
      res->gap_rel = gap_rel; res->infeas_rel = inf_rel; res->gamma = gk;
      res->restarts = restarts;
    }
  }
  free(D); free(lam); free(y); free(yp); free(G); free(Gp); free(mu); free(grad); free(lamn);
  return rc;
}

int oracle_set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
  return omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}
