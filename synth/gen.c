/*
 * Seeded synthetic matching-LP instances (shared input generator).
 *
 * This file draws random problem data only: per-source degrees, distinct
 * destinations per source, edge costs c, constraint coefficients a and
 * destination budgets b.  It contains none of the dual-ascent arithmetic and
 * is used, unchanged, to feed both the FP64 CPU oracle and the CUDA path.
 *
 * Randomness is counter based: every source i owns its own SplitMix64 stream
 * keyed by (seed, purpose, i), so the output does not depend on the number of
 * threads or on the machine.  SplitMix64 is Steele, Lea and Flood,
 * "Fast splittable pseudorandom number generators" (OOPSLA 2014).
 *
 * Layout produced (source-major, the CSC-by-source layout of the paper's
 * Section 6, "Sparse tensor computation"):
 *   off[I+1] int64   edges of source i are off[i] .. off[i+1]-1
 *   dst[E]   int32   destination j of each edge, 0 <= j < J
 *   c[E]     float32 cost (minimisation sign, so values enter as -value)
 *   a[E]     float32 constraint coefficient a_ij
 *   b[J]     float32 budget b_j = frac * sum of a over the edges into j
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SYN_OK 0
#define SYN_EINVAL 1
#define SYN_ENOMEM 2

/* ---- SplitMix64 --------------------------------------------------------- */
static inline uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
typedef struct { uint64_t s; } rng_t;
static inline rng_t rng_for(uint64_t seed, uint64_t purpose, uint64_t idx) {
  rng_t r;
  r.s = sm_mix(sm_mix(seed ^ (purpose * 0xD1B54A32D192ED03ULL)) + idx * 0x9E3779B97F4A7C15ULL);
  return r;
}
static inline uint64_t rng_next(rng_t* r) {
  r->s += 0x9E3779B97F4A7C15ULL;
  return sm_mix(r->s);
}
/* uniform double in [0, 1) with 53 random bits */
static inline double rng_u01(rng_t* r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }
/* uniform double in (0, 1] */
static inline double rng_u01_open0(rng_t* r) { return ((double)(rng_next(r) >> 11) + 1.0) * 0x1.0p-53; }
/* standard normal by the Box-Muller transform */
static inline double rng_normal(rng_t* r) {
  double u1 = rng_u01_open0(r), u2 = rng_u01(r);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2);
}
/* uniform integer in [0, n) (n > 0), by rejection to avoid modulo bias */
static inline uint64_t rng_below(rng_t* r, uint64_t n) {
  uint64_t lim = UINT64_MAX - (UINT64_MAX % n);
  uint64_t v;
  do { v = rng_next(r); } while (v >= lim);
  return v % n;
}

enum { PURPOSE_DEG = 1, PURPOSE_EDGE = 2, PURPOSE_PERM = 3, PURPOSE_RHO = 4 };
enum { DEG_FIXED = 0, DEG_POISSON = 1, DEG_UNIFORM = 2 };
enum { DST_UNIFORM = 0, DST_ZIPF = 1 };
enum { C_NEG_UNIFORM = 0, C_NEG_LOGNORMAL = 1 };

/* ---- degrees ------------------------------------------------------------ */
/*
 * kind DEG_FIXED:   d = p1
 * kind DEG_POISSON: d ~ Poisson(p1), by inversion of a precomputed CDF
 * kind DEG_UNIFORM: d ~ UniformInt[p1, p2]
 * then clipped to [lo, hi].
 */
int synth_degrees(int64_t I, uint64_t seed, int kind, double p1, double p2, int64_t lo, int64_t hi,
                  int64_t* deg) {
  if (I < 0 || lo < 0 || hi < lo) return SYN_EINVAL;
  double* cdf = NULL;
  int64_t ncdf = 0;
  if (kind == DEG_POISSON) {
    if (!(p1 > 0)) return SYN_EINVAL;
    ncdf = (int64_t)(p1 + 40.0 * sqrt(p1) + 64.0);
    cdf = (double*)malloc(sizeof(double) * (size_t)ncdf);
    if (!cdf) return SYN_ENOMEM;
    /* pmf(k) = exp(k log p1 - p1 - lgamma(k+1)) */
    double acc = 0.0;
    for (int64_t k = 0; k < ncdf; ++k) {
      acc += exp((double)k * log(p1) - p1 - lgamma((double)k + 1.0));
      cdf[k] = acc;
    }
  } else if (kind != DEG_FIXED && kind != DEG_UNIFORM) {
    return SYN_EINVAL;
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < I; ++i) {
    rng_t r = rng_for(seed, PURPOSE_DEG, (uint64_t)i);
    int64_t d;
    if (kind == DEG_FIXED) {
      d = (int64_t)p1;
    } else if (kind == DEG_UNIFORM) {
      int64_t a = (int64_t)p1, b = (int64_t)p2;
      d = a + (int64_t)rng_below(&r, (uint64_t)(b - a + 1));
    } else {
      double u = rng_u01(&r) * cdf[ncdf - 1];
      int64_t L = 0, H = ncdf - 1; /* first k with cdf[k] > u */
      while (L < H) {
        int64_t m = (L + H) / 2;
        if (cdf[m] > u) H = m; else L = m + 1;
      }
      d = L;
    }
    if (d < lo) d = lo;
    if (d > hi) d = hi;
    deg[i] = d;
  }
  free(cdf);
  return SYN_OK;
}

/* ---- edges -------------------------------------------------------------- */
typedef struct {
  uint32_t* key;  /* stored destination + 1, 0 = empty */
  uint32_t* stamp;
  uint32_t cur;
  uint32_t mask;
} pickset_t;

static int pickset_init(pickset_t* s, int64_t dmax) {
  uint32_t n = 64;
  while ((int64_t)n < 4 * dmax) n <<= 1;
  s->key = (uint32_t*)calloc(n, sizeof(uint32_t));
  s->stamp = (uint32_t*)calloc(n, sizeof(uint32_t));
  s->cur = 0;
  s->mask = n - 1;
  return (s->key && s->stamp) ? 0 : -1;
}
static void pickset_free(pickset_t* s) { free(s->key); free(s->stamp); }
static void pickset_clear(pickset_t* s) { s->cur++; }
/* returns 1 if inserted, 0 if already present */
static int pickset_insert(pickset_t* s, uint32_t v) {
  uint32_t h = (v * 2654435761u) & s->mask;
  for (;;) {
    if (s->stamp[h] != s->cur) { s->stamp[h] = s->cur; s->key[h] = v + 1; return 1; }
    if (s->key[h] == v + 1) return 0;
    h = (h + 1) & s->mask;
  }
}
static int pickset_has(pickset_t* s, uint32_t v) {
  uint32_t h = (v * 2654435761u) & s->mask;
  for (;;) {
    if (s->stamp[h] != s->cur) return 0;
    if (s->key[h] == v + 1) return 1;
    h = (h + 1) & s->mask;
  }
}

/*
 * Fill dst, c, a for every source.  Destinations of one source are distinct
 * (degree must be <= J).  Uniform law: j uniform over [0, J).  Zipf law: a
 * rank k in 1..J with P(k) proportional to k^(-zipf_s), mapped through a
 * seeded random permutation to a destination id, so ids carry no hotness
 * order.  Repeats are rejected; after 64*d + 64 rejected draws the rest of
 * the source's destinations are drawn uniformly among those not yet picked.
 */
int synth_edges(int64_t I, int32_t J, const int64_t* off, uint64_t seed, int dst_law, double zipf_s,
                int c_law, double a_lo, double a_hi, int32_t* dst, float* c, float* a) {
  if (I < 0 || J <= 0) return SYN_EINVAL;
  int64_t dmax = 0;
  for (int64_t i = 0; i < I; ++i) {
    int64_t d = off[i + 1] - off[i];
    if (d < 0 || d > J) return SYN_EINVAL;
    if (d > dmax) dmax = d;
  }
  double* zcdf = NULL;
  int32_t* perm = NULL;
  if (dst_law == DST_ZIPF) {
    zcdf = (double*)malloc(sizeof(double) * (size_t)J);
    perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)J);
    if (!zcdf || !perm) { free(zcdf); free(perm); return SYN_ENOMEM; }
    double acc = 0.0;
    for (int32_t k = 0; k < J; ++k) { acc += pow((double)(k + 1), -zipf_s); zcdf[k] = acc; }
    for (int32_t k = 0; k < J; ++k) perm[k] = k;
    rng_t r = rng_for(seed, PURPOSE_PERM, 0);
    for (int32_t k = J - 1; k > 0; --k) { /* Fisher-Yates */
      int32_t m = (int32_t)rng_below(&r, (uint64_t)k + 1);
      int32_t t = perm[k]; perm[k] = perm[m]; perm[m] = t;
    }
  } else if (dst_law != DST_UNIFORM) {
    return SYN_EINVAL;
  }
  int err = 0;
#pragma omp parallel
  {
    pickset_t ps;
    int ok = pickset_init(&ps, dmax) == 0;
    if (!ok) {
#pragma omp atomic write
      err = 1;
    }
#pragma omp for schedule(dynamic, 1024)
    for (int64_t i = 0; i < I; ++i) {
      if (!ok) continue;
      rng_t r = rng_for(seed, PURPOSE_EDGE, (uint64_t)i);
      int64_t e0 = off[i], d = off[i + 1] - off[i];
      pickset_clear(&ps);
      int64_t got = 0, tries = 0;
      while (got < d && tries < 64 * d + 64) {
        int32_t j;
        if (dst_law == DST_ZIPF) {
          double u = rng_u01(&r) * zcdf[J - 1];
          int32_t L = 0, H = J - 1;
          while (L < H) {
            int32_t m = L + (H - L) / 2;
            if (zcdf[m] > u) H = m; else L = m + 1;
          }
          j = perm[L];
        } else {
          j = (int32_t)rng_below(&r, (uint64_t)J);
        }
        ++tries;
        if (pickset_insert(&ps, (uint32_t)j)) dst[e0 + got++] = j;
      }
      if (got < d) { /* fallback: uniform over the destinations not yet picked */
        int64_t left = (int64_t)J - got;
        while (got < d) {
          int64_t pick = (int64_t)rng_below(&r, (uint64_t)left), seen = 0;
          for (int32_t j = 0; j < J; ++j) {
            if (pickset_has(&ps, (uint32_t)j)) continue;
            if (seen++ == pick) { pickset_insert(&ps, (uint32_t)j); dst[e0 + got++] = j; break; }
          }
          --left;
        }
      }
      for (int64_t k = 0; k < d; ++k) {
        double cv = (c_law == C_NEG_LOGNORMAL) ? -exp(rng_normal(&r)) : -rng_u01(&r);
        double av = a_lo + (a_hi - a_lo) * rng_u01(&r);
        c[e0 + k] = (float)cv;
        a[e0 + k] = (float)av;
      }
    }
    if (ok) pickset_free(&ps);
  }
  free(zcdf);
  free(perm);
  return err ? SYN_ENOMEM : SYN_OK;
}

/* b_j = frac * sum of a_e over the edges e into j, summed in edge order in
 * double on one thread (so the result never depends on the thread count). */
int synth_budgets(int64_t E, int32_t J, const int32_t* dst, const float* a, double frac, float* b) {
  double* acc = (double*)calloc((size_t)J, sizeof(double));
  if (!acc) return SYN_ENOMEM;
  for (int64_t e = 0; e < E; ++e) acc[dst[e]] += (double)a[e];
  for (int32_t j = 0; j < J; ++j) b[j] = (float)(frac * acc[j]);
  free(acc);
  return SYN_OK;
}

/* Greedy-load budgets (the paper's Appendix B right-hand-side rule): every
 * source sends the coefficient of its largest-a edge (first one on ties) to
 * that edge's destination; l_j sums what j receives, and
 * b_j = rho_j (l_j + eps) with rho_j ~ U[rho_lo, rho_hi] drawn per destination. */
int synth_budgets_greedy(int64_t I, int32_t J, const int64_t* off, const int32_t* dst,
                         const float* a, uint64_t seed, double rho_lo, double rho_hi, double eps,
                         float* b) {
  double* acc = (double*)calloc((size_t)J, sizeof(double));
  if (!acc) return SYN_ENOMEM;
  for (int64_t i = 0; i < I; ++i) {
    int64_t best = -1;
    for (int64_t e = off[i]; e < off[i + 1]; ++e)
      if (best < 0 || a[e] > a[best]) best = e;
    if (best >= 0) acc[dst[best]] += (double)a[best];
  }
  for (int32_t j = 0; j < J; ++j) {
    rng_t r = rng_for(seed, PURPOSE_RHO, (uint64_t)j);
    double rho = rho_lo + (rho_hi - rho_lo) * rng_u01(&r);
    b[j] = (float)(rho * (acc[j] + eps));
  }
  free(acc);
  return SYN_OK;
}

/* ---- the paper's Appendix B generator ------------------------------------ */
/*
 * Resource-major draw (Appendix B, "Synthetic LP construction"), stored
 * source-major: requests are the sources i, resources the destinations j.
 * The paper names the families of its laws but not their parameters; every
 * one is an argument here:
 *   breadth_j ~ LogNormal(0, sig_breadth), p_j = breadth_j / sum_k breadth_k
 *   K_j ~ Poisson(p_j I nu), truncated at I (nu: mean edges per request);
 *         by inversion for means below 64, else by the rounded normal
 *         approximation mean + sqrt(mean) N(0,1) (clipped to [0, I])
 *   the K_j requests of j: distinct, uniform (Floyd's sampling)
 *   v_j ~ LogNormal(0, sig_v), u_i ~ LogNormal(0, sig_u),
 *   eps_ij ~ LogNormal(0, sig_eps): value_ij = min(v_j u_i eps_ij, c_max)
 *   s_j ~ LogNormal(mu_s, sig_s): a_ij = s_j value_ij
 *   c_ij = -value_ij (values enter the minimisation with their sign flipped)
 * appb_degrees fills K[J] and returns E = sum K; appb_fill then writes the
 * source-major arrays (off[I+1], dst, c, a; within a request, its resources
 * in increasing id).  Every random number is keyed by (seed, purpose, index),
 * so the result does not depend on the thread count.
 */
enum { PURPOSE_APPB_BREADTH = 11, PURPOSE_APPB_K = 12, PURPOSE_APPB_PICK = 13,
       PURPOSE_APPB_V = 14, PURPOSE_APPB_U = 15, PURPOSE_APPB_S = 16 };

static int cmp_u32(const void* p, const void* q) {
  uint32_t x = *(const uint32_t*)p, y = *(const uint32_t*)q;
  return (x > y) - (x < y);
}

static int64_t poisson_draw(rng_t* r, double mean, int64_t cap) {
  int64_t k;
  if (mean <= 0.0) return 0;
  if (mean < 64.0) {  /* inversion: the first k with F(k) > u */
    double u = rng_u01(r), p = exp(-mean), F = p;
    k = 0;
    while (F <= u && k < cap) {
      ++k;
      p *= mean / (double)k;
      F += p;
    }
  } else {
    k = (int64_t)floor(mean + sqrt(mean) * rng_normal(r) + 0.5);
  }
  if (k < 0) k = 0;
  if (k > cap) k = cap;
  return k;
}

int synth_appb_degrees(int64_t I, int32_t J, double nu, uint64_t seed, double sig_breadth,
                       int64_t* K, int64_t* E_out) {
  if (I < 0 || J <= 0 || !(nu >= 0)) return SYN_EINVAL;
  double* w = (double*)malloc(sizeof(double) * (size_t)J);
  if (!w) return SYN_ENOMEM;
  double tot = 0.0;
  for (int32_t j = 0; j < J; ++j) {
    rng_t r = rng_for(seed, PURPOSE_APPB_BREADTH, (uint64_t)j);
    w[j] = exp(sig_breadth * rng_normal(&r));
    tot += w[j];
  }
  int64_t E = 0;
  for (int32_t j = 0; j < J; ++j) {
    rng_t r = rng_for(seed, PURPOSE_APPB_K, (uint64_t)j);
    K[j] = poisson_draw(&r, w[j] / tot * (double)I * nu, I);
    E += K[j];
  }
  free(w);
  *E_out = E;
  return SYN_OK;
}

int synth_appb_fill(int64_t I, int32_t J, const int64_t* K, uint64_t seed, double sig_v,
                    double sig_u, double sig_eps, double c_max, double mu_s, double sig_s,
                    int64_t* off, int32_t* dst, float* c, float* a) {
  if (I < 0 || J <= 0) return SYN_EINVAL;
  int64_t* roff = (int64_t*)malloc(sizeof(int64_t) * ((size_t)J + 1));
  if (!roff) return SYN_ENOMEM;
  roff[0] = 0;
  int64_t kmax = 0;
  for (int32_t j = 0; j < J; ++j) {
    if (K[j] < 0 || K[j] > I) { free(roff); return SYN_EINVAL; }
    roff[j + 1] = roff[j] + K[j];
    if (K[j] > kmax) kmax = K[j];
  }
  const int64_t E = roff[J];
  int32_t* req = (int32_t*)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
  float* val = (float*)malloc(sizeof(float) * (size_t)(E > 0 ? E : 1));
  float* coef = (float*)malloc(sizeof(float) * (size_t)(E > 0 ? E : 1));
  double* u = (double*)malloc(sizeof(double) * (size_t)(I > 0 ? I : 1));
  if (!req || !val || !coef || !u) {
    free(roff); free(req); free(val); free(coef); free(u);
    return SYN_ENOMEM;
  }
  for (int64_t i = 0; i < I; ++i) {
    rng_t r = rng_for(seed, PURPOSE_APPB_U, (uint64_t)i);
    u[i] = exp(sig_u * rng_normal(&r));
  }
  int err = 0;
#pragma omp parallel
  {
    /* Floyd's sampling of min(K, I - K) distinct requests (the complement when
     * K > I / 2), in a hash set sized for the largest K */
    pickset_t ps;
    const int64_t mmax = kmax < I - kmax ? kmax : I - kmax;
    uint32_t* pick = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(mmax + 1));
    int ok = pickset_init(&ps, mmax) == 0 && pick;
    if (!ok) {
#pragma omp atomic write
      err = 1;
    }
#pragma omp for schedule(dynamic, 16)
    for (int32_t j = 0; j < J; ++j) {
      if (!ok) continue;
      rng_t r = rng_for(seed, PURPOSE_APPB_PICK, (uint64_t)j);
      const int64_t k = K[j], m = k <= I - k ? k : I - k;
      pickset_clear(&ps);
      int64_t np = 0;
      for (int64_t t = I - m; t < I; ++t) { /* Floyd */
        uint32_t v = (uint32_t)rng_below(&r, (uint64_t)t + 1);
        if (!pickset_insert(&ps, v)) {
          v = (uint32_t)t;
          pickset_insert(&ps, v);
        }
        pick[np++] = v;
      }
      int64_t pos = roff[j];
      if (m == k) {  /* the picks, in increasing request id */
        qsort(pick, (size_t)np, sizeof(uint32_t), cmp_u32);
        for (int64_t q = 0; q < np; ++q) req[pos++] = (int32_t)pick[q];
      } else {       /* more than half of the requests: all but the picks */
        for (int64_t i = 0; i < I && pos < roff[j + 1]; ++i)
          if (!pickset_has(&ps, (uint32_t)i)) req[pos++] = (int32_t)i;
      }
      rng_t rv = rng_for(seed, PURPOSE_APPB_V, (uint64_t)j);
      rng_t rs = rng_for(seed, PURPOSE_APPB_S, (uint64_t)j);
      const double vj = exp(sig_v * rng_normal(&rv));
      const double sj = exp(mu_s + sig_s * rng_normal(&rs));
      for (int64_t e = roff[j]; e < roff[j + 1]; ++e) {
        double x = vj * u[req[e]] * exp(sig_eps * rng_normal(&r));
        if (x > c_max) x = c_max;
        val[e] = (float)x;
        coef[e] = (float)(sj * x);
      }
    }
    if (ok) pickset_free(&ps);
    free(pick);
  }
  if (!err) {
    /* source-major by a stable counting sort on the request */
    for (int64_t i = 0; i <= I; ++i) off[i] = 0;
    for (int64_t e = 0; e < E; ++e) off[req[e] + 1]++;
    for (int64_t i = 0; i < I; ++i) off[i + 1] += off[i];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(I > 0 ? I : 1));
    if (!fill) {
      err = 1;
    } else {
      for (int64_t i = 0; i < I; ++i) fill[i] = off[i];
      for (int32_t j = 0; j < J; ++j)
        for (int64_t e = roff[j]; e < roff[j + 1]; ++e) {
          const int64_t p = fill[req[e]]++;
          dst[p] = j;
          c[p] = -val[e];
          a[p] = coef[e];
        }
      free(fill);
    }
  }
  free(roff); free(req); free(val); free(coef); free(u);
  return err ? SYN_ENOMEM : SYN_OK;
}

int synth_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}
