/*
 * Pair-HMM oracle: plain, slow, FP64 CPU reference for the batched Pair-HMM forward
 * algorithm of gpuPairHMM (Schmidt et al., arXiv 2411.11547) and its adjoint.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls this file:
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark do.  It shares no
 * source, header, table or constant with the CUDA path.
 *
 * What it computes (Sec. II-A):
 *   Eq. 1  M(i,j) = lambda(i,j) * ( alpha_i M(i-1,j-1) + beta (I(i-1,j-1) + D(i-1,j-1)) )
 *   Eq. 2  I(i,j) = delta_i M(i-1,j) + eps I(i-1,j)
 *   Eq. 3  D(i,j) = zeta_i  M(i,j-1) + eps D(i,j-1)
 *   (with a per-base gap-continuation track, eps and beta become eps_i and beta_i of the row
 *   being computed, like alpha_i, delta_i and zeta_i)
 *   init   M(i,0)=I(i,0)=D(i,0)=0 (i>=1); M(0,j)=I(0,j)=0, D(0,j)=1/n (0<=j<=n)
 *   Eq. 4  lambda(i,j) = 1-Q_i if r_i == h_j else Q_i/3
 *   result L = sum_{j=1..n} M(m,j) + I(m,j);  reported as log10 L.
 *
 * Readings of points the paper leaves open (each one is listed in the design notes):
 *   - transitions (Sec. III-A only says quality scores and gap probabilities are inputs):
 *       Q_i = 10^(-bq_i/10), delta_i = 10^(-iq_i/10), zeta_i = 10^(-dq_i/10),
 *       eps = 10^(-gcp/10), beta = 1 - eps  (per-base track: eps_i = 10^(-gcp_i/10),
 *       beta_i = 1 - eps_i, every transition of row i taken from read position i),
 *       alpha_i = 1 - (delta_i + zeta_i)            (alpha_mode 0, default)
 *       alpha_i = 1 - 10^(-(iq_i + dq_i)/10)        (alpha_mode 1, alternative)
 *   - D(0,0) = 1/n (the init line gives D(0,j)=1/n for every j including 0);
 *   - 'N' on either side matches every base (emission 1-Q_i); bases are case-insensitive.
 *
 * Numerics: FP64 row sweep.  After each row the three row vectors are divided by 2^e_i, with
 * e_i the binary exponent of the row maximum (frexp; an exact scaling), and the exponents are
 * summed, so no value ever underflows.  log10 L = log10(L~) + (sum e_i) log10 2.
 *
 * Adjoint: all scaled rows are stored; the reverse sweep works with normalised adjoints
 * A^(i,j) = dL/dA(i,j) * 2^{c_i} / L (c_i = sum of e_1..e_i), for which the posterior
 * occupancy of a cell is simply A~(i,j) * A^(i,j).  Parameter partials follow by the chain
 * rule through the definitions above.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL -1
#define OR_ENOMEM -3

static const double LN10 = 2.302585092994045684017991454684364208;
static const double LOG10_2 = 0.301029995663981195213738894724493027;

static int upcase(int c) { return (c >= 'a' && c <= 'z') ? c - 32 : c; }

static int valid_base(int c) {
  c = upcase(c);
  return c == 'A' || c == 'C' || c == 'G' || c == 'T' || c == 'N';
}

/* Phred value q -> probability 10^(-q/10). */
static double phred(double q) { return pow(10.0, -q / 10.0); }

/* Eq. 4 with the N reading: is (r_i, h_j) treated as a match? */
static int is_match(int r, int h) {
  r = upcase(r);
  h = upcase(h);
  return r == h || r == 'N' || h == 'N';
}

typedef struct {
  int m, n;
  const uint8_t *r, *h;
  const double *bq, *iq, *dq;
  double gcp;
  int alpha_mode;
  const double *gq; /* per-base gap-continuation Phred values [m], or NULL: gcp everywhere */
} or_pair;

/* Per-row transition parameters of one read (index i = 1..m). */
typedef struct {
  double *Q, *alpha, *delta, *zeta, *eps, *beta;
} or_params;

static int params_init(const or_pair *p, or_params *t) {
  t->Q = (double *)malloc(sizeof(double) * 6 * (size_t)(p->m + 1));
  if (!t->Q) return OR_ENOMEM;
  t->alpha = t->Q + (p->m + 1);
  t->delta = t->alpha + (p->m + 1);
  t->zeta = t->delta + (p->m + 1);
  t->eps = t->zeta + (p->m + 1);
  t->beta = t->eps + (p->m + 1);
  t->eps[0] = t->beta[0] = 0.0;
  for (int i = 1; i <= p->m; ++i) {
    t->eps[i] = phred(p->gq ? p->gq[i - 1] : p->gcp);
    t->beta[i] = 1.0 - t->eps[i];
    t->Q[i] = phred(p->bq[i - 1]);
    t->delta[i] = phred(p->iq[i - 1]);
    t->zeta[i] = phred(p->dq[i - 1]);
    if (p->alpha_mode == 1)
      t->alpha[i] = 1.0 - phred(p->iq[i - 1] + p->dq[i - 1]);
    else
      t->alpha[i] = 1.0 - (t->delta[i] + t->zeta[i]);
  }
  return OR_OK;
}

static void params_free(or_params *t) { free(t->Q); }

static double lambda_of(const or_pair *p, const or_params *t, int i, int j) {
  return is_match(p->r[i - 1], p->h[j - 1]) ? 1.0 - t->Q[i] : t->Q[i] / 3.0;
}

/* Scale row vectors by 2^-e where e = exponent of their max; return e. */
static int renorm_row(double *M, double *I, double *D, int n) {
  double mx = 0.0;
  for (int j = 0; j <= n; ++j) {
    if (M[j] > mx) mx = M[j];
    if (I[j] > mx) mx = I[j];
    if (D[j] > mx) mx = D[j];
  }
  if (mx == 0.0) return 0;
  int e;
  frexp(mx, &e);
  for (int j = 0; j <= n; ++j) {
    M[j] = ldexp(M[j], -e);
    I[j] = ldexp(I[j], -e);
    D[j] = ldexp(D[j], -e);
  }
  return e;
}

/*
 * Fill scaled rows 0..m.  If store is non-null it has room for (m+1)*(n+1) entries per matrix
 * and all rows are kept; otherwise two rolling rows are used.  e[i] receives the row exponent.
 * Returns log10 L (or -inf when L == 0).
 */
static double forward_rows(const or_pair *p, const or_params *t, double *SM, double *SI,
                           double *SD, int *e, double *Ltilde_out, long *csum_out) {
  const int m = p->m, n = p->n;
  const size_t W = (size_t)n + 1;
  double *buf = NULL;
  int keep = SM != NULL;
  if (!keep) {
    buf = (double *)calloc(6 * W, sizeof(double));
    if (!buf) return NAN;
  }
  double *pM = keep ? SM : buf, *pI = keep ? SI : buf + W, *pD = keep ? SD : buf + 2 * W;
  /* row 0 */
  for (size_t j = 0; j <= (size_t)n; ++j) {
    pM[j] = 0.0;
    pI[j] = 0.0;
    pD[j] = 1.0 / n;
  }
  if (e) e[0] = 0;
  long csum = 0;
  for (int i = 1; i <= m; ++i) {
    double *cM = keep ? SM + (size_t)i * W : (i & 1 ? buf + 3 * W : buf);
    double *cI = keep ? SI + (size_t)i * W : (i & 1 ? buf + 4 * W : buf + W);
    double *cD = keep ? SD + (size_t)i * W : (i & 1 ? buf + 5 * W : buf + 2 * W);
    cM[0] = cI[0] = cD[0] = 0.0;
    for (int j = 1; j <= n; ++j) {
      double lam = lambda_of(p, t, i, j);
      cM[j] = lam * (t->alpha[i] * pM[j - 1] + t->beta[i] * (pI[j - 1] + pD[j - 1]));
      cI[j] = t->delta[i] * pM[j] + t->eps[i] * pI[j];
      cD[j] = t->zeta[i] * cM[j - 1] + t->eps[i] * cD[j - 1];
    }
    int ei = renorm_row(cM, cI, cD, n);
    if (e) e[i] = ei;
    csum += ei;
    pM = cM;
    pI = cI;
    pD = cD;
  }
  double Lt = 0.0;
  for (int j = 1; j <= n; ++j) Lt += pM[j] + pI[j];
  free(buf);
  if (Ltilde_out) *Ltilde_out = Lt;
  if (csum_out) *csum_out = csum;
  if (Lt <= 0.0) return -INFINITY;
  return log10(Lt) + (double)csum * LOG10_2;
}

static int check_pair(const or_pair *p) {
  if (p->m <= 0 || p->n <= 0) return OR_EINVAL;
  if (!(p->gcp > 0.0)) return OR_EINVAL;
  for (int i = 0; i < p->m; ++i)
    if (!valid_base(p->r[i])) return OR_EINVAL;
  for (int j = 0; j < p->n; ++j)
    if (!valid_base(p->h[j])) return OR_EINVAL;
  for (int i = 0; i < p->m; ++i) {
    if (isnan(p->bq[i]) || isnan(p->iq[i]) || isnan(p->dq[i])) return OR_EINVAL;
    if (p->bq[i] < 0 || p->iq[i] < 0 || p->dq[i] < 0) return OR_EINVAL;
    if (p->alpha_mode == 0 && phred(p->iq[i]) + phred(p->dq[i]) > 1.0) return OR_EINVAL;
    if (p->gq && !(p->gq[i] > 0.0)) return OR_EINVAL;
  }
  return OR_OK;
}

/* log10 P(R | H) for one pair.  gq: per-base gap-continuation Phred values [m] or NULL (gcp
 * everywhere).  Returns NAN for invalid input. */
double oracle_forward_pair(int m, const uint8_t *r, const double *bq, const double *iq,
                           const double *dq, int n, const uint8_t *h, double gcp,
                           int alpha_mode, const double *gq) {
  or_pair p = {m, n, r, h, bq, iq, dq, gcp, alpha_mode, gq};
  if (check_pair(&p) != OR_OK) return NAN;
  or_params t;
  if (params_init(&p, &t) != OR_OK) return NAN;
  double res = forward_rows(&p, &t, NULL, NULL, NULL, NULL, NULL, NULL);
  params_free(&t);
  return res;
}

/*
 * Adjoint of one pair.  dy = d(loss)/d(log10 L).  Writes gradients of the loss w.r.t. the
 * Phred inputs: g_bq[m], g_iq[m], g_dq[m] (overwritten), g_gq[m] (per-base gap-continuation
 * values, overwritten; may be NULL) and *g_gcp = the sum of g_gq (the derivative for one gap-
 * continuation value shared by every row); returns log10 L.
 */
double oracle_backward_pair(int m, const uint8_t *r, const double *bq, const double *iq,
                            const double *dq, int n, const uint8_t *h, double gcp,
                            int alpha_mode, const double *gq, double dy, double *g_bq,
                            double *g_iq, double *g_dq, double *g_gq, double *g_gcp) {
  or_pair p = {m, n, r, h, bq, iq, dq, gcp, alpha_mode, gq};
  if (check_pair(&p) != OR_OK) return NAN;
  or_params t;
  if (params_init(&p, &t) != OR_OK) return NAN;
  const size_t W = (size_t)n + 1, cells = (size_t)(m + 1) * W;
  double *SM = (double *)malloc(sizeof(double) * 3 * cells);
  double *A = (double *)calloc(6 * W, sizeof(double)); /* adjoint rows i+1 and i */
  int *e = (int *)malloc(sizeof(int) * (size_t)(m + 1));
  double *gA = (double *)calloc(7 * (size_t)(m + 1), sizeof(double));
  if (!SM || !A || !e || !gA) {
    free(SM);
    free(A);
    free(e);
    free(gA);
    params_free(&t);
    return NAN;
  }
  double *SI = SM + cells, *SD = SI + cells;
  double Lt = 0.0;
  long csum = 0;
  double res = forward_rows(&p, &t, SM, SI, SD, e, &Lt, &csum);
  if (!(Lt > 0.0)) {
    /* L == 0: log-likelihood has no finite gradient. */
    for (int i = 0; i < m; ++i) {
      g_bq[i] = g_iq[i] = g_dq[i] = NAN;
      if (g_gq) g_gq[i] = NAN;
    }
    *g_gcp = NAN;
    free(SM);
    free(A);
    free(e);
    free(gA);
    params_free(&t);
    return res;
  }
  /* Per-row accumulators of (1/L) dL/dtheta. */
  double *gal = gA, *gdel = gA + (m + 1), *gzet = gA + 2 * (m + 1), *gQ = gA + 3 * (m + 1);
  double *gbeta = gA + 4 * (m + 1), *geps = gA + 5 * (m + 1);
  double *nM = A, *nI = A + W, *nD = A + 2 * W; /* row i+1 (normalised adjoints) */
  double *aM = A + 3 * W, *aI = A + 4 * W, *aD = A + 5 * W; /* row i */
  for (int i = m; i >= 1; --i) {
    const double *Mi = SM + (size_t)i * W, *Di = SD + (size_t)i * W;
    const double *Mp = SM + (size_t)(i - 1) * W, *Ip = SI + (size_t)(i - 1) * W,
                 *Dp = SD + (size_t)(i - 1) * W;
    const double down = (i < m) ? ldexp(1.0, -e[i + 1]) : 0.0; /* 2^{c_i - c_{i+1}} */
    const double seed = (i == m) ? 1.0 / Lt : 0.0;
    for (int j = n; j >= 1; --j) {
      double fromM = 0.0, fromIv = 0.0;
      if (i < m) {
        if (j < n) {
          double lam1 = lambda_of(&p, &t, i + 1, j + 1);
          fromM = lam1 * nM[j + 1];
        }
        fromIv = nI[j];
      }
      double dnext = (j < n) ? aD[j + 1] : 0.0;
      /* row i+1's transitions where the edge enters row i+1, row i's within row i */
      const double beta1 = (i < m) ? t.beta[i + 1] : 0.0, eps1 = (i < m) ? t.eps[i + 1] : 0.0;
      aD[j] = (beta1 * fromM) * down + t.eps[i] * dnext;
      aI[j] = seed + (beta1 * fromM + eps1 * fromIv) * down;
      double alpha1 = (i < m) ? t.alpha[i + 1] : 0.0;
      double delta1 = (i < m) ? t.delta[i + 1] : 0.0;
      aM[j] = seed + (alpha1 * fromM + delta1 * fromIv) * down + t.zeta[i] * dnext;
    }
    /* Parameter partials for row i: terms of Eq. 1 carry 2^{-e_i}, as do those of Eq. 2. */
    const double up = ldexp(1.0, -e[i]);
    for (int j = 1; j <= n; ++j) {
      double lam = lambda_of(&p, &t, i, j);
      double mdiag = Mp[j - 1], sdiag = Ip[j - 1] + Dp[j - 1];
      double a = aM[j] * lam * up;
      gal[i] += a * mdiag;
      gbeta[i] += a * sdiag;
      double G = t.alpha[i] * mdiag + t.beta[i] * sdiag;
      double dlam_dQ = is_match(p.r[i - 1], p.h[j - 1]) ? -1.0 : 1.0 / 3.0;
      gQ[i] += aM[j] * up * G * dlam_dQ;
      gdel[i] += aI[j] * up * Mp[j];
      geps[i] += aI[j] * up * Ip[j];
      gzet[i] += aD[j] * Mi[j - 1];
      geps[i] += aD[j] * Di[j - 1];
    }
    double *tmp;
    tmp = nM; nM = aM; aM = tmp;
    tmp = nI; nI = aI; aI = tmp;
    tmp = nD; nD = aD; aD = tmp;
  }
  /* Chain rule to the Phred inputs; scale d ln L -> d log10 L and by dy. */
  const double k = dy / LN10;
  const double dP = -LN10 / 10.0; /* dP/dq = dP * P for P = 10^(-q/10) */
  for (int i = 1; i <= m; ++i) {
    g_bq[i - 1] = k * gQ[i] * dP * t.Q[i];
    if (alpha_mode == 1) {
      double pa = phred(iq[i - 1] + dq[i - 1]); /* alpha = 1 - pa, dalpha/dq = -dP * pa */
      g_iq[i - 1] = k * (gdel[i] * dP * t.delta[i] - gal[i] * dP * pa);
      g_dq[i - 1] = k * (gzet[i] * dP * t.zeta[i] - gal[i] * dP * pa);
    } else {
      g_iq[i - 1] = k * (gdel[i] - gal[i]) * dP * t.delta[i];
      g_dq[i - 1] = k * (gzet[i] - gal[i]) * dP * t.zeta[i];
    }
  }
  /* beta_i = 1 - eps_i: d/d gcp_i = (d/d eps_i - d/d beta_i) * dP * eps_i */
  double gsum = 0.0;
  for (int i = 1; i <= m; ++i) {
    const double g = k * (geps[i] - gbeta[i]) * dP * t.eps[i];
    if (g_gq) g_gq[i - 1] = g;
    gsum += g;
  }
  *g_gcp = gsum;
  free(SM);
  free(A);
  free(e);
  free(gA);
  params_free(&t);
  return res;
}

/* ---------------------------------------------------------------- batch drivers ---- */

typedef struct {
  int64_t n_reads, n_haps, n_pairs;
  const uint8_t *read_bases;
  const double *bq, *iq, *dq;
  const int64_t *read_off;
  const uint8_t *hap_bases;
  const int64_t *hap_off;
  const int32_t *pair_read, *pair_hap;
  double gcp;
  int32_t alpha_mode;
  const double *gq; /* per-base gap-continuation Phred values [sum m], or NULL */
} oracle_batch;

typedef struct {
  const oracle_batch *b;
  const double *dy;
  double *out;
  double *gpair; /* per pair, 4*m values at pair_goff[p] (bq, iq, dq, gq), or NULL */
  const int64_t *goff;
  double *ggcp;
  int64_t next;
  pthread_mutex_t mu;
} job_t;

static void run_pair(job_t *J, int64_t p) {
  const oracle_batch *b = J->b;
  int32_t ri = b->pair_read[p], hi = b->pair_hap[p];
  if (ri < 0 || ri >= b->n_reads || hi < 0 || hi >= b->n_haps) {
    J->out[p] = NAN;
    return;
  }
  int64_t r0 = b->read_off[ri], r1 = b->read_off[ri + 1];
  int64_t h0 = b->hap_off[hi], h1 = b->hap_off[hi + 1];
  int m = (int)(r1 - r0), n = (int)(h1 - h0);
  if (!J->gpair) {
    J->out[p] = oracle_forward_pair(m, b->read_bases + r0, b->bq + r0, b->iq + r0, b->dq + r0, n,
                                    b->hap_bases + h0, b->gcp, b->alpha_mode,
                                    b->gq ? b->gq + r0 : NULL);
  } else {
    double *g = J->gpair + J->goff[p];
    J->out[p] = oracle_backward_pair(m, b->read_bases + r0, b->bq + r0, b->iq + r0, b->dq + r0,
                                     n, b->hap_bases + h0, b->gcp, b->alpha_mode,
                                     b->gq ? b->gq + r0 : NULL, J->dy[p], g, g + m, g + 2 * m,
                                     g + 3 * m, J->ggcp + p);
  }
}

static void *worker(void *arg) {
  job_t *J = (job_t *)arg;
  for (;;) {
    pthread_mutex_lock(&J->mu);
    int64_t p = J->next++;
    pthread_mutex_unlock(&J->mu);
    if (p >= J->b->n_pairs) break;
    run_pair(J, p);
  }
  return NULL;
}

static void run_all(job_t *J, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
  J->next = 0;
  pthread_mutex_init(&J->mu, NULL);
  int started = 0;
  for (int k = 0; th && k < nthreads; ++k)
    if (pthread_create(&th[k], NULL, worker, J) == 0) ++started;
  if (started == 0) worker(J);
  for (int k = 0; k < started; ++k) pthread_join(th[k], NULL);
  pthread_mutex_destroy(&J->mu);
  free(th);
}

/* Forward over every pair of the batch; out[n_pairs] = log10 L (NAN for invalid pairs). */
int oracle_forward_batch(const oracle_batch *b, double *out, int nthreads) {
  job_t J;
  memset(&J, 0, sizeof(J));
  J.b = b;
  J.out = out;
  run_all(&J, nthreads);
  return OR_OK;
}

/*
 * Forward + adjoint over every pair.  dy[n_pairs] = d(loss)/d(log10 L_p).  Per-read gradient
 * arrays g_bq/g_iq/g_dq[sum m] (and g_gq[sum m] when not NULL: the per-base gap-continuation
 * values) are overwritten with the sum over pairs in pair order; *g_gcp with the sum over
 * pairs and rows.  out[n_pairs] receives log10 L.
 */
int oracle_backward_batch(const oracle_batch *b, const double *dy, double *out, double *g_bq,
                          double *g_iq, double *g_dq, double *g_gq, double *g_gcp,
                          int nthreads) {
  int64_t *goff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(b->n_pairs + 1));
  double *ggcp = (double *)calloc((size_t)b->n_pairs + 1, sizeof(double));
  if (!goff || !ggcp) {
    free(goff);
    free(ggcp);
    return OR_ENOMEM;
  }
  goff[0] = 0;
  for (int64_t p = 0; p < b->n_pairs; ++p) {
    int32_t ri = b->pair_read[p];
    int64_t m = (ri >= 0 && ri < b->n_reads) ? b->read_off[ri + 1] - b->read_off[ri] : 0;
    goff[p + 1] = goff[p] + 4 * m;
  }
  double *gpair = (double *)calloc((size_t)goff[b->n_pairs] + 1, sizeof(double));
  if (!gpair) {
    free(goff);
    free(ggcp);
    return OR_ENOMEM;
  }
  job_t J;
  memset(&J, 0, sizeof(J));
  J.b = b;
  J.dy = dy;
  J.out = out;
  J.gpair = gpair;
  J.goff = goff;
  J.ggcp = ggcp;
  run_all(&J, nthreads);
  int64_t total = b->read_off[b->n_reads];
  for (int64_t i = 0; i < total; ++i) {
    g_bq[i] = g_iq[i] = g_dq[i] = 0.0;
    if (g_gq) g_gq[i] = 0.0;
  }
  double gg = 0.0;
  for (int64_t p = 0; p < b->n_pairs; ++p) {
    int32_t ri = b->pair_read[p];
    if (ri < 0 || ri >= b->n_reads) continue;
    int64_t r0 = b->read_off[ri];
    int64_t m = b->read_off[ri + 1] - r0;
    const double *g = gpair + goff[p];
    for (int64_t i = 0; i < m; ++i) {
      g_bq[r0 + i] += g[i];
      g_iq[r0 + i] += g[m + i];
      g_dq[r0 + i] += g[2 * m + i];
      if (g_gq) g_gq[r0 + i] += g[3 * m + i];
    }
    gg += ggcp[p];
  }
  *g_gcp = gg;
  free(goff);
  free(ggcp);
  free(gpair);
  return OR_OK;
}
