/*
 * ls_oracle.c -- plain single-threaded CPU LearnedSort.
 *
 * TEST INFRASTRUCTURE ONLY (see ls_oracle.h): loaded by tests/, the smoke
 * check and bench.py's cpu_baseline / reference leg, never by the product.
 *
 * Compile with -O2 -ffp-contract=off: every floating-point statement below is
 * one IEEE-754 binary64 operation, round-to-nearest-even, in the order
 * written.  max(p,q) is (p < q ? q : p) and min(p,q) is (q < p ? q : p).
 */
#include "ls_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN_GAMMA 0x9E3779B97F4A7C15ull
#define CHUNK 256          /* canonical summation chunk (fixed reading) */
#define REFINE_LIMIT 1125899906842624.0 /* 2^50: largest B^(k+1) refined */

static double dmax(double p, double q) { return (p < q) ? q : p; }
static double dmin(double p, double q) { return (q < p) ? q : p; }

/* Integer index from a floored double: values that are not > 0 (negatives,
 * zeros, NaN from a non-finite model) give 0, values >= hi give hi.  Equal
 * to min(max(t, 0), hi) for every non-NaN t. */
static uint32_t clamp_index(double t, uint32_t hi) {
  if (!(t > 0.0)) return 0;
  if (!(t < (double)hi)) return hi;
  return (uint32_t)t;
}

/* ------------------------------------------------------------------ keys */

/* Order-preserving map to uint64: for doubles this is IEEE totalOrder
 * (-0.0 before +0.0); for unsigned integers the identity.  The float-to-int
 * key extractor idea is the one the paper uses for radix sorting floats
 * (Sec. 5). */
uint64_t lsref_ord(uint64_t bits, int dtype) {
  if (dtype == LSREF_U64) return bits;
  return (bits >> 63) ? ~bits : (bits ^ 0x8000000000000000ull);
}

uint64_t lsref_unord(uint64_t u, int dtype) {
  if (dtype == LSREF_U64) return u;
  return (u >> 63) ? (u ^ 0x8000000000000000ull) : ~u;
}

/* v(x): the value the model reads.  A u64 key is converted by
 * round-to-nearest (C's conversion under the default rounding mode). */
double lsref_key_value(uint64_t bits, int dtype) {
  if (dtype == LSREF_U64) return (double)bits;
  double d;
  memcpy(&d, &bits, sizeof d);
  return d;
}

static double ord_value(uint64_t u, int dtype) { return lsref_key_value(lsref_unord(u, dtype), dtype); }

/* ------------------------------------------------------------- sampling */

/* SplitMix64 output function (Vigna, public domain): the value the
 * generator returns once its state has been advanced to `z`. */
uint64_t lsref_splitmix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

uint64_t lsref_seed_item(uint64_t seed, uint64_t segment, uint32_t level, uint64_t gidx) {
  uint64_t tag = (segment << 40) + ((uint64_t)level << 32) + (gidx & 0xFFFFFFFFull);
  return lsref_splitmix64(seed ^ tag);
}

/* Sec. 2.2: the RMI is trained on a sample of 1% of N.  S = ceil(r n),
 * raised to min_sample and capped at n. */
uint64_t lsref_sample_size(uint64_t n, const lsref_params* p) {
  if (n == 0) return 0;
  double want = ceil(p->sample_rate * (double)n);
  uint64_t S;
  if (!(want < (double)n)) S = n;
  else if (want < 1.0) S = 0;
  else S = (uint64_t)want;
  if (S < p->min_sample) S = p->min_sample;
  if (S > n) S = n;
  return S;
}

/* Sample(A, l, r) of Alg. 2-5: S positions drawn with replacement from a
 * counter-based SplitMix64 stream; position j = floor(u_j * n / 2^64).
 * When S == n every key is taken, in index order. */
void lsref_sample_positions(uint64_t h, uint64_t n, uint64_t S, uint64_t* pos) {
  if (S >= n) {
    for (uint64_t j = 0; j < n; ++j) pos[j] = j;
    return;
  }
  for (uint64_t j = 0; j < S; ++j) {
    uint64_t r = lsref_splitmix64(h + (j + 1) * GOLDEN_GAMMA);
    pos[j] = (uint64_t)(((unsigned __int128)r * (unsigned __int128)n) >> 64);
  }
}

void lsref_params_default(lsref_params* p) {
  memset(p, 0, sizeof *p);
  p->fanout = 1000;            /* LearnedSort's B (Sec. 2.1) */
  p->splitter_fanout = 1024;
  p->basecase_threshold = 16;  /* SampleSort's insertion-sort size (Sec. 3.3) */
  p->max_depth = 16;
  p->min_sample = 256;
  p->auto_splitter_fanout = 256; /* Alg. 5 default tree size (Sec. 4) */
  p->sample_rate = 0.01;       /* 1% sample (Sec. 2.2) */
  p->dup_frac = 0.10;          /* "more than 10% of duplicates" (Sec. 4) */
  p->imbalance_tau = 8.0;
  p->min_learned_n = 100000;   /* "smaller than N = 10^5" (Sec. 4) */
  p->seed = 0x5EEDull;
  p->partitioner = LSREF_PART_AUTO;
  p->recurse_model = LSREF_RECURSE_REFINE_GLOBAL;
}

size_t lsref_sizeof_model(void) { return sizeof(lsref_model); }
size_t lsref_sizeof_trace(void) { return sizeof(lsref_trace); }
size_t lsref_sizeof_params(void) { return sizeof(lsref_params); }
size_t lsref_sizeof_splitter(void) { return sizeof(lsref_splitter); }

/* ------------------------------------------------------------- sorting */

static void insertion_sort_u64(uint64_t* a, uint64_t n) {
  for (uint64_t i = 1; i < n; ++i) {
    uint64_t v = a[i];
    uint64_t j = i;
    while (j > 0 && a[j - 1] > v) {
      a[j] = a[j - 1];
      --j;
    }
    a[j] = v;
  }
}

static void sift_down(uint64_t* a, uint64_t root, uint64_t n) {
  for (;;) {
    uint64_t child = 2 * root + 1;
    if (child >= n) return;
    if (child + 1 < n && a[child] < a[child + 1]) ++child;
    if (!(a[root] < a[child])) return;
    uint64_t t = a[root];
    a[root] = a[child];
    a[child] = t;
    root = child;
  }
}

/* HeapSort (the sample sort named in Alg. 2-4). */
static void heapsort_u64(uint64_t* a, uint64_t n) {
  if (n < 2) return;
  for (uint64_t i = n / 2; i-- > 0;) sift_down(a, i, n);
  for (uint64_t end = n - 1; end > 0; --end) {
    uint64_t t = a[0];
    a[0] = a[end];
    a[end] = t;
    sift_down(a, 0, end);
  }
}

/* Base case: insertion sort (Sec. 2.2, Alg. 1), heap sort for larger runs.
 * The sorted result is unique, so the choice only changes speed. */
static void base_sort_u64(uint64_t* a, uint64_t n) {
  if (n <= 32) insertion_sort_u64(a, n);
  else heapsort_u64(a, n);
}

/* ----------------------------------------------------------------- RMI */

/* Fixed pairwise tree over chunk partials: while more than one value is
 * left, p[i] = p[2i] + p[2i+1] for each pair, an odd last value is carried
 * up unchanged.  Empty input sums to +0.0. */
static double tree_sum(double* p, uint64_t m) {
  if (m == 0) return 0.0;
  while (m > 1) {
    uint64_t h = m / 2;
    for (uint64_t i = 0; i < h; ++i) p[i] = p[2 * i] + p[2 * i + 1];
    if (m & 1) p[h] = p[m - 1];
    m = h + (m & 1);
  }
  return p[0];
}

/* The four least-squares sums over sample positions j in [st, en) of the
 * sorted sample, with X_j = v(s_j) - x0 and y_j = j / S (the empirical CDF
 * of Sec. 2.1: pos = N * P(A <= x)).  Canonical order: consecutive chunks
 * of 256 positions from st, each summed by tree_sum over its terms; the
 * chunk partials are then combined by tree_sum again.  (The paper fixes no
 * summation order; a fixed pairwise tree is deterministic and accurate.) */
static void ls_sums(const uint64_t* s_ord, int dtype, uint64_t st, uint64_t en, double x0, uint64_t S,
                    double out[4]) {
  uint64_t nch = (en - st + CHUNK - 1) / CHUNK;
  double* part = (double*)malloc(4 * (nch ? nch : 1) * sizeof(double));
  double t[4][CHUNK];
  uint64_t c = 0;
  for (uint64_t c0 = st; c0 < en; c0 += CHUNK, ++c) {
    uint64_t c1 = (en - c0 > CHUNK) ? c0 + CHUNK : en;
    for (uint64_t j = c0; j < c1; ++j) {
      double X = ord_value(s_ord[j], dtype) - x0;
      double y = (double)j / (double)S;
      t[0][j - c0] = X;
      t[1][j - c0] = y;
      t[2][j - c0] = X * y;
      t[3][j - c0] = X * X;
    }
    for (int k = 0; k < 4; ++k) part[k * nch + c] = tree_sum(t[k], c1 - c0);
  }
  for (int k = 0; k < 4; ++k) out[k] = tree_sum(part + k * nch, nch);
  free(part);
}

/* Closed-form simple linear regression y = a X + b from the sums, slope
 * clamped at 0 so every model is non-decreasing (Sec. 3.1 monotonicity). */
static void linfit(double n, const double s[4], double* a, double* b) {
  double t1 = n * s[3];
  double t2 = s[0] * s[0];
  double D = t1 - t2;
  double A = 0.0;
  if (D > 0.0) {
    double u1 = n * s[2];
    double u2 = s[0] * s[1];
    double num = u1 - u2;
    A = num / D;
  }
  A = dmax(A, 0.0);
  double ax = A * s[0];
  double r = s[1] - ax;
  *a = A;
  *b = r / n;
}

/* Root model f1 routes x to leaf floor(L f1(x)) clamped to [0, L-1] (Sec. 2.1). */
static uint32_t root_leaf(const lsref_model* m, double xc) {
  double t = xc - m->root_x0;
  t = m->root_a * t;
  t = t + m->root_b;
  t = t * (double)m->L;
  t = floor(t);
  return clamp_index(t, m->L - 1);
}

uint32_t lsref_model_leaf(const lsref_model* m, double x) {
  double xc = dmax(x, m->xmin);
  xc = dmin(xc, m->xmax);
  return root_leaf(m, xc);
}

/* F(x) = f2^{leaf(x)}(x) clamped to the leaf's [lo, hi] (Sec. 2.1 + the
 * monotone-RMI constraint of Sec. 4). */
double lsref_model_F(const lsref_model* m, double x) {
  double xc = dmax(x, m->xmin);
  xc = dmin(xc, m->xmax);
  uint32_t i = root_leaf(m, xc);
  double f = xc - m->leaf_x0[i];
  f = m->leaf_a[i] * f;
  f = f + m->leaf_b[i];
  f = dmax(f, m->leaf_lo[i]);
  f = dmin(f, m->leaf_hi[i]);
  return f;
}

static double leaf_eval(const lsref_model* m, uint32_t i, double xc) {
  double f = xc - m->leaf_x0[i];
  f = m->leaf_a[i] * f;
  f = f + m->leaf_b[i];
  return f;
}

static int model_finite(const lsref_model* m) {
  if (!isfinite(m->xmin) || !isfinite(m->xmax)) return 0;
  double range = m->xmax - m->xmin;
  if (!isfinite(range)) return 0;
  if (!isfinite(m->root_a) || !isfinite(m->root_b)) return 0;
  for (uint32_t i = 0; i < m->L; ++i) {
    if (!isfinite(m->leaf_a[i]) || !isfinite(m->leaf_b[i]) || !isfinite(m->leaf_lo[i]) ||
        !isfinite(m->leaf_hi[i]))
      return 0;
  }
  return 1;
}

/* TrainCDFModel (Alg. 2-4) for the two-layer linear RMI of Sec. 2.1-2.2 on a
 * sample sorted by ord.  Returns 1 if the model is finite (usable). */
static int fit_ord(const uint64_t* s_ord, uint64_t S, int dtype, uint32_t L, lsref_model* m) {
  memset(m, 0, sizeof *m);
  m->L = L;
  m->S = (uint32_t)S;
  if (S == 0 || L == 0 || L > LSREF_MAX_FANOUT) return 0;
  m->xmin = ord_value(s_ord[0], dtype);
  m->xmax = ord_value(s_ord[S - 1], dtype);
  double sums[4];
  /* Root: anchor x0 = v(s_0), fit over all S points. */
  m->root_x0 = m->xmin;
  ls_sums(s_ord, dtype, 0, S, m->root_x0, S, sums);
  linfit((double)S, sums, &m->root_a, &m->root_b);
  /* Route the sample to the leaves; routing is monotone, so each leaf owns
   * a contiguous run of the sorted sample. */
  uint64_t j = 0;
  double hprev = 0.0;
  for (uint32_t i = 0; i < L; ++i) {
    uint64_t st = j;
    while (j < S && root_leaf(m, ord_value(s_ord[j], dtype)) == i) ++j;
    uint64_t en = j;
    uint64_t cnt = en - st;
    m->leaf_count[i] = (uint32_t)cnt;
    double raw_lo = 0.0, raw_hi = 0.0;
    if (cnt == 0) {
      m->leaf_x0[i] = m->xmin;
      m->leaf_a[i] = 0.0;
      m->leaf_b[i] = 0.0;
    } else {
      double x_first = ord_value(s_ord[st], dtype);
      double x_last = ord_value(s_ord[en - 1], dtype);
      m->leaf_x0[i] = x_first;
      ls_sums(s_ord, dtype, st, en, x_first, S, sums);
      linfit((double)cnt, sums, &m->leaf_a[i], &m->leaf_b[i]);
      raw_lo = leaf_eval(m, i, x_first);
      raw_hi = leaf_eval(m, i, x_last);
    }
    /* Monotone RMI (Sec. 4): max f2^(i) <= min f2^(i+1), as a running max. */
    if (cnt == 0) {
      m->leaf_lo[i] = hprev;
      m->leaf_hi[i] = hprev;
    } else {
      m->leaf_lo[i] = dmax(raw_lo, hprev);
      m->leaf_hi[i] = dmax(raw_hi, m->leaf_lo[i]);
    }
    hprev = m->leaf_hi[i];
  }
  /* Points the root sends past leaf L-1 cannot exist (clamped), so j == S. */
  return model_finite(m);
}

int lsref_fit(const uint64_t* sorted_sample, uint64_t S, int dtype, uint32_t L, lsref_model* m) {
  uint64_t* s = (uint64_t*)malloc((S ? S : 1) * sizeof(uint64_t));
  if (!s) return -1;
  for (uint64_t j = 0; j < S; ++j) s[j] = lsref_ord(sorted_sample[j], dtype);
  int ok = fit_ord(s, S, dtype, L, m);
  free(s);
  return ok;
}

static double pow_exact(uint32_t B, uint32_t e) {
  double P = 1.0;
  for (uint32_t i = 0; i < e; ++i) P = P * (double)B;
  return P;
}

/* Bucket of a key at refinement depth k below the model's item, inside
 * parent bucket g (global index at depth k):
 *   id = clamp(floor(F(x) * B^(k+1)) - B g, 0, B-1).
 * k = 0, g = 0 is b(x) = min(floor(B F(x)), B-1) of Sec. 2.2. */
static uint32_t refine_id_value(const lsref_model* m, double x, uint32_t B, double P, double Bg) {
  double F = lsref_model_F(m, x);
  double t = F * P;
  t = floor(t);
  t = t - Bg;
  return clamp_index(t, B - 1);
}

uint32_t lsref_refine_id(const lsref_model* m, uint64_t bits, int dtype, uint32_t B, uint32_t k, uint64_t g) {
  double P = pow_exact(B, k + 1);
  double Bg = (double)((uint64_t)B * g);
  return refine_id_value(m, lsref_key_value(bits, dtype), B, P, Bg);
}

void lsref_classify(const lsref_model* m, const uint64_t* keys, uint64_t n, int dtype, uint32_t B, uint32_t k,
                    uint64_t g, uint32_t* ids, uint64_t* hist) {
  double P = pow_exact(B, k + 1);
  double Bg = (double)((uint64_t)B * g);
  if (hist) memset(hist, 0, B * sizeof(uint64_t));
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t b = refine_id_value(m, lsref_key_value(keys[i], dtype), B, P, Bg);
    if (ids) ids[i] = b;
    if (hist) hist[b] += 1;
  }
}

/* ------------------------------------------------- training fwd / bwd */

/* Forward pass of the least-squares objective that the fit minimises:
 * prediction of the raw (unclamped) linear leaf the root routes s_j to, and
 * residual pred - y_j with y_j = j / S. */
void lsref_fit_forward(const lsref_model* m, const uint64_t* sorted_sample, uint64_t S, int dtype, double* pred,
                       double* resid) {
  for (uint64_t j = 0; j < S; ++j) {
    double x = lsref_key_value(sorted_sample[j], dtype);
    double xc = dmax(x, m->xmin);
    xc = dmin(xc, m->xmax);
    uint32_t i = root_leaf(m, xc);
    double p = leaf_eval(m, i, xc);
    double y = (double)j / (double)S;
    if (pred) pred[j] = p;
    if (resid) resid[j] = p - y;
  }
}

/* Backward pass: gradient of MSE = (1/S) sum_j (pred_j - y_j)^2 with respect
 * to each leaf's (a_i, b_i) and the root's (a, b):
 *   dMSE/da_i = 2/S sum_{j in leaf i} r_j X_j,  dMSE/db_i = 2/S sum r_j,
 * X_j = xc_j - x0_i.  Each leaf's member list (index order) is summed in
 * chunks of 256 members left to right, chunks combined by tree_sum; the
 * root term likewise over all S points. */
static void grad_sums(const double* r, const double* X, const uint64_t* idx, uint64_t m, double* s_rx, double* s_r) {
  uint64_t nch = (m + CHUNK - 1) / CHUNK;
  double* part = (double*)malloc(2 * (nch ? nch : 1) * sizeof(double));
  for (uint64_t c = 0; c < nch; ++c) {
    uint64_t e = (m - c * CHUNK > CHUNK) ? (c + 1) * CHUNK : m;
    double prx = 0.0, pr = 0.0;
    for (uint64_t q = c * CHUNK; q < e; ++q) {
      uint64_t j = idx ? idx[q] : q;
      double rx = r[j] * X[j];
      prx = prx + rx;
      pr = pr + r[j];
    }
    part[c] = prx;
    part[nch + c] = pr;
  }
  *s_rx = tree_sum(part, nch);
  *s_r = tree_sum(part + nch, nch);
  free(part);
}

void lsref_fit_backward(const lsref_model* m, const uint64_t* sorted_sample, uint64_t S, int dtype, double* grad_a,
                        double* grad_b, double* grad_root) {
  uint32_t L = m->L;
  uint64_t n1 = S ? S : 1;
  uint32_t* leaf = (uint32_t*)malloc(n1 * sizeof(uint32_t));
  double* rl = (double*)malloc(n1 * sizeof(double));
  double* Xl = (double*)malloc(n1 * sizeof(double));
  double* rr = (double*)malloc(n1 * sizeof(double));
  double* Xr = (double*)malloc(n1 * sizeof(double));
  uint64_t* start = (uint64_t*)calloc((size_t)L + 1, sizeof(uint64_t));
  uint64_t* fill = (uint64_t*)calloc((size_t)L + 1, sizeof(uint64_t));
  uint64_t* members = (uint64_t*)malloc(n1 * sizeof(uint64_t));
  double Sd = (double)S;
  for (uint64_t j = 0; j < S; ++j) {
    double x = lsref_key_value(sorted_sample[j], dtype);
    double xc = dmax(x, m->xmin);
    xc = dmin(xc, m->xmax);
    uint32_t i = root_leaf(m, xc);
    leaf[j] = i;
    double y = (double)j / Sd;
    double X = xc - m->leaf_x0[i];
    double p = m->leaf_a[i] * X;
    p = p + m->leaf_b[i];
    rl[j] = p - y;
    Xl[j] = X;
    double XR = xc - m->root_x0;
    double pr = m->root_a * XR;
    pr = pr + m->root_b;
    rr[j] = pr - y;
    Xr[j] = XR;
    start[i + 1] += 1;
  }
  for (uint32_t i = 0; i < L; ++i) start[i + 1] += start[i];
  for (uint64_t j = 0; j < S; ++j) members[start[leaf[j]] + fill[leaf[j]]++] = j;
  for (uint32_t i = 0; i < L; ++i) {
    double srx, sr;
    grad_sums(rl, Xl, members + start[i], start[i + 1] - start[i], &srx, &sr);
    double ga = 2.0 * srx;
    double gb = 2.0 * sr;
    grad_a[i] = ga / Sd;
    grad_b[i] = gb / Sd;
  }
  if (grad_root) {
    double srx, sr;
    grad_sums(rr, Xr, NULL, S, &srx, &sr);
    double ga = 2.0 * srx;
    double gb = 2.0 * sr;
    grad_root[0] = ga / Sd;
    grad_root[1] = gb / Sd;
  }
  free(leaf);
  free(rl);
  free(Xl);
  free(rr);
  free(Xr);
  free(start);
  free(fill);
  free(members);
}

/* ------------------------------------------------------------ splitter */

/* SampleSort splitters (Sec. 2.4): B_s - 1 equally spaced elements of the
 * sorted sample, B_s = largest power of two <= min(bs_max, S).  If two
 * splitters are equal the tree gets IPS4o equality buckets (Sec. 2.4). */
static void splitter_build_ord(const uint64_t* s_ord, uint64_t S, uint32_t bs_max, int force_eq,
                               lsref_splitter* t) {
  memset(t, 0, sizeof *t);
  uint32_t bs = 1;
  while ((uint64_t)bs * 2 <= bs_max && (uint64_t)bs * 2 <= S && bs * 2 <= LSREF_MAX_FANOUT) bs *= 2;
  if (bs < 2) bs = 2;
  uint32_t ns = bs - 1;
  int dup = 0;
  for (uint32_t k = 0; k < ns; ++k) {
    uint64_t idx = ((uint64_t)(k + 1) * S) / bs;
    t->split[k] = s_ord[idx];
    if (k > 0 && t->split[k] == t->split[k - 1]) dup = 1;
  }
  if (dup || force_eq) {
    uint32_t m = 0;
    for (uint32_t k = 0; k < ns; ++k) {
      if (m == 0 || t->split[m - 1] != t->split[k]) t->split[m++] = t->split[k];
    }
    t->nsplit = m;
    t->nbuckets = 2 * m + 1;
    t->equality = 1;
  } else {
    t->nsplit = ns;
    t->nbuckets = bs;
    t->equality = 0;
  }
}

void lsref_splitter_build(const uint64_t* sorted_sample, uint64_t S, int dtype, uint32_t bs_max, int force_equality,
                          lsref_splitter* t) {
  uint64_t* s = (uint64_t*)malloc((S ? S : 1) * sizeof(uint64_t));
  for (uint64_t j = 0; j < S; ++j) s[j] = lsref_ord(sorted_sample[j], dtype);
  splitter_build_ord(s, S, bs_max, force_equality, t);
  free(s);
}

/* #{k : split_k < u} by binary search (lower bound). */
static uint32_t count_less(const uint64_t* a, uint32_t n, uint64_t u) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    uint32_t mid = lo + (hi - lo) / 2;
    if (a[mid] < u) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

uint32_t lsref_splitter_bucket(const lsref_splitter* t, uint64_t u) {
  uint32_t k = count_less(t->split, t->nsplit, u);
  if (!t->equality) return k; /* keys equal to a splitter go left */
  if (k < t->nsplit && t->split[k] == u) return 2 * k + 1;
  return 2 * k;
}

void lsref_splitter_classify(const lsref_splitter* t, const uint64_t* keys, uint64_t n, int dtype, uint32_t* ids,
                             uint64_t* hist) {
  if (hist) memset(hist, 0, t->nbuckets * sizeof(uint64_t));
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t b = lsref_splitter_bucket(t, lsref_ord(keys[i], dtype));
    if (ids) ids[i] = b;
    if (hist) hist[b] += 1;
  }
}

/* ------------------------------------------------------ the full sort */

enum { KIND_FRESH = 0, KIND_FORCE_SPLITTER = 1, KIND_REFINE = 2, KIND_RADIX = 3 };

typedef struct mslot {
  lsref_model m;
  int refs;
} mslot;

typedef struct {
  uint64_t lo, hi;
  uint64_t segment;
  uint64_t gidx;
  uint64_t mg;
  mslot* model;
  uint32_t level;
  uint32_t mk;  /* REFINE: refinement depth k; RADIX: keys agree above this many low bits */
  int kind;
  int is_root;
} item_t;

typedef struct {
  item_t* v;
  size_t n, cap;
} stack_t_;

static int push(stack_t_* s, const item_t* it) {
  if (s->n == s->cap) {
    size_t nc = s->cap ? 2 * s->cap : 1024;
    item_t* nv = (item_t*)realloc(s->v, nc * sizeof(item_t));
    if (!nv) return -1;
    s->v = nv;
    s->cap = nc;
  }
  s->v[s->n++] = *it;
  return 0;
}

typedef struct {
  uint64_t* a;   /* ord values being sorted */
  uint64_t* tmp; /* scatter buffer */
  int dtype;
  const lsref_params* p;
  lsref_trace* tr;
  lsref_model* root_model_out;
  uint64_t* root_hist_out;
  int32_t* seg_decision;
  uint64_t* sbuf;   /* sample buffer (ord values) */
  uint64_t sbuf_cap;
  uint64_t* cnt;    /* bucket counts */
  uint32_t* ids;    /* per-key bucket ids of the current item */
  lsref_splitter split;
} sctx;

static lsref_level_stats* lvl(sctx* c, uint32_t level) {
  static lsref_level_stats dummy;
  if (!c->tr) return &dummy;
  uint32_t l = level < LSREF_MAX_LEVELS ? level : LSREF_MAX_LEVELS - 1;
  return &c->tr->level[l];
}

static void draw_sample(sctx* c, const item_t* it, uint64_t n, uint64_t S) {
  uint64_t h = lsref_seed_item(c->p->seed, it->segment, it->level, it->gidx);
  if (S >= n) {
    for (uint64_t j = 0; j < n; ++j) c->sbuf[j] = c->a[it->lo + j];
  } else {
    for (uint64_t j = 0; j < S; ++j) {
      uint64_t r = lsref_splitmix64(h + (j + 1) * GOLDEN_GAMMA);
      uint64_t pos = (uint64_t)(((unsigned __int128)r * (unsigned __int128)n) >> 64);
      c->sbuf[j] = c->a[it->lo + pos];
    }
  }
  heapsort_u64(c->sbuf, S);
}

static uint64_t count_dups(const uint64_t* s, uint64_t S) {
  uint64_t d = 0;
  for (uint64_t j = 1; j < S; ++j) d += (s[j] == s[j - 1]);
  return d;
}

/* Sample imbalance: classify the sample itself with the RMI and return the
 * largest bucket count. */
static uint64_t sample_imbalance(const lsref_model* m, const uint64_t* s, uint64_t S, int dtype, uint32_t B,
                                 uint64_t* cnt) {
  memset(cnt, 0, B * sizeof(uint64_t));
  double P = (double)B;
  for (uint64_t j = 0; j < S; ++j) cnt[refine_id_value(m, ord_value(s[j], dtype), B, P, 0.0)] += 1;
  uint64_t mx = 0;
  for (uint32_t b = 0; b < B; ++b)
    if (cnt[b] > mx) mx = cnt[b];
  return mx;
}

static int process_item(sctx* c, stack_t_* st, item_t it) {
  const lsref_params* p = c->p;
  uint64_t n = it.hi - it.lo;
  uint64_t* a = c->a + it.lo;
  lsref_level_stats* ls = lvl(c, it.level);
  int dtype = c->dtype;
  mslot* inherited = it.model;

#define RELEASE_INHERITED()                         \
  do {                                              \
    if (inherited && --inherited->refs == 0) free(inherited); \
  } while (0)

  /* the first segment's root fills the trace's root fields */
  int record_root = it.is_root && it.segment == 0;
  if (n <= 1) {
    RELEASE_INHERITED();
    return 0;
  }
  if (n <= p->basecase_threshold) {
    base_sort_u64(a, n);
    ls->base_items += 1;
    ls->base_keys += n;
    RELEASE_INHERITED();
    return 0;
  }
  if (it.level > p->max_depth) {
    heapsort_u64(a, n);
    ls->fallback_items += 1;
    ls->fallback_keys += n;
    RELEASE_INHERITED();
    return 0;
  }
  /* Homogeneity check (Sec. 2.2): an all-equal range is already sorted.
   * odiff, the OR over the keys of ord(x) XOR ord(first key), is zero for
   * an all-equal range; its highest set bit is the highest bit in which two
   * keys differ (whatever their order), so every key agrees with every
   * other above bit_length(odiff). */
  uint64_t odiff = 0;
  for (uint64_t i = 1; i < n; ++i) odiff |= a[i] ^ a[0];
  if (odiff == 0) {
    ls->homogeneous += 1;
    if (record_root && c->tr) c->tr->root_decision = LSREF_DEC_HOMOGENEOUS;
    if (it.is_root && c->seg_decision) c->seg_decision[it.segment] = LSREF_DEC_HOMOGENEOUS;
    RELEASE_INHERITED();
    return 0;
  }

  uint32_t B = p->fanout;
  int decision;
  mslot* model = NULL; /* model this item classifies with */
  uint32_t mk = 0;
  uint64_t mg = 0;
  int fresh = 1;
  /* Radix split (a prediction-less partitioner for buckets the model could
   * not split, Sec. 2.4's IPS2Ra radix partitioning): the keys agree above
   * bit `top`; bucket = the bits [s, top) of ord(x), s = max(top - 10, 0). */
  uint32_t rshift = 0;
  if (it.kind == KIND_RADIX) {
    fresh = 0;
    decision = LSREF_DEC_RADIX;
    rshift = it.mk > 10 ? it.mk - 10 : 0;
  }
  if (it.kind == KIND_REFINE) {
    double P = pow_exact(B, it.mk + 1);
    if (P <= REFINE_LIMIT) {
      fresh = 0;
      model = inherited;
      mk = it.mk;
      mg = it.mg;
      decision = LSREF_DEC_LEARNED;
    }
  }
  if (fresh) {
    /* BuildPartitionModel (Alg. 5): sample, sort, duplicate test, model. */
    uint64_t S = lsref_sample_size(n, p);
    if (S > c->sbuf_cap) return LSREF_ENOMEM;
    draw_sample(c, &it, n, S);
    uint64_t dups = count_dups(c->sbuf, S);
    int learned = 0;
    uint64_t imb = 0;
    if (it.kind == KIND_FORCE_SPLITTER) {
      splitter_build_ord(c->sbuf, S, p->splitter_fanout, 1, &c->split);
    } else {
      int want = 0;
      if (p->partitioner == LSREF_PART_LEARNED) want = 1;
      else if (p->partitioner == LSREF_PART_AUTO) {
        double frac = (double)dups / (double)S;
        want = (n >= p->min_learned_n) && (frac <= p->dup_frac);
      }
      if (want) {
        mslot* ms = (mslot*)malloc(sizeof(mslot));
        if (!ms) return LSREF_ENOMEM;
        ms->refs = 0;
        int ok = fit_ord(c->sbuf, S, dtype, B, &ms->m);
        if (ok && p->partitioner == LSREF_PART_AUTO) {
          imb = sample_imbalance(&ms->m, c->sbuf, S, dtype, B, c->cnt);
          double thr = p->imbalance_tau * (double)S;
          thr = thr / (double)B;
          thr = dmax(thr, 16.0);
          if ((double)imb > thr) ok = 0;
        } else if (ok) {
          imb = sample_imbalance(&ms->m, c->sbuf, S, dtype, B, c->cnt);
        }
        if (ok) {
          learned = 1;
          model = ms;
          if (record_root && c->root_model_out) *c->root_model_out = ms->m;
        } else {
          free(ms);
        }
      }
      if (!learned) {
        uint32_t bs = p->splitter_fanout;
        if (p->partitioner == LSREF_PART_AUTO && p->auto_splitter_fanout < bs) bs = p->auto_splitter_fanout;
        splitter_build_ord(c->sbuf, S, bs, 0, &c->split);
      }
    }
    if (learned) decision = LSREF_DEC_LEARNED;
    else decision = c->split.equality ? LSREF_DEC_SPLITTER_EQ : LSREF_DEC_SPLITTER;
    if (record_root && c->tr) {
      c->tr->root_sample_size = S;
      c->tr->root_dups = dups;
      c->tr->root_imbalance_max = imb;
    }
  }

  /* Classify every key, histogram, stable scatter (Sec. 2.2 partitioning). */
  uint32_t nb = (decision == LSREF_DEC_LEARNED) ? B
                : (decision == LSREF_DEC_RADIX) ? (it.mk > rshift ? 1u << (it.mk - rshift) : 2u)
                                                : c->split.nbuckets;
  memset(c->cnt, 0, nb * sizeof(uint64_t));
  if (decision == LSREF_DEC_RADIX) {
    for (uint64_t i = 0; i < n; ++i) {
      uint32_t b = (uint32_t)((a[i] >> rshift) & (uint64_t)(nb - 1));
      c->ids[i] = b;
      c->cnt[b] += 1;
    }
  } else if (decision == LSREF_DEC_LEARNED) {
    double P = pow_exact(B, mk + 1);
    double Bg = (double)((uint64_t)B * mg);
    for (uint64_t i = 0; i < n; ++i) {
      uint32_t b = refine_id_value(&model->m, ord_value(a[i], dtype), B, P, Bg);
      c->ids[i] = b;
      c->cnt[b] += 1;
    }
  } else {
    for (uint64_t i = 0; i < n; ++i) {
      uint32_t b = lsref_splitter_bucket(&c->split, a[i]);
      c->ids[i] = b;
      c->cnt[b] += 1;
    }
  }
  if (record_root && c->tr) {
    c->tr->root_decision = decision;
    c->tr->root_nbuckets = nb;
  }
  if (record_root && c->root_hist_out) memcpy(c->root_hist_out, c->cnt, nb * sizeof(uint64_t));
  if (it.is_root && c->seg_decision) c->seg_decision[it.segment] = decision;
  /* exclusive scan + stable scatter */
  uint64_t run = 0;
  uint64_t* start = (uint64_t*)malloc((nb + 1) * sizeof(uint64_t));
  if (!start) return LSREF_ENOMEM;
  for (uint32_t b = 0; b < nb; ++b) {
    start[b] = run;
    run += c->cnt[b];
  }
  start[nb] = run;
  uint64_t* cur = (uint64_t*)malloc(nb * sizeof(uint64_t));
  if (!cur) {
    free(start);
    return LSREF_ENOMEM;
  }
  memcpy(cur, start, nb * sizeof(uint64_t));
  for (uint64_t i = 0; i < n; ++i) c->tmp[cur[c->ids[i]]++] = a[i];
  memcpy(a, c->tmp, n * sizeof(uint64_t));
  free(cur);

  ls->items += 1;
  ls->keys += n;
  if (decision == LSREF_DEC_LEARNED) ls->learned += 1;
  else if (decision == LSREF_DEC_RADIX) ls->radix += 1;
  else if (decision == LSREF_DEC_SPLITTER) ls->splitter += 1;
  else ls->splitter_eq += 1;
  int noprog = 0;
  for (uint32_t b = 0; b < nb; ++b) {
    uint64_t sz = c->cnt[b];
    if (sz > ls->max_child) ls->max_child = sz;
    ls->sumsq_child += sz * sz;
    if (sz == n) noprog = 1;
  }
  int eq = (decision == LSREF_DEC_SPLITTER || decision == LSREF_DEC_SPLITTER_EQ) && c->split.equality;
  if (noprog) {
    /* an all-in-one equality bucket is final, not a failed split */
    int only_eq = 0;
    for (uint32_t b = 0; b < nb; ++b)
      if (c->cnt[b] == n && eq && (b & 1)) only_eq = 1;
    if (!only_eq) ls->noprogress += 1;
  }

  /* Children, pushed in reverse so they are processed in bucket order. */
  int refine_children = (decision == LSREF_DEC_LEARNED) && (p->recurse_model == LSREF_RECURSE_REFINE_GLOBAL);
  for (uint32_t bb = nb; bb-- > 0;) {
    uint64_t sz = c->cnt[bb];
    if (eq && (bb & 1)) {
      ls->eq_keys += sz;
      continue; /* equality bucket: final (Sec. 2.4) */
    }
    if (sz <= 1) continue;
    item_t ch;
    memset(&ch, 0, sizeof ch);
    ch.lo = it.lo + start[bb];
    ch.hi = ch.lo + sz;
    ch.segment = it.segment;
    ch.level = it.level + 1;
    ch.gidx = it.gidx * nb + bb;
    /* Under REFINE_GLOBAL no bucket below a learned item draws a new sample
     * (LearnedSort 2.0 trains once, Sec. 2.2): a child the model did not
     * split (no progress), or one that would refine past the FP64 limit
     * B^(k+1) > 2^50, takes the radix split on the bits where this item's
     * keys differ; a radix item's children split the next bits down. */
    if (decision == LSREF_DEC_RADIX) {
      ch.kind = KIND_RADIX;
      ch.mk = rshift;
    } else if (refine_children && (sz == n || pow_exact(B, mk + 2) > REFINE_LIMIT)) {
      ch.kind = KIND_RADIX;
      ch.mk = 64 - (uint32_t)__builtin_clzll(odiff);
    } else if (sz == n) {
      ch.kind = KIND_FORCE_SPLITTER; /* no-progress guard */
    } else if (refine_children) {
      ch.kind = KIND_REFINE;
      ch.model = model;
      ch.mk = mk + 1;
      ch.mg = mg * B + bb;
      model->refs += 1;
    } else {
      ch.kind = KIND_FRESH;
    }
    if (push(st, &ch)) {
      free(start);
      return LSREF_ENOMEM;
    }
  }
  free(start);
  /* Drop this item's reference; a freshly fitted model lives while refine
   * children reference it. */
  if (fresh && model && model->refs == 0) free(model);
  RELEASE_INHERITED();
#undef RELEASE_INHERITED
  return 0;
}

static int run_sort(uint64_t* keys, const uint64_t* off, uint32_t nseg, int dtype, const lsref_params* p,
                    lsref_trace* tr, lsref_model* root_model, uint64_t* root_hist, int32_t* seg_decision) {
  if (!keys && off[nseg] > 0) return LSREF_EINVAL;
  if (!p || p->fanout < 2 || p->fanout > LSREF_MAX_FANOUT || p->splitter_fanout < 2 ||
      p->splitter_fanout > LSREF_MAX_FANOUT || (dtype != LSREF_F64 && dtype != LSREF_U64))
    return LSREF_EINVAL;
  uint64_t n = off[nseg];
  if (tr) {
    memset(tr, 0, sizeof *tr);
    tr->root_decision = LSREF_DEC_NONE;
  }
  /* Validate: NaN keys have no place in the order. */
  if (dtype == LSREF_F64) {
    for (uint64_t i = 0; i < n; ++i) {
      uint64_t b = keys[i];
      if ((b & 0x7FF0000000000000ull) == 0x7FF0000000000000ull && (b & 0x000FFFFFFFFFFFFFull)) {
        if (tr) tr->status = LSREF_ENAN;
        return LSREF_ENAN;
      }
    }
  }
  sctx c;
  memset(&c, 0, sizeof c);
  c.dtype = dtype;
  c.p = p;
  c.tr = tr;
  c.root_model_out = root_model;
  c.root_hist_out = root_hist;
  c.seg_decision = seg_decision;
  uint64_t maxseg = 0;
  for (uint32_t s = 0; s < nseg; ++s)
    if (off[s + 1] - off[s] > maxseg) maxseg = off[s + 1] - off[s];
  c.a = keys;
  c.tmp = (uint64_t*)malloc((maxseg ? maxseg : 1) * sizeof(uint64_t));
  c.ids = (uint32_t*)malloc((maxseg ? maxseg : 1) * sizeof(uint32_t));
  c.cnt = (uint64_t*)malloc((2 * LSREF_MAX_FANOUT + 2) * sizeof(uint64_t));
  c.sbuf_cap = maxseg ? maxseg : 1;
  c.sbuf = (uint64_t*)malloc(c.sbuf_cap * sizeof(uint64_t));
  stack_t_ st = {0, 0, 0};
  int rc = 0;
  if (!c.tmp || !c.ids || !c.cnt || !c.sbuf) rc = LSREF_ENOMEM;
  for (uint64_t i = 0; i < n && !rc; ++i) keys[i] = lsref_ord(keys[i], dtype);
  for (uint32_t s = 0; s < nseg && !rc; ++s) {
    item_t root;
    memset(&root, 0, sizeof root);
    root.lo = off[s];
    root.hi = off[s + 1];
    root.segment = s;
    root.kind = KIND_FRESH;
    root.is_root = 1;
    if (seg_decision) seg_decision[s] = LSREF_DEC_NONE;
    if (push(&st, &root)) rc = LSREF_ENOMEM;
    while (st.n > 0 && !rc) {
      item_t it = st.v[--st.n];
      rc = process_item(&c, &st, it);
    }
  }
  /* release any models still referenced if we stopped early */
  while (st.n > 0) {
    item_t it = st.v[--st.n];
    if (it.model && --it.model->refs == 0) free(it.model);
  }
  for (uint64_t i = 0; i < n; ++i) keys[i] = lsref_unord(keys[i], dtype);
  if (tr) {
    /* levels used: the deepest level where anything was recorded */
    tr->levels_used = 0;
    for (uint32_t l = 0; l < LSREF_MAX_LEVELS; ++l) {
      const lsref_level_stats* q = &tr->level[l];
      if (q->items || q->base_items || q->homogeneous || q->fallback_items) tr->levels_used = l + 1;
    }
    tr->status = rc;
  }
  free(st.v);
  free(c.tmp);
  free(c.ids);
  free(c.cnt);
  free(c.sbuf);
  return rc;
}

int lsref_sort(uint64_t* keys, uint64_t n, int dtype, const lsref_params* p, lsref_trace* tr,
               lsref_model* root_model, uint64_t* root_hist) {
  uint64_t off[2] = {0, n};
  return run_sort(keys, off, 1, dtype, p, tr, root_model, root_hist, NULL);
}

int lsref_sort_segmented(uint64_t* keys, const uint64_t* off, uint32_t nseg, int dtype, const lsref_params* p,
                         lsref_trace* tr, int32_t* seg_decision) {
  for (uint32_t s = 0; s < nseg; ++s)
    if (off[s + 1] < off[s]) return LSREF_EINVAL;
  return run_sort(keys, off, nseg, dtype, p, tr, NULL, NULL, seg_decision);
}

int lsref_root_decision(const uint64_t* keys, uint64_t n, int dtype, const lsref_params* p, uint64_t segment,
                        lsref_trace* tr, lsref_model* m, lsref_splitter* t, uint64_t* sorted_sample_out) {
  if (n == 0) return LSREF_EINVAL;
  uint64_t S = lsref_sample_size(n, p);
  uint64_t* s = (uint64_t*)malloc(S * sizeof(uint64_t));
  uint64_t* cnt = (uint64_t*)malloc(LSREF_MAX_FANOUT * sizeof(uint64_t));
  if (!s || !cnt) return LSREF_ENOMEM;
  uint64_t h = lsref_seed_item(p->seed, segment, 0, 0);
  if (S >= n) {
    for (uint64_t j = 0; j < n; ++j) s[j] = lsref_ord(keys[j], dtype);
  } else {
    for (uint64_t j = 0; j < S; ++j) {
      uint64_t r = lsref_splitmix64(h + (j + 1) * GOLDEN_GAMMA);
      uint64_t pos = (uint64_t)(((unsigned __int128)r * (unsigned __int128)n) >> 64);
      s[j] = lsref_ord(keys[pos], dtype);
    }
  }
  heapsort_u64(s, S);
  if (sorted_sample_out)
    for (uint64_t j = 0; j < S; ++j) sorted_sample_out[j] = lsref_unord(s[j], dtype);
  uint64_t dups = count_dups(s, S);
  int ok = fit_ord(s, S, dtype, p->fanout, m);
  uint64_t imb = ok ? sample_imbalance(m, s, S, dtype, p->fanout, cnt) : 0;
  int learned = 0;
  if (p->partitioner == LSREF_PART_LEARNED) learned = ok;
  else if (p->partitioner == LSREF_PART_AUTO) {
    double frac = (double)dups / (double)S;
    double thr = p->imbalance_tau * (double)S;
    thr = thr / (double)p->fanout;
    thr = dmax(thr, 16.0);
    learned = ok && n >= p->min_learned_n && frac <= p->dup_frac && !((double)imb > thr);
  }
  uint32_t bs = p->splitter_fanout;
  if (p->partitioner == LSREF_PART_AUTO && p->auto_splitter_fanout < bs) bs = p->auto_splitter_fanout;
  splitter_build_ord(s, S, bs, 0, t);
  if (tr) {
    memset(tr, 0, sizeof *tr);
    tr->root_sample_size = S;
    tr->root_dups = dups;
    tr->root_imbalance_max = imb;
    tr->root_decision = learned ? LSREF_DEC_LEARNED : (t->equality ? LSREF_DEC_SPLITTER_EQ : LSREF_DEC_SPLITTER);
    tr->root_nbuckets = learned ? p->fanout : t->nbuckets;
  }
  free(s);
  free(cnt);
  return LSREF_OK;
}
