/*
 * Seeded synthetic inputs for the global Curveball super step.
 *
 * Degree sequences follow the integer power-law distribution PLD([a,b), gamma)
 * of Section 2 ("Randomisation and Distributions": P[X=k] proportional to
 * k^-gamma for a <= k < b); graphs are realised with Havel-Hakimi, as in the
 * runtime experiments of Section 5.2.  This module holds none of the Curveball
 * method's arithmetic: it only builds the seeded input graphs that both the
 * CUDA path and the CPU oracle consume.
 *
 * Determinism across machines: the same seed must give the same graph on the
 * x86 build host and on the aarch64 GPU host.  Everything below uses only
 * integer arithmetic and IEEE-754 +,-,*,/ in a fixed order (the file is built
 * with -ffp-contract=off), and no libm transcendental function.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- counter-based uniform draws: SplitMix64 (Steele, Lea, Flood 2014) ---- */
static uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
/* i-th 64-bit draw of stream `stream` under `seed`. */
static uint64_t sm_draw(uint64_t seed, uint64_t stream, uint64_t i) {
  uint64_t base = sm_mix(seed + stream * 0x632be59bd9b4e019ULL + 0x9e3779b97f4a7c15ULL);
  return sm_mix(base + (i + 1) * 0x9e3779b97f4a7c15ULL);
}
/* uniform double in [0,1) with 53 random bits */
static double sm_unif(uint64_t seed, uint64_t stream, uint64_t i) {
  return (double)(sm_draw(seed, stream, i) >> 11) * (1.0 / 9007199254740992.0);
}

/* ---- portable natural log / exp (series; only + - * / in fixed order) ---- */
static const double LN2 = 0.693147180559945309417232121458176568; /* ln 2 */

/* ln x for x >= 1 via x = m 2^e, ln m = 2 atanh((m-1)/(m+1)). */
static double p_ln(double x) {
  int e = 0;
  while (x >= 2.0) { x *= 0.5; e++; }
  if (x > 1.4142135623730951) { x *= 0.5; e++; }
  double s = (x - 1.0) / (x + 1.0), s2 = s * s, term = s, sum = 0.0;
  for (int k = 1; k < 80; k += 2) { sum += term / (double)k; term *= s2; }
  return 2.0 * sum + (double)e * LN2;
}
/* e^y for y <= 0 via y = q ln2 + r, |r| < ln2, Taylor series for e^r. */
static double p_exp_neg(double y) {
  int q = (int)(y / LN2);           /* truncation toward zero, q <= 0 */
  double r = y - (double)q * LN2;    /* r in (-ln2, ln2) */
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 40; k++) { term *= r / (double)k; sum += term; }
  for (; q < 0; q++) sum *= 0.5;     /* exact scaling */
  return sum;
}
/* k^-gamma; exact IEEE paths for gamma = 2 and 3. */
static double p_pow_neg(int64_t k, double gamma) {
  double dk = (double)k;
  if (gamma == 2.0) return 1.0 / (dk * dk);
  if (gamma == 3.0) return 1.0 / (dk * dk * dk);
  return p_exp_neg(-gamma * p_ln(dk));
}

/* Uniform double in [0,1): exported so that ensemble / serving parameter
 * draws (graph sizes, exponents, arrival times) use the same portable stream. */
double cb_synth_uniform(uint64_t seed, uint64_t stream, uint64_t i) {
  return sm_unif(seed, stream, i);
}
/* 2^x for x >= 0 (portable), used for log-uniform graph sizes. */
double cb_synth_exp2(double x) {
  int q = (int)x;
  double r = x - (double)q;          /* r in [0,1) */
  double v = (r == 0.0) ? 1.0 : 1.0 / p_exp_neg(-r * LN2);
  for (; q > 0; q--) v *= 2.0;
  return v;
}

/*
 * Draw n i.i.d. degrees from PLD([a,b), gamma) with stream 0 of `seed`
 * (inverse CDF over the exact pmf table); if the sum is odd, add 1 to the last
 * degree.  Returns the degree sum, or -1 on bad arguments.
 */
int64_t cb_synth_pld(int64_t n, int32_t a, int32_t b, double gamma, uint64_t seed,
                     int32_t* deg_out) {
  if (n < 0 || a < 0 || b <= a || !deg_out) return -1;
  int64_t K = (int64_t)b - a;
  double* cdf = (double*)malloc(sizeof(double) * (size_t)K);
  if (!cdf) return -1;
  double z = 0.0;
  for (int64_t j = 0; j < K; j++) {
    z += (a + j == 0) ? 0.0 : p_pow_neg(a + j, gamma);
    cdf[j] = z;
  }
  int64_t sum = 0;
  for (int64_t i = 0; i < n; i++) {
    double u = sm_unif(seed, 0, (uint64_t)i) * z;
    int64_t lo = 0, hi = K - 1;
    while (lo < hi) {                 /* smallest j with cdf[j] > u */
      int64_t mid = (lo + hi) >> 1;
      if (cdf[mid] > u) hi = mid; else lo = mid + 1;
    }
    deg_out[i] = (int32_t)(a + lo);
    sum += deg_out[i];
  }
  if ((sum & 1) && n > 0) { deg_out[n - 1] += 1; sum += 1; }
  free(cdf);
  return sum;
}

static int cmp_i32(const void* p, const void* q) {
  int32_t x = *(const int32_t*)p, y = *(const int32_t*)q;
  return (x > y) - (x < y);
}

/*
 * Havel-Hakimi realisation of degree sequence deg[0..n-1] (sum even).
 * Repeatedly take a node x of maximum residual degree d and join it to the d
 * nodes of next-highest residual degree.  Nodes are kept in an array ordered by
 * residual degree (descending) with one contiguous bucket per residual value,
 * so each step costs O(d + number of distinct residuals among the targets):
 * O(n + m + max degree) overall.  Ties inside a bucket follow the array order,
 * which this procedure defines deterministically.
 *
 * Output: CSR with rows sorted ascending; row_ptr has n+1 entries, col has
 * sum(deg) entries (both caller-allocated).  Returns m = sum/2, or -1 if the
 * sequence is not graphical (the Havel-Hakimi test fails), -2 on bad input,
 * -3 on allocation failure.
 */
int64_t cb_synth_hh(int64_t n, const int32_t* deg, int64_t* row_ptr, int32_t* col) {
  if (n < 0 || (n > 0 && (!deg || !col)) || !row_ptr) return -2;
  int64_t S = 0;
  int32_t D = 0;
  for (int64_t i = 0; i < n; i++) {
    if (deg[i] < 0 || deg[i] >= n) return (deg[i] < 0) ? -2 : -1;
    S += deg[i];
    if (deg[i] > D) D = deg[i];
  }
  if (S & 1) return -1;
  row_ptr[0] = 0;
  for (int64_t i = 0; i < n; i++) row_ptr[i + 1] = row_ptr[i] + deg[i];
  if (n == 0) return 0;

  int64_t* ord = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int32_t* res = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int64_t* bs = (int64_t*)calloc((size_t)D + 2, sizeof(int64_t));
  int64_t* cnt = (int64_t*)calloc((size_t)D + 2, sizeof(int64_t));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!ord || !res || !bs || !cnt || !fill) {
    free(ord); free(res); free(bs); free(cnt); free(fill);
    return -3;
  }
  for (int64_t i = 0; i < n; i++) { res[i] = deg[i]; cnt[deg[i]]++; fill[i] = row_ptr[i]; }
  /* buckets laid out from residual D down to 0 */
  bs[D] = 0;
  for (int64_t r = (int64_t)D - 1; r >= 0; r--) bs[r] = bs[r + 1] + cnt[r + 1];
  {
    int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * ((size_t)D + 1));
    if (!cur) { free(ord); free(res); free(bs); free(cnt); free(fill); return -3; }
    for (int64_t r = 0; r <= D; r++) cur[r] = bs[r];
    for (int64_t i = 0; i < n; i++) ord[cur[deg[i]]++] = i;   /* ties by id */
    free(cur);
  }

  int64_t front = 0, result = S / 2;
  while (front < n) {
    int64_t x = ord[front];
    int32_t d = res[x];
    if (d == 0) break;                       /* everything left is exhausted */
    bs[d]++; cnt[d]--; res[x] = 0; front++;  /* consume x */
    if (front + d > n || res[ord[front + d - 1]] == 0) { result = -1; break; }
    int32_t r_top = res[ord[front]];
    int32_t r_last = res[ord[front + d - 1]];
    int64_t start = bs[r_last], c = cnt[r_last];
    int64_t k = front + d - start;           /* targets inside bucket r_last */
    for (int64_t i = 0; i < d; i++) {
      int64_t y = ord[front + i];
      col[fill[x]++] = (int32_t)y;
      col[fill[y]++] = (int32_t)x;
      res[y] -= 1;
    }
    /* move the k decremented members of bucket r_last to its end */
    if (k < c) {
      if (2 * k <= c) {
        for (int64_t i = 0; i < k; i++) {
          int64_t t = ord[start + i]; ord[start + i] = ord[start + c - k + i]; ord[start + c - k + i] = t;
        }
      } else {
        for (int64_t i = 0; i < c - k; i++) {
          int64_t t = ord[start + i]; ord[start + i] = ord[start + k + i]; ord[start + k + i] = t;
        }
      }
    }
    int64_t keep = c - k;
    /* bucket r_last-1 gains the k decremented members at its front */
    bs[r_last - 1] = start + keep;
    cnt[r_last - 1] += k;
    if (r_top > r_last) {
      /* buckets r_last+1..r_top were fully decremented: relabel them down */
      bs[r_last] = (cnt[r_last + 1] > 0) ? bs[r_last + 1] : start;
      cnt[r_last] = cnt[r_last + 1] + keep;
      for (int64_t r = (int64_t)r_last + 2; r <= r_top; r++) { bs[r - 1] = bs[r]; cnt[r - 1] = cnt[r]; }
      cnt[r_top] = 0;
    } else {
      cnt[r_last] = keep;
    }
  }
  if (result >= 0) {
    for (int64_t i = 0; i < n; i++) if (res[i] != 0) { result = -1; break; }
  }
  free(ord); free(res); free(bs); free(cnt);
  if (result >= 0) {
    for (int64_t i = 0; i < n; i++)
      if (fill[i] != row_ptr[i + 1]) { result = -1; break; }
  }
  free(fill);
  if (result < 0) return result;
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < n; i++) {
    int64_t len = row_ptr[i + 1] - row_ptr[i];
    if (len > 1) qsort(col + row_ptr[i], (size_t)len, sizeof(int32_t), cmp_i32);
  }
  return result;
}
