/*
 * tr_oracle.c -- CPU oracle for the transform-reduce-scan path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load it (through oracle/__init__.py).  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * What it computes (plain definitions, FP64 and exact integers, plain loops):
 *   - the map family  y = f(x): Horner polynomial, rational P/Q, fixed-step
 *     Newton cube-root iterate, square, xorshift32, splitmix32;
 *   - full and segmented sum / min / max of f over an array;
 *   - inclusive scans of f (u32 modulo 2^32, u32 widened to u64, and floating
 *     point with the exact prefix rounded once per element);
 *   - the dense Vandermonde product Y = V(x) C evaluated by FP64 Horner, plus
 *     the normwise scale S = |V| |C| used for error metrics.
 *
 * The paper (Mejstrik, "__host__ __device__ -- Generic programming in Cuda")
 * prescribes none of this arithmetic: it is about writing such functions once
 * for host, device and compile time (its "hdc" functions, Sec. 2 and the hdc
 * helper of Sec. 4).  The definitions below therefore follow the named
 * textbook methods cited at each function.
 *
 * Floating-point sums are EXACT: every addend (a double) is accumulated into a
 * fixed-point register that covers the whole double range (Kulisch & Miranker,
 * "The arithmetic of the digital computer", 1986), and the result is rounded
 * once, to nearest-even, to the requested precision.  So sums do not depend on
 * order.  Map values themselves are FP64 results of the stated operation
 * sequence (explicit fma in Horner, one IEEE division in P/Q), which is the
 * closest plain reading of "evaluate f in FP64".
 *
 * The *_mt functions at the end run the same arithmetic on several host
 * threads (to time the oracle on all cores and to check whole benchmark
 * outputs); their results are identical to the single-thread functions.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared -pthread (no SIMD
 * intrinsics, no -ffast-math); the C library's fma() is correctly rounded
 * (C99 7.12.13.1).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Exact accumulator                                                         */
/* ------------------------------------------------------------------------ */

/* Bit b of the register weighs 2^(b - ORC_BIAS); bit 0 is the smallest
 * subnormal double 2^-1074.  68 limbs of 32 bits (2176 bits) hold any double
 * (top bit 2^1023 sits at bit 2097, plus 53 mantissa bits shifted in) with
 * room for ~2^40 maximal addends; the top limb is a signed 64-bit integer and
 * carries the sign. */
#define ORC_BIAS 1074
#define ORC_LIMBS 68

typedef struct {
  int64_t d[ORC_LIMBS];
  int64_t pending; /* additions since the last carry propagation */
} orc_acc;

static void acc_clear(orc_acc* a) { memset(a, 0, sizeof(*a)); }

/* floor(v / 2^32) without relying on the sign behaviour of >> */
static int64_t floor_div32(int64_t v) {
  if (v >= 0) return v / 4294967296LL;
  return -((-v + 4294967295LL) / 4294967296LL);
}

/* Propagate carries so that limbs 0..LIMBS-2 lie in [0, 2^32). */
static void acc_norm(orc_acc* a) {
  for (int i = 0; i < ORC_LIMBS - 1; ++i) {
    int64_t c = floor_div32(a->d[i]);
    a->d[i] -= c * 4294967296LL;
    a->d[i + 1] += c;
  }
  a->pending = 0;
}

static void acc_add(orc_acc* a, double v) {
  if (v == 0.0) return;
  int e;
  double f = frexp(fabs(v), &e);        /* |v| = f * 2^e, f in [0.5, 1) */
  uint64_t m = (uint64_t)ldexp(f, 53);  /* exact: f has <= 53 significant bits */
  int sh = e - 53 + ORC_BIAS;           /* weight of m's least bit */
  while (sh < 0) { m >>= 1; ++sh; }     /* subnormals: the dropped bits are 0 */
  int li = sh / 32, off = sh % 32;
  unsigned __int128 w = (unsigned __int128)m << off; /* < 2^85: three limbs */
  int64_t s = v < 0 ? -1 : 1;
  a->d[li] += s * (int64_t)(uint32_t)w;
  a->d[li + 1] += s * (int64_t)(uint32_t)(w >> 32);
  a->d[li + 2] += s * (int64_t)(uint32_t)(w >> 64);
  if (++a->pending >= (1LL << 29)) acc_norm(a);
}

static int acc_bit(const orc_acc* a, int b) { return (int)((a->d[b / 32] >> (b % 32)) & 1); }

/* Round the exact value to a binary floating-point number with p significant
 * bits whose smallest quantum is bit qmin (qmin = 0: double subnormals;
 * qmin = 1074 - 149: float subnormals).  Round to nearest, ties to even. */
static double acc_round(const orc_acc* src, int p, int qmin) {
  orc_acc a = *src;
  acc_norm(&a);
  int neg = a.d[ORC_LIMBS - 1] < 0;
  if (neg) {
    for (int i = 0; i < ORC_LIMBS; ++i) a.d[i] = -a.d[i];
    acc_norm(&a);
  }
  int top = -1;
  for (int i = ORC_LIMBS - 1; i >= 0 && top < 0; --i)
    if (a.d[i] != 0)
      for (int b = 31; b >= 0; --b)
        if ((a.d[i] >> b) & 1) { top = i * 32 + b; break; }
  if (top < 0) return 0.0;
  if (top >= ORC_LIMBS * 32 - 32) return neg ? -INFINITY : INFINITY; /* never on these inputs */
  int lsb = top - p + 1;
  if (lsb < qmin) lsb = qmin;
  uint64_t mant = 0;
  for (int b = top; b >= lsb; --b) mant = (mant << 1) | (uint64_t)acc_bit(&a, b);
  int guard = (lsb >= 1 && lsb - 1 <= top) ? acc_bit(&a, lsb - 1) : 0;
  int sticky = 0;
  for (int b = lsb - 2; b >= 0 && !sticky; --b) sticky = acc_bit(&a, b);
  if (guard && (sticky || (mant & 1))) mant += 1;
  double r = ldexp((double)mant, lsb - ORC_BIAS);
  return neg ? -r : r;
}

/* Exact sum of v[0..n) rounded once to p bits (p = 53: double, p = 24: float). */
double orc_exact_sum(const double* v, int64_t n, int p) {
  orc_acc a;
  acc_clear(&a);
  for (int64_t i = 0; i < n; ++i) acc_add(&a, v[i]);
  return acc_round(&a, p, p == 24 ? ORC_BIAS - 149 : 0);
}

/* ------------------------------------------------------------------------ */
/* Map family                                                                */
/* ------------------------------------------------------------------------ */

enum { ORC_IDENTITY = 0, ORC_SQUARE, ORC_HORNER, ORC_RATIONAL, ORC_NEWTON_CBRT, ORC_XORSHIFT32, ORC_SPLITMIX32 };

typedef struct {
  int32_t kind;
  int32_t deg_p, deg_q, iters;
  const double* cp; /* deg_p + 1 coefficients, ascending powers */
  const double* cq; /* deg_q + 1 coefficients, ascending powers */
} orc_map;

/* Horner's rule with ascending coefficients c[0..d]:
 * p = c_d;  p = fma(p, x, c_k) for k = d-1 .. 0. */
static double horner(const double* c, int d, double x) {
  double p = c[d];
  for (int k = d - 1; k >= 0; --k) p = fma(p, x, c[k]);
  return p;
}

/* Fixed-step Newton iteration for y^3 = x started at y_0 = sign(x):
 * y <- (2y + x / y^2) / 3, `iters` times.  The result is the iterate. */
static double newton_cbrt(double x, int iters) {
  double y = copysign(1.0, x);
  for (int k = 0; k < iters; ++k) y = (2.0 * y + x / (y * y)) / 3.0;
  return y;
}

static double map_f64(const orc_map* m, double x) {
  switch (m->kind) {
    case ORC_IDENTITY: return x;
    case ORC_SQUARE: return x * x;
    case ORC_HORNER: return horner(m->cp, m->deg_p, x);
    case ORC_RATIONAL: return horner(m->cp, m->deg_p, x) / horner(m->cq, m->deg_q, x);
    case ORC_NEWTON_CBRT: return newton_cbrt(x, m->iters);
    default: return NAN;
  }
}

/* Marsaglia, "Xorshift RNGs", J. Stat. Softw. 8(14), 2003: the 32-bit
 * generator step with shift triple (13, 17, 5). */
static uint32_t xorshift32(uint32_t x) {
  x ^= x << 13;
  x ^= x >> 17;
  x ^= x << 5;
  return x;
}

/* 32-bit splitmix-style finaliser: add a Weyl increment, then two rounds of
 * xor-shift-right followed by an odd multiply, then a final xor-shift.
 * Increment floor(2^32 / golden ratio); multipliers are the first 32 bits of
 * the fractional parts of sqrt(2) and sqrt(3).  All arithmetic mod 2^32. */
static uint32_t splitmix32(uint32_t x) {
  uint32_t z = x + 0x9E3779B9u;
  z = (z ^ (z >> 16)) * 0x6A09E667u;
  z = (z ^ (z >> 13)) * 0xBB67AE85u;
  return z ^ (z >> 16);
}

static uint32_t map_u32(int kind, uint32_t x) {
  switch (kind) {
    case ORC_IDENTITY: return x;
    case ORC_XORSHIFT32: return xorshift32(x);
    case ORC_SPLITMIX32: return splitmix32(x);
    default: return 0;
  }
}

/* The same maps evaluated in IEEE binary32 (the precision of the FP32-compute
 * paths): coefficients and inputs are binary32 values (the callers pass doubles
 * that are exactly representable), every operation is one binary32 operation
 * of the stated sequence -- fmaf in Horner, one float division in P/Q, the
 * Newton step RN(RN(2y + RN(x / RN(y*y))) / 3) with 2y exact -- and the result
 * is returned widened exactly to double. */
static float horner_f32(const double* c, int d, float x) {
  float p = (float)c[d];
  for (int k = d - 1; k >= 0; --k) p = fmaf(p, x, (float)c[k]);
  return p;
}

static float map_f32(const orc_map* m, float x) {
  switch (m->kind) {
    case ORC_IDENTITY: return x;
    case ORC_SQUARE: return x * x;
    case ORC_HORNER: return horner_f32(m->cp, m->deg_p, x);
    case ORC_RATIONAL: return horner_f32(m->cp, m->deg_p, x) / horner_f32(m->cq, m->deg_q, x);
    case ORC_NEWTON_CBRT: {
      float y = copysignf(1.0f, x);
      for (int k = 0; k < m->iters; ++k) y = fmaf(2.0f, y, x / (y * y)) / 3.0f;
      return y;
    }
    default: return NAN;
  }
}

void orc_map_f32(const orc_map* m, const double* x, double* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] = (double)map_f32(m, (float)x[i]);
}

void orc_map_f64(const orc_map* m, const double* x, double* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] = map_f64(m, x[i]);
}

void orc_map_u32(int32_t kind, const uint32_t* x, uint32_t* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] = map_u32(kind, x[i]);
}

/* ------------------------------------------------------------------------ */
/* Reductions                                                                */
/* ------------------------------------------------------------------------ */

/* out[0] = exact sum of f(x_i) rounded to double, out[1] = min, out[2] = max.
 * Empty input: 0, +inf, -inf. */
void orc_reduce_f64(const orc_map* m, const double* x, int64_t n, double* out) {
  orc_acc a;
  acc_clear(&a);
  double mn = INFINITY, mx = -INFINITY;
  for (int64_t i = 0; i < n; ++i) {
    double f = map_f64(m, x[i]);
    acc_add(&a, f);
    if (f < mn) mn = f;
    if (f > mx) mx = f;
  }
  out[0] = acc_round(&a, 53, 0);
  out[1] = mn;
  out[2] = mx;
}

/* Exact u64 sum (no wraparound below 2^32 elements), min, max of f(x_i).
 * Empty input: 0, UINT32_MAX, 0. */
void orc_reduce_u32(int32_t kind, const uint32_t* x, int64_t n, uint64_t* sum, uint32_t* mn, uint32_t* mx) {
  uint64_t s = 0;
  uint32_t lo = 0xFFFFFFFFu, hi = 0;
  for (int64_t i = 0; i < n; ++i) {
    uint32_t f = map_u32(kind, x[i]);
    s += f;
    if (f < lo) lo = f;
    if (f > hi) hi = f;
  }
  *sum = s;
  *mn = lo;
  *mx = hi;
}

/* Segment s covers elements [off[s], off[s+1]).  Per segment: exact sum
 * rounded to double, min and max of f; an empty segment gets 0, +inf, -inf. */
void orc_segreduce_f64(const orc_map* m, const double* x, const int64_t* off, int64_t nseg, double* sums,
                       double* mins, double* maxs) {
  for (int64_t s = 0; s < nseg; ++s) {
    double out[3];
    orc_reduce_f64(m, x + off[s], off[s + 1] - off[s], out);
    sums[s] = out[0];
    mins[s] = out[1];
    maxs[s] = out[2];
  }
}

/* Sum of the mixer over the integer range [lo, hi) (hi <= 2^32), exact in u64. */
uint64_t orc_mixer_range_sum(int32_t kind, uint64_t lo, uint64_t hi) {
  uint64_t s = 0;
  for (uint64_t v = lo; v < hi; ++v) s += map_u32(kind, (uint32_t)v);
  return s;
}

/* ------------------------------------------------------------------------ */
/* Inclusive scans                                                           */
/* ------------------------------------------------------------------------ */

/* y_i = f(x_0) + ... + f(x_i) modulo 2^32. */
void orc_scan_u32(int32_t kind, const uint32_t* x, uint32_t* y, int64_t n) {
  uint32_t s = 0;
  for (int64_t i = 0; i < n; ++i) { s += map_u32(kind, x[i]); y[i] = s; }
}

/* y_i = f(x_0) + ... + f(x_i) in u64 (exact for n < 2^32). */
void orc_scan_u32_u64(int32_t kind, const uint32_t* x, uint64_t* y, int64_t n) {
  uint64_t s = 0;
  for (int64_t i = 0; i < n; ++i) { s += map_u32(kind, x[i]); y[i] = s; }
}

/* y_i = exact prefix sum of f rounded once to p bits (p = 24 for a float
 * result, 53 for double). */
void orc_scan_f64(const orc_map* m, const double* x, double* y, int64_t n, int p) {
  orc_acc a;
  acc_clear(&a);
  int qmin = p == 24 ? ORC_BIAS - 149 : 0;
  for (int64_t i = 0; i < n; ++i) {
    acc_add(&a, map_f64(m, x[i]));
    y[i] = acc_round(&a, p, qmin);
  }
}

/* Exclusive scans: y_0 = 0 and y_i = f(x_0) + ... + f(x_{i-1}), each output
 * written before its own element is added (u32 modulo 2^32; u32 widened to
 * u64; floating point exact, rounded once to p bits). */
void orc_scan_u32_excl(int32_t kind, const uint32_t* x, uint32_t* y, int64_t n) {
  uint32_t s = 0;
  for (int64_t i = 0; i < n; ++i) { y[i] = s; s += map_u32(kind, x[i]); }
}

void orc_scan_u32_u64_excl(int32_t kind, const uint32_t* x, uint64_t* y, int64_t n) {
  uint64_t s = 0;
  for (int64_t i = 0; i < n; ++i) { y[i] = s; s += map_u32(kind, x[i]); }
}

void orc_scan_f64_excl(const orc_map* m, const double* x, double* y, int64_t n, int p) {
  orc_acc a;
  acc_clear(&a);
  int qmin = p == 24 ? ORC_BIAS - 149 : 0;
  for (int64_t i = 0; i < n; ++i) {
    y[i] = acc_round(&a, p, qmin);
    acc_add(&a, map_f64(m, x[i]));
  }
}

/* The same exact prefixes, rounded only at the sorted positions pos[0..m)
 * (for checking very long scans at sampled outputs). */
void orc_scan_f64_sampled(const orc_map* m, const double* x, int64_t n, const int64_t* pos, int64_t npos, double* out,
                          int p) {
  orc_acc a;
  acc_clear(&a);
  int qmin = p == 24 ? ORC_BIAS - 149 : 0;
  int64_t k = 0;
  for (int64_t i = 0; i < n && k < npos; ++i) {
    acc_add(&a, map_f64(m, x[i]));
    while (k < npos && pos[k] == i) out[k++] = acc_round(&a, p, qmin);
  }
}

/* ------------------------------------------------------------------------ */
/* Dense Vandermonde product                                                 */
/* ------------------------------------------------------------------------ */

/* Y[r][j] = sum_k C[k][j] x_i^k for the selected rows i = rows[r], computed
 * as FP64 Horner in k;  S[r][j] = sum_k |C[k][j]| |x_i|^k (normwise scale).
 * C is (deg+1) x npoly, row k holding the power-k coefficients. */
void orc_vandermonde(const double* x, const double* coef, int32_t deg, int64_t npoly, const int64_t* rows,
                     int64_t nrows, double* y, double* scale) {
  double* c = (double*)malloc(sizeof(double) * (size_t)(deg + 1));
  double* ca = (double*)malloc(sizeof(double) * (size_t)(deg + 1));
  for (int64_t r = 0; r < nrows; ++r) {
    double xi = x[rows[r]];
    for (int64_t j = 0; j < npoly; ++j) {
      for (int k = 0; k <= deg; ++k) {
        c[k] = coef[(int64_t)k * npoly + j];
        ca[k] = fabs(c[k]);
      }
      y[r * npoly + j] = horner(c, deg, xi);
      if (scale) scale[r * npoly + j] = horner(ca, deg, fabs(xi));
    }
  }
  free(c);
  free(ca);
}

/* ------------------------------------------------------------------------ */
/* Multi-threaded drivers                                                    */
/* ------------------------------------------------------------------------ */

/* Storage types of the input array: the values are widened exactly to FP64. */
enum { ORC_IN_F64 = 0, ORC_IN_F32 = 1, ORC_IN_F16 = 2 };

/* IEEE 754 binary16 bit pattern -> its exact value: sign, 5-bit exponent
 * (bias 15), 10-bit fraction; exponent 0 holds zeros and subnormals
 * (fraction * 2^-24), exponent 31 infinities and NaN. */
static double half_value(uint16_t h) {
  int sign = h >> 15, e = (h >> 10) & 31, f = h & 1023;
  double v;
  if (e == 0) v = ldexp((double)f, -24);
  else if (e == 31) v = f ? NAN : INFINITY;
  else v = ldexp((double)(1024 + f), e - 25);
  return sign ? -v : v;
}

void orc_widen_f16(const uint16_t* h, double* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] = half_value(h[i]);
}

static double load_in(const void* x, int xt, int64_t i) {
  if (xt == ORC_IN_F32) return (double)((const float*)x)[i];
  if (xt == ORC_IN_F16) return half_value(((const uint16_t*)x)[i]);
  return ((const double*)x)[i];
}

/* dst += src, exactly */
static void acc_merge(orc_acc* dst, const orc_acc* src) {
  orc_acc t = *src;
  acc_norm(&t);
  for (int i = 0; i < ORC_LIMBS; ++i) dst->d[i] += t.d[i];
  if (++dst->pending >= (1LL << 29)) acc_norm(dst);
}

/* One pass over x[lo, hi): exact sums of f and of |f|, min and max of f, with
 * f evaluated in FP64 (f32 = 0) or in binary32 (f32 = 1). */
static void reduce_span(const orc_map* m, int f32, const void* x, int xt, int64_t lo, int64_t hi, orc_acc* sum,
                        orc_acc* abs_sum, double* mn, double* mx) {
  for (int64_t i = lo; i < hi; ++i) {
    double v = load_in(x, xt, i);
    double f = f32 ? (double)map_f32(m, (float)v) : map_f64(m, v);
    acc_add(sum, f);
    acc_add(abs_sum, fabs(f));
    if (f < *mn) *mn = f;
    if (f > *mx) *mx = f;
  }
}

typedef struct {
  const orc_map* m;
  int f32;                      /* evaluate f in binary32 */
  const void* x;
  int xt;
  const int64_t* off;           /* segmented: offsets; NULL for a full reduction */
  int64_t lo, hi;               /* element span (full) or segment span (segmented) */
  double *sums, *mins, *maxs, *abss;
  orc_acc sum, abs_sum;         /* full reduction: this thread's accumulators */
  double mn, mx;
} orc_job;

static void* job_run(void* p) {
  orc_job* j = (orc_job*)p;
  if (!j->off) {
    reduce_span(j->m, j->f32, j->x, j->xt, j->lo, j->hi, &j->sum, &j->abs_sum, &j->mn, &j->mx);
    return NULL;
  }
  orc_acc* a = (orc_acc*)malloc(2 * sizeof(orc_acc));
  for (int64_t s = j->lo; s < j->hi; ++s) {
    double mn = INFINITY, mx = -INFINITY;
    acc_clear(&a[0]);
    acc_clear(&a[1]);
    reduce_span(j->m, j->f32, j->x, j->xt, j->off[s], j->off[s + 1], &a[0], &a[1], &mn, &mx);
    j->sums[s] = acc_round(&a[0], 53, 0);
    j->mins[s] = mn;
    j->maxs[s] = mx;
    if (j->abss) j->abss[s] = acc_round(&a[1], 53, 0);
  }
  free(a);
  return NULL;
}

static void run_jobs(orc_job* jobs, int nt) {
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nt);
  int* started = (int*)calloc((size_t)nt, sizeof(int));
  for (int t = 1; t < nt; ++t) started[t] = pthread_create(&th[t], NULL, job_run, &jobs[t]) == 0;
  job_run(&jobs[0]);
  for (int t = 1; t < nt; ++t) {
    if (started[t]) pthread_join(th[t], NULL);
    else job_run(&jobs[t]);  /* no thread could be made: run it here */
  }
  free(started);
  free(th);
}

/* out[0] = exact sum of f rounded to double, out[1] = min, out[2] = max,
 * out[3] = exact sum of |f| rounded to double; x has storage type xt; f in
 * FP64, or in binary32 when f32 != 0.  The
 * array is cut into nthreads contiguous pieces; the pieces' exact
 * accumulators are merged exactly, so the result does not depend on
 * nthreads. */
void orc_reduce_mt(const orc_map* m, int32_t f32, const void* x, int32_t xt, int64_t n, double* out,
                   int32_t nthreads) {
  int nt = nthreads < 1 ? 1 : nthreads;
  orc_job* jobs = (orc_job*)calloc((size_t)nt, sizeof(orc_job));
  for (int t = 0; t < nt; ++t) {
    jobs[t].m = m;
    jobs[t].f32 = f32;
    jobs[t].x = x;
    jobs[t].xt = xt;
    jobs[t].lo = n * t / nt;
    jobs[t].hi = n * (t + 1) / nt;
    jobs[t].mn = INFINITY;
    jobs[t].mx = -INFINITY;
  }
  run_jobs(jobs, nt);
  double mn = INFINITY, mx = -INFINITY;
  for (int t = 1; t < nt; ++t) {
    acc_merge(&jobs[0].sum, &jobs[t].sum);
    acc_merge(&jobs[0].abs_sum, &jobs[t].abs_sum);
  }
  for (int t = 0; t < nt; ++t) {
    if (jobs[t].mn < mn) mn = jobs[t].mn;
    if (jobs[t].mx > mx) mx = jobs[t].mx;
  }
  out[0] = acc_round(&jobs[0].sum, 53, 0);
  out[1] = mn;
  out[2] = mx;
  out[3] = acc_round(&jobs[0].abs_sum, 53, 0);
  free(jobs);
}

/* orc_segreduce_f64 on nthreads threads, for input of storage type xt, plus
 * abss[s] = exact sum of |f| over segment s rounded to double (abss may be
 * NULL).  Thread t takes the segments starting in the t-th of nthreads equal
 * element spans; every segment is reduced whole by one thread. */
void orc_segreduce_mt(const orc_map* m, int32_t f32, const void* x, int32_t xt, const int64_t* off, int64_t nseg,
                      double* sums, double* mins, double* maxs, double* abss, int32_t nthreads) {
  int nt = nthreads < 1 ? 1 : nthreads;
  orc_job* jobs = (orc_job*)calloc((size_t)nt, sizeof(orc_job));
  int64_t n = off[nseg] - off[0], s = 0;
  for (int t = 0; t < nt; ++t) {
    int64_t end = off[0] + n * (t + 1) / nt;
    jobs[t].m = m;
    jobs[t].f32 = f32;
    jobs[t].x = x;
    jobs[t].xt = xt;
    jobs[t].off = off;
    jobs[t].lo = s;
    while (s < nseg && (t == nt - 1 || off[s] < end)) ++s;
    jobs[t].hi = s;
    jobs[t].sums = sums;
    jobs[t].mins = mins;
    jobs[t].maxs = maxs;
    jobs[t].abss = abss;
  }
  run_jobs(jobs, nt);
  free(jobs);
}
