/*
 * Plain CPU oracle for fast polynomial evaluation and composition (Moroz,
 * "Fast polynomial evaluation and composition", arXiv:1307.5655).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path: it rebuilds the evaluation tree
 * from the paper's definitions, literally and slowly.
 *
 * What each function computes, and the passage it follows:
 *   or_build_tree      Def. 1.2 (function scheme), Sec. 1.1 ordering, Remark on
 *                      multivariate recursion, Def. 1.3 (lazy height).
 *   or_eval_f64_plain  p(x) = sum c_e x^e (the plain definition), plus the
 *                      condition scale sum |c_e||x^e|.
 *   or_eval_modp_plain the same sum over Z/pZ, p = 2^64 - 2^32 + 1, in
 *                      unsigned __int128 with '%'.
 *   or_walk_f64 / or_walk_modp / or_walk_iv64
 *                      the coefficient walk of Sec. 2.1, node by node in
 *                      index order with the accumulators m[0..L]; IV64 runs it
 *                      in directed-rounding interval arithmetic (fesetround).
 *   or_compose_*_plain r(y) = sum_e c_e q(y)^e, schoolbook, exact for mod p.
 *
 * Readings of the paper (where it is silent or garbled):
 *   - f is applied to n = (#terms - 1); the split keeps the f(n) lowest terms
 *     in b and the rest in a (Def. 1.2 needs both non-empty: 0 < f(n) <= n).
 *   - Balanced B splits off floor(#terms/2) = ceil(n/2) low terms (Sec. 1.2).
 *   - Estrin E(n) = 2^floor(log2 n).
 *   - Multivariate: terms are grouped by the exponent of the first variable,
 *     the scheme is applied to the list of groups, each group is compiled
 *     recursively over the next variable and represented by its lowest term.
 *     Missing group roots (prefix followed by zeros) are inserted as virtual
 *     nodes with coefficient 0.
 *   - Lazy height: lh(leaf) = 0, lh(N) = max(lh(C1), 1 + max_{i>=2} lh(C_i)),
 *     C1 the lowest-index child (the printed rule, which ignores C1, is kept
 *     selectable with lh_rule = 1 to show that it breaks the walk).
 *   - The walk's loop runs to i = n inclusive (the root returns).
 *   - Interval product: the nine sign cases of Moore's table; interval square
 *     is tight ([+0, max] when 0 is inside); powers x^d are computed by
 *     x^1 = x, x^(2k) = sq(x^k), x^(2k+1) = x^(2k) * x.
 *
 * Build: gcc -O1 -frounding-math -ffp-contract=off -fPIC -shared.
 */
#include <fenv.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#pragma STDC FENV_ACCESS ON

#define OR_OK 0
#define OR_EBAD_VALUE (-1)
#define OR_EDUP (-2)
#define OR_EBAD_SCHEME (-3)
#define OR_ECAP (-4)
#define OR_ENOMEM (-5)

enum { OR_D = 0, OR_H = 1, OR_E = 2, OR_B = 3, OR_CUSTOM = 4 };

typedef unsigned __int128 u128;
static const uint64_t OR_P = 0xFFFFFFFF00000001ull; /* 2^64 - 2^32 + 1 */

/* ------------------------------------------------------------------ */
/* Function schemes, Sec. 1.1 (D, H, E) and Sec. 1.2 (B).              */
/* ------------------------------------------------------------------ */
int64_t or_scheme_f(int scheme, const int32_t* ftab, int64_t ftab_len, int64_t n) {
  if (n < 1) return OR_EBAD_VALUE;
  switch (scheme) {
    case OR_D: return n;
    case OR_H: return 1;
    case OR_E: {
      int64_t f = 1;
      while (f * 2 <= n) f *= 2;
      return f;
    }
    case OR_B: return (n + 1) / 2;
    case OR_CUSTOM:
      if (!ftab || n >= ftab_len) return OR_EBAD_SCHEME;
      return ftab[n];
    default: return OR_EBAD_SCHEME;
  }
}

/* ------------------------------------------------------------------ */
/* Tree construction                                                   */
/* ------------------------------------------------------------------ */
typedef struct {
  int nvars;
  int64_t n;        /* node count */
  int32_t* e;       /* n * nvars exponents, decreasing lex order */
  int64_t* parent;
  int32_t* pd_var;
  int64_t* pd;
  int scheme;
  const int32_t* ftab;
  int64_t ftab_len;
  int err;
} or_ctx;

static int g_nvars_for_cmp;
/* decreasing lex order: a before b when a > b */
static int cmp_lex_desc(const void* pa, const void* pb) {
  const int32_t* a = (const int32_t*)pa;
  const int32_t* b = (const int32_t*)pb;
  for (int v = 0; v < g_nvars_for_cmp; ++v) {
    if (a[v] != b[v]) return a[v] > b[v] ? -1 : 1;
  }
  return 0;
}

/* units a..b (b is the lowest), roots[u] = node index representing unit u */
static void build_units(or_ctx* c, const int64_t* roots, int64_t a, int64_t b, int var) {
  if (c->err || a >= b) return;
  int64_t n = b - a;
  int64_t f = or_scheme_f(c->scheme, c->ftab, c->ftab_len, n);
  if (f < 1 || f > n) { c->err = OR_EBAD_SCHEME; return; }
  /* p = a(x) x^f(n) + b(x): b = the f(n) lowest units, a = the others. */
  build_units(c, roots, b - f + 1, b, var);
  build_units(c, roots, a, b - f, var);
  int64_t child = roots[b - f], par = roots[b];
  c->parent[child] = par;
  c->pd_var[child] = var;
  c->pd[child] = (int64_t)c->e[child * c->nvars + var] - c->e[par * c->nvars + var];
}

/* nodes lo..hi share their exponents in the variables before var */
static void build_level(or_ctx* c, int64_t lo, int64_t hi, int var) {
  if (c->err) return;
  int64_t ngroups = 0;
  for (int64_t i = lo; i <= hi; ++i)
    if (i == hi || c->e[i * c->nvars + var] != c->e[(i + 1) * c->nvars + var]) ngroups++;
  int64_t* roots = (int64_t*)malloc(sizeof(int64_t) * (size_t)ngroups);
  if (!roots) { c->err = OR_ENOMEM; return; }
  int64_t g = 0, start = lo;
  for (int64_t i = lo; i <= hi; ++i) {
    if (i == hi || c->e[i * c->nvars + var] != c->e[(i + 1) * c->nvars + var]) {
      if (var + 1 < c->nvars) build_level(c, start, i, var + 1);
      roots[g++] = i; /* the group's lowest term represents it */
      start = i + 1;
    }
  }
  build_units(c, roots, 0, ngroups - 1, var);
  free(roots);
}

/*
 * Build the evaluation tree of a polynomial given by its exponent vectors
 * (terms in any order, no duplicates, no negative exponents).
 * Outputs (capacity `cap` nodes): node exponents in decreasing lex order,
 * term_of_node (-1 for a virtual node), parent (-1 for the root), the partial
 * degree as (variable, degree), and the lazy height.  Returns the node count,
 * or a negative error.
 */
int64_t or_build_tree(int nvars, int64_t nterms, const int32_t* exps, int scheme,
                      const int32_t* ftab, int64_t ftab_len, int lh_rule, int64_t cap,
                      int32_t* node_e, int64_t* term_of_node, int64_t* parent,
                      int32_t* pd_var, int64_t* pd, int32_t* lh) {
  if (nvars < 1 || nterms < 1) return OR_EBAD_VALUE;
  for (int64_t i = 0; i < nterms * nvars; ++i)
    if (exps[i] < 0) return OR_EBAD_VALUE;
  /* candidate rows: every term, plus each prefix followed by zeros; a row is
     nvars exponents then the term id (or -1) */
  int W = nvars + 1;
  int64_t ncand = nterms * nvars;
  int32_t* rows = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ncand * W));
  if (!rows) return OR_ENOMEM;
  int64_t r = 0;
  for (int64_t t = 0; t < nterms; ++t) {
    int32_t* row = rows + r * W;
    memcpy(row, exps + t * nvars, sizeof(int32_t) * nvars);
    row[nvars] = (int32_t)t;
    r++;
    for (int j = 1; j < nvars; ++j) {
      int32_t* vr = rows + r * W;
      for (int v = 0; v < nvars; ++v) vr[v] = v < j ? exps[t * nvars + v] : 0;
      vr[nvars] = -1;
      r++;
    }
  }
  /* sort by exponent (decreasing lex); among equal exponents real terms first */
  g_nvars_for_cmp = W; /* the trailing term id breaks ties: larger id first, -1 last */
  qsort(rows, (size_t)r, sizeof(int32_t) * W, cmp_lex_desc);
  g_nvars_for_cmp = nvars;
  int64_t n = 0;
  for (int64_t i = 0; i < r; ++i) {
    const int32_t* row = rows + i * W;
    if (n > 0) {
      const int32_t* prev = node_e + (n - 1) * nvars;
      if (cmp_lex_desc(prev, row) == 0) {
        if (row[nvars] >= 0 && term_of_node[n - 1] >= 0) { free(rows); return OR_EDUP; }
        continue;
      }
    }
    if (n >= cap) { free(rows); return OR_ECAP; }
    memcpy(node_e + n * nvars, row, sizeof(int32_t) * nvars);
    term_of_node[n] = row[nvars];
    n++;
  }
  free(rows);
  for (int64_t i = 0; i < n; ++i) { parent[i] = -1; pd_var[i] = 0; pd[i] = 0; }
  or_ctx c = {nvars, n, node_e, parent, pd_var, pd, scheme, ftab, ftab_len, 0};
  build_level(&c, 0, n - 1, 0);
  if (c.err) return c.err;
  /* the root's own degree: all of its exponents but the first are zero */
  pd_var[n - 1] = 0;
  pd[n - 1] = node_e[(n - 1) * nvars];

  /* lazy heights, Def. 1.3; children of a node have lower indices, so one
     ascending pass sees every child before its parent */
  int32_t* first_child_lh = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* max_other_lh = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int64_t* nchildren = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!first_child_lh || !max_other_lh || !nchildren) return OR_ENOMEM;
  for (int64_t i = 0; i < n; ++i) { nchildren[i] = 0; first_child_lh[i] = 0; max_other_lh[i] = -1; }
  for (int64_t i = 0; i < n; ++i) {
    int32_t h;
    if (nchildren[i] == 0) h = 0;
    else if (lh_rule == 1) h = nchildren[i] == 1 ? 0 : max_other_lh[i] + 1;
    else if (nchildren[i] == 1) h = first_child_lh[i];
    else h = first_child_lh[i] > max_other_lh[i] + 1 ? first_child_lh[i] : max_other_lh[i] + 1;
    lh[i] = h;
    int64_t q = parent[i];
    if (q >= 0) {
      if (nchildren[q] == 0) first_child_lh[q] = h;
      else if (h > max_other_lh[q]) max_other_lh[q] = h;
      nchildren[q]++;
    }
  }
  free(first_child_lh); free(max_other_lh); free(nchildren);
  return n;
}

/* ------------------------------------------------------------------ */
/* Plain definition p(x) = sum c_e x^e                                 */
/* ------------------------------------------------------------------ */
/* points: SoA, pts[v * npts + j].  Powers by repeated multiplication. */
int or_eval_f64_plain(int nvars, int64_t nterms, const int32_t* exps, const double* coef,
                      int64_t npts, const double* pts, double* out, double* absum) {
  int32_t maxd = 0;
  for (int64_t i = 0; i < nterms * nvars; ++i) if (exps[i] > maxd) maxd = exps[i];
  double* tab = (double*)malloc(sizeof(double) * (size_t)nvars * (maxd + 1));
  if (!tab) return OR_ENOMEM;
  for (int64_t j = 0; j < npts; ++j) {
    for (int v = 0; v < nvars; ++v) {
      double x = pts[(int64_t)v * npts + j];
      double* t = tab + (int64_t)v * (maxd + 1);
      t[0] = 1.0;
      for (int32_t d = 1; d <= maxd; ++d) t[d] = t[d - 1] * x;
    }
    double s = 0.0, a = 0.0;
    for (int64_t i = 0; i < nterms; ++i) {
      double m = coef[i];
      for (int v = 0; v < nvars; ++v) m *= tab[(int64_t)v * (maxd + 1) + exps[i * nvars + v]];
      s += m;
      a += fabs(m);
    }
    out[j] = s;
    if (absum) absum[j] = a;
  }
  free(tab);
  return OR_OK;
}

static uint64_t mulmod(uint64_t a, uint64_t b) { return (uint64_t)(((u128)a * b) % OR_P); }
static uint64_t addmod(uint64_t a, uint64_t b) { return (uint64_t)(((u128)a + b) % OR_P); }

int or_eval_modp_plain(int nvars, int64_t nterms, const int32_t* exps, const uint64_t* coef,
                       int64_t npts, const uint64_t* pts, uint64_t* out) {
  int32_t maxd = 0;
  for (int64_t i = 0; i < nterms * nvars; ++i) if (exps[i] > maxd) maxd = exps[i];
  for (int64_t i = 0; i < nterms; ++i) if (coef[i] >= OR_P) return OR_EBAD_VALUE;
  for (int64_t i = 0; i < npts * nvars; ++i) if (pts[i] >= OR_P) return OR_EBAD_VALUE;
  uint64_t* tab = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)nvars * (maxd + 1));
  if (!tab) return OR_ENOMEM;
  for (int64_t j = 0; j < npts; ++j) {
    for (int v = 0; v < nvars; ++v) {
      uint64_t x = pts[(int64_t)v * npts + j];
      uint64_t* t = tab + (int64_t)v * (maxd + 1);
      t[0] = 1;
      for (int32_t d = 1; d <= maxd; ++d) t[d] = mulmod(t[d - 1], x);
    }
    uint64_t s = 0;
    for (int64_t i = 0; i < nterms; ++i) {
      uint64_t m = coef[i];
      for (int v = 0; v < nvars; ++v) m = mulmod(m, tab[(int64_t)v * (maxd + 1) + exps[i * nvars + v]]);
      s = addmod(s, m);
    }
    out[j] = s;
  }
  free(tab);
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* The coefficient walk, Sec. 2.1, in RN double and in Z/pZ            */
/* ------------------------------------------------------------------ */
static int32_t max_lh(int64_t n, const int32_t* lh) {
  int32_t L = 0;
  for (int64_t i = 0; i < n; ++i) if (lh[i] > L) L = lh[i];
  return L;
}

/* node coefficients c[i] (0 for virtual nodes); x^d by repeated multiplication */
int or_walk_f64(int nvars, int64_t n, const int64_t* parent, const int32_t* pd_var, const int64_t* pd,
                const int32_t* lh, const double* c, int64_t npts, const double* pts, double* out) {
  int32_t L = max_lh(n, lh);
  double* m = (double*)calloc((size_t)L + 1, sizeof(double));
  if (!m) return OR_ENOMEM;
  for (int64_t j = 0; j < npts; ++j) {
    for (int32_t h = 0; h <= L; ++h) m[h] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double x = pts[(int64_t)pd_var[i] * npts + j], xd = 1.0;
      for (int64_t k = 0; k < pd[i]; ++k) xd *= x;
      int32_t h = lh[i];
      double p = (m[h] + c[i]) * xd;
      m[h] = 0.0;
      if (i == n - 1) out[j] = p;
      else m[lh[parent[i]]] += p;
    }
  }
  free(m);
  return OR_OK;
}

int or_walk_modp(int nvars, int64_t n, const int64_t* parent, const int32_t* pd_var, const int64_t* pd,
                 const int32_t* lh, const uint64_t* c, int64_t npts, const uint64_t* pts, uint64_t* out) {
  int32_t L = max_lh(n, lh);
  uint64_t* m = (uint64_t*)calloc((size_t)L + 1, sizeof(uint64_t));
  if (!m) return OR_ENOMEM;
  for (int64_t j = 0; j < npts; ++j) {
    for (int32_t h = 0; h <= L; ++h) m[h] = 0;
    for (int64_t i = 0; i < n; ++i) {
      uint64_t x = pts[(int64_t)pd_var[i] * npts + j], xd = 1;
      for (int64_t k = 0; k < pd[i]; ++k) xd = mulmod(xd, x);
      int32_t h = lh[i];
      uint64_t p = mulmod(addmod(m[h], c[i]), xd);
      m[h] = 0;
      if (i == n - 1) out[j] = p;
      else m[lh[parent[i]]] = addmod(m[lh[parent[i]]], p);
    }
  }
  free(m);
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Directed-rounding intervals (the paper's "boost intervals" type)    */
/* ------------------------------------------------------------------ */
typedef struct { double lo, hi; } iv;

static double add_dn(double a, double b) { volatile double x = a, y = b; fesetround(FE_DOWNWARD); volatile double r = x + y; fesetround(FE_TONEAREST); return r; }
static double add_up(double a, double b) { volatile double x = a, y = b; fesetround(FE_UPWARD); volatile double r = x + y; fesetround(FE_TONEAREST); return r; }
static double mul_dn(double a, double b) { volatile double x = a, y = b; fesetround(FE_DOWNWARD); volatile double r = x * y; fesetround(FE_TONEAREST); return r; }
static double mul_up(double a, double b) { volatile double x = a, y = b; fesetround(FE_UPWARD); volatile double r = x * y; fesetround(FE_TONEAREST); return r; }

static iv iv_add(iv a, iv b) { iv r = {add_dn(a.lo, b.lo), add_up(a.hi, b.hi)}; return r; }

/* class: 0 = non-negative (lo >= 0), 1 = non-positive (hi <= 0), 2 = straddles zero */
static int iv_class(iv a) { return a.lo >= 0.0 ? 0 : (a.hi <= 0.0 ? 1 : 2); }

/* Moore's nine-case product; each endpoint is the directed rounding of the
   exact extreme product */
static iv iv_mul(iv a, iv b) {
  int ca = iv_class(a), cb = iv_class(b);
  iv r;
  if (ca == 0 && cb == 0) { r.lo = mul_dn(a.lo, b.lo); r.hi = mul_up(a.hi, b.hi); }
  else if (ca == 0 && cb == 1) { r.lo = mul_dn(a.hi, b.lo); r.hi = mul_up(a.lo, b.hi); }
  else if (ca == 0 && cb == 2) { r.lo = mul_dn(a.hi, b.lo); r.hi = mul_up(a.hi, b.hi); }
  else if (ca == 1 && cb == 0) { r.lo = mul_dn(a.lo, b.hi); r.hi = mul_up(a.hi, b.lo); }
  else if (ca == 1 && cb == 1) { r.lo = mul_dn(a.hi, b.hi); r.hi = mul_up(a.lo, b.lo); }
  else if (ca == 1 && cb == 2) { r.lo = mul_dn(a.lo, b.hi); r.hi = mul_up(a.lo, b.lo); }
  else if (ca == 2 && cb == 0) { r.lo = mul_dn(a.lo, b.hi); r.hi = mul_up(a.hi, b.hi); }
  else if (ca == 2 && cb == 1) { r.lo = mul_dn(a.hi, b.lo); r.hi = mul_up(a.lo, b.lo); }
  else {
    double l1 = mul_dn(a.lo, b.hi), l2 = mul_dn(a.hi, b.lo);
    double h1 = mul_up(a.lo, b.lo), h2 = mul_up(a.hi, b.hi);
    r.lo = l1 < l2 ? l1 : l2;
    r.hi = h1 > h2 ? h1 : h2;
  }
  return r;
}

static iv iv_sq(iv a) {
  iv r;
  int ca = iv_class(a);
  if (ca == 0) { r.lo = mul_dn(a.lo, a.lo); r.hi = mul_up(a.hi, a.hi); }
  else if (ca == 1) { r.lo = mul_dn(a.hi, a.hi); r.hi = mul_up(a.lo, a.lo); }
  else {
    double h1 = mul_up(a.lo, a.lo), h2 = mul_up(a.hi, a.hi);
    r.lo = 0.0;
    r.hi = h1 > h2 ? h1 : h2;
  }
  return r;
}

static iv iv_pow(iv x, int64_t d) {
  if (d == 1) return x;
  if (d % 2 == 0) return iv_sq(iv_pow(x, d / 2));
  return iv_mul(iv_pow(x, d - 1), x);
}

void or_iv_pow(int64_t npts, const double* lo, const double* hi, int64_t d, double* olo, double* ohi) {
  for (int64_t j = 0; j < npts; ++j) {
    iv x = {lo[j], hi[j]};
    iv r = iv_pow(x, d);
    olo[j] = r.lo; ohi[j] = r.hi;
  }
}

void or_iv_mul(int64_t npts, const double* alo, const double* ahi, const double* blo, const double* bhi,
               double* olo, double* ohi) {
  for (int64_t j = 0; j < npts; ++j) {
    iv a = {alo[j], ahi[j]}, b = {blo[j], bhi[j]};
    iv r = iv_mul(a, b);
    olo[j] = r.lo; ohi[j] = r.hi;
  }
}

/* the walk of Sec. 2.1 in interval arithmetic; coefficients are degenerate
   intervals [c, c]; points are boxes given as SoA lo/hi per variable */
int or_walk_iv64(int nvars, int64_t n, const int64_t* parent, const int32_t* pd_var, const int64_t* pd,
                 const int32_t* lh, const double* c, int64_t npts, const double* lo, const double* hi,
                 double* out_lo, double* out_hi) {
  int32_t L = max_lh(n, lh);
  iv* m = (iv*)calloc((size_t)L + 1, sizeof(iv));
  if (!m) return OR_ENOMEM;
  for (int64_t j = 0; j < npts; ++j) {
    for (int32_t h = 0; h <= L; ++h) { m[h].lo = 0.0; m[h].hi = 0.0; }
    for (int64_t i = 0; i < n; ++i) {
      int32_t h = lh[i];
      iv ci = {c[i], c[i]};
      iv p = iv_add(m[h], ci);
      if (pd[i] > 0) {
        iv x = {lo[(int64_t)pd_var[i] * npts + j], hi[(int64_t)pd_var[i] * npts + j]};
        p = iv_mul(p, iv_pow(x, pd[i]));
      }
      m[h].lo = 0.0; m[h].hi = 0.0;
      if (i == n - 1) { out_lo[j] = p.lo; out_hi[j] = p.hi; }
      else { int32_t hp = lh[parent[i]]; m[hp] = iv_add(m[hp], p); }
    }
  }
  free(m);
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Composition r(y) = p(q(y)) = sum_e c_e q(y)^e (plain definition)    */
/* p dense by degree: pc[0..np-1] (pc[e] = coefficient of x^e);        */
/* q dense: qc[0..nq-1]; r has (np-1)(nq-1)+1 coefficients.            */
/* ------------------------------------------------------------------ */
int or_compose_modp_plain(int64_t np, const uint64_t* pc, int64_t nq, const uint64_t* qc, uint64_t* out) {
  int64_t dq = nq - 1, nr = (np - 1) * dq + 1;
  uint64_t* pw = (uint64_t*)calloc((size_t)nr, sizeof(uint64_t));
  uint64_t* nx = (uint64_t*)calloc((size_t)nr, sizeof(uint64_t));
  if (!pw || !nx) return OR_ENOMEM;
  for (int64_t j = 0; j < nr; ++j) out[j] = 0;
  pw[0] = 1; /* q^0 */
  for (int64_t e = 0; e < np; ++e) {
    int64_t deg = e * dq;
    for (int64_t j = 0; j <= deg; ++j) out[j] = addmod(out[j], mulmod(pc[e], pw[j]));
    if (e + 1 == np) break;
    for (int64_t j = 0; j <= deg + dq; ++j) nx[j] = 0;
    for (int64_t j = 0; j <= deg; ++j)
      for (int64_t k = 0; k < nq; ++k) nx[j + k] = addmod(nx[j + k], mulmod(pw[j], qc[k]));
    uint64_t* t = pw; pw = nx; nx = t;
  }
  free(pw); free(nx);
  return OR_OK;
}

/* FP64 version; also returns the same computation on |c| and |q| (the
   componentwise condition scale) */
int or_compose_f64_plain(int64_t np, const double* pc, int64_t nq, const double* qc, double* out, double* absout) {
  int64_t dq = nq - 1, nr = (np - 1) * dq + 1;
  double* pw = (double*)calloc((size_t)nr, sizeof(double));
  double* nx = (double*)calloc((size_t)nr, sizeof(double));
  double* apw = (double*)calloc((size_t)nr, sizeof(double));
  double* anx = (double*)calloc((size_t)nr, sizeof(double));
  if (!pw || !nx || !apw || !anx) return OR_ENOMEM;
  for (int64_t j = 0; j < nr; ++j) { out[j] = 0.0; absout[j] = 0.0; }
  pw[0] = 1.0; apw[0] = 1.0;
  for (int64_t e = 0; e < np; ++e) {
    int64_t deg = e * dq;
    for (int64_t j = 0; j <= deg; ++j) {
      out[j] += pc[e] * pw[j];
      absout[j] += fabs(pc[e]) * apw[j];
    }
    if (e + 1 == np) break;
    for (int64_t j = 0; j <= deg + dq; ++j) { nx[j] = 0.0; anx[j] = 0.0; }
    for (int64_t j = 0; j <= deg; ++j)
      for (int64_t k = 0; k < nq; ++k) {
        nx[j + k] += pw[j] * qc[k];
        anx[j + k] += apw[j] * fabs(qc[k]);
      }
    double* t = pw; pw = nx; nx = t;
    t = apw; apw = anx; anx = t;
  }
  free(pw); free(nx); free(apw); free(anx);
  return OR_OK;
}
