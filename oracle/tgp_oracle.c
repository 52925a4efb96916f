/*
 * tgp_oracle.c -- FP64 reference interpreter for tensorized tree-based GP.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness oracle that the
 * CUDA library is checked against.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it; the library itself never
 * links, calls or falls back to it.  It shares no code, header, table or
 * helper with the CUDA path (the opcode numbers below are restated here from
 * the encoding rules, not included from the library header).
 *
 * What it computes (paper sections cited per function):
 *   - the node semantics of Sec. II-A (constant, variable and function nodes,
 *     bottom-up evaluation, the root's result is the output);
 *   - the population encoding of Sec. III-A: three NaN-padded arrays per tree
 *     (types, values, subtree sizes), len(T) = size[0];
 *   - the SR fitness of Sec. III-C: mean squared error of the predictions
 *     against the targets over all data points;
 *   - Modi multi-output nodes of Sec. IV-C: a Modi node adds its function
 *     value into its output slot (outputs sum their contributions) and hands
 *     its parent the value of its rightmost child;
 *   - reverse-mode derivatives of the MSE with respect to constants and input
 *     features (not in the paper; the plain chain rule on the same tree).
 *
 * Evaluation is a plain recursion in prefix order: the first child starts at
 * i+1 and each recursive call returns the index one past its subtree, so the
 * subtree-size array is NOT used for evaluation; it is only checked by the
 * validator against the structure the recursion finds.  All arithmetic is
 * IEEE double; the float inputs are widened exactly.
 *
 * Readings of points the paper leaves open (the binding encoding table):
 *   type  : 0 variable, 1 constant, 2 unary function, 3 binary function,
 *           +16 marks a function node as a Modi node (18, 19).
 *   value : variable -> feature index; constant -> the constant;
 *           function -> func_id + 256 * output_index (output_index only on
 *           Modi nodes, 0 otherwise); an integer below 65536.
 *   func  : 0 add, 1 sub, 2 mul, 3 protected div, 4 max (binary);
 *           5 sin, 6 cos, 7 protected log, 8 clamped exp, 9 tan (unary);
 *           10 ite (ternary; type 4, 20 on a Modi node).
 *   ite(a, b, c) = a > 0 ? b : c (a NaN condition selects c): the paper's
 *   encoding admits any arity fixed by (type, value), Sec. III-A.
 *   The first prefix child is the left operand: [sub, a, b] = a - b.
 *   pdiv(a,b) = |b| > 1e-6f ? a/b : 1 ;  plog(a) = |a| > 1e-6f ? log|a| : 0 ;
 *   cexp(a)   = exp(min(a, 80)) ; max = IEEE fmax (a NaN operand yields the
 *   other one).  The guard threshold is the float value 1e-6f widened.
 *   Output rule: with one output and no Modi node the output is the root
 *   value; otherwise the outputs are the Modi sums (an output without a
 *   contribution is 0) and a non-Modi root value is discarded.
 *
 * Error bound (condition-aware comparison): alongside each double value the
 * interpreter can carry a first-order bound on how far an FP32 evaluation of
 * the same tree may land from it: every leaf is exact in FP32, every function
 * node adds the propagated child errors (through its local derivatives) and a
 * per-function rounding allowance of an FP32 implementation (unit roundoff
 * u = 2^-24).  A guard whose operand lies within its error of the threshold,
 * or any value that may leave the FP32 range, makes the bound infinite.
 */
#include <math.h>
#include <float.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* ---- encoding restated from the paper's Sec. III-A and the readings above ---- */
enum { T_VAR = 0, T_CONST = 1, T_UFUNC = 2, T_BFUNC = 3, T_TFUNC = 4, T_MODI = 16 };
enum { F_ADD = 0, F_SUB, F_MUL, F_PDIV, F_MAX, F_SIN, F_COS, F_PLOG, F_CEXP, F_TAN, F_ITE, F_COUNT };

/* validator status bits (restated; the library defines its own) */
enum {
  ST_OK = 0,
  ST_LEN = 1,      /* size[0] is not an integer in [1, max_len]          */
  ST_TYPE = 2,     /* a type code is not one of 0,1,2,3,18,19             */
  ST_FUNC = 4,     /* function id unknown or its arity disagrees with type */
  ST_VAR = 8,      /* variable index not an integer in [0, n_features)    */
  ST_MODI = 16,    /* Modi output index not in [0, n_outputs)             */
  ST_CONST = 32,   /* constant is not finite                              */
  ST_SIZE = 64,    /* subtree sizes disagree with the prefix structure    */
};

static const double GUARD = (double)1e-6f;
static const double EXP_CLAMP = 80.0;
static const double U32 = 5.9604644775390625e-08; /* 2^-24 */

static int arity_of(int f) { return f <= F_MAX ? 2 : f == F_ITE ? 3 : 1; }

static int is_int(double v) { return isfinite(v) && v == floor(v); }

/* One tree's view into the population arrays. */
typedef struct {
  const float *type, *val, *size;
  int len;
} tree_t;

/* ------------------------------------------------------------------ validator */
/* Structural parse by arity from position i; returns one past the subtree or
 * -1 when the prefix runs past len.  Records the true subtree size. */
static int parse(const tree_t* t, int i, int* true_size) {
  if (i >= t->len) return -1;
  int ty = (int)t->type[i] & ~T_MODI;
  int nxt = i + 1;
  if (ty == T_UFUNC || ty == T_BFUNC || ty == T_TFUNC) {
    int f = ((int)t->val[i]) % 256;
    for (int c = 0; c < arity_of(f); ++c) {
      nxt = parse(t, nxt, true_size);
      if (nxt < 0) return -1;
    }
  }
  true_size[i] = nxt - i;
  return nxt;
}

/* Sec. III-A encoding rules, checked per tree.  Returns the status bitmask. */
int orc_validate_one(const float* type, const float* val, const float* size,
                     int max_len, int n_features, int n_outputs, int* len_out) {
  double s0 = size[0];
  *len_out = 0;
  if (!is_int(s0) || s0 < 1 || s0 > max_len) return ST_LEN;
  int len = (int)s0;
  *len_out = len;
  int st = 0;
  for (int i = 0; i < len; ++i) {
    double tv = type[i], vv = val[i];
    int ty = (is_int(tv) && tv >= 0 && tv < 64) ? (int)tv : -1;
    int base = ty >= 0 ? (ty & ~T_MODI) : -1;
    int modi = ty >= 0 && (ty & T_MODI);
    if (!(ty == 0 || ty == 1 || ty == 2 || ty == 3 || ty == 4 || ty == 18 || ty == 19 || ty == 20)) {
      st |= ST_TYPE;
      continue;
    }
    if (base == T_VAR) {
      if (!is_int(vv) || vv < 0 || vv >= n_features) st |= ST_VAR;
    } else if (base == T_CONST) {
      if (!isfinite(vv)) st |= ST_CONST;
    } else {
      if (!is_int(vv) || vv < 0 || vv >= 65536) { st |= ST_FUNC; continue; }
      long iv = (long)vv;
      int f = (int)(iv % 256);
      long o = iv / 256;
      /* the type names the arity: 2 unary, 3 binary, 4 ternary */
      if (f >= F_COUNT || arity_of(f) != base - 1) st |= ST_FUNC;
      if (modi) { if (o >= n_outputs) st |= ST_MODI; }
      else if (o != 0) st |= ST_FUNC;
    }
  }
  if (st & (ST_TYPE | ST_FUNC)) return st; /* arity unknown: structure not checked */
  tree_t t = {type, val, size, len};
  int* ts = (int*)malloc(sizeof(int) * (size_t)len);
  int end = parse(&t, 0, ts);
  if (end != len) st |= ST_SIZE;
  else
    for (int i = 0; i < len; ++i)
      if (!is_int(size[i]) || (int)size[i] != ts[i]) { st |= ST_SIZE; break; }
  free(ts);
  return st;
}

/* ----------------------------------------------------------------- evaluation */
typedef struct {
  const tree_t* t;
  const float* x; /* one data point's feature row */
  double* out;    /* [n_outputs] Modi sums for this point */
  double* eout;   /* [n_outputs] error bounds, or NULL */
  int want_err;
  /* reverse-mode tape (grad only) */
  double* v;      /* value seen by the parent, per node          */
  double* fv;     /* function value (differs from v on Modi)     */
  int* c2;        /* index of the second child, per binary node  */
  double* ev;     /* FP32 error bound of v, per node (or NULL)   */
  int* c3;        /* index of the third child, per ternary node  */
  /* per output: sum of |contribution| and number of contributions, for the
   * rounding of a Modi sum taken in any order (bound mode only) */
  double msum[64];
  int mcnt[64];
} ctx_t;

/* The bound of a Modi output summed in FP32 in any order: the
 * contributions' own bounds plus (m - 1) u times the sum of their
 * magnitudes (recursive summation of m terms). */
static void finish_outputs(ctx_t* c, int O) {
  if (!c->want_err || !c->eout) return;
  for (int k = 0; k < O && k < 64; ++k) {
    if (c->mcnt[k] > 1) c->eout[k] += (double)(c->mcnt[k] - 1) * U32 * c->msum[k];
    if (!isfinite(c->out[k]) || !(c->eout[k] < INFINITY) || fabs(c->out[k]) + c->eout[k] > FLT_MAX)
      c->eout[k] = INFINITY;
  }
}

static double apply3(int f, double a, double b, double c) {
  return f == F_ITE ? (a > 0 ? b : c) : NAN;
}

static double apply(int f, double a, double b) {
  switch (f) {
    case F_ADD: return a + b;
    case F_SUB: return a - b;
    case F_MUL: return a * b;
    case F_PDIV: return fabs(b) > GUARD ? a / b : 1.0;
    case F_MAX: return fmax(a, b);
    case F_SIN: return sin(a);
    case F_COS: return cos(a);
    case F_PLOG: return fabs(a) > GUARD ? log(fabs(a)) : 0.0;
    case F_CEXP: return exp(fmin(a, EXP_CLAMP));
    case F_TAN: return tan(a);
  }
  return NAN;
}

/* Per-function allowances of an FP32 implementation, in units of the unit
 * roundoff u = 2^-24 (relative to |v|) plus an absolute part:
 *   add, sub, mul : 1 u |v|              (correctly rounded: half an ulp)
 *   pdiv          : 4 u |v|              (approximate reciprocal, 1 ulp, and a rounded product)
 *                   + |a| 2^-126 where |b| > 2^126 (in flush-to-zero arithmetic
 *                   the subnormal reciprocal is flushed to 0)
 *   max           : exact
 *   sin, cos      : 2^-20.5 absolute + 1 u |v|  (approximation on the reduced
 *                   argument plus a two-part argument reduction)
 *   plog          : 2^-22 absolute + 5 u |v|    (a base-2 logarithm accurate to
 *                   2^-22 relative, 2^-22 absolute near 1, times ln 2 with a
 *                   rounded product)
 *   cexp          : (6 + 1.25 |a|) u |v| (exp2 approximation, 2 ulp, and the
 *                   rounding of a*log2(e) with log2(e) itself rounded to
 *                   float, which scales the result by up to 1.22 |a| u)
 *   tan           : the sin/cos allowance divided by |cos a|, (1+|t|)^2
 *                   scaled; infinite where the possible error of cos a
 *                   reaches half of |cos a| (the first-order bound no longer
 *                   holds: the quotient may take any size or sign)
 * The FP32 implementation's own accuracy is checked against these numbers
 * function by function over sweeps of exact arguments. */
static double trig_abs(void) { return 6.9053396600248786e-07; /* 2^-20.5 */ }

/* First-order FP32 error bound of f(a,b) given the operand bounds ea, eb.
 * Every function result may also underflow (or be flushed) to zero in FP32,
 * an absolute error of at most FLT_MIN. */
static double err_of_raw(int f, double a, double ea, double b, double eb, double v);
static double err_of(int f, double a, double ea, double b, double eb, double v) {
  /* an operand whose own bound is infinite (or undefined) may be anything:
   * so may the result (this also keeps 0 * inf from turning into NaN) */
  if (!(ea < INFINITY) || !(eb < INFINITY)) return INFINITY;
  double e = err_of_raw(f, a, ea, b, eb, v);
  return e != e ? INFINITY : e + FLT_MIN;
}
static double err_of_raw(int f, double a, double ea, double b, double eb, double v) {
  double av = fabs(v);
  switch (f) {
    case F_ADD:
    case F_SUB: return ea + eb + U32 * av;
    case F_MUL: return fabs(b) * ea + fabs(a) * eb + ea * eb + U32 * av;
    case F_PDIV: {
      if (eb > 0 && fabs(fabs(b) - GUARD) <= eb) return INFINITY; /* guard branch ambiguous */
      if (!(fabs(b) > GUARD)) return 0.0;                          /* guard taken: exactly 1 */
      if (fabs(b) <= eb) return INFINITY;
      /* flush-to-zero arithmetic forms a/b as a times a reciprocal that is
       * subnormal, hence flushed to 0, for |b| > 2^126: |a| 2^-126 at most */
      double ftz = fabs(b) + eb > 0x1p126 ? fabs(a) * 0x1p-126 + ea * 0x1p-126 : 0.0;
      return (ea + av * eb) / (fabs(b) - eb) + 4 * U32 * av + ftz;
    }
    case F_MAX: return ea > eb ? ea : eb;
    case F_SIN: {
      double e = fabs(cos(a)) * ea + 0.5 * ea * ea;
      return (e < 2 ? e : 2) + trig_abs() + U32 * av;
    }
    case F_COS: {
      double e = fabs(sin(a)) * ea + 0.5 * ea * ea;
      return (e < 2 ? e : 2) + trig_abs() + U32 * av;
    }
    case F_PLOG: {
      if (ea > 0 && fabs(fabs(a) - GUARD) <= ea) return INFINITY;
      if (!(fabs(a) > GUARD)) return 0.0;
      if (fabs(a) <= ea) return INFINITY;
      return ea / (fabs(a) - ea) + ldexp(1.0, -22) + 5 * U32 * av;
    }
    case F_CEXP: {
      double am = fmin(a, EXP_CLAMP);
      return av * expm1(ea) + av * (6 + 1.25 * fabs(am)) * U32;
    }
    case F_TAN: {
      if (2 * (fabs(sin(a)) * ea + 0.5 * ea * ea + trig_abs()) >= fabs(cos(a))) return INFINITY;
      double g = 1 + v * v, s = 1 + fabs(v);
      return g * ea + 2 * trig_abs() * s * s + U32 * av;
    }
  }
  return INFINITY;
}

/* Evaluates the subtree at i; returns the value its parent sees and stores
 * one-past-the-subtree in *next.  *err receives the FP32 error bound. */
static double eval_node(ctx_t* c, int i, int* next, double* err) {
  const tree_t* t = c->t;
  int ty = (int)t->type[i];
  int base = ty & ~T_MODI;
  double v, e = 0.0;
  if (base == T_VAR) {
    v = (double)c->x[(int)t->val[i]];
    *next = i + 1;
    if (c->v) { c->v[i] = v; c->fv[i] = v; }
    if (c->ev) c->ev[i] = 0.0;
  } else if (base == T_CONST) {
    v = (double)t->val[i];
    *next = i + 1;
    if (c->v) { c->v[i] = v; c->fv[i] = v; }
    if (c->ev) c->ev[i] = 0.0;
  } else {
    long iv = (long)t->val[i];
    int f = (int)(iv % 256);
    int o = (int)(iv / 256);
    double a, b = 0.0, ea = 0.0, eb = 0.0, c3v = 0.0, ec = 0.0;
    int n1, n2, n3;
    a = eval_node(c, i + 1, &n1, &ea);
    double right = a, eright = ea; /* rightmost child's value */
    if (arity_of(f) >= 2) {
      if (c->c2) c->c2[i] = n1;
      b = eval_node(c, n1, &n2, &eb);
      right = b; eright = eb;
    } else {
      n2 = n1;
    }
    if (arity_of(f) == 3) {
      if (c->c3) c->c3[i] = n2;
      c3v = eval_node(c, n2, &n3, &ec);
      right = c3v; eright = ec;
    } else {
      n3 = n2;
    }
    *next = n3;
    double fv, fe = 0.0;
    if (f == F_ITE) {
      fv = apply3(f, a, b, c3v);
      /* the chosen branch's error, or anything when the sign of a is
       * undecided by its error (the FP32 path may take the other branch) */
      if (c->want_err) fe = (ea > 0 && fabs(a) <= ea) || !(ea < INFINITY) ? INFINITY : (a > 0 ? eb : ec);
    } else {
      fv = apply(f, a, b);
      fe = c->want_err ? err_of(f, a, ea, b, eb, fv) : 0.0;
    }
    if (c->want_err && (!isfinite(fv) || fabs(fv) + fe > FLT_MAX)) fe = INFINITY;
    if (ty & T_MODI) {
      /* Sec. IV-C: the function value is summed into output o and the parent
       * sees the rightmost child's value. */
      c->out[o] += fv;
      if (c->want_err) {
        c->eout[o] += fe;
        if (o < 64) {
          c->msum[o] += fabs(fv);
          c->mcnt[o] += 1;
        }
      }
      v = right;
      e = eright;
    } else {
      v = fv;
      e = fe;
    }
    if (c->v) { c->v[i] = v; c->fv[i] = fv; }
    if (c->ev) c->ev[i] = e;
  }
  *err = e;
  return v;
}

static int tree_has_modi(const tree_t* t) {
  for (int i = 0; i < t->len; ++i)
    if ((int)t->type[i] & T_MODI) return 1;
  return 0;
}

/* Evaluates one tree at one point into out[0..O) (and eout if want_err). */
static void eval_point(const tree_t* t, int has_modi, const float* x, int O,
                       double* out, double* eout, int want_err) {
  for (int k = 0; k < O; ++k) { out[k] = 0.0; if (eout) eout[k] = 0.0; }
  ctx_t c = {t, x, out, eout, want_err, NULL, NULL, NULL, NULL, NULL};
  int nx;
  double e;
  double r = eval_node(&c, 0, &nx, &e);
  if (!has_modi && O == 1) {
    out[0] = r;
    if (eout) eout[0] = e;
  } else {
    finish_outputs(&c, O);
  }
}

/* ----------------------------------------------------------- population jobs */
typedef struct {
  /* population */
  const float *type, *val, *size;
  long pop, ld;
  int max_len;
  /* data */
  const float* X;
  long D, ldx;
  int F;
  const float* y; /* [D][ldy], may be NULL for eval */
  long ldy;
  int O;
  /* outputs */
  double* out;       /* eval: [pop][O][D]                      */
  double* err;       /* eval: [pop][O][D] bound, or NULL       */
  double* mse;       /* [pop][O]                               */
  double* mse_allow; /* [pop][O] MSE allowance, or NULL        */
  double rel_tol;    /* per-point tolerance used by mse_allow  */
  const double* g;   /* grad: [pop][O] upstream gradient       */
  double* grad_val;  /* grad: [pop][ld]                        */
  double* grad_X;    /* grad: [D][F] (summed over threads)     */
  double* egrad_val; /* grad: [pop][ld] FP32 error bound, or NULL */
  double* egrad_X;   /* grad: [D][F] FP32 error bound, or NULL    */
  double acc_terms;  /* grad bound: FP32 partial-sum length       */
  int* status;       /* [pop] validator status                 */
  int mode;          /* 0 eval, 1 mse, 2 grad                  */
  int nthreads;
} job_t;

typedef struct {
  job_t* j;
  int tid;
  double* gx;  /* private grad_X                                   */
  double* egx; /* private [D][F] error bound sums and [D][F] sums of
                  |contribution| (bound mode only)                  */
} worker_t;

static void do_eval_tree(job_t* j, long p) {
  tree_t t = {j->type + p * j->ld, j->val + p * j->ld, j->size + p * j->ld, 0};
  int len;
  int st = orc_validate_one(t.type, t.val, t.size, j->max_len, j->F, j->O, &len);
  if (j->status) j->status[p] = st;
  int O = j->O;
  double* out = (double*)malloc(sizeof(double) * O * 2);
  double* eo = out + O;
  if (st != ST_OK) {
    for (long d = 0; d < j->D; ++d)
      for (int k = 0; k < O; ++k) {
        j->out[(p * O + k) * j->D + d] = NAN;
        if (j->err) j->err[(p * O + k) * j->D + d] = INFINITY;
      }
    free(out);
    return;
  }
  t.len = len;
  int hm = tree_has_modi(&t);
  for (long d = 0; d < j->D; ++d) {
    eval_point(&t, hm, j->X + d * j->ldx, O, out, j->err ? eo : NULL, j->err != NULL);
    for (int k = 0; k < O; ++k) {
      j->out[(p * O + k) * j->D + d] = out[k];
      if (j->err) j->err[(p * O + k) * j->D + d] = eo[k];
    }
  }
  free(out);
}

/* Sec. III-C fitness: MSE[p,k] = (1/D) sum_d (o_k(x_d) - y_{d,k})^2. */
static void do_mse_tree(job_t* j, long p) {
  tree_t t = {j->type + p * j->ld, j->val + p * j->ld, j->size + p * j->ld, 0};
  int len;
  int st = orc_validate_one(t.type, t.val, t.size, j->max_len, j->F, j->O, &len);
  if (j->status) j->status[p] = st;
  int O = j->O;
  double* buf = (double*)calloc((size_t)O * 4, sizeof(double));
  double *out = buf, *eo = buf + O, *acc = buf + 2 * O, *allow = buf + 3 * O;
  if (st == ST_OK) {
    t.len = len;
    int hm = tree_has_modi(&t);
    int we = j->mse_allow != NULL;
    for (long d = 0; d < j->D; ++d) {
      eval_point(&t, hm, j->X + d * j->ldx, O, out, we ? eo : NULL, we);
      for (int k = 0; k < O; ++k) {
        double r = out[k] - (double)j->y[d * j->ldy + k];
        acc[k] += r * r;
        if (we) {
          /* deviation the FP32 path may show at this point: the north-star
           * tolerance, or 2x the bound where the point is ill-conditioned */
          double tol = j->rel_tol * (fabs(out[k]) > 1 ? fabs(out[k]) : 1.0);
          double eps = 2 * eo[k] > tol ? 2 * eo[k] : tol;
          allow[k] += 2 * fabs(r) * eps + eps * eps;
        }
      }
    }
  }
  for (int k = 0; k < O; ++k) {
    j->mse[p * O + k] = st == ST_OK ? acc[k] / (double)j->D : NAN;
    if (j->mse_allow) j->mse_allow[p * O + k] = st == ST_OK ? allow[k] / (double)j->D : INFINITY;
  }
  free(buf);
}

/* Reverse sweep: adj is d(loss)/d(value the parent sees at node i). */
static void backprop(ctx_t* c, int i, double adj, const double* seed,
                     double* gval, double* gx) {
  const tree_t* t = c->t;
  int ty = (int)t->type[i];
  int base = ty & ~T_MODI;
  if (base == T_CONST) { gval[i] += adj; return; }
  if (base == T_VAR) { gx[(int)t->val[i]] += adj; return; }
  long iv = (long)t->val[i];
  int f = (int)(iv % 256);
  int o = (int)(iv / 256);
  int ia = i + 1;
  int ib = arity_of(f) >= 2 ? c->c2[i] : -1;
  int ic = arity_of(f) == 3 ? c->c3[i] : -1;
  double a = c->v[ia], b = ib >= 0 ? c->v[ib] : 0.0;
  /* adjoint of the function value: the parent's on a plain node, the
   * output's seed on a Modi node (whose parent sees the rightmost child) */
  double af = (ty & T_MODI) ? seed[o] : adj;
  double pass_b = 0.0, pass_a = 0.0, pass_c = 0.0;
  if (ty & T_MODI) {
    if (ic >= 0) pass_c = adj; else if (ib >= 0) pass_b = adj; else pass_a = adj;
  }
  double da = 0.0, db = 0.0, dc = 0.0;
  switch (f) {
    case F_ITE:
      /* the adjoint goes to the branch ite chose; the condition gets none */
      if (a > 0) db = 1; else dc = 1;
      break;
    case F_ADD: da = 1; db = 1; break;
    case F_SUB: da = 1; db = -1; break;
    case F_MUL: da = b; db = a; break;
    case F_PDIV:
      if (fabs(b) > GUARD) { da = 1.0 / b; db = -a / (b * b); }
      break;
    case F_MAX:
      /* the gradient goes to the operand fmax returned; ties go left */
      if (a >= b || isnan(b)) da = 1; else db = 1;
      break;
    case F_SIN: da = cos(a); break;
    case F_COS: da = -sin(a); break;
    case F_PLOG: if (fabs(a) > GUARD) da = 1.0 / a; break;
    case F_CEXP: if (a <= EXP_CLAMP) da = exp(a); break;
    case F_TAN: { double tn = tan(a); da = 1 + tn * tn; } break;
  }
  /* a zero local derivative contributes nothing, even when the upstream
   * adjoint is not finite */
  double ga = pass_a + (da != 0.0 ? af * da : 0.0);
  backprop(c, ia, ga, seed, gval, gx);
  if (ib >= 0) {
    double gb = pass_b + (db != 0.0 ? af * db : 0.0);
    backprop(c, ib, gb, seed, gval, gx);
  }
  if (ic >= 0) {
    double gc = pass_c + (dc != 0.0 ? af * dc : 0.0);
    backprop(c, ic, gc, seed, gval, gx);
  }
}

/* Local derivatives of f at (a, b) -- exactly those of backprop -- with
 * first-order bounds of how far an FP32 evaluation of them may land, given
 * the operand bounds ea, eb: the operands' errors carried through the second
 * derivatives plus the allowance of the FP32 function that forms them.  A
 * guard, clamp or max tie that the operand errors leave undecided makes
 * both bounds infinite (the FP32 path may take the other branch). */
static void dlocal(int f, double a, double ea, double b, double eb, double* da, double* eda,
                   double* db, double* edb) {
  *da = *db = *eda = *edb = 0.0;
  int undecided = 0;
  switch (f) {
    case F_ADD: *da = 1; *db = 1; break;
    case F_SUB: *da = 1; *db = -1; break;
    case F_MUL: *da = b; *eda = eb; *db = a; *edb = ea; break;
    case F_PDIV:
      undecided = eb > 0 && fabs(fabs(b) - GUARD) <= eb;
      if (fabs(b) > GUARD) {
        double m = fabs(b) - eb;
        *da = 1.0 / b;
        *db = -a / (b * b);
        if (!(m > 0)) { undecided = 1; break; }
        *eda = eb / (fabs(b) * m) + 2 * U32 / fabs(b);
        *edb = (ea + 2 * fabs(a) * eb / m) / (m * m) + 4 * U32 * fabs(a) / (b * b);
      }
      break;
    case F_MAX:
      if (a >= b || isnan(b)) *da = 1; else *db = 1;
      /* an FP32 evaluation may route the adjoint to the other operand when
       * the operands' errors leave the comparison undecided (exact operands
       * compare exactly): each derivative may then be off by 1 (max itself
       * is continuous, so its value's bound stays finite) */
      if (!isnan(a) && !isnan(b) && ea + eb > 0 && fabs(a - b) <= ea + eb) *eda = *edb = 1.0;
      break;
    case F_SIN:
      *da = cos(a);
      *eda = fabs(sin(a)) * ea + 0.5 * ea * ea + trig_abs() + U32 * fabs(*da);
      break;
    case F_COS:
      *da = -sin(a);
      *eda = fabs(cos(a)) * ea + 0.5 * ea * ea + trig_abs() + U32 * fabs(*da);
      break;
    case F_PLOG:
      undecided = ea > 0 && fabs(fabs(a) - GUARD) <= ea;
      if (fabs(a) > GUARD) {
        double m = fabs(a) - ea;
        *da = 1.0 / a;
        if (!(m > 0)) { undecided = 1; break; }
        *eda = ea / (fabs(a) * m) + 2 * U32 / fabs(a);
      }
      break;
    case F_CEXP:
      undecided = ea > 0 && fabs(a - EXP_CLAMP) <= ea;
      if (a <= EXP_CLAMP) {
        *da = exp(a);
        *eda = fabs(*da) * (expm1(ea) + (6 + 1.25 * fabs(a)) * U32);
      }
      break;
    case F_TAN: {
      double t = tan(a);
      double et = err_of(F_TAN, a, ea, 0.0, 0.0, t);
      *da = 1 + t * t;
      *eda = 2 * fabs(t) * et + et * et + 2 * U32 * fabs(*da);
      break;
    }
  }
  if (undecided) *eda = *edb = INFINITY;
}

/* The reverse sweep of backprop carrying a first-order bound eadj on how far
 * the FP32 adjoint of the value the parent sees at node i may be from adj.
 * Per leaf it adds the adjoint, its bound and |adjoint| (for the allowance
 * of the FP32 sums) into the constant and input-gradient accumulators. */
static void backprop_err(ctx_t* c, int i, double adj, double eadj, const double* seed,
                         const double* eseed, double* gval, double* egval, double* sgval,
                         double* gx, double* egx, double* sgx) {
  const tree_t* t = c->t;
  int ty = (int)t->type[i];
  int base = ty & ~T_MODI;
  if (base == T_CONST) { gval[i] += adj; egval[i] += eadj; sgval[i] += fabs(adj); return; }
  if (base == T_VAR) {
    int f = (int)t->val[i];
    gx[f] += adj; egx[f] += eadj; sgx[f] += fabs(adj);
    return;
  }
  long iv = (long)t->val[i];
  int f = (int)(iv % 256);
  int o = (int)(iv / 256);
  int ia = i + 1;
  int ib = arity_of(f) >= 2 ? c->c2[i] : -1;
  int ic = arity_of(f) == 3 ? c->c3[i] : -1;
  double a = c->v[ia], ea = c->ev[ia];
  double b = ib >= 0 ? c->v[ib] : 0.0, eb = ib >= 0 ? c->ev[ib] : 0.0;
  double af = (ty & T_MODI) ? seed[o] : adj;
  double eaf = (ty & T_MODI) ? eseed[o] : eadj;
  double pass_a = 0.0, pass_b = 0.0, pass_c = 0.0, epass_a = 0.0, epass_b = 0.0, epass_c = 0.0;
  if (ty & T_MODI) {
    if (ic >= 0) { pass_c = adj; epass_c = eadj; }
    else if (ib >= 0) { pass_b = adj; epass_b = eadj; }
    else { pass_a = adj; epass_a = eadj; }
  }
  double da, eda, db, edb, dc = 0.0, edc = 0.0;
  if (f == F_ITE) {
    /* the adjoint goes to the chosen branch; an undecided sign of the
     * condition may send it to the other one */
    da = eda = 0.0;
    db = a > 0 ? 1.0 : 0.0;
    dc = a > 0 ? 0.0 : 1.0;
    edb = edc = (ea > 0 && fabs(a) <= ea) ? INFINITY : 0.0;
  } else {
    dlocal(f, a, ea, b, eb, &da, &eda, &db, &edb);
  }
  /* one FP32 product (and one sum on a Modi node's pass-through) per child */
  /* a zero local derivative contributes nothing (as in backprop), but its
   * bound still counts: the FP32 path may see a non-zero one */
  double ga = pass_a + (da != 0.0 ? af * da : 0.0);
  double ega = epass_a + fabs(af) * eda + eaf * fabs(da) + eaf * eda + U32 * fabs(af * da) +
               U32 * fabs(ga);
  /* NaN (0 * inf) included; an adjoint that may leave the FP32 range too */
  if (!(ega < INFINITY) || fabs(ga) + ega > FLT_MAX) ega = INFINITY;
  backprop_err(c, ia, ga, ega, seed, eseed, gval, egval, sgval, gx, egx, sgx);
  if (ib >= 0) {
    double gb = pass_b + (db != 0.0 ? af * db : 0.0);
    double egb = epass_b + fabs(af) * edb + eaf * fabs(db) + eaf * edb + U32 * fabs(af * db) +
                 U32 * fabs(gb);
    if (!(egb < INFINITY) || fabs(gb) + egb > FLT_MAX) egb = INFINITY;
    backprop_err(c, ib, gb, egb, seed, eseed, gval, egval, sgval, gx, egx, sgx);
  }
  if (ic >= 0) {
    double gc = pass_c + (dc != 0.0 ? af * dc : 0.0);
    double egc = epass_c + fabs(af) * edc + eaf * fabs(dc) + eaf * edc + U32 * fabs(af * dc) +
                 U32 * fabs(gc);
    if (!(egc < INFINITY) || fabs(gc) + egc > FLT_MAX) egc = INFINITY;
    backprop_err(c, ic, gc, egc, seed, eseed, gval, egval, sgval, gx, egx, sgx);
  }
}

static void do_grad_tree(job_t* j, long p, double* gx_priv, double* egx_priv) {
  tree_t t = {j->type + p * j->ld, j->val + p * j->ld, j->size + p * j->ld, 0};
  int len;
  int st = orc_validate_one(t.type, t.val, t.size, j->max_len, j->F, j->O, &len);
  if (j->status) j->status[p] = st;
  int O = j->O;
  double* gval = j->grad_val + p * j->ld;
  for (long i = 0; i < j->ld; ++i) gval[i] = 0.0;
  if (st != ST_OK) {
    for (int k = 0; k < O; ++k) j->mse[p * O + k] = NAN;
    if (j->egrad_val)
      for (long i = 0; i < j->ld; ++i) j->egrad_val[p * j->ld + i] = INFINITY;
    return;
  }
  t.len = len;
  int hm = tree_has_modi(&t);
  const int we = j->egrad_val != NULL;
  double* v = (double*)malloc(sizeof(double) * (size_t)len * 4);
  double* fv = v + len;
  double* ev = v + 2 * (size_t)len;
  double* sgval = v + 3 * (size_t)len;
  int* c2 = (int*)malloc(sizeof(int) * (size_t)len * 2);
  int* c3 = c2 + len;
  double* buf = (double*)calloc((size_t)O * 5, sizeof(double));
  double *out = buf, *acc = buf + O, *seed = buf + 2 * O, *eout = buf + 3 * O, *eseed = buf + 4 * O;
  double* egval = we ? j->egrad_val + p * j->ld : NULL;
  if (we)
    for (long i = 0; i < j->ld; ++i) egval[i] = 0.0;
  for (int i = 0; i < len; ++i) sgval[i] = 0.0;
  int skip = 1;
  for (int k = 0; k < O; ++k) if (j->g[p * O + k] != 0.0) skip = 0;
  double inv_d = 1.0 / (double)j->D;
  for (long d = 0; d < j->D; ++d) {
    for (int k = 0; k < O; ++k) { out[k] = 0.0; eout[k] = 0.0; }
    ctx_t c = {&t, j->X + d * j->ldx, out, we ? eout : NULL, we, v, fv, c2, we ? ev : NULL, c3};
    int nx;
    double e;
    double r0 = eval_node(&c, 0, &nx, &e);
    if (!hm && O == 1) { out[0] = r0; eout[0] = e; }
    else finish_outputs(&c, O);
    for (int k = 0; k < O; ++k) {
      double r = out[k] - (double)j->y[d * j->ldy + k];
      acc[k] += r * r;
      seed[k] = j->g[p * O + k] * 2.0 * r * inv_d;
      /* the FP32 seed: (2g/D rounded) x (output - target, rounded) */
      double s2 = fabs(j->g[p * O + k] * 2.0 * inv_d);
      eseed[k] = s2 * (eout[k] + U32 * fabs(r)) + 2 * U32 * fabs(seed[k]);
      if (!(eseed[k] < INFINITY)) eseed[k] = INFINITY;
    }
    if (skip) continue; /* zero upstream gradient: nothing to propagate */
    double* gxd = gx_priv + d * j->F;
    if (we) {
      double* egxd = egx_priv + d * j->F;
      double* sgxd = egx_priv + (size_t)j->D * j->F + d * j->F;
      if (!hm && O == 1)
        backprop_err(&c, 0, seed[0], eseed[0], seed, eseed, gval, egval, sgval, gxd, egxd, sgxd);
      else
        backprop_err(&c, 0, 0.0, 0.0, seed, eseed, gval, egval, sgval, gxd, egxd, sgxd);
    } else if (!hm && O == 1) {
      backprop(&c, 0, seed[0], seed, gval, gxd);
    } else {
      /* the root's parent-visible value feeds no output */
      backprop(&c, 0, 0.0, seed, gval, gxd);
    }
  }
  for (int k = 0; k < O; ++k) j->mse[p * O + k] = acc[k] / (double)j->D;
  /* an FP32 sum of at most acc_terms contributions before the widening to
   * FP64 adds up to (acc_terms - 1) u times the sum of their magnitudes */
  if (we)
    for (int i = 0; i < len; ++i) {
      egval[i] += (j->acc_terms > 1 ? j->acc_terms - 1 : 0) * U32 * sgval[i];
      /* the gradient is delivered in FP32 */
      if (!(egval[i] < INFINITY) || fabs(gval[i]) + egval[i] > FLT_MAX) egval[i] = INFINITY;
    }
  free(v); free(c2); free(buf);
}

static void* worker(void* arg) {
  worker_t* w = (worker_t*)arg;
  job_t* j = w->j;
  for (long p = w->tid; p < j->pop; p += j->nthreads) {
    if (j->mode == 0) do_eval_tree(j, p);
    else if (j->mode == 1) do_mse_tree(j, p);
    else do_grad_tree(j, p, w->gx, w->egx);
  }
  return NULL;
}

static void run_job(job_t* j) {
  int nt = j->nthreads > 0 ? j->nthreads : 1;
  if (nt > j->pop) nt = j->pop > 0 ? (int)j->pop : 1;
  j->nthreads = nt;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nt);
  worker_t* ws = (worker_t*)calloc(nt, sizeof(worker_t));
  size_t gxn = (size_t)j->D * (size_t)j->F;
  for (int i = 0; i < nt; ++i) {
    ws[i].j = j;
    ws[i].tid = i;
    ws[i].gx = j->mode == 2 ? (double*)calloc(gxn > 0 ? gxn : 1, sizeof(double)) : NULL;
    ws[i].egx = (j->mode == 2 && j->egrad_val) ? (double*)calloc(gxn > 0 ? 2 * gxn : 1, sizeof(double))
                                                : NULL;
  }
  for (int i = 1; i < nt; ++i) pthread_create(&th[i], NULL, worker, &ws[i]);
  worker(&ws[0]);
  for (int i = 1; i < nt; ++i) pthread_join(th[i], NULL);
  if (j->mode == 2) {
    for (size_t q = 0; q < gxn; ++q) {
      double s = 0.0;
      for (int i = 0; i < nt; ++i) s += ws[i].gx[q];
      j->grad_X[q] = s;
      if (j->egrad_X) {
        /* the FP32 sum over the trees adds (pop - 1) u |terms| */
        double e = 0.0, m = 0.0;
        for (int i = 0; i < nt; ++i) { e += ws[i].egx[q]; m += ws[i].egx[gxn + q]; }
        e += (j->pop > 1 ? (double)(j->pop - 1) : 0.0) * U32 * m;
        j->egrad_X[q] = (e < INFINITY && fabs(s) + e <= FLT_MAX) ? e : INFINITY;
      }
    }
    for (int i = 0; i < nt; ++i) { free(ws[i].gx); free(ws[i].egx); }
  }
  free(th);
  free(ws);
}

/* ------------------------------------------------------------- C interface */
/* Validates every tree; status[pop], lens[pop]. */
void orc_validate(const float* type, const float* val, const float* size, long pop, long ld,
                  int max_len, int n_features, int n_outputs, int* status, int* lens) {
  for (long p = 0; p < pop; ++p)
    status[p] = orc_validate_one(type + p * ld, val + p * ld, size + p * ld, max_len,
                                 n_features, n_outputs, &lens[p]);
}

/* Forward outputs out[pop][O][D] (NaN rows for invalid trees) and, when err is
 * not NULL, the FP32 error bound per output point. */
void orc_eval(const float* type, const float* val, const float* size, long pop, long ld,
              int max_len, const float* X, long D, int F, long ldx, int O,
              double* out, double* err, int* status, int nthreads) {
  job_t j;
  memset(&j, 0, sizeof j);
  j.type = type; j.val = val; j.size = size; j.pop = pop; j.ld = ld; j.max_len = max_len;
  j.X = X; j.D = D; j.F = F; j.ldx = ldx; j.O = O;
  j.out = out; j.err = err; j.status = status; j.mode = 0; j.nthreads = nthreads;
  if (pop > 0) run_job(&j);
}

/* MSE[pop][O]; mse_allow (nullable) receives the MSE deviation that the
 * per-point tolerance rel_tol (and, at ill-conditioned points, 4x the FP32
 * bound) permits; it is infinite when some point is ambiguous. */
void orc_mse(const float* type, const float* val, const float* size, long pop, long ld,
             int max_len, const float* X, long D, int F, long ldx, const float* y, long ldy,
             int O, double* mse, double* mse_allow, double rel_tol, int* status, int nthreads) {
  job_t j;
  memset(&j, 0, sizeof j);
  j.type = type; j.val = val; j.size = size; j.pop = pop; j.ld = ld; j.max_len = max_len;
  j.X = X; j.D = D; j.F = F; j.ldx = ldx; j.y = y; j.ldy = ldy; j.O = O;
  j.mse = mse; j.mse_allow = mse_allow; j.rel_tol = rel_tol; j.status = status;
  j.mode = 1; j.nthreads = nthreads;
  if (pop > 0) run_job(&j);
}

/* Reverse mode of L = sum_{p,k} g[p,k] * MSE[p,k]: grad_val[pop][ld] (nonzero
 * only at constant nodes) and grad_X[D][F]; also returns MSE[pop][O].
 * With egrad_val / egrad_X (both non-NULL) it also returns a first-order
 * bound per element on how far an FP32 evaluation of the same gradient may
 * land: the forward bounds of every node value and output, propagated
 * through the seeds 2 g (o - y) / D and the local derivatives (dlocal), one
 * FP32 rounding per product and sum, and FP32 partial sums of at most
 * acc_terms contributions per constant (all trees' contributions per input
 * element) before FP64.  Infinite where a guard, clamp or max tie is
 * undecided or a value may leave the FP32 range. */
void orc_grad_bound(const float* type, const float* val, const float* size, long pop, long ld,
                    int max_len, const float* X, long D, int F, long ldx, const float* y, long ldy,
                    int O, const double* g, double* mse, double* grad_val, double* grad_X,
                    double* egrad_val, double* egrad_X, double acc_terms, int* status,
                    int nthreads) {
  job_t j;
  memset(&j, 0, sizeof j);
  j.type = type; j.val = val; j.size = size; j.pop = pop; j.ld = ld; j.max_len = max_len;
  j.X = X; j.D = D; j.F = F; j.ldx = ldx; j.y = y; j.ldy = ldy; j.O = O;
  j.g = g; j.mse = mse; j.grad_val = grad_val; j.grad_X = grad_X; j.status = status;
  j.egrad_val = egrad_X ? egrad_val : NULL;
  j.egrad_X = egrad_val ? egrad_X : NULL;
  j.acc_terms = acc_terms;
  j.mode = 2; j.nthreads = nthreads;
  for (long q = 0; q < D * F; ++q) {
    grad_X[q] = 0.0;
    if (j.egrad_X) j.egrad_X[q] = 0.0;
  }
  if (pop > 0) run_job(&j);
}

void orc_grad(const float* type, const float* val, const float* size, long pop, long ld,
              int max_len, const float* X, long D, int F, long ldx, const float* y, long ldy,
              int O, const double* g, double* mse, double* grad_val, double* grad_X,
              int* status, int nthreads) {
  orc_grad_bound(type, val, size, pop, ld, max_len, X, D, F, ldx, y, ldy, O, g, mse, grad_val,
                 grad_X, NULL, NULL, 0.0, status, nthreads);
}

/* Single-function evaluation in FP64 (used to pin the function table). */
double orc_apply(int f, double a, double b) { return apply(f, a, b); }
double orc_apply3(int f, double a, double b, double c) { return apply3(f, a, b, c); }
