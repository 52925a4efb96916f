/*
 * treegen.c -- seeded random prefix trees in the three-array population
 * encoding of Sec. III-A (types, values, subtree sizes; NaN padding).
 *
 * Input construction only: nothing here evaluates a tree.  Each tree draws
 * from its own splitmix64 stream (Steele, Lea and Flood, 2014) seeded by the
 * population seed and the tree index, so trees are generated in parallel and
 * reproducibly.
 *
 * Shape ("grow" with an exact target length n and a depth cap d): a subtree
 * of n nodes fits under depth d iff n <= 2^(d+1)-1 and, when the function set
 * has no unary function, n is odd.  A node with n = 1 is a leaf; otherwise a
 * function id is drawn uniformly from the set, and if its arity cannot
 * produce n nodes under the cap the other arity is used.  A binary node splits
 * its n-1 descendants uniformly over the feasible (left, right) pairs; a
 * ternary node (id 10) draws its first and second child sizes uniformly over
 * their feasible ranges in turn (function sets with a ternary id also hold a
 * unary one, so every size fits).
 * Leaves: the number of constants is Binomial(n_leaves, 1 - p_var) capped at
 * max_consts, placed on uniformly chosen leaves; the rest are variables with
 * a uniform feature index.  Constants are uniform on [c_lo, c_hi).
 * Modi trees: the root plus (m-1) further random function nodes carry the
 * Modi flag, m uniform on [max(1,O), min(modi_max, n_func)]; the first O of
 * them (in random order) cover outputs 0..O-1 and the rest draw an output
 * uniformly.  A tree with fewer function nodes than outputs is redrawn with a
 * new length.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef struct { uint64_t s; } sm64_t;

static uint64_t sm64_next(sm64_t* r) {
  uint64_t z = (r->s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static double sm64_unif(sm64_t* r) { return (double)(sm64_next(r) >> 11) * (1.0 / 9007199254740992.0); }
static int sm64_int(sm64_t* r, int lo, int hi) { /* inclusive */
  return lo + (int)(sm64_unif(r) * (double)(hi - lo + 1));
}

typedef struct {
  long pop, ld;
  int len_lo, len_hi, max_depth;
  const int* fset; int n_fset;
  int n_features;
  double c_lo, c_hi, p_var;
  int max_consts;
  int n_outputs, modi, modi_max;
  uint64_t seed;
  float *type, *val, *size;
  int nthreads;
} gen_t;

enum { T_VAR = 0, T_CONST = 1, T_UFUNC = 2, T_BFUNC = 3, T_TFUNC = 4, T_MODI = 16 };

static int arity(int f) { return f <= 4 ? 2 : f == 10 ? 3 : 1; }

typedef struct {
  int* kind;   /* 0 leaf, 1 unary, 2 binary, 3 ternary */
  int* func;
  int* size;
  int n;
} shape_t;

static int fits(long n, int d, int has_u) {
  if (n < 1 || d < 0) return 0;
  if (d > 30) d = 30;
  if (n > (1L << (d + 1)) - 1) return 0;
  return has_u || (n & 1);
}

/* iterative grow: stack of (position, n, depth_left) */
static void grow(const gen_t* g, sm64_t* r, int n0, shape_t* s, int has_u, int has_b) {
  int stk_n[2048], stk_d[2048], sp = 0;
  int pos = 0;
  stk_n[sp] = n0; stk_d[sp] = g->max_depth; sp++;
  while (sp > 0) {
    --sp;
    int n = stk_n[sp], d = stk_d[sp];
    int i = pos++;
    s->size[i] = n;
    if (n == 1) { s->kind[i] = 0; s->func[i] = -1; continue; }
    int f = g->fset[sm64_int(r, 0, g->n_fset - 1)];
    int ar = arity(f);
    int u_ok = has_u && fits(n - 1, d - 1, has_u);
    int b_ok = 0;
    long M = d - 1 >= 30 ? (1L << 30) : (1L << d) - 1; /* max child size */
    int a_lo = 1, a_hi = n - 2;
    if (has_b && n >= 3) {
      if (a_lo < n - 1 - M) a_lo = (int)(n - 1 - M);
      if (a_hi > M) a_hi = (int)M;
      b_ok = a_lo <= a_hi;
      if (!has_u && b_ok) { /* both children odd */
        if (!(a_lo & 1)) a_lo++;
        if (!(a_hi & 1)) a_hi--;
        b_ok = a_lo <= a_hi;
      }
    }
    if (ar == 3) {
      /* three children of at most M nodes each, only with a unary id in the
       * set (no parity constraint on the sizes) */
      long lo1 = n - 1 - 2 * M, hi1 = M < n - 3 ? M : n - 3;
      if (lo1 < 1) lo1 = 1;
      if (has_u && n >= 4 && lo1 <= hi1) {
        int a = sm64_int(r, (int)lo1, (int)hi1);
        long lo2 = n - 1 - a - M, hi2 = M < n - 2 - a ? M : n - 2 - a;
        if (lo2 < 1) lo2 = 1;
        int b = sm64_int(r, (int)lo2, (int)hi2);
        s->kind[i] = 3; s->func[i] = f;
        stk_n[sp] = n - 1 - a - b; stk_d[sp] = d - 1; sp++;
        stk_n[sp] = b; stk_d[sp] = d - 1; sp++;
        stk_n[sp] = a; stk_d[sp] = d - 1; sp++;
        continue;
      }
      ar = b_ok ? 2 : 1;
    }
    if (ar == 1 && !u_ok) ar = 2;
    if (ar == 2 && !b_ok) ar = 1;
    if (ar == 1) {
      if (arity(f) != 1) { /* redraw within the unary ids */
        int k; do { k = g->fset[sm64_int(r, 0, g->n_fset - 1)]; } while (arity(k) != 1);
        f = k;
      }
      s->kind[i] = 1; s->func[i] = f;
      stk_n[sp] = n - 1; stk_d[sp] = d - 1; sp++;
    } else {
      if (arity(f) != 2) {
        int k; do { k = g->fset[sm64_int(r, 0, g->n_fset - 1)]; } while (arity(k) != 2);
        f = k;
      }
      int a;
      if (has_u) a = sm64_int(r, a_lo, a_hi);
      else a = a_lo + 2 * sm64_int(r, 0, (a_hi - a_lo) / 2);
      s->kind[i] = 2; s->func[i] = f;
      /* push right first so the left child is emitted next (prefix order) */
      stk_n[sp] = n - 1 - a; stk_d[sp] = d - 1; sp++;
      stk_n[sp] = a; stk_d[sp] = d - 1; sp++;
    }
  }
  s->n = pos;
}

static void gen_tree(const gen_t* g, long p) {
  sm64_t r = {g->seed * 0xD1B54A32D192ED03ULL + (uint64_t)p * 0x9E3779B97F4A7C15ULL + 1};
  int has_u = 0, has_b = 0;
  for (int k = 0; k < g->n_fset; ++k) { if (arity(g->fset[k]) == 1) has_u = 1; else if (arity(g->fset[k]) == 2) has_b = 1; }
  int cap = g->len_hi;
  shape_t s;
  s.kind = (int*)malloc(sizeof(int) * cap * 3);
  s.func = s.kind + cap;
  s.size = s.kind + 2 * cap;
  int n;
  for (int tries = 0;; ++tries) {
    do { n = sm64_int(&r, g->len_lo, g->len_hi); } while (!fits(n, g->max_depth, has_u) && tries++ < 100000);
    grow(g, &r, n, &s, has_u, has_b);
    if (!g->modi) break;
    int nf = 0;
    for (int i = 0; i < n; ++i) nf += s.kind[i] != 0;
    if (nf >= g->n_outputs && s.kind[0] != 0) break;
  }
  float* ty = g->type + p * g->ld;
  float* va = g->val + p * g->ld;
  float* sz = g->size + p * g->ld;
  for (long i = 0; i < g->ld; ++i) { ty[i] = NAN; va[i] = NAN; sz[i] = NAN; }
  /* leaves: constants vs variables */
  int n_leaf = 0;
  for (int i = 0; i < n; ++i) n_leaf += s.kind[i] == 0;
  int* leaves = (int*)malloc(sizeof(int) * (n_leaf + 1));
  int q = 0;
  for (int i = 0; i < n; ++i) if (s.kind[i] == 0) leaves[q++] = i;
  int n_const = 0;
  for (int k = 0; k < n_leaf; ++k) n_const += sm64_unif(&r) >= g->p_var;
  if (g->max_consts >= 0 && n_const > g->max_consts) n_const = g->max_consts;
  /* partial Fisher-Yates: the first n_const leaves become constants */
  for (int k = 0; k < n_const; ++k) {
    int j = sm64_int(&r, k, n_leaf - 1);
    int t = leaves[k]; leaves[k] = leaves[j]; leaves[j] = t;
  }
  for (int i = 0; i < n; ++i) {
    sz[i] = (float)s.size[i];
    if (s.kind[i] == 0) { ty[i] = T_VAR; va[i] = (float)sm64_int(&r, 0, g->n_features - 1); }
    else { ty[i] = s.kind[i] == 1 ? T_UFUNC : s.kind[i] == 2 ? T_BFUNC : T_TFUNC; va[i] = (float)s.func[i]; }
  }
  for (int k = 0; k < n_const; ++k) {
    int i = leaves[k];
    ty[i] = T_CONST;
    va[i] = (float)(g->c_lo + (g->c_hi - g->c_lo) * sm64_unif(&r));
  }
  free(leaves);
  if (g->modi) {
    int nf = 0;
    int* fn = (int*)malloc(sizeof(int) * n);
    for (int i = 1; i < n; ++i) if (s.kind[i] != 0) fn[nf++] = i;
    int lo = g->n_outputs > 1 ? g->n_outputs : 1;
    int hi = g->modi_max < nf + 1 ? g->modi_max : nf + 1;
    if (hi < lo) hi = lo;
    int m = sm64_int(&r, lo, hi);
    for (int k = 0; k < m - 1 && k < nf; ++k) { /* choose m-1 non-root function nodes */
      int j = sm64_int(&r, k, nf - 1);
      int t = fn[k]; fn[k] = fn[j]; fn[j] = t;
    }
    /* chosen list: root, fn[0..m-2]; shuffle it, then outputs 0..O-1 first */
    int* ch = (int*)malloc(sizeof(int) * m);
    ch[0] = 0;
    for (int k = 1; k < m; ++k) ch[k] = fn[k - 1];
    for (int k = m - 1; k > 0; --k) {
      int j = sm64_int(&r, 0, k);
      int t = ch[k]; ch[k] = ch[j]; ch[j] = t;
    }
    for (int k = 0; k < m; ++k) {
      int i = ch[k];
      int o = k < g->n_outputs ? k : sm64_int(&r, 0, g->n_outputs - 1);
      ty[i] = (float)((int)ty[i] | T_MODI);
      va[i] = (float)(s.func[i] + 256 * o);
    }
    free(ch);
    free(fn);
  }
  free(s.kind);
}

static void* gen_worker(void* arg) {
  void** a = (void**)arg;
  const gen_t* g = (const gen_t*)a[0];
  long tid = (long)(intptr_t)a[1];
  for (long p = tid; p < g->pop; p += g->nthreads) gen_tree(g, p);
  return NULL;
}

/* Fills type/val/size [pop][ld] (ld >= len_hi).  Returns 0 on success. */
int tg_population(long pop, long ld, int len_lo, int len_hi, int max_depth,
                  const int* fset, int n_fset, int n_features, double c_lo, double c_hi,
                  double p_var, int max_consts, int n_outputs, int modi, int modi_max,
                  uint64_t seed, float* type, float* val, float* size, int nthreads) {
  if (len_lo < 1 || len_hi < len_lo || ld < len_hi || n_fset < 1 || n_features < 1) return 1;
  if (len_hi > 2000 || max_depth < 0) return 1;
  {
    int has_u = 0, ok = 0;
    for (int k = 0; k < n_fset; ++k) if (arity(fset[k]) == 1) has_u = 1;
    for (int n = len_lo; n <= len_hi && !ok; ++n) ok = fits(n, max_depth, has_u);
    if (!ok) return 2;                                   /* no length fits the depth cap */
    if (modi && (n_outputs < 1 || len_hi < 2 * n_outputs + 1)) return 3;
  }
  gen_t g = {pop, ld, len_lo, len_hi, max_depth, fset, n_fset, n_features, c_lo, c_hi, p_var,
             max_consts, n_outputs, modi, modi_max, seed, type, val, size, nthreads > 0 ? nthreads : 1};
  if (g.nthreads > pop) g.nthreads = pop > 0 ? (int)pop : 1;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * g.nthreads);
  void*** args = (void***)malloc(sizeof(void**) * g.nthreads);
  for (int t = 0; t < g.nthreads; ++t) {
    args[t] = (void**)malloc(sizeof(void*) * 2);
    args[t][0] = &g;
    args[t][1] = (void*)(intptr_t)t;
  }
  for (int t = 1; t < g.nthreads; ++t) pthread_create(&th[t], NULL, gen_worker, args[t]);
  if (pop > 0) gen_worker(args[0]);
  for (int t = 1; t < g.nthreads; ++t) pthread_join(th[t], NULL);
  for (int t = 0; t < g.nthreads; ++t) free(args[t]);
  free(args);
  free(th);
  return 0;
}
