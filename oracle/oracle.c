/* Oracle: plain CPU implementation of the kernel property counts, access
 * classification, feature layouts, prediction, ranking and weight fit of the
 * linear run-time model (arXiv:1604.04997).  TEST INFRASTRUCTURE ONLY: loaded by
 * the tests, the smoke check and the bench's CPU-baseline leg; never by the
 * product path.  Shares no code with the CUDA library.
 *
 * Counting follows Alg. 1 (Sec. 3.2): n_ops = sum over instructions i of
 * |pi_i(D_i)| * n_ops,i, where |pi_i(D_i)| is the number of integer points of the
 * instruction's loop domain.  orc_count_brute obtains |pi_i(D_i)| by visiting every
 * point; orc_count_struct evaluates the same number per axis, numerically, at the
 * given parameter values (a box intersected with per-axis guards; where guards couple
 * indices, by visiting all indices but one and counting the last one's interval), and
 * is pinned to the brute force by the tests.
 */
#include "oracle.h"

#include <ctype.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef __int128 i128;

#define MAXP 4
#define MAXD 32
#define MAXARR 16
#define MAXST 48
#define MAXBAR 48
#define MAXGU 16
#define MAXFL 8
#define MAXACC 32
#define MAXIDX 4
#define MAXNODE 8192
#define NAMELEN 40

enum { N_INT, N_PAR, N_DIM, N_ADD, N_SUB, N_MUL, N_NEG, N_FLOOR, N_CEIL };
typedef struct { int kind; int64_t v; int a, b; } node_t;

enum { TAG_G0 = 0, TAG_G1, TAG_G2, TAG_L0, TAG_L1, TAG_L2, TAG_SEQ };

typedef struct { char name[NAMELEN]; int tag; int lo, hi; } dim_t;
typedef struct { char name[NAMELEN]; int global, f64, n_ext; int ext[MAXIDX]; } arr_t;
typedef struct { int arr, store, width, n_idx; int idx[MAXIDX]; } acc_t;
typedef struct { int e; int64_t coef[MAXD]; } guard_t; /* e(par, dims) >= 0; coef = per stmt-dim slot */
typedef struct { int dtype, kind; int64_t count; } flop_t;
typedef struct {
  char name[NAMELEN];
  int n_dims; int dims[MAXD];
  int n_guards; guard_t guards[MAXGU];
  int n_flops; flop_t flops[MAXFL];
  int n_acc; acc_t acc[MAXACC];
} stmt_t;
typedef struct { char name[NAMELEN]; int n_dims; int dims[MAXD]; } bar_t;

struct orc_kernel {
  char name[NAMELEN];
  int n_params; char params[MAXP][NAMELEN];
  int n_arr; arr_t arr[MAXARR];
  int n_dims; dim_t dims[MAXD];
  int n_st; stmt_t st[MAXST];
  int n_bar; bar_t bar[MAXBAR];
  int n_nodes; node_t nodes[MAXNODE];
  int cls_done; int cls_err;
  int8_t cls[MAXST][MAXACC];
};

/* ------------------------------------------------------------------ arithmetic */

static i128 floordiv(i128 x, i128 c) { /* c > 0, mathematical floor */
  i128 q = x / c;
  if ((x % c) != 0 && x < 0) q -= 1;
  return q;
}

static i128 ev(const orc_kernel *k, int n, const int64_t *par, const int64_t *dimv) {
  const node_t *x = &k->nodes[n];
  switch (x->kind) {
    case N_INT: return x->v;
    case N_PAR: return par[x->a];
    case N_DIM: return dimv[x->a];
    case N_ADD: return ev(k, x->a, par, dimv) + ev(k, x->b, par, dimv);
    case N_SUB: return ev(k, x->a, par, dimv) - ev(k, x->b, par, dimv);
    case N_MUL: return ev(k, x->a, par, dimv) * ev(k, x->b, par, dimv);
    case N_NEG: return -ev(k, x->a, par, dimv);
    case N_FLOOR: return floordiv(ev(k, x->a, par, dimv), x->v);
    case N_CEIL: return -floordiv(-ev(k, x->a, par, dimv), x->v);
  }
  return 0;
}

/* polynomial degree in params+dims (floor/ceil count as degree-1 atoms) */
static int degree(const orc_kernel *k, int n) {
  const node_t *x = &k->nodes[n];
  int da, db;
  switch (x->kind) {
    case N_INT: return 0;
    case N_PAR: case N_DIM: return 1;
    case N_ADD: case N_SUB: da = degree(k, x->a); db = degree(k, x->b); return da > db ? da : db;
    case N_MUL: return degree(k, x->a) + degree(k, x->b);
    case N_NEG: return degree(k, x->a);
    case N_FLOOR: case N_CEIL: return degree(k, x->a) > 1 ? 9 : 1;
  }
  return 9;
}

static int uses_dims(const orc_kernel *k, int n) {
  const node_t *x = &k->nodes[n];
  switch (x->kind) {
    case N_DIM: return 1;
    case N_ADD: case N_SUB: case N_MUL: return uses_dims(k, x->a) || uses_dims(k, x->b);
    case N_NEG: case N_FLOOR: case N_CEIL: return uses_dims(k, x->a);
    default: return 0;
  }
}
static int uses_floor(const orc_kernel *k, int n) {
  const node_t *x = &k->nodes[n];
  switch (x->kind) {
    case N_FLOOR: case N_CEIL: return 1;
    case N_ADD: case N_SUB: case N_MUL: return uses_floor(k, x->a) || uses_floor(k, x->b);
    case N_NEG: return uses_floor(k, x->a);
    default: return 0;
  }
}

/* ------------------------------------------------------------------ parser */

typedef struct {
  orc_kernel *k;
  const char *s; int pos;
  const stmt_t *st;        /* statement whose dims may be named (NULL: params only) */
  char *err; int errlen; int bad;
} ps_t;

static void perr(ps_t *p, const char *msg) {
  if (!p->bad && p->err) snprintf(p->err, p->errlen, "%s near '%s'", msg, p->s + p->pos);
  p->bad = 1;
}

static int mk(ps_t *p, int kind, int64_t v, int a, int b) {
  orc_kernel *k = p->k;
  if (k->n_nodes >= MAXNODE) { perr(p, "expression pool full"); return 0; }
  node_t *x = &k->nodes[k->n_nodes];
  x->kind = kind; x->v = v; x->a = a; x->b = b;
  return k->n_nodes++;
}

static int p_expr(ps_t *p);

static int p_factor(ps_t *p) {
  const char *s = p->s;
  if (p->bad) return 0;
  if (isdigit((unsigned char)s[p->pos])) {
    int64_t v = 0;
    while (isdigit((unsigned char)s[p->pos])) { v = v * 10 + (s[p->pos] - '0'); p->pos++; if (v > (1LL << 40)) { perr(p, "integer too large"); return 0; } }
    return mk(p, N_INT, v, 0, 0);
  }
  if (s[p->pos] == '(') {
    p->pos++;
    int e = p_expr(p);
    if (s[p->pos] != ')') { perr(p, "expected ')'"); return 0; }
    p->pos++;
    return e;
  }
  if (isalpha((unsigned char)s[p->pos]) || s[p->pos] == '_') {
    char nm[NAMELEN]; int n = 0;
    while ((isalnum((unsigned char)s[p->pos]) || s[p->pos] == '_') && n < NAMELEN - 1) nm[n++] = s[p->pos++];
    nm[n] = 0;
    if ((!strcmp(nm, "floor") || !strcmp(nm, "ceil")) && s[p->pos] == '(') {
      int isfloor = !strcmp(nm, "floor");
      p->pos++;
      int e = p_expr(p);
      if (s[p->pos] != '/') { perr(p, "expected '/' in floor/ceil"); return 0; }
      p->pos++;
      int64_t c = 0;
      if (!isdigit((unsigned char)s[p->pos])) { perr(p, "divisor must be a positive integer"); return 0; }
      while (isdigit((unsigned char)s[p->pos])) { c = c * 10 + (s[p->pos] - '0'); p->pos++; }
      if (c <= 0 || s[p->pos] != ')') { perr(p, "bad floor/ceil"); return 0; }
      p->pos++;
      return mk(p, isfloor ? N_FLOOR : N_CEIL, c, e, 0);
    }
    for (int i = 0; i < p->k->n_params; i++)
      if (!strcmp(nm, p->k->params[i])) return mk(p, N_PAR, 0, i, 0);
    if (p->st) {
      for (int j = 0; j < p->st->n_dims; j++)
        if (!strcmp(nm, p->k->dims[p->st->dims[j]].name)) return mk(p, N_DIM, 0, p->st->dims[j], 0);
    }
    perr(p, "unknown name");
    return 0;
  }
  perr(p, "unexpected character");
  return 0;
}

static int p_term(ps_t *p) {
  int neg = 0;
  if (p->s[p->pos] == '-') { neg = 1; p->pos++; }
  int a = p_factor(p);
  while (!p->bad && p->s[p->pos] == '*') {
    p->pos++;
    int b = p_factor(p);
    a = mk(p, N_MUL, 0, a, b);
  }
  return neg ? mk(p, N_NEG, 0, a, 0) : a;
}

static int p_expr(ps_t *p) {
  int a = p_term(p);
  while (!p->bad && (p->s[p->pos] == '+' || p->s[p->pos] == '-')) {
    char op = p->s[p->pos++];
    int b = p_term(p);
    a = mk(p, op == '+' ? N_ADD : N_SUB, 0, a, b);
  }
  return a;
}

/* parse a full token as an expression; mode 0: params only, floor allowed (bounds/extents);
   mode 1: params + statement dims, affine, no floor (guards/indices) */
static int parse_tok(ps_t *p, const char *tok, const stmt_t *st, int mode) {
  ps_t q = *p;
  q.s = tok; q.pos = 0; q.st = st;
  int e = p_expr(&q);
  if (!q.bad && tok[q.pos] != 0) perr(&q, "trailing characters");
  if (!q.bad && degree(q.k, e) > 1) perr(&q, "expression is not affine");
  if (!q.bad && mode == 1 && uses_floor(q.k, e)) perr(&q, "floor/ceil not allowed here");
  if (!q.bad && mode == 0 && uses_dims(q.k, e)) perr(&q, "loop indices not allowed here");
  p->bad = q.bad;
  return e;
}

static int split(char *line, char **tok, int maxtok) {
  int n = 0;
  char *s = line;
  while (*s && n < maxtok) {
    while (*s && isspace((unsigned char)*s)) s++;
    if (!*s) break;
    tok[n++] = s;
    while (*s && !isspace((unsigned char)*s)) s++;
    if (*s) *s++ = 0;
  }
  return n;
}

static int find_dim(const orc_kernel *k, const char *nm) {
  for (int i = 0; i < k->n_dims; i++) if (!strcmp(k->dims[i].name, nm)) return i;
  return -1;
}
static int find_arr(const orc_kernel *k, const char *nm) {
  for (int i = 0; i < k->n_arr; i++) if (!strcmp(k->arr[i].name, nm)) return i;
  return -1;
}

static int parse_dimlist(ps_t *p, char *list, int *out, int *n) {
  *n = 0;
  if (!strcmp(list, "-")) return 0;
  char *s = list;
  while (*s) {
    char nm[NAMELEN]; int m = 0;
    while (*s && *s != ',' && m < NAMELEN - 1) nm[m++] = *s++;
    nm[m] = 0;
    if (*s == ',') s++;
    int d = find_dim(p->k, nm);
    if (d < 0) { perr(p, "unknown dim in list"); return -1; }
    for (int j = 0; j < *n; j++) if (out[j] == d) { perr(p, "dim listed twice"); return -1; }
    if (*n >= MAXD) { perr(p, "too many dims"); return -1; }
    out[(*n)++] = d;
  }
  return 0;
}

static void parse_access(ps_t *p, stmt_t *st, char **tok, int nt, int store) {
  if (nt < 2 || nt > 3) { perr(p, "load/store takes ARRAY[IDX,...] [x2|x4]"); return; }
  if (st->n_acc >= MAXACC) { perr(p, "too many accesses"); return; }
  acc_t *a = &st->acc[st->n_acc];
  memset(a, 0, sizeof *a);
  char *br = strchr(tok[1], '[');
  size_t L = strlen(tok[1]);
  if (!br || tok[1][L - 1] != ']') { perr(p, "expected ARRAY[...]"); return; }
  *br = 0; tok[1][L - 1] = 0;
  a->arr = find_arr(p->k, tok[1]);
  if (a->arr < 0) { perr(p, "unknown array"); return; }
  a->store = store;
  a->width = 1;
  if (nt == 3) {
    if (!strcmp(tok[2], "x2")) a->width = 2;
    else if (!strcmp(tok[2], "x4")) a->width = 4;
    else { perr(p, "vector width must be x2 or x4"); return; }
  }
  /* split indices on commas (no commas occur inside an affine index) */
  char *s = br + 1;
  while (1) {
    char *c = strchr(s, ',');
    if (c) *c = 0;
    if (a->n_idx >= MAXIDX) { perr(p, "too many indices"); return; }
    a->idx[a->n_idx++] = parse_tok(p, s, st, 1);
    if (p->bad) return;
    if (!c) break;
    s = c + 1;
  }
  const arr_t *ar = &p->k->arr[a->arr];
  if (a->n_idx != ar->n_ext) { perr(p, "index count does not match array rank"); return; }
  int bits = (ar->f64 ? 64 : 32) * a->width;
  if (bits > 128) { perr(p, "access wider than 128 bits"); return; }
  st->n_acc++;
}

/* guard coefficients per statement dim slot (affine: constant coefficients) */
static void guard_coefs(orc_kernel *k, const stmt_t *st, guard_t *g) {
  int64_t par[MAXP] = {0}, dimv[MAXD] = {0};
  i128 e0 = ev(k, g->e, par, dimv);
  for (int j = 0; j < st->n_dims; j++) {
    dimv[st->dims[j]] = 1;
    g->coef[j] = (int64_t)(ev(k, g->e, par, dimv) - e0);
    dimv[st->dims[j]] = 0;
  }
}

orc_kernel *orc_parse(const char *text, char *err, int errlen) {
  orc_kernel *k = (orc_kernel *)calloc(1, sizeof(orc_kernel));
  if (!k) return NULL;
  ps_t p; memset(&p, 0, sizeof p);
  p.k = k; p.err = err; p.errlen = errlen;
  if (err && errlen) err[0] = 0;
  size_t n = strlen(text);
  char *buf = (char *)malloc(n + 1);
  memcpy(buf, text, n + 1);
  char *save = NULL;
  stmt_t *cur = NULL;
  int have_kernel = 0, lineno = 0;
  for (char *line = strtok_r(buf, "\n", &save); line && !p.bad; line = strtok_r(NULL, "\n", &save)) {
    lineno++;
    char *h = strchr(line, '#');
    if (h) *h = 0;
    char *tok[16];
    int nt = split(line, tok, 16);
    if (nt == 0) continue;
    const char *kw = tok[0];
    if (cur) {
      if (!strcmp(kw, "end")) { cur = NULL; k->n_st++; continue; }
      if (!strcmp(kw, "guard")) {
        if (nt != 4) { perr(&p, "guard takes LHS OP RHS"); break; }
        if (cur->n_guards >= MAXGU) { perr(&p, "too many guards"); break; }
        int l = parse_tok(&p, tok[1], cur, 1), r = parse_tok(&p, tok[3], cur, 1);
        if (p.bad) break;
        int e;
        const char *op = tok[2];
        if (!strcmp(op, "<")) e = mk(&p, N_SUB, 0, mk(&p, N_SUB, 0, r, l), mk(&p, N_INT, 1, 0, 0));
        else if (!strcmp(op, "<=")) e = mk(&p, N_SUB, 0, r, l);
        else if (!strcmp(op, ">")) e = mk(&p, N_SUB, 0, mk(&p, N_SUB, 0, l, r), mk(&p, N_INT, 1, 0, 0));
        else if (!strcmp(op, ">=")) e = mk(&p, N_SUB, 0, l, r);
        else { perr(&p, "guard operator must be < <= > >="); break; }
        guard_t *g = &cur->guards[cur->n_guards++];
        g->e = e;
        guard_coefs(k, cur, g);
        continue;
      }
      if (!strcmp(kw, "flop")) {
        if (nt != 4) { perr(&p, "flop takes DTYPE KIND COUNT"); break; }
        if (cur->n_flops >= MAXFL) { perr(&p, "too many flop lines"); break; }
        flop_t *f = &cur->flops[cur->n_flops];
        if (!strcmp(tok[1], "f32")) f->dtype = 0; else if (!strcmp(tok[1], "f64")) f->dtype = 1;
        else { perr(&p, "flop dtype must be f32|f64"); break; }
        static const char *kinds[5] = {"add", "mul", "div", "pow", "spec"};
        f->kind = -1;
        for (int i = 0; i < 5; i++) if (!strcmp(tok[2], kinds[i])) f->kind = i;
        if (f->kind < 0) { perr(&p, "flop kind must be add|mul|div|pow|spec"); break; }
        char *endp;
        long long c = strtoll(tok[3], &endp, 10);
        if (*endp || c < 0) { perr(&p, "flop count must be a non-negative integer"); break; }
        f->count = c;
        cur->n_flops++;
        continue;
      }
      if (!strcmp(kw, "load") || !strcmp(kw, "store")) {
        parse_access(&p, cur, tok, nt, kw[0] == 's');
        continue;
      }
      perr(&p, "unknown directive inside stmt");
      break;
    }
    if (!strcmp(kw, "kernel")) {
      if (nt != 2 || have_kernel) { perr(&p, "kernel NAME (once)"); break; }
      snprintf(k->name, NAMELEN, "%s", tok[1]);
      have_kernel = 1;
    } else if (!strcmp(kw, "param")) {
      if (nt < 2 || nt - 1 > MAXP || k->n_params) { perr(&p, "param takes 1..4 names (once)"); break; }
      for (int i = 1; i < nt; i++) snprintf(k->params[k->n_params++], NAMELEN, "%s", tok[i]);
    } else if (!strcmp(kw, "array")) {
      if (nt != 5 || k->n_arr >= MAXARR) { perr(&p, "array NAME SPACE DTYPE EXTENTS"); break; }
      arr_t *a = &k->arr[k->n_arr];
      snprintf(a->name, NAMELEN, "%s", tok[1]);
      if (!strcmp(tok[2], "global")) a->global = 1; else if (!strcmp(tok[2], "local")) a->global = 0;
      else { perr(&p, "array space must be global|local"); break; }
      if (!strcmp(tok[3], "f32")) a->f64 = 0; else if (!strcmp(tok[3], "f64")) a->f64 = 1;
      else { perr(&p, "array dtype must be f32|f64"); break; }
      char *s = tok[4];
      while (1) {
        char *c = strchr(s, ',');
        if (c) *c = 0;
        if (a->n_ext >= MAXIDX) { perr(&p, "too many extents"); break; }
        a->ext[a->n_ext++] = parse_tok(&p, s, NULL, 0);
        if (p.bad || !c) break;
        s = c + 1;
      }
      k->n_arr++;
    } else if (!strcmp(kw, "dim")) {
      if (nt != 5 || k->n_dims >= MAXD) { perr(&p, "dim NAME TAG LO HI"); break; }
      dim_t *d = &k->dims[k->n_dims];
      snprintf(d->name, NAMELEN, "%s", tok[1]);
      static const char *tags[7] = {"g0", "g1", "g2", "l0", "l1", "l2", "seq"};
      d->tag = -1;
      for (int i = 0; i < 7; i++) if (!strcmp(tok[2], tags[i])) d->tag = i;
      if (d->tag < 0) { perr(&p, "unknown dim tag"); break; }
      d->lo = parse_tok(&p, tok[3], NULL, 0);
      d->hi = parse_tok(&p, tok[4], NULL, 0);
      if (p.bad) break;
      for (int i = 0; i < k->n_dims; i++) if (!strcmp(k->dims[i].name, d->name)) { perr(&p, "duplicate dim"); break; }
      if (d->tag >= TAG_L0 && d->tag <= TAG_L2) {
        /* work-item index ranges are fixed by the group size */
        int64_t z[MAXP] = {0}, o[MAXP] = {1, 1, 1, 1};
        if (uses_floor(k, d->lo) || uses_floor(k, d->hi) || degree(k, d->lo) || degree(k, d->hi) ||
            ev(k, d->lo, z, NULL) != 0 || ev(k, d->hi, o, NULL) <= 0) {
          (void)o; perr(&p, "local dims need constant range [0, W)"); break;
        }
      }
      k->n_dims++;
    } else if (!strcmp(kw, "stmt")) {
      if (nt != 3 || k->n_st >= MAXST) { perr(&p, "stmt NAME DIMS"); break; }
      cur = &k->st[k->n_st];
      memset(cur, 0, sizeof *cur);
      snprintf(cur->name, NAMELEN, "%s", tok[1]);
      parse_dimlist(&p, tok[2], cur->dims, &cur->n_dims);
    } else if (!strcmp(kw, "barrier")) {
      if (nt != 3 || k->n_bar >= MAXBAR) { perr(&p, "barrier NAME DIMS"); break; }
      bar_t *b = &k->bar[k->n_bar];
      snprintf(b->name, NAMELEN, "%s", tok[1]);
      parse_dimlist(&p, tok[2], b->dims, &b->n_dims);
      for (int j = 0; j < b->n_dims && !p.bad; j++) {
        int t = k->dims[b->dims[j]].tag;
        if (t >= TAG_L0 && t <= TAG_L2) perr(&p, "barrier may not depend on work-item indices");
      }
      k->n_bar++;
    } else {
      perr(&p, "unknown directive");
    }
  }
  if (!p.bad && cur) perr(&p, "missing end");
  if (!p.bad && (!have_kernel || !k->n_params)) perr(&p, "missing kernel/param line");
  /* every statement and barrier runs in every work-group */
  for (int s = 0; s < k->n_st && !p.bad; s++)
    for (int d = 0; d < k->n_dims; d++)
      if (k->dims[d].tag <= TAG_G2) {
        int found = 0;
        for (int j = 0; j < k->st[s].n_dims; j++) found |= k->st[s].dims[j] == d;
        if (!found) { perr(&p, "statement does not list every group dim"); break; }
      }
  for (int s = 0; s < k->n_bar && !p.bad; s++)
    for (int d = 0; d < k->n_dims; d++)
      if (k->dims[d].tag <= TAG_G2) {
        int found = 0;
        for (int j = 0; j < k->bar[s].n_dims; j++) found |= k->bar[s].dims[j] == d;
        if (!found) { perr(&p, "barrier does not list every group dim"); break; }
      }
  free(buf);
  if (p.bad) {
    if (err && errlen && !err[0]) snprintf(err, errlen, "parse error at line %d", lineno);
    free(k);
    return NULL;
  }
  return k;
}

void orc_free(orc_kernel *k) { free(k); }
int orc_n_params(const orc_kernel *k) { return k->n_params; }
int orc_n_stmts(const orc_kernel *k) { return k->n_st; }
int orc_n_access(const orc_kernel *k, int s) { return (s >= 0 && s < k->n_st) ? k->st[s].n_acc : -1; }

/* ------------------------------------------------------------------ domains */

static void dim_range(const orc_kernel *k, int d, const int64_t *par, i128 *lo, i128 *hi) {
  *lo = ev(k, k->dims[d].lo, par, NULL);
  *hi = ev(k, k->dims[d].hi, par, NULL);
}

/* Enumerate every point of statement s's domain; call fn for each point satisfying the guards.
   Returns number of points visited or -1 if more than max_points would be visited. */
typedef void (*visit_fn)(const orc_kernel *, int s, const int64_t *par, const int64_t *dimv, void *ctx);

static i128 enumerate_stmt(const orc_kernel *k, int s, const int64_t *par, int64_t max_points,
                           visit_fn fn, void *ctx, i128 *n_in) {
  const stmt_t *st = &k->st[s];
  i128 lo[MAXD], hi[MAXD], total = 1;
  int64_t dimv[MAXD] = {0};
  for (int j = 0; j < st->n_dims; j++) {
    dim_range(k, st->dims[j], par, &lo[j], &hi[j]);
    i128 r = hi[j] - lo[j];
    if (r <= 0) { *n_in = 0; return 0; }
    total *= r;
    if (total > max_points) return -1;
  }
  for (int j = 0; j < st->n_dims; j++) dimv[st->dims[j]] = (int64_t)lo[j];
  i128 cnt = 0;
  for (i128 it = 0; it < total; it++) {
    int ok = 1;
    for (int g = 0; g < st->n_guards && ok; g++) ok = ev(k, st->guards[g].e, par, dimv) >= 0;
    if (ok) { cnt++; if (fn) fn(k, s, par, dimv, ctx); }
    for (int j = st->n_dims - 1; j >= 0; j--) {           /* odometer */
      int d = st->dims[j];
      if (++dimv[d] < hi[j]) break;
      dimv[d] = (int64_t)lo[j];
    }
  }
  *n_in = cnt;
  return total;
}

/* Numeric per-axis count of statement s at par (see header comment).
   Returns 0 and *out, or -3 if the guards couple axes in a way this evaluator does not handle. */
static int struct_stmt(const orc_kernel *k, int s, const int64_t *par, i128 *out) {
  const stmt_t *st = &k->st[s];
  int nd = st->n_dims;
  i128 lo[MAXD], hi[MAXD];
  int owner[MAXD];                 /* -1 free, -2 single-dim guards, >=0 composite group id */
  for (int j = 0; j < nd; j++) {
    dim_range(k, st->dims[j], par, &lo[j], &hi[j]);
    if (hi[j] <= lo[j]) { *out = 0; return 0; }
    owner[j] = -1;
  }
  int64_t zero[MAXD] = {0};
  /* composite groups */
  int ng = 0;
  int gmask[MAXGU];                /* bitmask of stmt dim slots */
  int gref[MAXGU];                 /* guard defining the coefficient ratios */
  i128 glo[MAXGU], ghi[MAXGU];     /* j-range bounds [glo, ghi) before clamping to [0, N) */
  i128 single_lo[MAXD], single_hi[MAXD];
  for (int j = 0; j < nd; j++) { single_lo[j] = lo[j]; single_hi[j] = hi[j]; }
  for (int g = 0; g < st->n_guards; g++) {
    const guard_t *gu = &st->guards[g];
    i128 e0 = ev(k, gu->e, par, zero);
    int mask = 0, cnt = 0, only = -1;
    for (int j = 0; j < nd; j++) if (gu->coef[j]) { mask |= 1 << j; cnt++; only = j; }
    if (cnt == 0) { if (e0 < 0) { *out = 0; return 0; } continue; }
    if (cnt == 1) {
      if (owner[only] >= 0) return -3;
      owner[only] = -2;
      i128 c = gu->coef[only];
      if (c > 0) { i128 b = -floordiv(e0, c); if (b > single_lo[only]) single_lo[only] = b; }          /* d >= ceil(-e0/c) */
      else { i128 b = floordiv(e0, -c) + 1; if (b < single_hi[only]) single_hi[only] = b; }            /* d <= floor(e0/|c|) */
      continue;
    }
    int gi = -1;
    for (int q = 0; q < ng; q++) if (gmask[q] == mask) gi = q;
    for (int j = 0; j < nd; j++)
      if ((mask >> j) & 1) {
        if (owner[j] == -2) return -3;
        if (owner[j] >= 0 && owner[j] != (gi < 0 ? ng : gi)) return -3;
      }
    if (gi < 0) {
      if (ng >= MAXGU) return -3;
      gi = ng++;
      gmask[gi] = mask; gref[gi] = g;
      glo[gi] = 0; ghi[gi] = ((i128)1) << 100;
      for (int j = 0; j < nd; j++) if ((mask >> j) & 1) owner[j] = gi;
    }
    /* proportional to the reference guard? */
    const guard_t *rf = &st->guards[gref[gi]];
    int j1 = -1;
    for (int j = 0; j < nd; j++) if ((mask >> j) & 1) { j1 = j; break; }
    for (int j = 0; j < nd; j++)
      if ((mask >> j) & 1) {
        if ((i128)gu->coef[j] * rf->coef[j1] != (i128)rf->coef[j] * gu->coef[j1]) return -3;
      }
    /* order the dims by (|coef|, range) and check the mixed-radix chain */
    int ord[MAXD], no = 0;
    for (int j = 0; j < nd; j++) if ((mask >> j) & 1) ord[no++] = j;
    for (int a = 0; a < no; a++)
      for (int b = a + 1; b < no; b++) {
        i128 ca = rf->coef[ord[a]] < 0 ? -(i128)rf->coef[ord[a]] : rf->coef[ord[a]];
        i128 cb = rf->coef[ord[b]] < 0 ? -(i128)rf->coef[ord[b]] : rf->coef[ord[b]];
        i128 ra = hi[ord[a]] - lo[ord[a]], rb = hi[ord[b]] - lo[ord[b]];
        if (cb < ca || (cb == ca && rb < ra)) { int t = ord[a]; ord[a] = ord[b]; ord[b] = t; }
      }
    i128 sgn0 = rf->coef[ord[0]] > 0 ? 1 : -1;
    for (int a = 0; a < no; a++)
      if ((rf->coef[ord[a]] > 0 ? 1 : -1) != sgn0) return -3;
    i128 a1 = rf->coef[ord[0]] * sgn0;
    i128 N = 1;
    for (int a = 0; a < no; a++) {
      int j = ord[a];
      i128 aj = rf->coef[j] * sgn0;
      if (a < no - 1) {
        if (lo[j] != 0) return -3;
        i128 anext = rf->coef[ord[a + 1]] * sgn0;
        if (anext != aj * (hi[j] - lo[j])) return -3;
      }
      N *= hi[j] - lo[j];
    }
    int top = ord[no - 1];
    i128 J0 = (rf->coef[top] * sgn0 / a1) * lo[top];
    /* this guard in j: c1 (j + J0) + e0 >= 0 with c1 = gu coefficient of ord[0] */
    i128 c1 = gu->coef[ord[0]];
    if (c1 > 0) { i128 b = -floordiv(e0, c1) - J0; if (b > glo[gi]) glo[gi] = b; }
    else { i128 b = floordiv(e0, -c1) - J0 + 1; if (b < ghi[gi]) ghi[gi] = b; }
    (void)N;
  }
  i128 total = 1;
  for (int j = 0; j < nd; j++) {
    if (owner[j] == -1) total *= hi[j] - lo[j];
    else if (owner[j] == -2) { i128 r = single_hi[j] - single_lo[j]; total *= r > 0 ? r : 0; }
  }
  for (int q = 0; q < ng; q++) {
    i128 N = 1;
    for (int j = 0; j < nd; j++) if ((gmask[q] >> j) & 1) N *= hi[j] - lo[j];
    i128 a = glo[q] > 0 ? glo[q] : 0, b = ghi[q] < N ? ghi[q] : N;
    total *= b > a ? b - a : 0;
  }
  *out = total;
  return 0;
}

/* Count of statement s at par when its guards couple indices (j < i, a band, a sequential
   index bounded by a tiled one).  The indices fall into groups joined by shared guards;
   the count is the product of the groups' counts.  In each group, visit every point of
   all its indices but the one with the widest range, and take that index's interval
   from the guards directly (each guard is affine: c x + e >= 0 with the others fixed).
   Returns 0 and *out, or -3 if a group needs more than max_outer visits. */
static int semi_stmt(const orc_kernel *k, int s, const int64_t *par, i128 max_outer, i128 *out) {
  const stmt_t *st = &k->st[s];
  int nd = st->n_dims;
  i128 lo[MAXD], hi[MAXD];
  int grp[MAXD];
  for (int j = 0; j < nd; j++) {
    dim_range(k, st->dims[j], par, &lo[j], &hi[j]);
    if (hi[j] <= lo[j]) { *out = 0; return 0; }
    grp[j] = j;
  }
  for (int g = 0; g < st->n_guards; g++) {          /* join the indices of each guard */
    int first = -1;
    for (int j = 0; j < nd; j++) {
      if (!st->guards[g].coef[j]) continue;
      if (first < 0) { first = j; continue; }
      int a = grp[j], b = grp[first];
      for (int q = 0; q < nd; q++) if (grp[q] == a) grp[q] = b;
    }
  }
  i128 total = 1;
  int64_t dimv[MAXD] = {0};
  for (int g = 0; g < st->n_guards; g++) {          /* guards on the parameters alone */
    int param_only = 1;
    for (int j = 0; j < nd; j++) param_only &= !st->guards[g].coef[j];
    if (param_only && ev(k, st->guards[g].e, par, dimv) < 0) { *out = 0; return 0; }
  }
  for (int r = 0; r < nd; r++) {
    if (grp[r] != r) continue;                       /* r names its group */
    int last = -1;
    for (int j = 0; j < nd; j++)
      if (grp[j] == r && (last < 0 || hi[j] - lo[j] >= hi[last] - lo[last])) last = j;
    i128 outer = 1;
    for (int j = 0; j < nd; j++) {
      if (grp[j] != r || j == last) continue;
      outer *= hi[j] - lo[j];
      if (outer > max_outer) return -3;
      dimv[st->dims[j]] = (int64_t)lo[j];
    }
    dimv[st->dims[last]] = 0;
    i128 cnt = 0;
    for (i128 it = 0; it < outer; it++) {
      i128 a = lo[last], b = hi[last];
      for (int g = 0; g < st->n_guards && a < b; g++) {
        int mine = 0;
        for (int j = 0; j < nd; j++) mine |= st->guards[g].coef[j] && grp[j] == r;
        if (!mine) continue;
        i128 e0 = ev(k, st->guards[g].e, par, dimv);   /* the guard at x_last = 0 */
        i128 c = st->guards[g].coef[last];
        if (c == 0) { if (e0 < 0) b = a; }
        else if (c > 0) { i128 t = -floordiv(e0, c); if (t > a) a = t; }        /* x >= ceil(-e0/c) */
        else { i128 t = floordiv(e0, -c) + 1; if (t < b) b = t; }               /* x <= floor(e0/|c|) */
      }
      if (b > a) cnt += b - a;
      for (int j = nd - 1; j >= 0; j--) {                /* odometer over the group's other indices */
        if (grp[j] != r || j == last) continue;
        int d = st->dims[j];
        if (++dimv[d] < hi[j]) break;
        dimv[d] = (int64_t)lo[j];
      }
    }
    total *= cnt;
  }
  *out = total;
  return 0;
}

/* ------------------------------------------------------------------ classification (Sec. 2.1, Alg. 2) */

static i128 lin_offset(const orc_kernel *k, const acc_t *a, const int64_t *par, const int64_t *dimv) {
  const arr_t *ar = &k->arr[a->arr];
  i128 off = 0;
  for (int x = 0; x < a->n_idx; x++) off = off * ev(k, ar->ext[x], par, NULL) + ev(k, a->idx[x], par, dimv);
  return off;
}

typedef struct { int arr; uint8_t *bm; i128 size; int bad; } mark_ctx;

static void mark_visit(const orc_kernel *k, int s, const int64_t *par, const int64_t *dimv, void *vctx) {
  mark_ctx *c = (mark_ctx *)vctx;
  const stmt_t *st = &k->st[s];
  for (int i = 0; i < st->n_acc; i++) {
    const acc_t *a = &st->acc[i];
    if (a->arr != c->arr) continue;
    i128 off = lin_offset(k, a, par, dimv);
    if (off < 0 || off + a->width > c->size) { c->bad = 1; continue; }
    for (int w = 0; w < a->width; w++) c->bm[(int64_t)off + w] = 1;
  }
}

#define CLS_N 128
static int classify(orc_kernel *k) {
  if (k->cls_done) return k->cls_err;
  int64_t p1[MAXP], p2[MAXP];
  for (int i = 0; i < MAXP; i++) { p1[i] = CLS_N; p2[i] = 2 * CLS_N; }
  /* footprint bitmaps per global array, built on demand */
  uint8_t *bm[MAXARR] = {0};
  i128 size[MAXARR] = {0}, cells[MAXARR] = {0};
  int err = 0;
  for (int s = 0; s < k->n_st && !err; s++) {
    const stmt_t *st = &k->st[s];
    int l0 = -1;
    for (int j = 0; j < st->n_dims; j++) if (k->dims[st->dims[j]].tag == TAG_L0) l0 = st->dims[j];
    for (int i = 0; i < st->n_acc && !err; i++) {
      const acc_t *a = &st->acc[i];
      const arr_t *ar = &k->arr[a->arr];
      if (!ar->global) { k->cls[s][i] = -1; continue; }
      if (l0 < 0) { k->cls[s][i] = 0; continue; }
      int64_t dv[MAXD] = {0};
      i128 c1 = lin_offset(k, a, p1, dv), c2 = lin_offset(k, a, p2, dv);
      dv[l0] = 1;
      c1 = lin_offset(k, a, p1, dv) - c1;
      c2 = lin_offset(k, a, p2, dv) - c2;
      int param = c1 != c2;
      i128 se = c1 < 0 ? -c1 : c1;            /* stride in elements at the instance */
      if (!param && se % a->width) { err = -3; break; }
      i128 sv = param ? 1000 : se / a->width;  /* stride in units of the access size */
      if (!param && sv <= 1) { k->cls[s][i] = (int8_t)sv; continue; }
      int A = a->arr;
      if (!bm[A]) {
        i128 sz = 1;
        for (int x = 0; x < ar->n_ext; x++) sz *= ev(k, ar->ext[x], p1, NULL);
        if (sz <= 0 || sz > (1 << 26)) { err = -5; break; }
        size[A] = sz;
        bm[A] = (uint8_t *)calloc((size_t)sz, 1);
        mark_ctx mc = {A, bm[A], sz, 0};
        for (int t = 0; t < k->n_st && !err; t++) {
          i128 nin;
          if (enumerate_stmt(k, t, p1, (int64_t)1 << 25, mark_visit, &mc, &nin) < 0) err = -2;
        }
        if (mc.bad) err = -5;
        for (i128 x = 0; x < sz; x++) cells[A] += bm[A][x];
      }
      if (err) break;
      /* filled-in footprint: every cell within se-1 cells after an accessed cell */
      i128 filled = 0, last = -((i128)1 << 80);
      for (i128 x = 0; x < size[A] + se; x++) {
        if (x < size[A] && bm[A][x]) last = x;
        if (x - last < se) filled++;
      }
      i128 num = cells[A];
      /* no accessed cell, or a lane stride of 0 at the instance: the Sec. 2.1 fraction
         is undefined there, so the access is refused */
      if (num == 0 || filled == 0) { err = -3; break; }
      int cls;
      if (!param && sv <= 4) {
        i128 j = (sv * num + filled - 1) / filled;
        if (j < 1) j = 1;
        if (j > sv) j = (int)sv;
        cls = (sv == 2 ? 1 : sv == 3 ? 3 : 6) + (int)j;
      } else {
        i128 j = (4 * num + filled - 1) / filled;
        if (j < 1) j = 1;
        if (j > 4) j = 4;
        cls = 10 + (int)j;
      }
      k->cls[s][i] = (int8_t)cls;
    }
  }
  for (int A = 0; A < MAXARR; A++) free(bm[A]);
  k->cls_done = 1;
  k->cls_err = err;
  return err;
}

int orc_classify(orc_kernel *k, int32_t *out, int cap) {
  int e = classify(k);
  if (e) return e;
  int n = 0;
  for (int s = 0; s < k->n_st; s++)
    for (int i = 0; i < k->st[s].n_acc; i++) { if (n < cap) out[n] = k->cls[s][i]; n++; }
  return n;
}

/* ------------------------------------------------------------------ counts */

static int add_stmt_keys(const orc_kernel *k, int s, i128 cnt, i128 *keys) {
  const stmt_t *st = &k->st[s];
  for (int f = 0; f < st->n_flops; f++) keys[ORC_K_FLOP + st->flops[f].dtype * 5 + st->flops[f].kind] += cnt * st->flops[f].count;
  for (int i = 0; i < st->n_acc; i++) {
    const acc_t *a = &st->acc[i];
    const arr_t *ar = &k->arr[a->arr];
    if (!ar->global) {
      keys[(a->store ? ORC_K_LSTORE : ORC_K_LLOAD) + ar->f64] += cnt;
    } else {
      int bits = (ar->f64 ? 64 : 32) * a->width;
      int sz = bits == 32 ? 0 : bits == 64 ? 1 : 2;
      keys[ORC_K_GLOBAL + (a->store * 3 + sz) * ORC_NCLASS + k->cls[s][i]] += cnt;
    }
  }
  return 0;
}

static int kernel_common(const orc_kernel *k, const int64_t *par, i128 *keys) {
  keys[ORC_K_CONST] = 1;
  i128 groups = 1;
  for (int d = 0; d < k->n_dims; d++)
    if (k->dims[d].tag <= TAG_G2) {
      i128 lo, hi;
      dim_range(k, d, par, &lo, &hi);
      groups *= hi > lo ? hi - lo : 0;
    }
  keys[ORC_K_GROUPS] = groups;
  /* barriers: one per work-group per pass, i.e. one per point of the barrier's dims (Sec. 2.3) */
  for (int b = 0; b < k->n_bar; b++) {
    i128 c = 1;
    for (int j = 0; j < k->bar[b].n_dims; j++) {
      i128 lo, hi;
      dim_range(k, k->bar[b].dims[j], par, &lo, &hi);
      c *= hi > lo ? hi - lo : 0;
    }
    keys[ORC_K_BARRIERS] += c;
  }
  return 0;
}

static int finish_keys(const i128 *keys, int64_t *out) {
  for (int i = 0; i < ORC_NKEYS; i++) {
    if (keys[i] > INT64_MAX || keys[i] < INT64_MIN) return -4;
    out[i] = (int64_t)keys[i];
  }
  return 0;
}

int orc_count_brute(orc_kernel *k, const int64_t *par, int64_t max_points, int64_t *out) {
  int e = classify(k);
  if (e) return e;
  i128 keys[ORC_NKEYS];
  memset(keys, 0, sizeof keys);
  kernel_common(k, par, keys);
  for (int s = 0; s < k->n_st; s++) {
    i128 cnt;
    if (enumerate_stmt(k, s, par, max_points, NULL, NULL, &cnt) < 0) return -2;
    add_stmt_keys(k, s, cnt, keys);
  }
  return finish_keys(keys, out);
}

int orc_count_struct(orc_kernel *k, const int64_t *par, int64_t *out) {
  int e = classify(k);
  if (e) return e;
  i128 keys[ORC_NKEYS];
  memset(keys, 0, sizeof keys);
  kernel_common(k, par, keys);
  for (int s = 0; s < k->n_st; s++) {
    i128 cnt;
    int r = struct_stmt(k, s, par, &cnt);
    if (r == -3) r = semi_stmt(k, s, par, ((i128)1) << 30, &cnt);
    if (r) return r;
    add_stmt_keys(k, s, cnt, keys);
  }
  return finish_keys(keys, out);
}

/* ------------------------------------------------------------------ layouts */

static int64_t gkey(const int64_t *keys, int store, int size, int cls) {
  return keys[ORC_K_GLOBAL + (store * 3 + size) * ORC_NCLASS + cls];
}
static int is_filled(int c) { return c == 3 || c == 6 || c == 10; }
static int is_partial(int c) { return c == 2 || c == 4 || c == 5 || c == 7 || c == 8 || c == 9; }
static int is_wide(int c) { return c >= 11; }

int orc_layout(const int64_t *keys, int layout, int64_t *c) {
  if (layout == 32) {
    memset(c, 0, 32 * sizeof(int64_t));
    c[0] = keys[ORC_K_CONST]; c[1] = keys[ORC_K_GROUPS]; c[2] = keys[ORC_K_BARRIERS];
    for (int t = 0; t < 2; t++)
      for (int q = 0; q < 5; q++) c[3 + 5 * t + q] = keys[ORC_K_FLOP + 5 * t + q];
    c[13] = keys[ORC_K_LLOAD + 0]; c[14] = keys[ORC_K_LLOAD + 1];
    c[15] = keys[ORC_K_LSTORE + 0] + keys[ORC_K_LSTORE + 1];
    for (int cl = 0; cl < ORC_NCLASS; cl++) {
      int64_t l32 = gkey(keys, 0, 0, cl), l64 = gkey(keys, 0, 1, cl);
      int64_t s32 = gkey(keys, 1, 0, cl), s64 = gkey(keys, 1, 1, cl);
      if (cl == 0) c[16] += l32; else if (cl == 1) c[17] += l32;
      else if (is_filled(cl)) c[18] += l32; else if (is_partial(cl)) c[19] += l32; else if (is_wide(cl)) c[20] += l32;
      if (cl == 0) c[21] += l64; else if (cl == 1) c[22] += l64; else c[23] += l64;
      if (cl == 1) c[24] += s32; else if (cl == 0 || is_filled(cl)) c[25] += s32; else c[26] += s32;
      if (cl == 1) c[27] += s64; else c[28] += s64;
      c[31] += gkey(keys, 0, 2, cl) + gkey(keys, 1, 2, cl);
    }
    /* min(loads, stores) per access size, stride-1 accesses (Sec. 2.1) */
    c[29] = c[17] < c[24] ? c[17] : c[24];
    c[30] = c[22] < c[27] ? c[22] : c[27];
    return 32;
  }
  if (layout == 12) {
    memset(c, 0, 12 * sizeof(int64_t));
    c[0] = keys[ORC_K_CONST]; c[1] = keys[ORC_K_GROUPS]; c[2] = keys[ORC_K_BARRIERS];
    for (int q = 0; q < 5; q++) { c[3] += keys[ORC_K_FLOP + q]; c[4] += keys[ORC_K_FLOP + 5 + q]; }
    c[5] = keys[ORC_K_LLOAD] + keys[ORC_K_LLOAD + 1];
    c[6] = keys[ORC_K_LSTORE] + keys[ORC_K_LSTORE + 1];
    int64_t ld1 = 0, st1 = 0;
    for (int sz = 0; sz < 3; sz++)
      for (int cl = 0; cl < ORC_NCLASS; cl++) {
        int64_t l = gkey(keys, 0, sz, cl), s = gkey(keys, 1, sz, cl);
        if (cl <= 1) c[7] += l; else c[8] += l;
        if (cl == 1) c[9] += s; else c[10] += s;
        if (cl == 1) { ld1 += l; st1 += s; }
      }
    c[11] = ld1 < st1 ? ld1 : st1;
    return 12;
  }
  return -1;
}

int orc_eval(orc_kernel *k, int layout, int method, const int64_t *points, int64_t n_points,
             int64_t max_points, int64_t *out) {
  int kk = layout;
  int e = classify(k);
  if (e) return e;
  int np = k->n_params;
  for (int64_t p = 0; p < n_points; p++) {
    int64_t keys[ORC_NKEYS];
    int r = method == 0 ? orc_count_brute(k, points + p * np, max_points, keys)
                        : orc_count_struct(k, points + p * np, keys);
    if (r) return r;
    if (orc_layout(keys, layout, out + p * kk) < 0) return -1;
  }
  return 0;
}

/* ------------------------------------------------------------------ prediction */

/* Error-free transformations: TwoSum (Knuth) and TwoProduct via fma. */
static void two_sum(double a, double b, double *s, double *e) {
  *s = a + b;
  double z = *s - a;
  *e = (a - (*s - z)) + (b - z);
}
static void two_prod(double a, double b, double *p, double *e) {
  *p = a * b;
  *e = fma(a, b, -*p);
}

/* Dot2 of Ogita-Rump-Oishi: result as if accumulated in twice the working precision.
   Each int64 count is split exactly into two doubles (high part a multiple of 2^32). */
static double dot2(const int64_t *F, const double *w, int k, double *absum) {
  double s = 0, c = 0, a = 0;
  for (int i = 0; i < k; i++) {
    int64_t f = F[i];
    int64_t hi = (f >> 32) * ((int64_t)1 << 32);
    double parts[2] = {(double)hi, (double)(f - hi)};
    for (int q = 0; q < 2; q++) {
      double p, ep, es;
      two_prod(parts[q], w[i], &p, &ep);
      two_sum(s, p, &s, &es);
      c += ep + es;
    }
    a += fabs((double)f * w[i]);
  }
  if (absum) *absum = a;
  return s + c;
}

void orc_predict(const int64_t *F, int64_t R, int k, const double *W, int M, double *T) {
  for (int64_t r = 0; r < R; r++)
    for (int m = 0; m < M; m++) T[r * M + m] = dot2(F + r * k, W + (int64_t)m * k, k, NULL);
}

void orc_predict_abs(const int64_t *F, int64_t R, int k, const double *W, int M, double *A) {
  for (int64_t r = 0; r < R; r++)
    for (int m = 0; m < M; m++) dot2(F + r * k, W + (int64_t)m * k, k, &A[r * M + m]);
}

/* ------------------------------------------------------------------ top-k */

static const double *g_sort_t;
static int cmp_idx(const void *a, const void *b) {
  int32_t i = *(const int32_t *)a, j = *(const int32_t *)b;
  double x = g_sort_t[i], y = g_sort_t[j];
  if (x < y) return -1;
  if (x > y) return 1;
  return (i > j) - (i < j);
}

void orc_topk(const double *t, int64_t n_groups, int64_t seg, int topk, int32_t *idx, double *val) {
  int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * (seg > 0 ? seg : 1));
  for (int64_t g = 0; g < n_groups; g++) {
    for (int64_t i = 0; i < seg; i++) ord[i] = (int32_t)i;
    g_sort_t = t + g * seg;
    qsort(ord, (size_t)seg, sizeof(int32_t), cmp_idx);
    for (int q = 0; q < topk; q++) {
      idx[g * topk + q] = q < seg ? ord[q] : -1;
      val[g * topk + q] = q < seg ? g_sort_t[ord[q]] : INFINITY;
    }
  }
  free(ord);
}

/* ------------------------------------------------------------------ fit (Sec. 4.3) */

/* Householder QR with column pivoting of the m x n column-major matrix A, applied to b.
   Solves min ||A x - b||.  Returns rank; x[n]; cond = |R11|/|Rrr|; res = ||Ax-b||/||b||. */
static int qr_lstsq(double *A, int64_t m, int n, double *b, double *x, double *cond, double *res) {
  int perm[64];
  double *v = (double *)malloc(sizeof(double) * (size_t)m);
  double bnorm = 0;
  for (int64_t i = 0; i < m; i++) bnorm += b[i] * b[i];
  bnorm = sqrt(bnorm);
  for (int j = 0; j < n; j++) perm[j] = j;
  int steps = n < m ? n : (int)m;
  for (int j = 0; j < steps; j++) {
    /* pivot: the remaining column of largest norm */
    int best = j; double bn = -1;
    for (int c = j; c < n; c++) {
      double s = 0;
      for (int64_t i = j; i < m; i++) s += A[(int64_t)c * m + i] * A[(int64_t)c * m + i];
      if (s > bn) { bn = s; best = c; }
    }
    if (best != j) {
      for (int64_t i = 0; i < m; i++) { double t = A[(int64_t)j * m + i]; A[(int64_t)j * m + i] = A[(int64_t)best * m + i]; A[(int64_t)best * m + i] = t; }
      int t = perm[j]; perm[j] = perm[best]; perm[best] = t;
    }
    /* Householder vector for A[j:, j] */
    double *col = A + (int64_t)j * m;
    double alpha = 0;
    for (int64_t i = j; i < m; i++) alpha += col[i] * col[i];
    alpha = sqrt(alpha);
    if (alpha == 0) continue;
    if (col[j] > 0) alpha = -alpha;
    for (int64_t i = j; i < m; i++) v[i] = col[i];
    v[j] -= alpha;
    double vv = 0;
    for (int64_t i = j; i < m; i++) vv += v[i] * v[i];
    if (vv == 0) continue;
    for (int c = j; c < n; c++) {
      double *a = A + (int64_t)c * m, d = 0;
      for (int64_t i = j; i < m; i++) d += v[i] * a[i];
      d = 2 * d / vv;
      for (int64_t i = j; i < m; i++) a[i] -= d * v[i];
    }
    double d = 0;
    for (int64_t i = j; i < m; i++) d += v[i] * b[i];
    d = 2 * d / vv;
    for (int64_t i = j; i < m; i++) b[i] -= d * v[i];
  }
  double r00 = fabs(A[0]);
  double tol = (double)(m > n ? m : n) * 2.220446049250313e-16 * r00;
  int rank = 0;
  for (int j = 0; j < steps; j++) if (fabs(A[(int64_t)j * m + j]) > tol) rank = j + 1; else break;
  double z[64] = {0};
  for (int j = rank - 1; j >= 0; j--) {
    double s = b[j];
    for (int c = j + 1; c < rank; c++) s -= A[(int64_t)c * m + j] * z[c];
    z[j] = s / A[(int64_t)j * m + j];
  }
  for (int j = 0; j < n; j++) x[perm[j]] = z[j];
  double rr = 0;
  for (int64_t i = rank; i < m; i++) rr += b[i] * b[i];
  *res = bnorm > 0 ? sqrt(rr) / bnorm : 0;
  *cond = rank ? r00 / fabs(A[(int64_t)(rank - 1) * m + rank - 1]) : INFINITY;
  free(v);
  return rank;
}

int orc_fit(const int64_t *F, int64_t R, int k, const double *t, int objective,
            double *w_out, double *report) {
  if (k > 64 || R <= 0) return -1;
  /* The matrix of the least-squares problem: each property row divided by the
     kernel's measured time (relative objective, Sec. 4.3), or the properties
     themselves (absolute).  Its all-zero columns are dropped; the others are scaled
     by a power of two so that the largest entry of each lies in [1/2, 1). */
  int keep[64], nk = 0;
  double scale[64];
  for (int c = 0; c < k; c++) {
    double mx = 0;
    for (int64_t i = 0; i < R; i++) {
      double a = fabs((double)F[i * k + c]) / (objective == 0 ? t[i] : 1.0);
      if (a > mx) mx = a;
    }
    w_out[c] = 0;
    if (!(mx > 0)) continue;
    int e;
    frexp(mx, &e);
    scale[nk] = ldexp(1.0, -e);
    keep[nk++] = c;
  }
  double *A = (double *)malloc(sizeof(double) * (size_t)R * nk);
  double *b = (double *)malloc(sizeof(double) * (size_t)R);
  for (int64_t i = 0; i < R; i++) {
    double ri = objective == 0 ? 1.0 / t[i] : 1.0;
    for (int q = 0; q < nk; q++) A[(int64_t)q * R + i] = (double)F[i * k + keep[q]] * ri * scale[q];
    b[i] = objective == 0 ? 1.0 : t[i];
  }
  double x[64], cond, res;
  int rank = qr_lstsq(A, R, nk, b, x, &cond, &res);
  for (int q = 0; q < nk; q++) w_out[keep[q]] = x[q] * scale[q];
  report[0] = rank; report[1] = cond; report[2] = res;
  free(A); free(b);
  return rank < nk ? 1 : 0;
}

/* ------------------------------------------------------------------ batched CPU baseline */

int orc_eval_predict_topk(orc_kernel **kernels, int n_variants, const int64_t *points,
                          int64_t n_points, const double *w, int topk, int32_t *idx,
                          double *val, int n_threads) {
  int np = kernels[0]->n_params;
  for (int v = 0; v < n_variants; v++) { int e = classify(kernels[v]); if (e) return e; }
  int err = 0;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
  for (int64_t p = 0; p < n_points; p++) {
    double tv[64]; int32_t ti[64];
    int cnt = 0;
    for (int v = 0; v < n_variants; v++) {
      int64_t keys[ORC_NKEYS], F[32];
      if (orc_count_struct(kernels[v], points + p * np, keys)) { err = -3; continue; }
      orc_layout(keys, 32, F);
      double t = dot2(F, w, 32, NULL);
      /* insertion into the sorted list ordered by (t, v) */
      if (cnt == topk && !(t < tv[topk - 1])) continue;
      int q = cnt < topk ? cnt++ : topk - 1;
      while (q > 0 && t < tv[q - 1]) { tv[q] = tv[q - 1]; ti[q] = ti[q - 1]; q--; }
      tv[q] = t; ti[q] = v;
    }
    for (int q = 0; q < topk; q++) {
      idx[p * topk + q] = q < cnt ? ti[q] : -1;
      val[p * topk + q] = q < cnt ? tv[q] : INFINITY;
    }
  }
  return err;
}
