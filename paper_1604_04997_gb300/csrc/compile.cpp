// Count compiler: affine loop-nest IR -> compiled piecewise quasi-polynomial table.
//
// Alg. 1 (Sec. 3.2): the count of a per-instruction property is
//     n_ops = sum_i |pi_i(D_i)| * n_ops,i
// where |pi_i(D_i)| is the number of integer points of instruction i's loop
// domain.  The paper obtains |pi_i(D_i)| symbolically with isl/barvinok.  Here a
// domain is a box intersected with guards that bound one loop index, one
// "composite axis" (indices combined in mixed radix, such as x = T*g + l of a tiled
// axis), or several indices at once (coupled domains: triangles, bands).  Free
// axes contribute interval lengths max(0, min(U...) - max(L...)) whose bounds are
// quasi-affine in the parameters (atoms floor((a.n+b)/c)); coupled groups are
// counted by eliminating one index at a time with closed-form power sums (see
// "coupled domains" below), whose rational coefficients share one denominator per
// table.  Expanding the min/max choices gives pieces selected by affine conditions
// on the atoms; conditions that hold or fail everywhere on the declared parameter
// box are resolved at compile time.  Each piece is a quasi-polynomial in the atoms,
// kept as exact int64 monomials per feature column.
//
// Access categories follow Sec. 2.1: access size (32/64/128 bit), direction and
// the amortized stride fraction, whose denominator is the lid(0) stride and whose
// numerator is the quantised data utilisation of the array's footprint (Alg. 2).
#include <algorithm>
#include <array>
#include <cstdint>
#include <cstring>
#include <functional>
#include <map>
#include <set>
#include <string>
#include <vector>

#include "pm_table.h"

typedef __int128 i128;

namespace pmc {

struct Error {
  int code;
  std::string msg;
};
// codes mirror pm.h
constexpr int E_PARSE = -2, E_UNSUP = -3, E_RANGE = -4, E_ARG = -1;

[[noreturn]] static void fail(int code, const std::string &m) { throw Error{code, m}; }

static i128 fdiv(i128 x, i128 c) {  // floor(x / c), c > 0
  i128 q = x / c;
  if ((x % c) != 0 && x < 0) q -= 1;
  return q;
}
static i128 gcd128(i128 a, i128 b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b) { i128 t = a % b; a = b; b = t; }
  return a;
}

// ----------------------------------------------------------------------------------- parse tree

struct Node {
  enum K { INT, PAR, DIM, ADD, SUB, MUL, NEG, FLOOR, CEIL } k;
  int64_t v = 0;
  int a = -1, b = -1;
};

struct Access { int arr; bool store; int width; std::vector<int> idx; };
struct Guard { int expr; };  // expr >= 0
struct Flop { int dtype, kind; int64_t count; };
struct Stmt {
  std::string name;
  std::vector<int> dims;
  std::vector<Guard> guards;
  std::vector<Flop> flops;
  std::vector<Access> acc;
};
struct Dim { std::string name; int tag; int lo, hi; };
struct Array { std::string name; bool global, f64; std::vector<int> ext; };
struct Barrier { std::vector<int> dims; };

enum { TAG_G0 = 0, TAG_G1, TAG_G2, TAG_L0, TAG_L1, TAG_L2, TAG_SEQ };

struct Kernel {
  std::vector<std::string> params;
  std::vector<Array> arrays;
  std::vector<Dim> dims;
  std::vector<Stmt> stmts;
  std::vector<Barrier> bars;
  std::vector<Node> nodes;
};

class Parser {
 public:
  explicit Parser(Kernel &k) : K(k) {}
  int parse(const std::string &tok, const Stmt *st) {
    s = tok; pos = 0; cur = st;
    int e = expr();
    if (pos != s.size()) fail(E_PARSE, "trailing characters in '" + tok + "'");
    return e;
  }

 private:
  Kernel &K;
  std::string s;
  size_t pos = 0;
  const Stmt *cur = nullptr;
  int mk(Node::K k, int64_t v, int a, int b) {
    K.nodes.push_back(Node{k, v, a, b});
    return (int)K.nodes.size() - 1;
  }
  char peek() const { return pos < s.size() ? s[pos] : 0; }
  int expr() {
    int a = term();
    while (peek() == '+' || peek() == '-') {
      char op = s[pos++];
      int b = term();
      a = mk(op == '+' ? Node::ADD : Node::SUB, 0, a, b);
    }
    return a;
  }
  int term() {
    bool neg = false;
    if (peek() == '-') { neg = true; pos++; }
    int a = factor();
    while (peek() == '*') { pos++; int b = factor(); a = mk(Node::MUL, 0, a, b); }
    return neg ? mk(Node::NEG, 0, a, -1) : a;
  }
  int64_t integer() {
    if (!isdigit((unsigned char)peek())) fail(E_PARSE, "expected integer in '" + s + "'");
    int64_t v = 0;
    while (isdigit((unsigned char)peek())) {
      v = v * 10 + (s[pos++] - '0');
      if (v > (int64_t(1) << 40)) fail(E_PARSE, "integer too large");
    }
    return v;
  }
  int factor() {
    char c = peek();
    if (isdigit((unsigned char)c)) return mk(Node::INT, integer(), -1, -1);
    if (c == '(') {
      pos++;
      int e = expr();
      if (peek() != ')') fail(E_PARSE, "expected ')' in '" + s + "'");
      pos++;
      return e;
    }
    if (isalpha((unsigned char)c) || c == '_') {
      std::string nm;
      while (isalnum((unsigned char)peek()) || peek() == '_') nm += s[pos++];
      if ((nm == "floor" || nm == "ceil") && peek() == '(') {
        pos++;
        int e = expr();
        if (peek() != '/') fail(E_PARSE, "expected '/' in " + nm);
        pos++;
        int64_t d = integer();
        if (d <= 0 || peek() != ')') fail(E_PARSE, "bad " + nm);
        pos++;
        return mk(nm == "floor" ? Node::FLOOR : Node::CEIL, d, e, -1);
      }
      for (size_t i = 0; i < K.params.size(); i++)
        if (K.params[i] == nm) return mk(Node::PAR, 0, (int)i, -1);
      if (cur)
        for (int d : cur->dims)
          if (K.dims[d].name == nm) return mk(Node::DIM, 0, d, -1);
      fail(E_PARSE, "unknown name '" + nm + "'");
    }
    fail(E_PARSE, "unexpected character in '" + s + "'");
  }
};

static std::vector<std::string> split_ws(const std::string &line) {
  std::vector<std::string> t;
  size_t i = 0;
  while (i < line.size()) {
    while (i < line.size() && isspace((unsigned char)line[i])) i++;
    size_t j = i;
    while (j < line.size() && !isspace((unsigned char)line[j])) j++;
    if (j > i) t.push_back(line.substr(i, j - i));
    i = j;
  }
  return t;
}
static std::vector<std::string> split_c(const std::string &s, char c) {
  std::vector<std::string> out;
  size_t i = 0;
  while (true) {
    size_t j = s.find(c, i);
    out.push_back(s.substr(i, j == std::string::npos ? std::string::npos : j - i));
    if (j == std::string::npos) break;
    i = j + 1;
  }
  return out;
}

// ----------------------------------------------------------------------------------- affine forms

// Affine in parameters and loop indices: c + sum p[i] n_i + sum d[dim] x_dim.
struct Aff {
  i128 c = 0;
  i128 p[4] = {0, 0, 0, 0};
  std::map<int, i128> d;
  bool has_dims() const {
    for (auto &kv : d) if (kv.second) return true;
    return false;
  }
  bool is_const() const { return !has_dims() && !p[0] && !p[1] && !p[2] && !p[3]; }
};
static Aff aff_add(const Aff &a, const Aff &b, i128 sb) {
  Aff r = a;
  r.c += sb * b.c;
  for (int i = 0; i < 4; i++) r.p[i] += sb * b.p[i];
  for (auto &kv : b.d) r.d[kv.first] += sb * kv.second;
  return r;
}
static Aff aff_scale(const Aff &a, i128 s) {
  Aff r = a;
  r.c *= s;
  for (int i = 0; i < 4; i++) r.p[i] *= s;
  for (auto &kv : r.d) kv.second *= s;
  return r;
}
static Aff to_aff(const Kernel &K, int n) {
  const Node &x = K.nodes[n];
  Aff r;
  switch (x.k) {
    case Node::INT: r.c = x.v; return r;
    case Node::PAR: r.p[x.a] = 1; return r;
    case Node::DIM: r.d[x.a] = 1; return r;
    case Node::ADD: return aff_add(to_aff(K, x.a), to_aff(K, x.b), 1);
    case Node::SUB: return aff_add(to_aff(K, x.a), to_aff(K, x.b), -1);
    case Node::NEG: return aff_scale(to_aff(K, x.a), -1);
    case Node::MUL: {
      Aff a = to_aff(K, x.a), b = to_aff(K, x.b);
      if (a.is_const()) return aff_scale(b, a.c);
      if (b.is_const()) return aff_scale(a, b.c);
      fail(E_PARSE, "expression is not affine");
    }
    default: fail(E_PARSE, "floor/ceil not allowed in guards or indices");
  }
}

// Atom floor((a.n + b) / c), canonical: c >= 2, gcd(a, c) = 1, 0 <= b < c.
struct Atom {
  int64_t a[4];
  int64_t b, c;
  bool operator<(const Atom &o) const {
    return std::memcmp(this, &o, sizeof(Atom)) < 0;
  }
};

// Quasi-affine in parameters: c + sum p[i] n_i + sum over atoms at[j] * atom_j.
struct QAff {
  i128 c = 0;
  i128 p[4] = {0, 0, 0, 0};
  std::map<int, i128> at;
  void clean() {
    for (auto it = at.begin(); it != at.end();) it = it->second ? std::next(it) : at.erase(it);
  }
  bool is_const() const {
    if (p[0] || p[1] || p[2] || p[3]) return false;
    for (auto &kv : at) if (kv.second) return false;
    return true;
  }
  bool operator<(const QAff &o) const {
    if (c != o.c) return c < o.c;
    for (int i = 0; i < 4; i++) if (p[i] != o.p[i]) return p[i] < o.p[i];
    return at < o.at;
  }
  bool operator==(const QAff &o) const { return !(*this < o) && !(o < *this); }
};
static QAff q_add(const QAff &a, const QAff &b, i128 sb) {
  QAff r = a;
  r.c += sb * b.c;
  for (int i = 0; i < 4; i++) r.p[i] += sb * b.p[i];
  for (auto &kv : b.at) r.at[kv.first] += sb * kv.second;
  r.clean();
  return r;
}
static QAff q_scale(const QAff &a, i128 s) {
  QAff r = a;
  r.c *= s;
  for (int i = 0; i < 4; i++) r.p[i] *= s;
  for (auto &kv : r.at) kv.second *= s;
  r.clean();
  return r;
}
static QAff q_const(i128 c) { QAff r; r.c = c; return r; }
static QAff q_from_aff(const Aff &a) {
  if (a.has_dims()) fail(E_PARSE, "loop index in a parameter expression");
  QAff r;
  r.c = a.c;
  for (int i = 0; i < 4; i++) r.p[i] = a.p[i];
  return r;
}

// ----------------------------------------------------------------------------------- compiler state

struct Compiler {
  Kernel K;
  int P = 0;
  int layout = 32;
  int64_t box_lo[4] = {0, 0, 0, 0}, box_hi[4] = {0, 0, 0, 0};
  std::vector<Atom> atoms;
  std::map<Atom, int> atom_id;

  // --- atoms
  QAff floor_of(const Aff &num_in, i128 c) {  // floor(num / c), num affine in params
    if (num_in.has_dims()) fail(E_PARSE, "loop index inside floor/ceil");
    Aff num = num_in;
    if (c == 1) return q_from_aff(num);
    i128 g = c;
    for (int i = 0; i < 4; i++) g = gcd128(g, num.p[i]);
    if (g > 1) {
      for (int i = 0; i < 4; i++) num.p[i] /= g;
      num.c = fdiv(num.c, g);
      c /= g;
    }
    bool allzero = !num.p[0] && !num.p[1] && !num.p[2] && !num.p[3];
    if (allzero) return q_const(fdiv(num.c, c));
    if (c == 1) return q_from_aff(num);
    i128 q = fdiv(num.c, c);
    Atom A;
    std::memset(&A, 0, sizeof A);
    for (int i = 0; i < 4; i++) A.a[i] = (int64_t)num.p[i];
    A.b = (int64_t)(num.c - q * c);
    A.c = (int64_t)c;
    auto it = atom_id.find(A);
    int id;
    if (it == atom_id.end()) {
      id = (int)atoms.size();
      atoms.push_back(A);
      atom_id[A] = id;
    } else {
      id = it->second;
    }
    QAff r = q_const(q);
    r.at[id] = 1;
    return r;
  }
  QAff to_qaff(int n) {
    const Node &x = K.nodes[n];
    switch (x.k) {
      case Node::INT: return q_const(x.v);
      case Node::PAR: { QAff r; r.p[x.a] = 1; return r; }
      case Node::DIM: fail(E_PARSE, "loop index in a bound or extent");
      case Node::ADD: return q_add(to_qaff(x.a), to_qaff(x.b), 1);
      case Node::SUB: return q_add(to_qaff(x.a), to_qaff(x.b), -1);
      case Node::NEG: return q_scale(to_qaff(x.a), -1);
      case Node::MUL: {
        QAff a = to_qaff(x.a), b = to_qaff(x.b);
        if (a.is_const()) return q_scale(b, a.c);
        if (b.is_const()) return q_scale(a, b.c);
        fail(E_PARSE, "bound is not quasi-affine");
      }
      case Node::FLOOR: case Node::CEIL: {
        Aff num = to_aff(K, x.a);
        if (x.k == Node::CEIL) num.c += x.v - 1;
        return floor_of(num, x.v);
      }
    }
    fail(E_PARSE, "bad expression");
  }

  // --- value ranges over the box (values: params 0..P-1, atoms P..)
  void atom_num_range(const Atom &A, i128 &lo, i128 &hi) const {
    lo = hi = A.b;
    for (int i = 0; i < P; i++) {
      i128 x = (i128)A.a[i] * box_lo[i], y = (i128)A.a[i] * box_hi[i];
      lo += std::min(x, y);
      hi += std::max(x, y);
    }
  }
  void atom_range(int id, i128 &lo, i128 &hi) const {
    i128 nl, nh;
    atom_num_range(atoms[id], nl, nh);
    lo = fdiv(nl, atoms[id].c);
    hi = fdiv(nh, atoms[id].c);
  }

  // Sign of q over the box: +1 always >= 0, -1 always < 0, 0 unknown.
  // Two sound bounds are intersected: (A) each value in its own range;
  // (B) each atom replaced by (a.n + b - r)/c with r in [0, c-1], which keeps its
  // correlation with the parameters.
  int prove(const QAff &q) const {
    i128 lo = q.c, hi = q.c;
    for (int i = 0; i < P; i++) {
      i128 x = q.p[i] * box_lo[i], y = q.p[i] * box_hi[i];
      lo += std::min(x, y);
      hi += std::max(x, y);
    }
    for (auto &kv : q.at) {
      i128 al, ah;
      atom_range(kv.first, al, ah);
      i128 x = kv.second * al, y = kv.second * ah;
      lo += std::min(x, y);
      hi += std::max(x, y);
    }
    // (B): scale by L = lcm of the divisors
    i128 L = 1;
    bool okB = true;
    for (auto &kv : q.at) {
      i128 c = atoms[kv.first].c;
      L = L / gcd128(L, c) * c;
      if (L > (i128(1) << 40)) { okB = false; break; }
    }
    if (okB && !q.at.empty()) {
      i128 pc[4];
      i128 cst = q.c * L, rlo = 0, rhi = 0;
      for (int i = 0; i < 4; i++) pc[i] = q.p[i] * L;
      for (auto &kv : q.at) {
        const Atom &A = atoms[kv.first];
        i128 f = kv.second * (L / A.c);   // coefficient of (a.n + b - r)
        for (int i = 0; i < 4; i++) pc[i] += f * A.a[i];
        cst += f * A.b;
        i128 x = -f * 0, y = -f * (A.c - 1);
        rlo += std::min(x, y);
        rhi += std::max(x, y);
      }
      i128 blo = cst + rlo, bhi = cst + rhi;
      for (int i = 0; i < P; i++) {
        i128 x = pc[i] * box_lo[i], y = pc[i] * box_hi[i];
        blo += std::min(x, y);
        bhi += std::max(x, y);
      }
      // bounds on L*q: q >= ceil(blo/L), q <= floor(bhi/L)
      lo = std::max(lo, -fdiv(-blo, L));
      hi = std::min(hi, fdiv(bhi, L));
    }
    if (lo >= 0) return 1;
    if (hi < 0) return -1;
    return 0;
  }
  i128 upper_bound(const QAff &q) const {  // sound upper bound over the box (method A)
    i128 hi = q.c;
    for (int i = 0; i < P; i++) hi += std::max(q.p[i] * box_lo[i], q.p[i] * box_hi[i]);
    for (auto &kv : q.at) {
      i128 al, ah;
      atom_range(kv.first, al, ah);
      hi += std::max(kv.second * al, kv.second * ah);
    }
    return hi;
  }

  // --- conditions: q >= 0, interned up to a positive integer factor
  std::vector<QAff> conds;
  std::map<QAff, int> cond_id;
  static QAff normalize(const QAff &q) {
    i128 g = 0;
    for (int i = 0; i < 4; i++) g = gcd128(g, q.p[i]);
    for (auto &kv : q.at) g = gcd128(g, kv.second);
    if (g <= 1) return q;
    QAff r = q;
    for (int i = 0; i < 4; i++) r.p[i] /= g;
    for (auto &kv : r.at) kv.second /= g;
    r.c = fdiv(q.c, g);  // sum g*x + c >= 0  <=>  sum x + floor(c/g) >= 0
    return r;
  }
  // literal for "q >= 0": (cond index, polarity)
  std::pair<int, bool> literal(const QAff &q) {
    QAff n = normalize(q);
    auto it = cond_id.find(n);
    if (it != cond_id.end()) return {it->second, true};
    QAff neg = normalize(q_add(q_scale(q, -1), q_const(1), -1));  // not(q >= 0) <=> -q-1 >= 0
    it = cond_id.find(neg);
    if (it != cond_id.end()) return {it->second, false};
    int id = (int)conds.size();
    conds.push_back(n);
    cond_id[n] = id;
    return {id, true};
  }
};

// A polynomial in values: monomial (sorted value ids, 0xFF padded) -> coefficient.
typedef std::array<uint8_t, 4> Mono;
typedef std::map<Mono, i128> Poly;

static Poly poly_from(const QAff &q, int P) {
  Poly r;
  Mono one = {0xFF, 0xFF, 0xFF, 0xFF};
  if (q.c) r[one] += q.c;
  for (int i = 0; i < 4; i++)
    if (q.p[i]) { Mono m = {(uint8_t)i, 0xFF, 0xFF, 0xFF}; r[m] += q.p[i]; }
  for (auto &kv : q.at)
    if (kv.second) { Mono m = {(uint8_t)(P + kv.first), 0xFF, 0xFF, 0xFF}; r[m] += kv.second; }
  return r;
}
static int mono_deg(const Mono &m) {
  int d = 0;
  for (auto x : m) d += x != 0xFF;
  return d;
}
static Poly poly_mul(const Poly &a, const Poly &b) {
  Poly r;
  for (auto &x : a)
    for (auto &y : b) {
      int da = mono_deg(x.first), db = mono_deg(y.first);
      if (da + db > pmt::MAX_DEGREE) fail(E_UNSUP, "count polynomial degree above 4");
      std::vector<uint8_t> f;
      for (int i = 0; i < da; i++) f.push_back(x.first[i]);
      for (int i = 0; i < db; i++) f.push_back(y.first[i]);
      std::sort(f.begin(), f.end());
      Mono m = {0xFF, 0xFF, 0xFF, 0xFF};
      for (size_t i = 0; i < f.size(); i++) m[i] = f[i];
      r[m] += x.second * y.second;
    }
  for (auto it = r.begin(); it != r.end();) it = it->second ? std::next(it) : r.erase(it);
  return r;
}
static void poly_acc(Poly &a, const Poly &b, i128 s) {
  for (auto &kv : b) {
    i128 &x = a[kv.first];
    x += s * kv.second;
  }
  for (auto it = a.begin(); it != a.end();) it = it->second ? std::next(it) : a.erase(it);
}

// One case of a factor or of a statement count: literals that select it and its value.
struct Case {
  std::vector<std::pair<int, bool>> lits;
  Poly val;    // the value is val / den
  i128 bound;  // upper bound of the value over the box
  i128 den = 1;
};

static void poly_reduce(Poly &p, i128 &den) {  // divide val and den by their common factor
  if (p.empty()) { den = 1; return; }
  i128 g = den;
  for (auto &kv : p) g = gcd128(g, kv.second);
  if (g > 1) {
    for (auto &kv : p) kv.second /= g;
    den /= g;
  }
}

// Interval length max(0, min(U) - max(L)) -> cases.
static std::vector<Case> interval_cases(Compiler &C, std::vector<QAff> U, std::vector<QAff> L) {
  // prune dominated bounds
  auto prune = [&](std::vector<QAff> &v, bool upper) {
    std::vector<QAff> kept;
    for (auto &x : v) {
      bool drop = false;
      for (auto &y : kept) {
        // upper: drop x if x >= y everywhere; lower: drop x if y >= x everywhere
        if (C.prove(upper ? q_add(x, y, -1) : q_add(y, x, -1)) == 1) { drop = true; break; }
      }
      if (drop) continue;
      std::vector<QAff> k2;
      for (auto &y : kept)
        if (C.prove(upper ? q_add(y, x, -1) : q_add(x, y, -1)) != 1) k2.push_back(y);
      k2.push_back(x);
      kept.swap(k2);
    }
    v.swap(kept);
  };
  prune(U, true);
  prune(L, false);
  std::vector<Case> out;
  for (size_t i = 0; i < U.size(); i++) {
    for (size_t j = 0; j < L.size(); j++) {
      std::vector<std::pair<int, bool>> lits;
      bool dead = false;
      auto need = [&](const QAff &q, bool want) {  // require (q >= 0) == want
        int s = C.prove(q);
        if (s == 1) { if (!want) dead = true; return; }
        if (s == -1) { if (want) dead = true; return; }
        auto l = C.literal(q);
        lits.push_back({l.first, l.second == want});
      };
      // U[i] is the first minimiser: U[i'] >= U[i] for i' > i, U[i'] > U[i] for i' < i
      for (size_t i2 = 0; i2 < U.size() && !dead; i2++) {
        if (i2 > i) need(q_add(U[i2], U[i], -1), true);
        if (i2 < i) need(q_add(U[i], U[i2], -1), false);
      }
      // L[j] is the first maximiser
      for (size_t j2 = 0; j2 < L.size() && !dead; j2++) {
        if (j2 > j) need(q_add(L[j], L[j2], -1), true);
        if (j2 < j) need(q_add(L[j2], L[j], -1), false);
      }
      if (dead) continue;
      QAff D = q_add(U[i], L[j], -1);
      int s = C.prove(D);
      if (s == 1) {
        out.push_back({lits, poly_from(D, C.P), std::max<i128>(0, C.upper_bound(D))});
      } else if (s == -1) {
        out.push_back({lits, Poly(), 0});
      } else {
        auto l = C.literal(D);
        auto a = lits, b = lits;
        a.push_back({l.first, l.second});
        b.push_back({l.first, !l.second});
        out.push_back({a, poly_from(D, C.P), std::max<i128>(0, C.upper_bound(D))});
        out.push_back({b, Poly(), 0});
      }
    }
  }
  return out;
}

static std::vector<Case> case_product(const std::vector<Case> &A, const std::vector<Case> &B) {
  std::vector<Case> out;
  for (auto &a : A)
    for (auto &b : B) {
      Case c;
      c.lits = a.lits;
      bool bad = false;
      for (auto &l : b.lits) {
        bool dup = false;
        for (auto &m : c.lits)
          if (m.first == l.first) {
            dup = true;
            if (m.second != l.second) bad = true;
          }
        if (!dup) c.lits.push_back(l);
      }
      if (bad) continue;
      if (a.val.empty() || b.val.empty()) { c.val = Poly(); c.bound = 0; c.den = 1; }
      else {
        c.val = poly_mul(a.val, b.val);
        c.bound = a.bound * b.bound;
        c.den = a.den * b.den;
        poly_reduce(c.val, c.den);
      }
      out.push_back(c);
    }
  return out;
}

// ----------------------------------------------------------------------------------- coupled domains
//
// Guards that tie loop indices together (j < i, i + j < n, a band |i - j| <= w, a
// sequential index bounded by a tiled one) do not factor into per-axis intervals.
// Their count is taken by eliminating one index at a time, innermost first.  For
// each choice of the index's active bounds (the largest lower bound and the smallest
// upper bound, ties to the first listed) the index runs over [L, U); the choice and
// L < U become linear constraints on the indices still to be eliminated, and the
// summand is summed in closed form with Faulhaber's polynomials,
//     sum_{x=L}^{U-1} x^k = S_k(U) - S_k(L).
// When no index is left, the remaining constraints are conditions on the parameters
// (piece conditions) and the chambers whose conditions hold are added up.  S_k has
// rational coefficients (S_1(z) = (z^2 - z)/2), so values carry a denominator.

constexpr int VAR0 = 0xC0;             // polynomial factor ids >= VAR0 are loop variables
typedef std::vector<uint8_t> EMono;    // sorted factor ids
typedef std::map<EMono, i128> EPoly;
struct RPoly {                         // num / den, den > 0
  EPoly num;
  i128 den = 1;
};

static void ep_clean(EPoly &p) {
  for (auto it = p.begin(); it != p.end();) it = it->second ? std::next(it) : p.erase(it);
}
static void ep_acc(EPoly &a, const EPoly &b, i128 s) {
  for (auto &kv : b) a[kv.first] += s * kv.second;
  ep_clean(a);
}
static EPoly ep_const(i128 c) {
  EPoly r;
  if (c) r[EMono{}] = c;
  return r;
}
static EPoly ep_mul(const EPoly &a, const EPoly &b) {
  EPoly r;
  for (auto &x : a)
    for (auto &y : b) {
      EMono m(x.first);
      m.insert(m.end(), y.first.begin(), y.first.end());
      if (m.size() > 8) fail(E_UNSUP, "coupled-domain count of degree above 8");
      std::sort(m.begin(), m.end());
      r[m] += x.second * y.second;
    }
  ep_clean(r);
  return r;
}
static EPoly ep_qaff(const QAff &q, int P) {
  EPoly r = ep_const(q.c);
  for (int i = 0; i < 4; i++)
    if (q.p[i]) r[EMono{(uint8_t)i}] += q.p[i];
  for (auto &kv : q.at) {
    if (!kv.second) continue;
    if (P + kv.first >= VAR0) fail(E_UNSUP, "too many atoms");
    r[EMono{(uint8_t)(P + kv.first)}] += kv.second;
  }
  ep_clean(r);
  return r;
}
static RPoly rp_norm(RPoly r) {
  ep_clean(r.num);
  if (r.num.empty()) { r.den = 1; return r; }
  i128 g = r.den;
  for (auto &kv : r.num) g = gcd128(g, kv.second);
  if (g > 1) {
    for (auto &kv : r.num) kv.second /= g;
    r.den /= g;
  }
  return r;
}
static RPoly rp_add(const RPoly &a, const RPoly &b, i128 s) {
  RPoly r;
  r.den = a.den / gcd128(a.den, b.den) * b.den;
  ep_acc(r.num, a.num, r.den / a.den);
  ep_acc(r.num, b.num, s * (r.den / b.den));
  return rp_norm(r);
}
static RPoly rp_mul(const RPoly &a, const RPoly &b) {
  RPoly r;
  r.num = ep_mul(a.num, b.num);
  r.den = a.den * b.den;
  return rp_norm(r);
}

// S_k(z) = sum_{x=0}^{z-1} x^k = (sum_j FH[k][j] z^j) / FH_DEN[k].  S_k(z+1) - S_k(z) = z^k
// holds as a polynomial identity, so S_k(U) - S_k(L) is the sum over [L, U) for any L <= U.
static const int64_t FH[5][6] = {{0, 1, 0, 0, 0, 0}, {0, -1, 1, 0, 0, 0}, {0, 1, -3, 2, 0, 0},
                                 {0, 0, 1, -2, 1, 0}, {0, -1, 0, 10, -15, 6}};
static const int64_t FH_DEN[5] = {1, 2, 6, 4, 30};
static RPoly faulhaber(int k, const EPoly &z) {
  RPoly r;
  r.den = FH_DEN[k];
  EPoly pw = ep_const(1);
  for (int j = 1; j <= k + 1; j++) {
    pw = ep_mul(pw, z);
    ep_acc(r.num, pw, FH[k][j]);
  }
  return rp_norm(r);
}

struct Lin {  // sum_v a[v] x_v + e; as a constraint, Lin >= 0
  std::vector<i128> a;
  QAff e;
  bool var_free() const {
    for (auto x : a) if (x) return false;
    return true;
  }
  bool operator==(const Lin &o) const { return a == o.a && e == o.e; }
};
static Lin lin_add(const Lin &x, const Lin &y, i128 s) {
  Lin r = x;
  for (size_t v = 0; v < r.a.size(); v++) r.a[v] += s * y.a[v];
  r.e = q_add(x.e, y.e, s);
  return r;
}
static Lin lin_scale(const Lin &x, i128 s) {
  Lin r = x;
  for (auto &v : r.a) v *= s;
  r.e = q_scale(x.e, s);
  return r;
}
static Lin lin_plus(const Lin &x, i128 c) {
  Lin r = x;
  r.e = q_add(x.e, q_const(c), 1);
  return r;
}
static EPoly ep_lin(const Lin &l, int P) {
  EPoly r = ep_qaff(l.e, P);
  for (size_t v = 0; v < l.a.size(); v++)
    if (l.a[v]) r[EMono{(uint8_t)(VAR0 + v)}] += l.a[v];
  ep_clean(r);
  return r;
}

struct Chamber {  // one region of the index space: literals, constraints, summand
  std::vector<std::pair<int, bool>> lits;
  std::vector<Lin> cons;
  RPoly f;
};

struct CoupledCounter {
  Compiler &C;
  size_t m;                 // variables
  std::vector<int> depth;   // nesting depth of each variable (deeper ones go first)

  // Sound proof that x >= 0 on the chamber: x - c is provably non-negative for one of its
  // constraints c (or for c = 0), bounding each variable of x - c by its unit-coefficient
  // single-variable constraints.
  bool nonneg(const Chamber &t, const Lin &x) const {
    std::vector<std::vector<QAff>> lo(m), hi(m);  // x_v >= lo, x_v <= hi
    for (auto &c : t.cons) {
      int v = -1, nz = 0;
      for (size_t w = 0; w < m; w++)
        if (c.a[w]) { v = (int)w; nz++; }
      if (nz != 1) continue;
      if (c.a[v] == 1) lo[v].push_back(q_scale(c.e, -1));
      else if (c.a[v] == -1) hi[v].push_back(c.e);
    }
    std::vector<const Lin *> base = {nullptr};
    for (auto &c : t.cons) base.push_back(&c);
    for (auto *c : base) {
      Lin d = c ? lin_add(x, *c, -1) : x;
      // try every combination of bounds (few in practice)
      std::vector<const std::vector<QAff> *> opts;
      std::vector<size_t> vs;
      bool ok = true;
      for (size_t v = 0; v < m && ok; v++) {
        if (!d.a[v]) continue;
        const auto &o = d.a[v] > 0 ? lo[v] : hi[v];
        if (o.empty()) ok = false;
        opts.push_back(&o);
        vs.push_back(v);
      }
      if (!ok) continue;
      std::vector<size_t> idx(vs.size(), 0);
      for (int guard = 0; guard < 64; guard++) {
        QAff q = d.e;
        for (size_t k = 0; k < vs.size(); k++) q = q_add(q, (*opts[k])[idx[k]], d.a[vs[k]]);
        if (C.prove(q) == 1) return true;
        size_t k = 0;
        while (k < vs.size() && ++idx[k] == opts[k]->size()) idx[k++] = 0;
        if (k == vs.size()) break;
      }
    }
    return false;
  }
  // sum a x + e >= 0 with g = gcd(a) > 1 holds iff sum (a/g) x + floor(e/g) >= 0 (the
  // left side is a multiple of g); floor(e/g) must stay quasi-affine, else x is kept.
  Lin tighten(const Lin &x) const {
    i128 g = 0;
    for (auto v : x.a) g = gcd128(g, v);
    if (g <= 1) return x;
    Lin r = x;
    for (auto &v : r.a) v /= g;
    if (x.e.at.empty()) {
      Aff e;
      e.c = x.e.c;
      for (int i = 0; i < 4; i++) e.p[i] = x.e.p[i];
      r.e = C.floor_of(e, g);
      return r;
    }
    for (int i = 0; i < 4; i++) if (x.e.p[i] % g) return x;
    for (auto &kv : x.e.at) if (kv.second % g) return x;
    r.e = q_scale(x.e, 1);
    for (int i = 0; i < 4; i++) r.e.p[i] /= g;
    for (auto &kv : r.e.at) kv.second /= g;
    r.e.c = fdiv(x.e.c, g);
    return r;
  }
  // Add constraint x0 >= 0; false if the chamber is then empty.
  bool add(Chamber &t, const Lin &x0) {
    const Lin x = tighten(x0);
    if (x.var_free()) {
      int s = C.prove(x.e);
      if (s == 1) return true;
      if (s == -1) return false;
      auto l = C.literal(x.e);
      for (auto &q : t.lits)
        if (q.first == l.first) return q.second == l.second;
      t.lits.push_back({l.first, l.second});
      return true;
    }
    for (auto &c : t.cons)
      if (c == x) return true;
    if (nonneg(t, x)) return true;
    if (nonneg(t, lin_plus(lin_scale(x, -1), -1))) return false;
    t.cons.push_back(x);
    return true;
  }
  // Can x be eliminated from t: every constraint on x has coefficient +-1, or bounds x
  // alone by an atom-free parameter expression.
  bool eligible(const Chamber &t, size_t x) const {
    bool used = false;
    for (auto &c : t.cons) {
      i128 ax = c.a[x];
      if (!ax) continue;
      used = true;
      if (ax == 1 || ax == -1) continue;
      Lin r = c;
      r.a[x] = 0;
      if (!r.var_free() || !r.e.at.empty()) return false;
    }
    return used;
  }
  std::vector<Chamber> eliminate(const Chamber &t, size_t x) {
    std::vector<Lin> lows, ups, rest;  // x >= low, x < up
    for (auto &c : t.cons) {
      i128 ax = c.a[x];
      if (!ax) { rest.push_back(c); continue; }
      Lin r = c;
      r.a[x] = 0;
      if (ax == 1) { lows.push_back(lin_scale(r, -1)); continue; }
      if (ax == -1) { ups.push_back(lin_plus(r, 1)); continue; }
      Aff e;
      e.c = r.e.c;
      for (int i = 0; i < 4; i++) e.p[i] = r.e.p[i];
      Lin b = r;
      if (ax > 0) {  // x >= ceil(-e / ax)
        Aff num = aff_scale(e, -1);
        num.c += ax - 1;
        b.e = C.floor_of(num, ax);
        lows.push_back(b);
      } else {       // x <= floor(e / |ax|)
        b.e = q_add(C.floor_of(e, -ax), q_const(1), 1);
        ups.push_back(b);
      }
    }
    // drop bounds that another bound makes redundant wherever the other variables may
    // be: the proof may use only the constraints without x (those with x hold on the
    // chamber's points, not on its projection, so a bound they dominate there can still
    // cut the range of the other variables)
    Chamber tr;
    tr.lits = t.lits;
    tr.cons = rest;
    auto prune = [&](std::vector<Lin> &v, bool upper) {
      std::vector<Lin> kept;
      for (auto &b : v) {
        bool drop = false;
        for (auto &k : kept)
          if (k == b || nonneg(tr, upper ? lin_add(b, k, -1) : lin_add(k, b, -1))) { drop = true; break; }
        if (drop) continue;
        std::vector<Lin> k2;
        for (auto &k : kept)
          if (!nonneg(tr, upper ? lin_add(k, b, -1) : lin_add(b, k, -1))) k2.push_back(k);
        k2.push_back(b);
        kept.swap(k2);
      }
      v.swap(kept);
    };
    prune(ups, true);
    prune(lows, false);
    if (ups.empty() || lows.empty()) fail(E_UNSUP, "unbounded loop index");
    // the summand by powers of x
    std::vector<RPoly> g;
    for (auto &kv : t.f.num) {
      EMono rem;
      size_t k = 0;
      for (auto id : kv.first) {
        if (id == VAR0 + x) k++;
        else rem.push_back(id);
      }
      if (k > 4) fail(E_UNSUP, "coupled-domain summand of degree above 4 in one index");
      if (g.size() <= k) g.resize(k + 1);
      g[k].den = t.f.den;
      g[k].num[rem] += kv.second;
    }
    std::vector<Chamber> out;
    for (size_t iu = 0; iu < ups.size(); iu++)
      for (size_t il = 0; il < lows.size(); il++) {
        Chamber n;
        n.lits = t.lits;
        n.cons = rest;
        bool ok = true;
        for (size_t i2 = 0; i2 < ups.size() && ok; i2++)
          if (i2 != iu) ok = add(n, lin_plus(lin_add(ups[i2], ups[iu], -1), i2 < iu ? -1 : 0));
        for (size_t l2 = 0; l2 < lows.size() && ok; l2++)
          if (l2 != il) ok = add(n, lin_plus(lin_add(lows[il], lows[l2], -1), l2 < il ? -1 : 0));
        if (ok) ok = add(n, lin_plus(lin_add(ups[iu], lows[il], -1), -1));
        if (!ok) continue;
        const EPoly U = ep_lin(ups[iu], C.P), L = ep_lin(lows[il], C.P);
        RPoly f;
        for (size_t k = 0; k < g.size(); k++) {
          if (g[k].num.empty()) continue;
          f = rp_add(f, rp_mul(rp_norm(g[k]), rp_add(faulhaber((int)k, U), faulhaber((int)k, L), -1)), 1);
        }
        if (f.num.empty()) continue;
        n.f = f;
        out.push_back(n);
      }
    return out;
  }

  std::vector<Case> count(const std::vector<Lin> &cons, i128 bound) {
    Chamber t0;
    for (auto &c : cons) t0.cons.push_back(tighten(c));
    t0.f.num = ep_const(1);
    std::vector<Chamber> work = {t0}, done;
    while (!work.empty()) {
      Chamber t = work.back();
      work.pop_back();
      int x = -1;
      bool left = false;
      for (size_t v = 0; v < m; v++) {
        bool used = false;
        for (auto &c : t.cons) used = used || c.a[v] != 0;
        if (!used) continue;
        left = true;
        if (eligible(t, v) && (x < 0 || depth[v] > depth[x])) x = (int)v;
      }
      if (!left) { done.push_back(t); continue; }
      if (x < 0) fail(E_UNSUP, "coupled guards with non-unit coefficients on shared indices");
      for (auto &n : eliminate(t, (size_t)x)) work.push_back(n);
      if (work.size() + done.size() > 4096) fail(E_UNSUP, "coupled domain splits into too many chambers");
    }
    // chambers hold at once for one parameter point: add up those whose literals hold
    std::vector<int> ids;
    for (auto &t : done)
      for (auto &l : t.lits)
        if (std::find(ids.begin(), ids.end(), l.first) == ids.end()) ids.push_back(l.first);
    if (ids.size() > (size_t)pmt::MAX_CONDS) fail(E_UNSUP, "more than 10 piece conditions");
    std::vector<Case> out;
    for (uint32_t asg = 0; asg < (1u << ids.size()); asg++) {
      Case cs;
      for (size_t q = 0; q < ids.size(); q++) cs.lits.push_back({ids[q], ((asg >> q) & 1) != 0});
      RPoly sum;
      for (auto &t : done) {
        bool ok = true;
        for (auto &l : t.lits) {
          size_t q = std::find(ids.begin(), ids.end(), l.first) - ids.begin();
          if ((((asg >> q) & 1) != 0) != l.second) { ok = false; break; }
        }
        if (ok) sum = rp_add(sum, t.f, 1);
      }
      for (auto &kv : sum.num) {
        if (kv.first.size() > (size_t)pmt::MAX_DEGREE) fail(E_UNSUP, "count polynomial degree above 4");
        Mono mo = {0xFF, 0xFF, 0xFF, 0xFF};
        for (size_t q = 0; q < kv.first.size(); q++) mo[q] = kv.first[q];
        cs.val[mo] = kv.second;
      }
      cs.den = sum.den;
      cs.bound = cs.val.empty() ? 0 : bound;
      out.push_back(cs);
    }
    return out;
  }
};

// ----------------------------------------------------------------------------------- keys and layouts

// Key space of Sec. 2: const, groups, barriers, flops (dtype x kind), local loads/stores
// (dtype), global accesses (direction x size x stride class).
enum { KEY_CONST = 0, KEY_GROUPS, KEY_BARRIERS, KEY_FLOP = 3, KEY_LLOAD = 13, KEY_LSTORE = 15,
       KEY_GLOBAL = 17, N_KEYS = 17 + 90 };
// stride classes: 0 "0", 1 "1", 2..3 "j/2", 4..6 "j/3", 7..10 "j/4", 11..14 "j/>4"
static int gkey(int store, int size, int cls) { return KEY_GLOBAL + (store * 3 + size) * 15 + cls; }

struct LayoutDef {
  int k = 0, hidden = 0;
  std::vector<std::vector<int>> cols;                  // key -> columns
  std::vector<std::array<int, 3>> post;                 // out col, in col A, in col B
};

static LayoutDef make_layout(int layout) {
  LayoutDef D;
  D.cols.assign(N_KEYS, {});
  auto filled = [](int c) { return c == 3 || c == 6 || c == 10; };
  auto partial = [](int c) { return c == 2 || c == 4 || c == 5 || c == 7 || c == 8 || c == 9; };
  if (layout == 32) {
    D.k = 32;
    D.cols[KEY_CONST] = {0}; D.cols[KEY_GROUPS] = {1}; D.cols[KEY_BARRIERS] = {2};
    for (int t = 0; t < 2; t++) for (int q = 0; q < 5; q++) D.cols[KEY_FLOP + 5 * t + q] = {3 + 5 * t + q};
    D.cols[KEY_LLOAD] = {13}; D.cols[KEY_LLOAD + 1] = {14};
    D.cols[KEY_LSTORE] = {15}; D.cols[KEY_LSTORE + 1] = {15};
    for (int cl = 0; cl < 15; cl++) {
      D.cols[gkey(0, 0, cl)] = {cl == 0 ? 16 : cl == 1 ? 17 : filled(cl) ? 18 : partial(cl) ? 19 : 20};
      D.cols[gkey(0, 1, cl)] = {cl == 0 ? 21 : cl == 1 ? 22 : 23};
      D.cols[gkey(1, 0, cl)] = {cl == 1 ? 24 : (cl == 0 || filled(cl)) ? 25 : 26};
      D.cols[gkey(1, 1, cl)] = {cl == 1 ? 27 : 28};
      D.cols[gkey(0, 2, cl)] = {31};
      D.cols[gkey(1, 2, cl)] = {31};
    }
    D.post = {{29, 17, 24}, {30, 22, 27}};
  } else if (layout == 12) {
    D.k = 12; D.hidden = 1;  // column 12: stride-1 global loads of every size
    D.cols[KEY_CONST] = {0}; D.cols[KEY_GROUPS] = {1}; D.cols[KEY_BARRIERS] = {2};
    for (int q = 0; q < 5; q++) { D.cols[KEY_FLOP + q] = {3}; D.cols[KEY_FLOP + 5 + q] = {4}; }
    D.cols[KEY_LLOAD] = {5}; D.cols[KEY_LLOAD + 1] = {5};
    D.cols[KEY_LSTORE] = {6}; D.cols[KEY_LSTORE + 1] = {6};
    for (int sz = 0; sz < 3; sz++)
      for (int cl = 0; cl < 15; cl++) {
        if (cl == 1) D.cols[gkey(0, sz, cl)] = {7, 12};
        else D.cols[gkey(0, sz, cl)] = {cl == 0 ? 7 : 8};
        D.cols[gkey(1, sz, cl)] = {cl == 1 ? 9 : 10};
      }
    D.post = {{11, 12, 9}};
  } else {
    fail(E_ARG, "layout must be 12 or 32");
  }
  return D;
}

// ----------------------------------------------------------------------------------- numeric helpers

static i128 num_eval(const Kernel &K, int n, const int64_t *par, const int64_t *dimv) {
  const Node &x = K.nodes[n];
  switch (x.k) {
    case Node::INT: return x.v;
    case Node::PAR: return par[x.a];
    case Node::DIM: return dimv[x.a];
    case Node::ADD: return num_eval(K, x.a, par, dimv) + num_eval(K, x.b, par, dimv);
    case Node::SUB: return num_eval(K, x.a, par, dimv) - num_eval(K, x.b, par, dimv);
    case Node::MUL: return num_eval(K, x.a, par, dimv) * num_eval(K, x.b, par, dimv);
    case Node::NEG: return -num_eval(K, x.a, par, dimv);
    case Node::FLOOR: return fdiv(num_eval(K, x.a, par, dimv), x.v);
    case Node::CEIL: return -fdiv(-num_eval(K, x.a, par, dimv), x.v);
  }
  return 0;
}

// ----------------------------------------------------------------------------------- classification

struct LinAcc {  // an access's linear element offset as an affine function at a fixed instance
  i128 c;
  std::vector<i128> d;  // per kernel dim
};

static LinAcc lin_at(const Kernel &K, const Access &a, const int64_t *par) {
  const Array &ar = K.arrays[a.arr];
  LinAcc r;
  r.c = 0;
  r.d.assign(K.dims.size(), 0);
  for (size_t x = 0; x < a.idx.size(); x++) {
    i128 ext = num_eval(K, ar.ext[x], par, nullptr);
    Aff ia = to_aff(K, a.idx[x]);
    r.c = r.c * ext;
    for (auto &v : r.d) v *= ext;
    i128 c = ia.c;
    for (int i = 0; i < 4; i++) c += ia.p[i] * par[i];
    r.c += c;
    for (auto &kv : ia.d) r.d[kv.first] += kv.second;
  }
  return r;
}

// Footprint of one array at the classification instance: visit every point of every
// statement domain (guards applied) and mark the cells of each access (Alg. 2).
static void footprint(const Kernel &K, int arr, const int64_t *par, std::vector<uint8_t> &bm) {
  for (const Stmt &st : K.stmts) {
    std::vector<const Access *> accs;
    for (auto &a : st.acc) if (a.arr == arr) accs.push_back(&a);
    if (accs.empty()) continue;
    size_t nd = st.dims.size();
    std::vector<i128> lo(nd), hi(nd);
    bool empty = false;
    for (size_t j = 0; j < nd; j++) {
      lo[j] = num_eval(K, K.dims[st.dims[j]].lo, par, nullptr);
      hi[j] = num_eval(K, K.dims[st.dims[j]].hi, par, nullptr);
      if (hi[j] <= lo[j]) empty = true;
    }
    if (empty) continue;
    // the walk below visits every point of the box: keep it bounded (the templates and
    // the measurement kernels stay near 2^21 points at this instance)
    i128 pts = 1;
    for (size_t j = 0; j < nd; j++) {
      pts *= hi[j] - lo[j];
      if (pts > (i128(1) << 25)) fail(E_UNSUP, "statement domain too large at the classification instance");
    }
    // guards and offsets as affine functions of the statement's dims at this instance
    std::vector<Aff> g;
    for (auto &gu : st.guards) g.push_back(to_aff(K, gu.expr));
    std::vector<LinAcc> la;
    for (auto *a : accs) la.push_back(lin_at(K, *a, par));
    std::vector<int64_t> x(nd);
    for (size_t j = 0; j < nd; j++) x[j] = (int64_t)lo[j];
    while (true) {
      bool ok = true;
      for (auto &ga : g) {
        i128 v = ga.c;
        for (int i = 0; i < 4; i++) v += ga.p[i] * par[i];
        for (size_t j = 0; j < nd; j++) {
          auto it = ga.d.find(st.dims[j]);
          if (it != ga.d.end()) v += it->second * x[j];
        }
        if (v < 0) { ok = false; break; }
      }
      if (ok) {
        for (size_t q = 0; q < accs.size(); q++) {
          i128 off = la[q].c;
          for (size_t j = 0; j < nd; j++) off += la[q].d[st.dims[j]] * x[j];
          if (off < 0 || off + accs[q]->width > (i128)bm.size())
            fail(E_UNSUP, "access outside its array at the classification instance");
          for (int w = 0; w < accs[q]->width; w++) bm[(size_t)off + w] = 1;
        }
      }
      size_t j = nd;
      while (j > 0) {
        j--;
        if (++x[j] < hi[j]) break;
        x[j] = (int64_t)lo[j];
        if (j == 0) { j = (size_t)-1; break; }
      }
      if (j == (size_t)-1 || nd == 0) break;
    }
  }
}

// class of every access (-1 = local), evaluated with every parameter = 128;
// a lid(0) stride that changes when the parameters double is parametric (">4").
static std::vector<std::vector<int>> classify(const Kernel &K) {
  const int64_t I1[4] = {128, 128, 128, 128}, I2[4] = {256, 256, 256, 256};
  std::vector<std::vector<int>> cls(K.stmts.size());
  std::map<int, std::pair<std::vector<uint8_t>, i128>> fp;  // array -> (bitmap, #cells)
  for (size_t s = 0; s < K.stmts.size(); s++) {
    const Stmt &st = K.stmts[s];
    int l0 = -1;
    for (int d : st.dims) if (K.dims[d].tag == TAG_L0) l0 = d;
    for (auto &a : st.acc) {
      const Array &ar = K.arrays[a.arr];
      if (!ar.global) { cls[s].push_back(-1); continue; }
      if (l0 < 0) { cls[s].push_back(0); continue; }
      i128 c1 = lin_at(K, a, I1).d[l0], c2 = lin_at(K, a, I2).d[l0];
      bool param = c1 != c2;
      i128 se = c1 < 0 ? -c1 : c1;
      if (!param && se % a.width) fail(E_UNSUP, "lane stride not a multiple of the vector width");
      i128 sv = param ? 1000 : se / a.width;
      if (!param && sv <= 1) { cls[s].push_back((int)sv); continue; }
      auto it = fp.find(a.arr);
      if (it == fp.end()) {
        i128 sz = 1;
        for (int e : ar.ext) sz *= num_eval(K, e, I1, nullptr);
        if (sz <= 0 || sz > (i128(1) << 26)) fail(E_UNSUP, "array too large at the classification instance");
        std::vector<uint8_t> bm((size_t)sz, 0);
        footprint(K, a.arr, I1, bm);
        i128 cells = 0;
        for (auto b : bm) cells += b;
        it = fp.emplace(a.arr, std::make_pair(std::move(bm), cells)).first;
      }
      const auto &bm = it->second.first;
      i128 cells = it->second.second, filled = 0;
      // gaps of the stride filled in: a cell counts if an accessed cell lies within se-1 before it
      i128 last = -(i128(1) << 80), size = (i128)bm.size();
      for (i128 x = 0; x < size + se; x++) {
        if (x < size && bm[(size_t)x]) last = x;
        if (x - last < se) filled++;
      }
      // no accessed cell (an empty domain), or a parametric stride that vanishes at
      // the classification instance: the Sec. 2.1 fraction is undefined there
      if (cells == 0 || filled == 0)
        fail(E_UNSUP, "stride class undefined: the access touches no cell, or its lane stride is 0, "
                      "with every parameter = 128");
      int c;
      if (!param && sv <= 4) {
        i128 j = (sv * cells + filled - 1) / filled;
        j = std::max<i128>(1, std::min<i128>(j, sv));
        c = (sv == 2 ? 1 : sv == 3 ? 3 : 6) + (int)j;
      } else {
        i128 j = (4 * cells + filled - 1) / filled;
        j = std::max<i128>(1, std::min<i128>(j, 4));
        c = 10 + (int)j;
      }
      cls[s].push_back(c);
    }
  }
  return cls;
}

// ----------------------------------------------------------------------------------- parse

static void parse_kernel(Compiler &C, const std::string &text) {
  Kernel &K = C.K;
  Parser ps(K);
  Stmt *cur = nullptr;
  bool have_kernel = false;
  size_t i = 0;
  int lineno = 0;
  while (i <= text.size()) {
    size_t j = text.find('\n', i);
    if (j == std::string::npos) j = text.size();
    std::string line = text.substr(i, j - i);
    i = j + 1;
    lineno++;
    size_t h = line.find('#');
    if (h != std::string::npos) line = line.substr(0, h);
    auto t = split_ws(line);
    if (t.empty()) { if (j >= text.size()) break; continue; }
    const std::string &kw = t[0];
    auto dimlist = [&](const std::string &s) {
      std::vector<int> out;
      if (s == "-") return out;
      for (auto &nm : split_c(s, ',')) {
        int f = -1;
        for (size_t d = 0; d < K.dims.size(); d++) if (K.dims[d].name == nm) f = (int)d;
        if (f < 0) fail(E_PARSE, "unknown dim '" + nm + "'");
        if (std::find(out.begin(), out.end(), f) != out.end()) fail(E_PARSE, "dim listed twice");
        out.push_back(f);
      }
      return out;
    };
    if (cur) {
      if (kw == "end") { cur = nullptr; }
      else if (kw == "guard") {
        if (t.size() != 4) fail(E_PARSE, "guard takes LHS OP RHS");
        int l = ps.parse(t[1], cur), r = ps.parse(t[3], cur);
        auto sub = [&](int a, int b) { K.nodes.push_back(Node{Node::SUB, 0, a, b}); return (int)K.nodes.size() - 1; };
        auto one = [&]() { K.nodes.push_back(Node{Node::INT, 1, -1, -1}); return (int)K.nodes.size() - 1; };
        int e;
        if (t[2] == "<") e = sub(sub(r, l), one());
        else if (t[2] == "<=") e = sub(r, l);
        else if (t[2] == ">") e = sub(sub(l, r), one());
        else if (t[2] == ">=") e = sub(l, r);
        else fail(E_PARSE, "guard operator must be < <= > >=");
        to_aff(K, e);  // affine check
        cur->guards.push_back(Guard{e});
      } else if (kw == "flop") {
        if (t.size() != 4) fail(E_PARSE, "flop takes DTYPE KIND COUNT");
        Flop f;
        f.dtype = t[1] == "f32" ? 0 : t[1] == "f64" ? 1 : -1;
        const char *kinds[5] = {"add", "mul", "div", "pow", "spec"};
        f.kind = -1;
        for (int q = 0; q < 5; q++) if (t[2] == kinds[q]) f.kind = q;
        if (f.dtype < 0 || f.kind < 0) fail(E_PARSE, "bad flop line");
        char *endp;
        long long c = strtoll(t[3].c_str(), &endp, 10);
        if (*endp || c < 0) fail(E_PARSE, "bad flop count");
        f.count = c;
        cur->flops.push_back(f);
      } else if (kw == "load" || kw == "store") {
        if (t.size() < 2 || t.size() > 3) fail(E_PARSE, "load/store ARRAY[IDX] [x2|x4]");
        Access a;
        a.store = kw == "store";
        a.width = 1;
        if (t.size() == 3) {
          if (t[2] == "x2") a.width = 2;
          else if (t[2] == "x4") a.width = 4;
          else fail(E_PARSE, "vector width must be x2 or x4");
        }
        size_t br = t[1].find('[');
        if (br == std::string::npos || t[1].back() != ']') fail(E_PARSE, "expected ARRAY[...]");
        std::string nm = t[1].substr(0, br);
        a.arr = -1;
        for (size_t q = 0; q < K.arrays.size(); q++) if (K.arrays[q].name == nm) a.arr = (int)q;
        if (a.arr < 0) fail(E_PARSE, "unknown array '" + nm + "'");
        for (auto &ix : split_c(t[1].substr(br + 1, t[1].size() - br - 2), ',')) {
          int e = ps.parse(ix, cur);
          to_aff(K, e);
          a.idx.push_back(e);
        }
        const Array &ar = K.arrays[a.arr];
        if (a.idx.size() != ar.ext.size()) fail(E_PARSE, "index count does not match array rank");
        if ((ar.f64 ? 64 : 32) * a.width > 128) fail(E_PARSE, "access wider than 128 bits");
        cur->acc.push_back(a);
      } else {
        fail(E_PARSE, "unknown directive in stmt: " + kw);
      }
    } else if (kw == "kernel") {
      if (t.size() != 2 || have_kernel) fail(E_PARSE, "kernel NAME (once)");
      have_kernel = true;
    } else if (kw == "param") {
      if (t.size() < 2 || t.size() > 5 || !K.params.empty()) fail(E_PARSE, "param takes 1..4 names (once)");
      for (size_t q = 1; q < t.size(); q++) K.params.push_back(t[q]);
    } else if (kw == "array") {
      if (t.size() != 5) fail(E_PARSE, "array NAME SPACE DTYPE EXTENTS");
      Array a;
      a.name = t[1];
      if (t[2] != "global" && t[2] != "local") fail(E_PARSE, "array space");
      if (t[3] != "f32" && t[3] != "f64") fail(E_PARSE, "array dtype");
      a.global = t[2] == "global";
      a.f64 = t[3] == "f64";
      for (auto &e : split_c(t[4], ',')) a.ext.push_back(ps.parse(e, nullptr));
      if (a.ext.size() > 4) fail(E_PARSE, "too many extents");
      K.arrays.push_back(a);
    } else if (kw == "dim") {
      if (t.size() != 5) fail(E_PARSE, "dim NAME TAG LO HI");
      Dim d;
      d.name = t[1];
      const char *tags[7] = {"g0", "g1", "g2", "l0", "l1", "l2", "seq"};
      d.tag = -1;
      for (int q = 0; q < 7; q++) if (t[2] == tags[q]) d.tag = q;
      if (d.tag < 0) fail(E_PARSE, "unknown dim tag");
      for (auto &o : K.dims) if (o.name == d.name) fail(E_PARSE, "duplicate dim");
      d.lo = ps.parse(t[3], nullptr);
      d.hi = ps.parse(t[4], nullptr);
      if (d.tag >= TAG_L0 && d.tag <= TAG_L2) {
        QAff lo = C.to_qaff(d.lo), hi = C.to_qaff(d.hi);
        if (!lo.is_const() || !hi.is_const() || lo.c != 0 || hi.c <= 0)
          fail(E_PARSE, "local dims need a constant range [0, W)");
      }
      K.dims.push_back(d);
    } else if (kw == "stmt") {
      if (t.size() != 3) fail(E_PARSE, "stmt NAME DIMS");
      K.stmts.push_back(Stmt());
      cur = &K.stmts.back();
      cur->name = t[1];
      cur->dims = dimlist(t[2]);
    } else if (kw == "barrier") {
      if (t.size() != 3) fail(E_PARSE, "barrier NAME DIMS");
      Barrier b;
      b.dims = dimlist(t[2]);
      for (int d : b.dims)
        if (K.dims[d].tag >= TAG_L0 && K.dims[d].tag <= TAG_L2)
          fail(E_PARSE, "barrier may not depend on work-item indices");
      K.bars.push_back(b);
    } else {
      fail(E_PARSE, "unknown directive: " + kw);
    }
    if (j >= text.size()) break;
  }
  if (cur) fail(E_PARSE, "missing end");
  if (!have_kernel || K.params.empty()) fail(E_PARSE, "missing kernel/param line");
  for (int d = 0; d < (int)K.dims.size(); d++) {
    if (K.dims[d].tag > TAG_G2) continue;
    for (auto &s : K.stmts)
      if (std::find(s.dims.begin(), s.dims.end(), d) == s.dims.end())
        fail(E_PARSE, "statement '" + s.name + "' does not list every group dim");
    for (auto &b : K.bars)
      if (std::find(b.dims.begin(), b.dims.end(), d) == b.dims.end())
        fail(E_PARSE, "barrier does not list every group dim");
  }
}

// ----------------------------------------------------------------------------------- counting

// Symbolic |pi(D)| of one statement as a list of cases.
static std::vector<Case> stmt_count(Compiler &C, const Stmt &st) {
  const Kernel &K = C.K;
  size_t nd = st.dims.size();
  std::vector<QAff> lo(nd), hi(nd);
  for (size_t j = 0; j < nd; j++) {
    lo[j] = C.to_qaff(K.dims[st.dims[j]].lo);
    hi[j] = C.to_qaff(K.dims[st.dims[j]].hi);
  }
  // Composite axes that a coupling guard cuts through (it weighs their indices unlike
  // the axis' own guards, as jt <= g against 64 g + l < n) are split into their indices.
  std::set<uint32_t> split;
  for (;;) {
  std::vector<int> owner(nd, -1);  // -1 free, -2 single, >=0 composite
  std::vector<std::vector<QAff>> sU(nd), sL(nd);
  std::vector<Case> acc = {Case{{}, Poly{{Mono{0xFF, 0xFF, 0xFF, 0xFF}, 1}}, 1}};
  struct Comp { uint32_t mask; std::vector<int> ord; std::vector<i128> ref; QAff N, J0; std::vector<QAff> U, L; };
  std::vector<Comp> comps;
  struct Coupling { std::vector<i128> coef; QAff e; };
  std::vector<Coupling> coupled;   // guards left to the coupled-domain counter
  std::vector<Coupling> multi;     // every guard on two or more indices
  // A composite axis: indices in mixed radix, sorted by (|coef|, range); all but the top
  // one need a constant range [0, R).  The axis index j = J - J0 runs over [0, N), where
  // J = sum_d (|coef_d| / |coef_min|) x_d.  Returns false if the indices do not qualify.
  auto open_comp = [&](uint32_t mask, const std::vector<int> &slots, const std::vector<i128> &coef) {
    if (split.count(mask)) return false;
    Comp cp;
    cp.mask = mask;
    cp.ref = coef;
    std::vector<std::pair<std::pair<i128, i128>, int>> key;
    for (int j : slots) {
      QAff r = q_add(hi[j], lo[j], -1);
      i128 rv = r.is_const() ? r.c : (i128(1) << 100);
      key.push_back({{coef[j] < 0 ? -coef[j] : coef[j], rv}, j});
    }
    std::sort(key.begin(), key.end());
    for (auto &kv : key) cp.ord.push_back(kv.second);
    i128 sg = coef[cp.ord[0]] > 0 ? 1 : -1;
    for (int j : cp.ord) if ((coef[j] > 0 ? 1 : -1) != sg) return false;
    i128 a1 = coef[cp.ord[0]] * sg;
    i128 Nc = 1;
    for (size_t q = 0; q + 1 < cp.ord.size(); q++) {
      int j = cp.ord[q];
      if (!lo[j].is_const() || !hi[j].is_const() || lo[j].c != 0) return false;
      i128 R = hi[j].c;
      if (coef[cp.ord[q + 1]] * sg != coef[j] * sg * R) return false;
      Nc *= R;
    }
    int top = cp.ord.back();
    cp.N = q_scale(q_add(hi[top], lo[top], -1), Nc);
    cp.J0 = q_scale(lo[top], coef[top] * sg / a1);
    cp.U.push_back(cp.N);
    cp.L.push_back(q_const(0));
    comps.push_back(cp);
    return true;
  };
  bool split_redo = false;
  for (auto &g : st.guards) {
    Aff a = to_aff(K, g.expr);
    std::vector<int> slots;
    std::vector<i128> coef(nd, 0);
    for (size_t j = 0; j < nd; j++) {
      auto it = a.d.find(st.dims[j]);
      if (it != a.d.end() && it->second) { slots.push_back((int)j); coef[j] = it->second; }
    }
    Aff e = a;
    e.d.clear();
    QAff eq = q_from_aff(e);
    if (slots.empty()) {  // guard on the parameters only: indicator [e >= 0]
      int s = C.prove(eq);
      if (s == -1) return {};
      if (s == 0) {
        auto l = C.literal(eq);
        std::vector<Case> ind = {Case{{{l.first, l.second}}, Poly{{Mono{0xFF, 0xFF, 0xFF, 0xFF}, 1}}, 1},
                                 Case{{{l.first, !l.second}}, Poly(), 0}};
        acc = case_product(acc, ind);
      }
      continue;
    }
    if (slots.size() == 1) {
      int j = slots[0];
      if (owner[j] >= 0) {  // bounded alone and inside a composite axis: split the axis
        split.insert(comps[owner[j]].mask);
        split_redo = true;
        break;
      }
      owner[j] = -2;
      i128 c = coef[j];
      if (c > 0) {  // x >= ceil(-e/c)
        Aff num = aff_scale(e, -1);
        num.c += c - 1;
        sL[j].push_back(C.floor_of(num, c));
      } else {      // x <= floor(e/|c|)
        sU[j].push_back(q_add(C.floor_of(e, -c), q_const(1), 1));
      }
      continue;
    }
    multi.push_back({coef, eq});
    uint32_t mask = 0;
    for (int j : slots) mask |= 1u << j;
    int gi = -1;
    for (size_t q = 0; q < comps.size(); q++) if (comps[q].mask == mask) gi = (int)q;
    bool couple = false;
    if (gi < 0) {
      for (int j : slots) couple = couple || owner[j] != -1;
      if (!couple && open_comp(mask, slots, coef)) {
        gi = (int)comps.size() - 1;
        for (int j : slots) owner[j] = gi;
      } else {
        couple = true;
      }
    } else {
      int j1 = comps[gi].ord[0];
      for (int j : slots) couple = couple || coef[j] * comps[gi].ref[j1] != comps[gi].ref[j] * coef[j1];
    }
    if (couple) {
      coupled.push_back({coef, eq});
      continue;
    }
    Comp &cp = comps[gi];
    int j1 = cp.ord[0];
    i128 c1 = coef[j1];
    if (c1 > 0) {  // j >= ceil(-e/c1) - J0
      Aff num = aff_scale(e, -1);
      num.c += c1 - 1;
      cp.L.push_back(q_add(C.floor_of(num, c1), cp.J0, -1));
    } else {       // j <= floor(e/|c1|) - J0
      cp.U.push_back(q_add(q_add(C.floor_of(e, -c1), cp.J0, -1), q_const(1), 1));
    }
  }
  if (split_redo) continue;
  // variables: the indices outside composite axes, then the composite axes
  std::vector<int> var_of(nd, -1), var_dim, var_comp, var_depth;
  for (size_t j = 0; j < nd; j++)
    if (owner[j] < 0) {
      var_of[j] = (int)var_dim.size();
      var_dim.push_back((int)j);
      var_comp.push_back(-1);
      var_depth.push_back((int)j);
    }
  for (size_t q = 0; q < comps.size(); q++) {
    int v = (int)var_dim.size(), dmax = 0;
    for (int j : comps[q].ord) { var_of[j] = v; dmax = std::max(dmax, j); }
    var_dim.push_back(-1);
    var_comp.push_back((int)q);
    var_depth.push_back(dmax);
  }
  const size_t nv = var_dim.size();
  // A guard G that cuts a composite axis may be implied by another guard H and the index
  // ranges (as jt <= g by 16 jt + jj <= 16 g + l): c G - H + c - 1 >= 0 over the ranges for
  // an integer c >= 1 gives G >= (H - c + 1) / c > -1.  Such a G is dropped.
  auto implied = [&](const Coupling &G) {
    for (auto &H : multi) {
      if (H.coef == G.coef && H.e == G.e) continue;
      std::set<i128> cs = {1};
      for (size_t j = 0; j < nd; j++)
        if (G.coef[j] && H.coef[j] && H.coef[j] % G.coef[j] == 0 && H.coef[j] / G.coef[j] > 0)
          cs.insert(H.coef[j] / G.coef[j]);
      for (i128 c : cs) {
        QAff q = q_add(q_scale(G.e, c), H.e, -1);
        q.c += c - 1;
        for (size_t j = 0; j < nd; j++) {
          i128 a = c * G.coef[j] - H.coef[j];
          if (a > 0) q = q_add(q, lo[j], a);
          if (a < 0) q = q_add(q, q_add(hi[j], q_const(1), -1), a);
        }
        if (C.prove(q) == 1) return true;
      }
    }
    return false;
  };
  // coupling guards over the variables; a composite axis enters as c1 (j + J0)
  std::vector<Lin> glin;
  bool redo = false;
  for (auto &cg : coupled) {
    Lin L;
    L.a.assign(nv, 0);
    L.e = cg.e;
    bool drop = false;
    for (size_t q = 0; q < comps.size() && !drop; q++) {
      const Comp &cp = comps[q];
      int j1 = cp.ord[0];
      bool any = false;
      for (int j : cp.ord) any = any || cg.coef[j] != 0;
      if (!any) continue;
      bool cut = false;
      for (int j : cp.ord) cut = cut || cg.coef[j] * cp.ref[j1] != cp.ref[j] * cg.coef[j1];
      if (cut && implied(cg)) { drop = true; break; }
      if (cut) {
        split.insert(cp.mask);
        redo = true;
        continue;
      }
      L.a[var_of[j1]] = cg.coef[j1];
      L.e = q_add(L.e, cp.J0, cg.coef[j1]);
    }
    if (drop) continue;
    for (size_t j = 0; j < nd; j++)
      if (owner[j] < 0) L.a[var_of[j]] += cg.coef[j];
    glin.push_back(L);
  }
  if (redo) continue;
  // connected groups of coupled variables
  std::vector<int> root(nv);
  for (size_t v = 0; v < nv; v++) root[v] = (int)v;
  std::function<int(int)> find = [&](int v) { return root[v] == v ? v : root[v] = find(root[v]); };
  std::vector<char> in_coupled(nv, 0);
  for (auto &L : glin) {
    int first = -1;
    for (size_t v = 0; v < nv; v++) {
      if (!L.a[v]) continue;
      in_coupled[v] = 1;
      if (first < 0) first = (int)v;
      else root[find((int)v)] = find(first);
    }
  }
  for (size_t j = 0; j < nd; j++) {
    if (owner[j] >= 0 || in_coupled[var_of[j]]) continue;
    std::vector<QAff> U = {hi[j]}, L = {lo[j]};
    for (auto &u : sU[j]) U.push_back(u);
    for (auto &l : sL[j]) L.push_back(l);
    auto f = interval_cases(C, U, L);
    acc = case_product(acc, f);
  }
  for (size_t q = 0; q < comps.size(); q++)
    if (!in_coupled[var_of[comps[q].ord[0]]]) acc = case_product(acc, interval_cases(C, comps[q].U, comps[q].L));
  std::vector<char> seen(nv, 0);
  for (size_t v0 = 0; v0 < nv; v0++) {
    if (!in_coupled[v0] || seen[find((int)v0)]) continue;
    seen[find((int)v0)] = 1;
    std::vector<int> gvars;
    for (size_t v = 0; v < nv; v++)
      if (in_coupled[v] && find((int)v) == find((int)v0)) gvars.push_back((int)v);
    const size_t m = gvars.size();
    std::vector<int> local(nv, -1);
    for (size_t k = 0; k < m; k++) local[gvars[k]] = (int)k;
    std::vector<Lin> cons;
    i128 bound = 1;
    auto bound_con = [&](size_t k, const QAff &b, bool lower) {  // x_k >= b, or x_k < b
      Lin L;
      L.a.assign(m, 0);
      L.a[k] = lower ? 1 : -1;
      L.e = lower ? q_scale(b, -1) : q_add(b, q_const(1), -1);
      cons.push_back(L);
    };
    for (size_t k = 0; k < m; k++) {
      const int v = gvars[k];
      QAff ext;
      if (var_comp[v] < 0) {
        const int j = var_dim[v];
        bound_con(k, lo[j], true);
        bound_con(k, hi[j], false);
        for (auto &l : sL[j]) bound_con(k, l, true);
        for (auto &u : sU[j]) bound_con(k, u, false);
        ext = q_add(hi[j], lo[j], -1);
      } else {
        const Comp &cp = comps[var_comp[v]];
        for (auto &l : cp.L) bound_con(k, l, true);
        for (auto &u : cp.U) bound_con(k, u, false);
        ext = cp.N;
      }
      bound *= std::max<i128>(0, C.upper_bound(ext));
      if (bound > (i128(1) << 100)) bound = i128(1) << 100;
    }
    for (auto &L : glin) {
      bool mine = false;
      for (size_t v = 0; v < nv; v++) mine = mine || (L.a[v] && local[v] >= 0);
      if (!mine) continue;
      Lin M;
      M.a.assign(m, 0);
      M.e = L.e;
      for (size_t v = 0; v < nv; v++)
        if (L.a[v]) M.a[local[v]] = L.a[v];
      cons.push_back(M);
    }
    CoupledCounter cc{C, m, {}};
    for (size_t k = 0; k < m; k++) cc.depth.push_back(var_depth[gvars[k]]);
    acc = case_product(acc, cc.count(cons, bound));
  }
  return acc;
  }
}

struct Term {  // one contribution: a count (as cases) times per-column multiplicities
  std::vector<Case> cases;
  std::map<int, i128> colmul;  // column -> multiplicity
};

struct Result {
  std::vector<uint32_t> words;
  int n_atoms, n_conds, n_pieces, n_monos, degree;
};

static uint32_t magic_for(int64_t c, int &sh2) {
  // Granlund & Montgomery (1994), Fig. 4.1: unsigned division by an invariant
  // c >= 2: l = ceil(log2 c), m = floor(2^32 (2^l - c) / c) + 1,
  // q = (t + ((n - t) >> 1)) >> (l - 1) with t = umulhi(m, n).
  int l = 0;
  while ((int64_t(1) << l) < c) l++;
  unsigned __int128 m = ((unsigned __int128)1 << 32) * (((unsigned __int128)1 << l) - (unsigned __int128)c) /
                        (unsigned __int128)c + 1;
  sh2 = l - 1;
  return (uint32_t)m;
}

static Result compile(const std::string &text, int layout, const int64_t *plo, const int64_t *phi) {
  Compiler C;
  parse_kernel(C, text);
  C.layout = layout;
  C.P = (int)C.K.params.size();
  for (int i = 0; i < C.P; i++) {
    if (plo[i] > phi[i]) fail(E_ARG, "empty parameter box");
    if (plo[i] < -(int64_t(1) << 30) || phi[i] > (int64_t(1) << 30)) fail(E_RANGE, "parameter box beyond +-2^30");
    C.box_lo[i] = plo[i];
    C.box_hi[i] = phi[i];
  }
  LayoutDef LD = make_layout(layout);
  const Kernel &K = C.K;
  auto cls = classify(K);

  std::vector<Term> terms;
  // const
  { Term t; t.cases = {Case{{}, Poly{{Mono{0xFF, 0xFF, 0xFF, 0xFF}, 1}}, 1}}; for (int c : LD.cols[KEY_CONST]) t.colmul[c] += 1; terms.push_back(t); }
  // groups: product of the group-index ranges (Sec. 2.4)
  {
    Term t;
    t.cases = {Case{{}, Poly{{Mono{0xFF, 0xFF, 0xFF, 0xFF}, 1}}, 1}};
    for (size_t d = 0; d < K.dims.size(); d++)
      if (K.dims[d].tag <= TAG_G2)
        t.cases = case_product(t.cases, interval_cases(C, {C.to_qaff(K.dims[d].hi)}, {C.to_qaff(K.dims[d].lo)}));
    for (int c : LD.cols[KEY_GROUPS]) t.colmul[c] += 1;
    terms.push_back(t);
  }
  // barriers: one per point of the barrier's (group, sequential) indices (Sec. 2.3)
  for (auto &b : K.bars) {
    Term t;
    t.cases = {Case{{}, Poly{{Mono{0xFF, 0xFF, 0xFF, 0xFF}, 1}}, 1}};
    for (int d : b.dims)
      t.cases = case_product(t.cases, interval_cases(C, {C.to_qaff(K.dims[d].hi)}, {C.to_qaff(K.dims[d].lo)}));
    for (int c : LD.cols[KEY_BARRIERS]) t.colmul[c] += 1;
    terms.push_back(t);
  }
  // statements (Alg. 1)
  for (size_t s = 0; s < K.stmts.size(); s++) {
    const Stmt &st = K.stmts[s];
    std::map<int, i128> keymul;
    for (auto &f : st.flops) keymul[KEY_FLOP + 5 * f.dtype + f.kind] += f.count;
    for (size_t i = 0; i < st.acc.size(); i++) {
      const Access &a = st.acc[i];
      const Array &ar = K.arrays[a.arr];
      if (!ar.global) keymul[(a.store ? KEY_LSTORE : KEY_LLOAD) + (ar.f64 ? 1 : 0)] += 1;
      else {
        int bits = (ar.f64 ? 64 : 32) * a.width;
        keymul[gkey(a.store, bits == 32 ? 0 : bits == 64 ? 1 : 2, cls[s][i])] += 1;
      }
    }
    Term t;
    for (auto &kv : keymul)
      for (int c : LD.cols[kv.first]) t.colmul[c] += kv.second;
    if (t.colmul.empty()) continue;
    t.cases = stmt_count(C, st);
    terms.push_back(t);
  }

  int NC = (int)C.conds.size();
  if (NC > pmt::MAX_CONDS) fail(E_UNSUP, "more than 10 piece conditions");
  int ncols = LD.k + LD.hidden;

  // common denominator D of the counts: the table holds D * count, the evaluators divide
  i128 D = 1;
  for (auto &t : terms)
    for (auto &c : t.cases)
      if (!c.val.empty()) D = D / gcd128(D, c.den) * c.den;
  if (D > 4096) fail(E_UNSUP, "count denominator above 4096");

  // overflow check: per column, the sum of multiplicity * count bound, times D, stays
  // below 2^62, so every value D * count the evaluators form is below 2^62
  {
    const i128 lim = i128(1) << 62;
    std::vector<i128> bound(ncols, 0);
    for (auto &t : terms) {
      i128 mb = 0;
      for (auto &c : t.cases) mb = std::max(mb, c.bound);
      if (mb >= lim) fail(E_RANGE, "a count may reach 2^62 on the box");
      mb *= D;
      for (auto &kv : t.colmul) {
        i128 m = kv.second < 0 ? -kv.second : kv.second;
        if (m && mb >= (lim + m - 1) / m) fail(E_RANGE, "a count may reach 2^62 on the box");   // m * mb >= 2^62
        bound[kv.first] += m * mb;
        if (bound[kv.first] >= lim) fail(E_RANGE, "a count may reach 2^62 on the box");
      }
    }
  }

  // implications between parallel conditions: (f + c1 >= 0) => (f + c2 >= 0) when c1 <= c2
  std::vector<std::pair<int, int>> implies;  // (a true) => (b true)
  for (int a = 0; a < NC; a++)
    for (int b = 0; b < NC; b++) {
      if (a == b) continue;
      QAff fa = C.conds[a], fb = C.conds[b];
      i128 ca = fa.c, cb = fb.c;
      fa.c = fb.c = 0;
      if (fa == fb && ca <= cb) implies.push_back({a, b});
    }

  // pieces: every condition assignment -> column polynomials, deduplicated
  std::vector<std::vector<Poly>> pieces;
  std::map<std::vector<Poly>, int> piece_id;
  std::vector<uint8_t> lut(size_t(1) << NC, 0);
  for (uint32_t asg = 0; asg < (1u << NC); asg++) {
    bool feasible = true;
    for (auto &im : implies)
      if (((asg >> im.first) & 1) && !((asg >> im.second) & 1)) feasible = false;
    if (!feasible) continue;  // never produced by a real point; lut entry stays 0
    std::vector<Poly> cols(ncols);
    for (auto &t : terms) {
      const Case *hit = nullptr;
      for (auto &c : t.cases) {
        bool ok = true;
        for (auto &l : c.lits) if ((((asg >> l.first) & 1) != 0) != l.second) { ok = false; break; }
        if (ok) { hit = &c; break; }
      }
      if (!hit) continue;
      for (auto &kv : t.colmul) poly_acc(cols[kv.first], hit->val, kv.second * (D / hit->den));
    }
    auto it = piece_id.find(cols);
    int id;
    if (it == piece_id.end()) {
      id = (int)pieces.size();
      if (id > 255) fail(E_UNSUP, "more than 256 pieces");
      pieces.push_back(cols);
      piece_id[cols] = id;
    } else {
      id = it->second;
    }
    lut[asg] = (uint8_t)id;
  }

  // smallest denominator: divide out what every coefficient shares with D
  {
    i128 g = D;
    for (auto &pc : pieces)
      for (auto &poly : pc)
        for (auto &kv : poly) g = gcd128(g, kv.second);
    if (g > 1) {
      for (auto &pc : pieces)
        for (auto &poly : pc)
          for (auto &kv : poly) kv.second /= g;
      D /= g;
    }
  }

  // values used (params always kept), atom renumbering
  std::vector<int> used_atom(C.atoms.size(), 0);
  for (auto &q : C.conds) for (auto &kv : q.at) used_atom[kv.first] = 1;
  for (auto &pc : pieces)
    for (auto &poly : pc)
      for (auto &kv : poly)
        for (auto f : kv.first) if (f != 0xFF && f >= C.P) used_atom[f - C.P] = 1;
  std::vector<int> newid(C.atoms.size(), -1);
  int na = 0;
  for (size_t a = 0; a < C.atoms.size(); a++) if (used_atom[a]) newid[a] = na++;
  if (C.P + na > pmt::MAX_VALUES) fail(E_UNSUP, "more than 32 distinct atoms");
  auto vmap = [&](int v) { return v < C.P ? v : C.P + newid[v - C.P]; };

  // hold slots for post-op inputs
  std::map<int, int> hold;
  for (auto &po : LD.post) {
    if (!hold.count(po[1])) { int h = (int)hold.size(); hold[po[1]] = h; }
    if (!hold.count(po[2])) { int h = (int)hold.size(); hold[po[2]] = h; }
  }

  // ---- emit
  std::vector<uint32_t> W(pmt::HEADER_WORDS, 0);
  auto put64 = [&](std::vector<uint32_t> &v, i128 x) {
    int64_t y = (int64_t)x;
    v.push_back((uint32_t)((uint64_t)y & 0xffffffffu));
    v.push_back((uint32_t)((uint64_t)y >> 32));
  };
  W[pmt::H_MAGIC] = pmt::MAGIC;
  W[pmt::H_NPARAMS] = C.P;
  W[pmt::H_NATOMS] = na;
  W[pmt::H_NCONDS] = NC;
  W[pmt::H_NPIECES] = (uint32_t)pieces.size();
  W[pmt::H_K] = LD.k;
  W[pmt::H_NHIDDEN] = LD.hidden;
  W[pmt::H_NPOST] = (uint32_t)LD.post.size();
  for (int i = 0; i < 4; i++) {
    W[pmt::H_BOX_LO + i] = (uint32_t)(int32_t)(i < C.P ? C.box_lo[i] : 0);
    W[pmt::H_BOX_HI + i] = (uint32_t)(int32_t)(i < C.P ? C.box_hi[i] : 0);
  }
  // atoms
  W[pmt::H_OFF_ATOMS] = (uint32_t)W.size();
  for (size_t a = 0; a < C.atoms.size(); a++) {
    if (newid[a] < 0) continue;
    const Atom &A = C.atoms[a];
    i128 nl, nh;
    C.atom_num_range(A, nl, nh);
    if (nl < -(i128(1) << 31) + (i128(1) << 20) || nh > (i128(1) << 31) - (i128(1) << 20))
      fail(E_RANGE, "atom numerator leaves int32 on the box");
    int sh2;
    uint32_t m = magic_for(A.c, sh2);
    for (int i = 0; i < 4; i++) W.push_back((uint32_t)(int32_t)A.a[i]);
    W.push_back((uint32_t)(int32_t)A.b);
    W.push_back((uint32_t)(int32_t)A.c);
    W.push_back(m);
    W.push_back((uint32_t)(1 | (sh2 << 8) | ((nl < 0 ? 1 : 0) << 16)));
  }
  // conditions
  W[pmt::H_OFF_CONDS] = (uint32_t)W.size();
  for (auto &q : C.conds) {
    std::vector<std::pair<int, i128>> tm;
    for (int i = 0; i < C.P; i++) if (q.p[i]) tm.push_back({i, q.p[i]});
    for (auto &kv : q.at) if (kv.second) tm.push_back({vmap(C.P + kv.first), kv.second});
    W.push_back((uint32_t)tm.size());
    put64(W, q.c);
    for (auto &x : tm) {
      if (x.second > INT32_MAX || x.second < INT32_MIN) fail(E_RANGE, "condition coefficient beyond int32");
      W.push_back((uint32_t)x.first);
      W.push_back((uint32_t)(int32_t)x.second);
    }
  }
  // LUT
  W[pmt::H_OFF_LUT] = (uint32_t)W.size();
  for (size_t i = 0; i < lut.size(); i += 4) {
    uint32_t w = 0;
    for (size_t b = 0; b < 4 && i + b < lut.size(); b++) w |= (uint32_t)lut[i + b] << (8 * b);
    W.push_back(w);
  }
  // pieces: the distinct monomials of each piece become products (each one value times
  // an earlier product, prefixes added as needed); columns become coefficient entries
  std::vector<uint32_t> pw, prods, entries;
  int degree = 0, nentry = 0, maxprod = 0;
  for (auto &pc : pieces) {
    std::map<Mono, int> pid;  // monomial (new value ids, sorted) -> slot
    std::vector<uint32_t> plist;
    const int V = C.P + na;
    std::function<int(const Mono &)> need = [&](const Mono &m) -> int {
      int d = mono_deg(m);
      if (d == 0) return (int)pmt::CONST_SLOT;
      if (d == 1) return m[0];
      auto it = pid.find(m);
      if (it != pid.end()) return it->second;
      Mono pre = m;
      pre[d - 1] = 0xFF;
      int a = need(pre);
      int id = V + (int)plist.size();
      plist.push_back((uint32_t)a | ((uint32_t)m[d - 1] << 8));
      pid[m] = id;
      return id;
    };
    std::vector<std::array<uint32_t, 4>> ent;
    for (int col = 0; col < ncols; col++) {
      const Poly &p = pc[col];
      if (p.empty()) continue;
      int h = hold.count(col) ? hold[col] + 1 : 0;
      size_t first = ent.size();
      for (auto &kv : p) {
        Mono m = {0xFF, 0xFF, 0xFF, 0xFF};
        std::vector<uint8_t> f;
        for (auto x : kv.first) if (x != 0xFF) f.push_back((uint8_t)vmap(x));
        std::sort(f.begin(), f.end());
        for (size_t q = 0; q < f.size(); q++) m[q] = f[q];
        degree = std::max(degree, (int)f.size());
        int pr = need(m);
        int64_t cf = (int64_t)kv.second;
        ent.push_back({(uint32_t)((uint64_t)cf & 0xffffffffu), (uint32_t)((uint64_t)cf >> 32),
                       (uint32_t)col | ((uint32_t)pr << 8) | ((uint32_t)h << 16), 0u});
      }
      ent.back()[2] |= pmt::ENTRY_LAST;
      (void)first;
    }
    if (V + (int)plist.size() > pmt::MAX_PRODS) fail(E_UNSUP, "more than 19 values and products in a piece");
    maxprod = std::max(maxprod, (int)plist.size());
    pw.push_back((uint32_t)prods.size());
    pw.push_back((uint32_t)plist.size());
    pw.push_back((uint32_t)(entries.size() / pmt::ENTRY_WORDS));
    pw.push_back((uint32_t)ent.size());
    prods.insert(prods.end(), plist.begin(), plist.end());
    for (auto &e : ent) entries.insert(entries.end(), e.begin(), e.end());
    nentry += (int)ent.size();
  }
  while (W.size() % 4) W.push_back(0);  // 16-byte alignment of the piece headers
  W[pmt::H_OFF_PIECES] = (uint32_t)W.size();
  W.insert(W.end(), pw.begin(), pw.end());
  W[pmt::H_OFF_PRODS] = (uint32_t)W.size();
  W.insert(W.end(), prods.begin(), prods.end());
  while (W.size() % 4) W.push_back(0);  // 16-byte alignment of the entry block
  W[pmt::H_OFF_ENTRIES] = (uint32_t)W.size();
  W.insert(W.end(), entries.begin(), entries.end());
  W[pmt::H_OFF_POST] = (uint32_t)W.size();
  for (auto &po : LD.post) W.push_back((uint32_t)po[0] | ((uint32_t)hold[po[1]] << 8) | ((uint32_t)hold[po[2]] << 16));
  while (W.size() % 4) W.push_back(0);  // 16-byte multiple for bulk copies
  {  // D = 2^t d, d odd: exact division is a shift by t and a product with d^-1 mod 2^128
    int t = 0;
    uint64_t d = (uint64_t)D;
    while (!(d & 1)) { d >>= 1; t++; }
    unsigned __int128 inv = d;   // Newton: each step doubles the correct low bits (d*d = 1 mod 8)
    for (int it = 0; it < 7; it++) inv *= 2 - (unsigned __int128)d * inv;
    W[pmt::H_DEN] = (uint32_t)D;
    W[pmt::H_DEN_SHIFT] = (uint32_t)t;
    for (int i = 0; i < 4; i++) W[pmt::H_DEN_INV + i] = (uint32_t)(inv >> (32 * i));
  }
  W[pmt::H_NENTRIES] = nentry;
  W[pmt::H_DEGREE] = degree;
  W[pmt::H_NPRODS] = (uint32_t)prods.size();
  W[pmt::H_MAXPROD] = maxprod;
  W[pmt::H_WORDS] = (uint32_t)W.size();
  if (W.size() > (size_t)pmt::MAX_TABLE_WORDS) fail(E_UNSUP, "compiled table larger than 16 KB");
  Result r;
  r.words = W;
  r.n_atoms = na;
  r.n_conds = NC;
  r.n_pieces = (int)pieces.size();
  r.n_monos = nentry;
  r.degree = degree;
  return r;
}

}  // namespace pmc

// Entry used by the C ABI layer.  Returns 0 or a PM_ERR_* code; msg receives a description.
int pm_compile_table(const char *ir, size_t len, int layout, const int64_t *plo, const int64_t *phi,
                     std::vector<uint32_t> &words, int info[8], std::string &msg) {
  try {
    pmc::Result r = pmc::compile(std::string(ir, len), layout, plo, phi);
    words = r.words;
    info[0] = (int)words[pmt::H_NPARAMS];
    info[1] = r.n_atoms;
    info[2] = r.n_conds;
    info[3] = r.n_pieces;
    info[4] = r.n_monos;
    info[5] = (int)words[pmt::H_K];
    info[6] = (int)words.size();
    info[7] = r.degree;
    return 0;
  } catch (const pmc::Error &e) {
    msg = e.msg;
    return e.code;
  } catch (const std::exception &e) {
    msg = e.what();
    return pmc::E_UNSUP;
  }
}

int pm_ir_param_count(const char *ir, size_t len) {
  try {
    pmc::Compiler C;
    pmc::parse_kernel(C, std::string(ir, len));
    return (int)C.K.params.size();
  } catch (...) {
    return -1;
  }
}
