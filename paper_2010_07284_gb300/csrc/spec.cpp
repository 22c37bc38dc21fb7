// Specification text front end (Sec. 3): a specification is a sequence of
// commands --
//   load x = "s"              bind image x (the images given at evaluation,
//                             in load order; "s" names it, nothing is read)
//   let f = e                 a constant
//   let f(x1, ..., xN) = e    a macro, expanded where it is applied; the
//                             expansion shares identical sub-expressions
//   save "s" e                an output of the formula (roots in save order)
//   import "s"                accepted: the derived operators are built in
// -- and an expression is a number, a name, an application f(e1, ..., eN),
// an infix application or a parenthesised expression.  `//` starts a
// comment.  The language's text is only described in the paper (its grammar
// is deferred to the tool's documentation); the vocabulary and precedences
// below are this library's reading, listed with the entry point.
#include "spec.h"

#include <cctype>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <exception>
#include <map>
#include <tuple>

namespace vl {

namespace {

// ---------------------------------------------------------------- lexer

enum TokKind { T_END, T_ID, T_NUM, T_STR, T_SYM };
struct Token {
  TokKind k = T_END;
  std::string s;
  double v = 0;
  int line = 1, col = 1;
};

struct SpecError {
  int line, col;
  std::string what;
};

[[noreturn]] void fail(int line, int col, const std::string& what) {
  throw SpecError{line, col, what};
}

std::vector<Token> lex(const char* src) {
  std::vector<Token> out;
  int line = 1, col = 1;
  const char* p = src;
  auto adv = [&](int n) {
    for (int i = 0; i < n; ++i, ++p) {
      if (*p == '\n') { ++line; col = 1; }
      else ++col;
    }
  };
  while (*p) {
    const char c = *p;
    if (c == ' ' || c == '\t' || c == '\r' || c == '\n') { adv(1); continue; }
    if (c == '/' && p[1] == '/') {
      while (*p && *p != '\n') adv(1);
      continue;
    }
    Token t;
    t.line = line;
    t.col = col;
    if (std::isalpha((unsigned char)c) || c == '_') {
      const char* q = p;
      while (std::isalnum((unsigned char)*q) || *q == '_') ++q;
      t.k = T_ID;
      t.s.assign(p, q);
      adv((int)(q - p));
    } else if (std::isdigit((unsigned char)c) || (c == '.' && std::isdigit((unsigned char)p[1]))) {
      char* end = nullptr;
      t.v = std::strtod(p, &end);
      if (end == p) fail(line, col, "bad number");
      t.k = T_NUM;
      adv((int)(end - p));
    } else if (c == '"') {
      const char* q = p + 1;
      while (*q && *q != '"' && *q != '\n') ++q;
      if (*q != '"') fail(line, col, "unterminated string");
      t.k = T_STR;
      t.s.assign(p + 1, q);
      adv((int)(q - p) + 1);
    } else if ((c == '>' || c == '<') && p[1] == '.') {
      t.k = T_SYM;
      t.s.assign(p, p + 2);
      adv(2);
    } else if (std::strchr("()=,&|!+-*/", c)) {
      t.k = T_SYM;
      t.s.assign(1, c);
      adv(1);
    } else {
      fail(line, col, std::string("unexpected character '") + c + "'");
    }
    out.push_back(t);
  }
  Token e;
  e.line = line;
  e.col = col;
  out.push_back(e);
  return out;
}

bool is_keyword(const std::string& s) {
  return s == "let" || s == "load" || s == "save" || s == "import" || s == "print";
}

// ------------------------------------------------------------ syntax tree

enum AstKind { A_NUM, A_ID, A_CALL, A_UN, A_BIN };
struct Ast {
  AstKind k;
  double v = 0;
  std::string s;           // name, or operator symbol
  std::vector<int> kids;
  int line = 0, col = 0;
};

struct Parser {
  std::vector<Token> t;
  size_t i = 0;
  std::vector<Ast> ast;
  int depth = 0;  // nesting of the expression being parsed (bounded: no stack overflow)

  const Token& cur() const { return t[i]; }
  bool sym(const char* s) const { return cur().k == T_SYM && cur().s == s; }
  int node(AstKind k, const Token& at) {
    Ast a;
    a.k = k;
    a.line = at.line;
    a.col = at.col;
    ast.push_back(a);
    return (int)ast.size() - 1;
  }
  void expect(const char* s) {
    if (!sym(s)) fail(cur().line, cur().col, std::string("expected '") + s + "'");
    ++i;
  }
  std::string ident(const char* what) {
    if (cur().k != T_ID || is_keyword(cur().s))
      fail(cur().line, cur().col, std::string("expected ") + what);
    return t[i++].s;
  }

  int binary(int l, const Token& at, const char* op, int r) {
    const int n = node(A_BIN, at);
    ast[n].s = op;
    ast[n].kids = {l, r};
    return n;
  }
  int expr() {
    if (++depth > 1000) fail(cur().line, cur().col, "expression nested deeper than 1000");
    const int e = or_();
    --depth;
    return e;
  }
  int or_() {
    int l = and_();
    while (sym("|")) { const Token at = t[i++]; l = binary(l, at, "|", and_()); }
    return l;
  }
  int and_() {
    int l = cmp();
    while (sym("&")) { const Token at = t[i++]; l = binary(l, at, "&", cmp()); }
    return l;
  }
  int cmp() {
    int l = add();
    if (sym(">.") || sym("<.")) {
      const Token at = t[i++];
      l = binary(l, at, at.s.c_str(), add());
      if (sym(">.") || sym("<.")) fail(cur().line, cur().col, "comparisons do not chain");
    }
    return l;
  }
  int add() {
    int l = mul();
    while (sym("+") || sym("-")) { const Token at = t[i++]; l = binary(l, at, at.s.c_str(), mul()); }
    return l;
  }
  int mul() {
    int l = unary();
    while (sym("*") || sym("/")) { const Token at = t[i++]; l = binary(l, at, at.s.c_str(), unary()); }
    return l;
  }
  int unary() {
    if (sym("!") || sym("-")) {
      const Token at = t[i++];
      if (++depth > 1000) fail(at.line, at.col, "expression nested deeper than 1000");
      const int n = node(A_UN, at);
      ast[n].s = at.s;
      const int k = unary();
      ast[n].kids = {k};
      --depth;
      return n;
    }
    return primary();
  }
  int primary() {
    const Token at = cur();
    if (at.k == T_NUM) {
      ++i;
      const int n = node(A_NUM, at);
      ast[n].v = at.v;
      return n;
    }
    if (sym("(")) {
      ++i;
      const int e = expr();
      expect(")");
      return e;
    }
    if (at.k == T_ID && !is_keyword(at.s)) {
      ++i;
      if (sym("(")) {
        ++i;
        const int n = node(A_CALL, at);
        ast[n].s = at.s;
        std::vector<int> args;
        if (!sym(")")) {
          args.push_back(expr());
          while (sym(",")) { ++i; args.push_back(expr()); }
        }
        expect(")");
        ast[n].kids = args;
        return n;
      }
      const int n = node(A_ID, at);
      ast[n].s = at.s;
      return n;
    }
    fail(at.line, at.col, at.k == T_END ? "unexpected end of text" : "expected an expression");
  }
};

// ------------------------------------------------------------- evaluation

// A value: a mask (node), a number term (node), a number literal, a loaded
// image, or a percentile of a number term (only as a comparison's bound).
enum ValKind { V_MASK, V_NUM, V_LIT, V_IMG, V_PCT };
struct Val {
  ValKind k = V_LIT;
  int node = -1;   // V_MASK, V_NUM; V_PCT: the number term
  double lit = 0;  // V_LIT; V_PCT: the level q
  int img = -1;    // V_IMG
};

struct Macro {
  std::vector<std::string> params;
  int body;
};

struct Eval {
  const std::vector<Ast>& ast;
  TextSpec& out;
  std::map<std::string, Val> globals;
  std::map<std::string, Macro> macros;
  std::vector<std::map<std::string, Val>> frames;  // parameters of the macros being expanded
  std::map<std::tuple<int, int, int, int, int, uint32_t, uint64_t>, int> shared;

  Eval(const std::vector<Ast>& a, TextSpec& o) : ast(a), out(o) {}

  int emit(int op, int a = -1, int b = -1, int image = 0, int channel = 0, float t = 0.f,
           double q = 0.0) {
    uint32_t tb;
    uint64_t qb;
    std::memcpy(&tb, &t, 4);
    std::memcpy(&qb, &q, 8);
    const auto key = std::make_tuple(op, a, b, image, channel, tb, qb);
    auto it = shared.find(key);
    if (it != shared.end()) return it->second;
    vl_node n{op, a, b, image, channel, t, q};
    out.nodes.push_back(n);
    const int idx = (int)out.nodes.size() - 1;
    shared[key] = idx;
    return idx;
  }
  Val mask(int node) { Val v; v.k = V_MASK; v.node = node; return v; }
  Val num(int node) { Val v; v.k = V_NUM; v.node = node; return v; }
  Val lit(double x) { Val v; v.k = V_LIT; v.lit = x; return v; }

  [[noreturn]] void err(int a, const std::string& what) { fail(ast[a].line, ast[a].col, what); }
  Val need(int a, ValKind k, const char* what) {
    Val v = eval(a);
    if (v.k != k) err(a, std::string("expected ") + what);
    return v;
  }

  // a threshold or percentile comparison of the number term l
  Val compare(int at, const Val& l, bool gt, const Val& r) {
    if (l.k != V_NUM) err(at, "a comparison needs a number term on its left (e.g. intensity(img))");
    const vl_node& ln = out.nodes[l.node];
    const bool bare = ln.op == VL_OP_VALUE;  // a channel as it is: the atom reads it directly
    if (r.k == V_LIT) {
      const float t = (float)r.lit;
      return bare ? mask(emit(gt ? VL_OP_THR_GT : VL_OP_THR_LT, -1, -1, ln.image, ln.channel, t))
                  : mask(emit(gt ? VL_OP_THR_GT : VL_OP_THR_LT, l.node, -1, 0, 0, t));
    }
    if (r.k == V_PCT) {
      if (r.node != l.node) err(at, "a percentile bound must be of the term it is compared with");
      return bare ? mask(emit(gt ? VL_OP_PCT_GT : VL_OP_PCT_LT, -1, -1, ln.image, ln.channel, 0.f, r.lit))
                  : mask(emit(gt ? VL_OP_PCT_GT : VL_OP_PCT_LT, l.node, -1, 0, 0, 0.f, r.lit));
    }
    err(at, "a comparison's bound is a number or percentile(term, q)");
  }

  Val arith(int at, char op, const Val& l, const Val& r) {
    const int code = op == '+' ? VL_OP_ADD : op == '-' ? VL_OP_SUB : op == '*' ? VL_OP_MUL : VL_OP_DIV;
    if (l.k == V_LIT && r.k == V_LIT) {  // literals: exact real arithmetic, rounded where used
      return lit(op == '+' ? l.lit + r.lit : op == '-' ? l.lit - r.lit
                 : op == '*' ? l.lit * r.lit : l.lit / r.lit);
    }
    if (l.k == V_NUM && r.k == V_NUM) return num(emit(code, l.node, r.node));
    if (l.k == V_NUM && r.k == V_LIT) return num(emit(code, l.node, -1, 0, 0, (float)r.lit));
    if (l.k == V_LIT && r.k == V_NUM) {
      if (op == '+' || op == '*') return num(emit(code, r.node, -1, 0, 0, (float)l.lit));
      if (op == '-') {  // t - x = (x * -1) + t, both exact steps of binary32
        const int neg = emit(VL_OP_MUL, r.node, -1, 0, 0, -1.f);
        return num(emit(VL_OP_ADD, neg, -1, 0, 0, (float)l.lit));
      }
      err(at, "a number divided by a number term is not supported");
    }
    err(at, "arithmetic takes number terms and numbers");
  }

  Val call(int a) {
    const Ast& n = ast[a];
    const std::string& f = n.s;
    const size_t na = n.kids.size();
    auto arity = [&](size_t k) {
      if (na != k) err(a, f + " takes " + std::to_string(k) + " argument" + (k == 1 ? "" : "s"));
    };
    auto m1 = [&]() { arity(1); return need(n.kids[0], V_MASK, "a mask").node; };
    auto m2 = [&](int op) {
      arity(2);
      const int x = need(n.kids[0], V_MASK, "a mask").node;
      const int y = need(n.kids[1], V_MASK, "a mask").node;
      return mask(emit(op, x, y));
    };
    auto chan = [&](int c) {
      arity(1);
      const Val im = need(n.kids[0], V_IMG, "a loaded image");
      return num(emit(VL_OP_VALUE, -1, -1, im.img, c));
    };
    auto mit = macros.find(f);
    if (mit != macros.end()) {
      const Macro& m = mit->second;
      if (na != m.params.size())
        err(a, f + " takes " + std::to_string(m.params.size()) + " arguments");
      if (frames.size() >= 64) err(a, "macros nested deeper than 64 (a recursive definition?)");
      std::map<std::string, Val> frame;
      for (size_t k = 0; k < na; ++k) frame[m.params[k]] = eval(n.kids[k]);
      frames.push_back(frame);
      const Val v = eval(m.body);
      frames.pop_back();
      return v;
    }
    if (f == "intensity") return chan(0);
    if (f == "red") return chan(0);
    if (f == "green") return chan(1);
    if (f == "blue") return chan(2);
    if (f == "alpha") return chan(3);
    if (f == "channel") {
      arity(2);
      const Val im = need(n.kids[0], V_IMG, "a loaded image");
      const Val c = need(n.kids[1], V_LIT, "a channel number");
      if (c.lit < 0 || c.lit != std::floor(c.lit) || c.lit > 1e6) err(n.kids[1], "bad channel");
      return num(emit(VL_OP_VALUE, -1, -1, im.img, (int)c.lit));
    }
    if (f == "mask") {
      arity(1);
      const Val im = need(n.kids[0], V_IMG, "a loaded image");
      return mask(emit(VL_OP_MASK, -1, -1, im.img));
    }
    if (f == "percentile") {
      arity(2);
      const Val x = need(n.kids[0], V_NUM, "a number term");
      const Val q = need(n.kids[1], V_LIT, "a level in [0, 1]");
      if (!(q.lit >= 0.0 && q.lit <= 1.0)) err(n.kids[1], "a percentile level lies in [0, 1]");
      Val v;
      v.k = V_PCT;
      v.node = x.node;
      v.lit = q.lit;
      return v;
    }
    if (f == "not") return mask(emit(VL_OP_NOT, m1()));
    if (f == "near" || f == "N") return mask(emit(VL_OP_NEAR, m1()));
    if (f == "interior") return mask(emit(VL_OP_INTERIOR, m1()));
    if (f == "and") return m2(VL_OP_AND);
    if (f == "or") return m2(VL_OP_OR);
    if (f == "reach" || f == "rho") return m2(VL_OP_REACH);
    if (f == "surrounded") return m2(VL_OP_SURROUNDED);
    if (f == "grow") return m2(VL_OP_GROW);
    if (f == "touch") return m2(VL_OP_TOUCH);
    err(a, "unknown function " + f);
  }

  Val name(int a) {
    const std::string& s = ast[a].s;
    if (!frames.empty()) {
      auto it = frames.back().find(s);
      if (it != frames.back().end()) return it->second;
    }
    auto it = globals.find(s);
    if (it != globals.end()) return it->second;
    if (s == "tt") return mask(emit(VL_OP_TRUE));
    if (s == "ff") return mask(emit(VL_OP_FALSE));
    if (macros.count(s)) err(a, s + " needs arguments");
    err(a, "unknown name " + s);
  }

  int edepth = 0;  // expansion depth (macros included): bounded, no stack overflow
  Val eval(int a) {
    struct Depth {
      int& d;
      explicit Depth(int& x) : d(x) { ++d; }
      ~Depth() { --d; }
    } guard(edepth);
    if (edepth > 4000) err(a, "expression expands deeper than 4000");
    const Ast& n = ast[a];
    switch (n.k) {
      case A_NUM: return lit(n.v);
      case A_ID: return name(a);
      case A_CALL: return call(a);
      case A_UN: {
        const Val x = eval(n.kids[0]);
        if (n.s == "!") {
          if (x.k != V_MASK) err(a, "'!' takes a mask");
          return mask(emit(VL_OP_NOT, x.node));
        }
        if (x.k == V_LIT) return lit(-x.lit);
        if (x.k == V_NUM) return num(emit(VL_OP_MUL, x.node, -1, 0, 0, -1.f));
        err(a, "'-' takes a number or a number term");
      }
      case A_BIN: {
        const Val l = eval(n.kids[0]), r = eval(n.kids[1]);
        if (n.s == "&" || n.s == "|") {
          if (l.k != V_MASK || r.k != V_MASK) err(a, "'" + n.s + "' takes masks");
          return mask(emit(n.s == "&" ? VL_OP_AND : VL_OP_OR, l.node, r.node));
        }
        if (n.s == ">." || n.s == "<.") return compare(a, l, n.s == ">.", r);
        return arith(a, n.s[0], l, r);
      }
    }
    err(a, "bad expression");
  }
};

}  // namespace

bool parse_spec(const char* src, TextSpec* out, std::string* err) {
  TextSpec spec;
  try {
    Parser p;
    p.t = lex(src ? src : "");
    Eval ev(p.ast, spec);
    while (p.cur().k != T_END) {
      const Token at = p.cur();
      if (at.k != T_ID || !is_keyword(at.s))
        fail(at.line, at.col, "expected a command (let, load, save, import)");
      ++p.i;
      if (at.s == "load") {
        const Token nt = p.cur();
        const std::string nm = p.ident("an image name");
        p.expect("=");
        if (p.cur().k != T_STR) fail(p.cur().line, p.cur().col, "expected a string");
        const std::string source = p.t[p.i++].s;
        if (ev.globals.count(nm) || ev.macros.count(nm)) fail(nt.line, nt.col, nm + " is already defined");
        Val v;
        v.k = V_IMG;
        v.img = (int)spec.loads.size();
        ev.globals[nm] = v;
        spec.loads.push_back(nm);
        spec.sources.push_back(source);
      } else if (at.s == "let") {
        const Token nt = p.cur();
        const std::string nm = p.ident("a name");
        if (ev.globals.count(nm) || ev.macros.count(nm)) fail(nt.line, nt.col, nm + " is already defined");
        if (p.sym("(")) {
          ++p.i;
          Macro m;
          if (!p.sym(")")) {
            m.params.push_back(p.ident("a parameter"));
            while (p.sym(",")) { ++p.i; m.params.push_back(p.ident("a parameter")); }
          }
          p.expect(")");
          p.expect("=");
          m.body = p.expr();
          ev.macros[nm] = m;
        } else {
          p.expect("=");
          const int e = p.expr();
          ev.globals[nm] = ev.eval(e);
        }
      } else if (at.s == "save") {
        if (p.cur().k != T_STR) fail(p.cur().line, p.cur().col, "expected a string");
        const std::string nm = p.t[p.i++].s;
        const int e = p.expr();
        const Val v = ev.eval(e);
        if (v.k != V_MASK) ev.err(e, "save takes a mask");
        spec.roots.push_back(v.node);
        spec.saves.push_back(nm);
      } else if (at.s == "import") {
        if (p.cur().k != T_STR) fail(p.cur().line, p.cur().col, "expected a string");
        ++p.i;  // the derived operators of a standard library are built in
      } else {
        fail(at.line, at.col, "print is not supported (formulas output masks: use save)");
      }
    }
    if (spec.roots.empty()) fail(p.cur().line, p.cur().col, "nothing saved: a specification needs a save");
  } catch (const SpecError& e) {
    if (err) *err = "line " + std::to_string(e.line) + ", column " + std::to_string(e.col) + ": " + e.what;
    return false;
  } catch (const std::exception& e) {  // (memory): nothing may cross the C boundary
    if (err) *err = std::string("specification not read: ") + e.what();
    return false;
  }
  *out = std::move(spec);
  return true;
}

}  // namespace vl
