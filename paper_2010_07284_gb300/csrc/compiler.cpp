// Host compiler: node array -> execution plan.
//
// 1. Expansion with sharing (Sec. 3.2: macros are expanded without
//    duplicating sub-expressions).  Derived connectives become primitives
//    (Eq. (1) of Sec. 2); identical nodes become one.  The resulting primitive
//    DAG is what the pixel-operation metric counts.
// 2. Lowering for execution: rho phi1[phi2] = N(phi1 or Z) with Z the
//    phi2-components meeting N phi1 (the reduction of Sec. 3.2), plus
//    local simplifications that do not change any mask (double negation,
//    constants, and-not, De Morgan for or), and dead-node removal.
// 3. Scheduling: component selects (Z) are global barriers; everything else
//    is grouped by "rho depth" into fused tile groups, split where the N
//    depth exceeds the halo budget or the shared-memory buffers run out.
//    Independent selects of the same depth run in one batch.
// 4. Materialised masks get global slots, reused by liveness over steps.
#include "compiler.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>

namespace vl {
namespace {

// ------------------------------------------------------------- step 1 --

struct Key {
  int op, a, b, img, ch, lt;
  uint32_t tb;
  uint64_t qb;
  bool operator<(const Key& o) const {
    return std::tie(op, a, b, img, ch, lt, tb, qb) <
           std::tie(o.op, o.a, o.b, o.img, o.ch, o.lt, o.tb, o.qb);
  }
};

uint32_t fbits(float f) { uint32_t u; std::memcpy(&u, &f, 4); return u; }
uint64_t dbits(double d) { uint64_t u; std::memcpy(&u, &d, 8); return u; }

struct PrimBuilder {
  std::vector<vl_node> nodes;
  std::map<Key, int> index;

  int add(const vl_node& n) {
    Key k{n.op, -1, -1, 0, 0, 0, 0, 0};
    vl_node c = n;
    switch (n.op) {
      case VL_OP_TRUE: case VL_OP_FALSE: break;
      case VL_OP_MASK: k.img = n.image; break;
      case VL_OP_THR_GT: case VL_OP_THR_LT: case VL_OP_PCT_GT: case VL_OP_PCT_LT:
        if (n.a >= 0) {  // compares a number term
          k.a = n.a; k.img = -1;
          c.image = c.channel = 0;
        } else {
          k.img = n.image; k.ch = n.channel;
          c.a = -1;
        }
        c.b = -1;
        if (n.op == VL_OP_THR_GT || n.op == VL_OP_THR_LT) { k.tb = fbits(n.t); c.q = 0; }
        else { k.qb = dbits(n.q); c.t = 0; }
        break;
      case VL_OP_VALUE:
        k.img = n.image; k.ch = n.channel;
        c.a = c.b = -1; c.t = 0; c.q = 0;
        break;
      case VL_OP_ADD: case VL_OP_SUB: case VL_OP_MUL: case VL_OP_DIV:
        k.a = n.a; k.b = n.b;
        if (n.b < 0) k.tb = fbits(n.t);
        else c.t = 0;
        c.image = c.channel = 0; c.q = 0;
        break;
      default:
        k.a = n.a; k.b = n.b;
        c.image = 0; c.channel = 0; c.t = 0; c.q = 0;
        break;
    }
    auto it = index.find(k);
    if (it != index.end()) return it->second;
    nodes.push_back(c);
    index.emplace(k, (int)nodes.size() - 1);
    return (int)nodes.size() - 1;
  }
  int op1(int op, int a) { vl_node n{op, a, -1, 0, 0, 0.f, 0.0}; return add(n); }
  int op2(int op, int a, int b) { vl_node n{op, a, b, 0, 0, 0.f, 0.0}; return add(n); }
  int NOT(int a) { return op1(VL_OP_NOT, a); }
  int AND(int a, int b) { return op2(VL_OP_AND, a, b); }
  int NEAR(int a) { return op1(VL_OP_NEAR, a); }
  int REACH(int a, int b) { return op2(VL_OP_REACH, a, b); }
  // derived connectives, written out in primitives
  int OR(int a, int b) { return NOT(AND(NOT(a), NOT(b))); }
  int INTERIOR(int a) { return NOT(NEAR(NOT(a))); }
  int SURROUNDED(int a, int b) { return AND(a, NOT(REACH(NOT(OR(a, b)), NOT(b)))); }
  int GROW(int a, int b) { return OR(a, AND(b, REACH(a, b))); }
  int TOUCH(int a, int b) { return AND(a, REACH(b, a)); }
};

// ------------------------------------------------------------- step 2 --

struct ExecBuilder {
  std::vector<ENode> nodes;
  std::map<Key, int> index;

  int add(ENode n) {
    Key k{n.op, n.a, n.b, n.img, n.ch, n.lt, fbits(n.t), dbits(n.q)};
    auto it = index.find(k);
    if (it != index.end()) return it->second;
    n.pct_slot = -1;
    nodes.push_back(n);
    index.emplace(k, (int)nodes.size() - 1);
    return (int)nodes.size() - 1;
  }
  ENode blank(int op) { ENode n{}; n.op = op; n.a = n.b = -1; return n; }
  int k(int id) const { return nodes[id].op; }
  int TRUE_() { return add(blank(E_TRUE)); }
  int FALSE_() { return add(blank(E_FALSE)); }

  int NOT(int x) {
    const ENode& v = nodes[x];
    if (v.op == E_NOT) return v.a;
    if (v.op == E_TRUE) return FALSE_();
    if (v.op == E_FALSE) return TRUE_();
    // not(not p and not y) = p or y
    if (v.op == E_ANDNOT && nodes[v.a].op == E_NOT) return OR(nodes[v.a].a, v.b);
    ENode n = blank(E_NOT); n.a = x; return add(n);
  }
  int AND(int p, int q) {
    if (p == q) return p;
    if (k(p) == E_FALSE || k(q) == E_FALSE) return FALSE_();
    if (k(p) == E_TRUE) return q;
    if (k(q) == E_TRUE) return p;
    if (k(q) == E_NOT) {
      if (nodes[q].a == p) return FALSE_();
      return ANDNOT(p, nodes[q].a);
    }
    if (k(p) == E_NOT) {
      if (nodes[p].a == q) return FALSE_();
      return ANDNOT(q, nodes[p].a);
    }
    ENode n = blank(E_AND); n.a = std::min(p, q); n.b = std::max(p, q); return add(n);
  }
  int ANDNOT(int p, int y) {  // p and not y
    if (p == y) return FALSE_();
    if (k(y) == E_FALSE) return p;
    if (k(y) == E_TRUE || k(p) == E_FALSE) return FALSE_();
    ENode n = blank(E_ANDNOT); n.a = p; n.b = y; return add(n);
  }
  int OR(int p, int q) {
    if (p == q) return p;
    if (k(p) == E_TRUE || k(q) == E_TRUE) return TRUE_();
    if (k(p) == E_FALSE) return q;
    if (k(q) == E_FALSE) return p;
    ENode n = blank(E_OR); n.a = std::min(p, q); n.b = std::max(p, q); return add(n);
  }
  int NEAR(int x) {
    if (k(x) == E_FALSE || k(x) == E_TRUE) return x;
    ENode n = blank(E_NEAR); n.a = x; return add(n);
  }
  int REACH(int a, int b) {
    if (k(a) == E_FALSE) return a;
    if (k(b) == E_FALSE) return NEAR(a);
    ENode z = blank(E_RZ); z.a = a; z.b = b;
    int zi = add(z);
    return NEAR(OR(a, zi));
  }
};

bool is_atom(int op) { return op == E_TRUE || op == E_FALSE || op == E_THR || op == E_PCT || op == E_MASK; }
bool is_number_op(int op) {
  return op == VL_OP_VALUE || op == VL_OP_ADD || op == VL_OP_SUB || op == VL_OP_MUL || op == VL_OP_DIV;
}
// Provisional image index of the k-th number image (renumbered to follow the
// formula's own images once the live nodes are known).
constexpr int kNumImageBase = 16384;
int arity(int op) {
  switch (op) {
    case E_NOT: case E_NEAR: case E_COPY: return 1;
    case E_AND: case E_OR: case E_ANDNOT: case E_RZ: return 2;
    default: return 0;
  }
}

}  // namespace

int compile_formula(const vl_node* in, int n_nodes, const int32_t* roots, int n_roots, int conn,
                    const PlanParams& pp, Plan* out, std::string* err) {
  if (n_nodes < 1 || !in) { *err = "formula needs at least one node"; return VL_ERR_ARG; }
  if (n_roots < 1 || !roots) { *err = "formula needs at least one root"; return VL_ERR_ARG; }
  if (conn != 4 && conn != 8 && conn != 6 && conn != 26) {
    *err = "connectivity must be 4 or 8 (images), 6 or 26 (volumes)";
    return VL_ERR_ARG;
  }
  if (pp.group_buffers < 4 || pp.hmax < 1 || pp.hmax > 31 || pp.scratch_sets < 1 ||
      pp.scratch_sets > 4096) { *err = "bad plan parameters"; return VL_ERR_ARG; }
  Plan P;
  P.conn = conn;
  P.params = pp;
  // ---- 1. expansion with sharing
  PrimBuilder pb;
  std::vector<int> prim_of(n_nodes);
  std::vector<char> num(n_nodes, 0);  // node i is a number term
  for (int i = 0; i < n_nodes; ++i) {
    const vl_node& n = in[i];
    auto bad_operand = [&](int x) { return x < 0 || x >= i; };
    const char* why = nullptr;
    const bool thr = n.op == VL_OP_THR_GT || n.op == VL_OP_THR_LT || n.op == VL_OP_PCT_GT ||
                     n.op == VL_OP_PCT_LT;
    if (thr && n.a >= 0) {  // comparison of a number term
      if (n.a >= i || !num[n.a]) why = "a compared operand must be an earlier number term";
      else if ((n.op == VL_OP_PCT_GT || n.op == VL_OP_PCT_LT) && !(n.q >= 0.0 && n.q <= 1.0))
        why = "percentile level outside [0, 1]";
      else if ((n.op == VL_OP_THR_GT || n.op == VL_OP_THR_LT) && std::isnan(n.t))
        why = "threshold is NaN";
      if (!why) {
        vl_node c = n;
        c.a = prim_of[n.a];
        prim_of[i] = pb.add(c);
      }
      if (why) { *err = "node " + std::to_string(i) + ": " + why; return VL_ERR_FORMULA; }
      continue;
    }
    if (is_number_op(n.op)) {
      num[i] = 1;
      if (n.op == VL_OP_VALUE) {
        if (n.image < 0 || n.image > 4095) why = "image index out of range";
        else if (n.channel < 0 || n.channel > 4095) why = "channel out of range";
        if (!why) prim_of[i] = pb.add(n);
      } else if (bad_operand(n.a) || !num[n.a] || (n.b >= 0 && (n.b >= i || !num[n.b]))) {
        why = "arithmetic operands must be earlier number terms";
      } else if (n.b < 0 && std::isnan(n.t)) {
        why = "arithmetic constant is NaN";
      } else {
        vl_node c = n;
        c.a = prim_of[n.a];
        c.b = n.b >= 0 ? prim_of[n.b] : -1;
        prim_of[i] = pb.add(c);
      }
      if (why) { *err = "node " + std::to_string(i) + ": " + why; return VL_ERR_FORMULA; }
      continue;
    }
    if (n.op >= VL_OP_NOT && n.op <= VL_OP_TOUCH) {
      const bool unary = n.op == VL_OP_NOT || n.op == VL_OP_NEAR || n.op == VL_OP_INTERIOR;
      if ((n.a >= 0 && n.a < i && num[n.a]) || (!unary && n.b >= 0 && n.b < i && num[n.b])) {
        *err = "node " + std::to_string(i) + ": connectives take masks, not number terms";
        return VL_ERR_FORMULA;
      }
    }
    switch (n.op) {
      case VL_OP_TRUE: case VL_OP_FALSE: prim_of[i] = pb.add(n); break;
      case VL_OP_THR_GT: case VL_OP_THR_LT: case VL_OP_PCT_GT: case VL_OP_PCT_LT:
      case VL_OP_MASK:
        if (n.image < 0 || n.image > 4095) why = "image index out of range";
        else if (n.op != VL_OP_MASK && (n.channel < 0 || n.channel > 4095)) why = "channel out of range";
        else if ((n.op == VL_OP_PCT_GT || n.op == VL_OP_PCT_LT) && !(n.q >= 0.0 && n.q <= 1.0))
          why = "percentile level outside [0, 1]";
        else if ((n.op == VL_OP_THR_GT || n.op == VL_OP_THR_LT) && std::isnan(n.t))
          why = "threshold is NaN";
        if (!why) prim_of[i] = pb.add(n);
        break;
      case VL_OP_NOT: case VL_OP_NEAR: case VL_OP_INTERIOR:
        if (bad_operand(n.a)) { why = "operand must precede the node"; break; }
        prim_of[i] = n.op == VL_OP_NOT ? pb.NOT(prim_of[n.a])
                   : n.op == VL_OP_NEAR ? pb.NEAR(prim_of[n.a]) : pb.INTERIOR(prim_of[n.a]);
        break;
      case VL_OP_AND: case VL_OP_REACH: case VL_OP_OR: case VL_OP_SURROUNDED:
      case VL_OP_GROW: case VL_OP_TOUCH: {
        if (bad_operand(n.a) || bad_operand(n.b)) { why = "operands must precede the node"; break; }
        int a = prim_of[n.a], b = prim_of[n.b];
        switch (n.op) {
          case VL_OP_AND: prim_of[i] = pb.AND(a, b); break;
          case VL_OP_REACH: prim_of[i] = pb.REACH(a, b); break;
          case VL_OP_OR: prim_of[i] = pb.OR(a, b); break;
          case VL_OP_SURROUNDED: prim_of[i] = pb.SURROUNDED(a, b); break;
          case VL_OP_GROW: prim_of[i] = pb.GROW(a, b); break;
          default: prim_of[i] = pb.TOUCH(a, b); break;
        }
        break;
      }
      default: why = "unknown operator";
    }
    if (why) { *err = "node " + std::to_string(i) + ": " + why; return VL_ERR_FORMULA; }
  }
  for (int r = 0; r < n_roots; ++r) {
    if (roots[r] < 0 || roots[r] >= n_nodes) { *err = "root index out of range"; return VL_ERR_FORMULA; }
    if (num[roots[r]]) { *err = "root " + std::to_string(r) + " is a number term, not a mask"; return VL_ERR_FORMULA; }
  }
  P.n_primitive = (int64_t)pb.nodes.size();
  for (const vl_node& n : pb.nodes) {
    if (is_number_op(n.op)) { P.n_num++; continue; }
    switch (n.op) {
      case VL_OP_REACH: P.n_reach++; break;
      case VL_OP_THR_GT: case VL_OP_THR_LT: case VL_OP_PCT_GT: case VL_OP_PCT_LT: P.n_thr++; break;
      case VL_OP_NOT: P.n_not++; break;
      case VL_OP_AND: P.n_and++; break;
      case VL_OP_NEAR: P.n_near++; break;
      default: P.n_other++; break;
    }
  }
  // ---- 2. lowering + simplification
  ExecBuilder eb;
  std::vector<int> e_of(pb.nodes.size(), -1);
  // a compared number term reads a number image: VALUE terms are the image
  // channel itself; every other term gets a number image of its own
  std::vector<int> num_image(pb.nodes.size(), -1);
  std::vector<int> num_root_prim;  // prim node of each provisional number image
  auto compared = [&](const vl_node& n, int* img, int* ch) {
    if (n.a < 0) { *img = n.image; *ch = n.channel; return; }
    const vl_node& v = pb.nodes[n.a];
    if (v.op == VL_OP_VALUE) { *img = v.image; *ch = v.channel; return; }
    if (num_image[n.a] < 0) {
      num_image[n.a] = kNumImageBase + (int)num_root_prim.size();
      num_root_prim.push_back(n.a);
    }
    *img = num_image[n.a];
    *ch = 0;
  };
  for (size_t i = 0; i < pb.nodes.size(); ++i) {
    const vl_node& n = pb.nodes[i];
    if (is_number_op(n.op)) continue;  // programs are built below
    switch (n.op) {
      case VL_OP_TRUE: e_of[i] = eb.TRUE_(); break;
      case VL_OP_FALSE: e_of[i] = eb.FALSE_(); break;
      case VL_OP_THR_GT: case VL_OP_THR_LT: {
        ENode e = eb.blank(E_THR); compared(n, &e.img, &e.ch); e.t = n.t;
        e.lt = n.op == VL_OP_THR_LT; e_of[i] = eb.add(e); break;
      }
      case VL_OP_PCT_GT: case VL_OP_PCT_LT: {
        ENode e = eb.blank(E_PCT); compared(n, &e.img, &e.ch); e.q = n.q;
        e.lt = n.op == VL_OP_PCT_LT; e_of[i] = eb.add(e); break;
      }
      case VL_OP_MASK: { ENode e = eb.blank(E_MASK); e.img = n.image; e_of[i] = eb.add(e); break; }
      case VL_OP_NOT: e_of[i] = eb.NOT(e_of[n.a]); break;
      case VL_OP_AND: e_of[i] = eb.AND(e_of[n.a], e_of[n.b]); break;
      case VL_OP_NEAR: e_of[i] = eb.NEAR(e_of[n.a]); break;
      case VL_OP_REACH: e_of[i] = eb.REACH(e_of[n.a], e_of[n.b]); break;
      default: *err = "internal: unexpected primitive"; return VL_ERR_INTERNAL;
    }
  }
  // dead-node removal + renumbering (creation order is topological)
  const int NE = (int)eb.nodes.size();
  std::vector<char> live(NE, 0);
  for (int r = 0; r < n_roots; ++r) live[e_of[prim_of[roots[r]]]] = 1;
  for (int i = NE - 1; i >= 0; --i)
    if (live[i]) {
      const ENode& e = eb.nodes[i];
      if (arity(e.op) >= 1) live[e.a] = 1;
      if (arity(e.op) == 2) live[e.b] = 1;
    }
  std::vector<int> ren(NE, -1);
  for (int i = 0; i < NE; ++i)
    if (live[i]) {
      ENode e = eb.nodes[i];
      if (arity(e.op) >= 1) e.a = ren[e.a];
      if (arity(e.op) == 2) e.b = ren[e.b];
      ren[i] = (int)P.exec.size();
      P.exec.push_back(e);
    }
  P.n_roots = n_roots;
  for (int r = 0; r < n_roots; ++r) P.exec_roots.push_back(ren[e_of[prim_of[roots[r]]]]);
  // a root that is an input mask is copied into its own output buffer
  for (int r = 0; r < n_roots; ++r)
    if (P.exec[P.exec_roots[r]].op == E_MASK) {
      int src = P.exec_roots[r], found = -1;
      for (int k = 0; k < (int)P.exec.size(); ++k)
        if (P.exec[k].op == E_COPY && P.exec[k].a == src) found = k;
      if (found < 0) {
        ENode c{}; c.op = E_COPY; c.a = src; c.b = -1;
        P.exec.push_back(c);
        found = (int)P.exec.size() - 1;
      }
      P.exec_roots[r] = found;
    }
  const int N = (int)P.exec.size();
  if (N > 32000) { *err = "formula too large after expansion (> 32000 nodes)"; return VL_ERR_FORMULA; }
  std::vector<ENode>& X = P.exec;

  // image requirements
  auto need_image = [&](int img, int kind, int ch) -> bool {
    if ((int)P.img_kind.size() <= img) { P.img_kind.resize(img + 1, 0); P.img_channels.resize(img + 1, 0); }
    if (P.img_kind[img] != 0 && P.img_kind[img] != kind) {
      *err = "image " + std::to_string(img) + " used both as a mask and as a number image";
      return false;
    }
    P.img_kind[img] = kind;
    if (kind == 1) P.img_channels[img] = std::max(P.img_channels[img], ch + 1);
    return true;
  };
  for (const ENode& e : X)
    if ((e.op == E_THR || e.op == E_PCT || e.op == E_MASK) && e.img < kNumImageBase)
      if (!need_image(e.img, e.op == E_MASK ? 2 : 1, e.ch)) return VL_ERR_FORMULA;
  // ---- number terms: the live compared terms, numbered after the
  // formula's images; the terms they need, in order, as one program with
  // registers reused after their last read
  {
    std::vector<int> live_num;  // provisional index -> final (or -1)
    live_num.assign(num_root_prim.size(), -1);
    std::vector<int> roots_in_order;
    for (const ENode& e : X)
      if ((e.op == E_THR || e.op == E_PCT) && e.img >= kNumImageBase && live_num[e.img - kNumImageBase] < 0) {
        live_num[e.img - kNumImageBase] = (int)roots_in_order.size();
        roots_in_order.push_back(num_root_prim[e.img - kNumImageBase]);
      }
    const int NP = (int)pb.nodes.size();
    std::vector<char> need(NP, 0);
    for (int r : roots_in_order) need[r] = 1;
    for (int i = NP - 1; i >= 0; --i)
      if (need[i] && pb.nodes[i].op != VL_OP_VALUE) {
        need[pb.nodes[i].a] = 1;
        if (pb.nodes[i].b >= 0) need[pb.nodes[i].b] = 1;
      }
    std::vector<int> uses(NP, 0), store_k(NP, -1);
    for (size_t k = 0; k < roots_in_order.size(); ++k) {
      store_k[roots_in_order[k]] = (int)k;
      uses[roots_in_order[k]]++;
    }
    for (int i = 0; i < NP; ++i)
      if (need[i] && pb.nodes[i].op != VL_OP_VALUE) {
        uses[pb.nodes[i].a]++;
        if (pb.nodes[i].b >= 0) uses[pb.nodes[i].b]++;
      }
    std::vector<int> reg(NP, -1);
    std::vector<char> busy(kArithMaxRegs, 0);
    auto release = [&](int v) {
      if (--uses[v] == 0) busy[reg[v]] = 0;
    };
    for (int i = 0; i < NP; ++i) {
      if (!need[i]) continue;
      const vl_node& n = pb.nodes[i];
      ArithInsn A{};
      A.b = kArithConst;
      if (n.op == VL_OP_VALUE) {
        A.op = A_VALUE;
        A.img = (int16_t)n.image;
        A.ch = (int16_t)n.channel;
        if (!need_image(n.image, 1, n.channel)) return VL_ERR_FORMULA;
      } else {
        A.op = n.op == VL_OP_ADD ? A_ADD : n.op == VL_OP_SUB ? A_SUB : n.op == VL_OP_MUL ? A_MUL : A_DIV;
        A.a = (uint8_t)reg[n.a];
        if (n.b >= 0) A.b = (uint8_t)reg[n.b];
        else A.c = n.t;
        release(n.a);  // operands are read before the result is written
        if (n.b >= 0) release(n.b);
      }
      int r = 0;
      while (r < kArithMaxRegs && busy[r]) ++r;
      if (r == kArithMaxRegs) {
        *err = "number terms need more than " + std::to_string(kArithMaxRegs) + " live values";
        return VL_ERR_FORMULA;
      }
      busy[r] = 1;
      reg[i] = r;
      A.dst = (uint8_t)r;
      P.arith_regs = std::max(P.arith_regs, r + 1);
      P.arith.push_back(A);
      if (store_k[i] >= 0) {
        ArithInsn S{};
        S.op = A_STORE;
        S.a = (uint8_t)r;
        S.b = kArithConst;
        S.img = (int16_t)store_k[i];
        P.arith.push_back(S);
        release(i);
      }
    }
    if ((int)P.arith.size() > kArithMaxInsns) {
      *err = "number terms need more than " + std::to_string(kArithMaxInsns) + " operations";
      return VL_ERR_FORMULA;
    }
    P.n_num_images = (int)roots_in_order.size();
    const int first = (int)P.img_kind.size();
    if (first + P.n_num_images > 32000) { *err = "too many images"; return VL_ERR_FORMULA; }
    for (ENode& e : X)
      if ((e.op == E_THR || e.op == E_PCT) && e.img >= kNumImageBase)
        e.img = first + live_num[e.img - kNumImageBase];
  }
  // percentile slots
  std::map<std::tuple<int, int, uint64_t>, int> pct_slot;
  for (ENode& e : X) {
    if (e.op == E_PCT) {
      auto key = std::make_tuple(e.img, e.ch, dbits(e.q));
      auto it = pct_slot.find(key);
      if (it == pct_slot.end()) {
        int s = (int)pct_slot.size();
        pct_slot.emplace(key, s);
        PctDesc d{}; d.img = (int16_t)e.img; d.ch = (int16_t)e.ch; d.slot = (int16_t)s; d.q = e.q;
        P.pct.push_back(d);
        e.pct_slot = s;
      } else {
        e.pct_slot = it->second;
      }
    }
  }
  P.n_pct_slots = (int)pct_slot.size();

  // consumers
  std::vector<std::vector<int>> cons(N);
  for (int i = 0; i < N; ++i) {
    const ENode& e = X[i];
    if (arity(e.op) >= 1) cons[e.a].push_back(i);
    if (arity(e.op) == 2 && e.b != e.a) cons[e.b].push_back(i);
  }
  std::vector<char> is_root(N, 0);
  for (int r : P.exec_roots) is_root[r] = 1;

  // ---- 3. levels: a component select sits one level above its operands
  std::vector<int> L(N, 0);
  for (int i = 0; i < N; ++i) {
    const ENode& e = X[i];
    if (is_atom(e.op)) continue;
    int l = 0;
    if (arity(e.op) >= 1) l = std::max(l, L[e.a]);
    if (arity(e.op) == 2) l = std::max(l, L[e.b]);
    L[i] = e.op == E_RZ ? l + 1 : l;
  }
  // atoms are computed in the group of their first consumer
  for (int i = 0; i < N; ++i) {
    if (!is_atom(X[i].op) || X[i].op == E_MASK) continue;
    int l = is_root[i] ? 0 : 1 << 30;
    for (int c : cons[i]) l = std::min(l, X[c].op == E_RZ ? L[c] - 1 : L[c]);
    L[i] = (l == 1 << 30) ? 0 : l;
  }
  int maxL = 0;
  for (int i = 0; i < N; ++i) maxL = std::max(maxL, L[i]);

  // slot bookkeeping: value -> slot, with definition/last-use steps
  const int NO = -1;
  std::vector<int> slot_of(N, NO), def_step(N, -1), last_step(N, -1);
  std::vector<char> mat(N, 0);  // materialised (has a global slot)
  // mask images are slots from the start
  std::map<int, int> mask_slot_idx;
  for (int i = 0; i < N; ++i)
    if (X[i].op == E_MASK) {
      mat[i] = 1;
      if (!mask_slot_idx.count(X[i].img)) {
        int s = (int)mask_slot_idx.size();
        mask_slot_idx[X[i].img] = s;
        P.mask_slot_image.push_back(X[i].img);
      }
    }
  auto note_read = [&](int v, int step) { last_step[v] = std::max(last_step[v], step); };

  // value ids used in instructions: we keep per-instruction value ids to
  // resolve slots after liveness.
  struct PendingInsn { Insn in; int val; int src; };  // val: value defined/stored; src: value read (LOAD)
  std::vector<PendingInsn> pins;

  if (!P.pct.empty()) {
    StepDesc s{}; s.kind = SK_PCT; s.pct_off = 0; s.pct_cnt = (int)P.pct.size();
    P.steps.push_back(s);
  }

  const int NB = pp.group_buffers;
  int next_set = 0, n_selects_total = 0;  // select scratch pool (round robin)
  for (int level = 0; level <= maxL; ++level) {
    // ---- groups of this level
    std::vector<int> nodes;
    for (int i = 0; i < N; ++i)
      if (L[i] == level && X[i].op != E_RZ && X[i].op != E_MASK) nodes.push_back(i);
    // consumers inside this level (pending uses) and out-of-group needs
    // uses at this level of every value (inputs from earlier steps included,
    // so a loaded input stays in its buffer until its last consumer here)
    std::vector<int> pending(N, 0);
    for (int c : nodes) {
      const ENode& e = X[c];
      if (arity(e.op) >= 1) pending[e.a]++;
      if (arity(e.op) == 2 && e.b != e.a) pending[e.b]++;
    }
    std::vector<char> needs_store(N, 0);
    for (int i : nodes) {
      if (is_root[i]) needs_store[i] = 1;
      for (int c : cons[i])
        if (X[c].op == E_RZ || L[c] != level) needs_store[i] = 1;
    }
    size_t g_first = pins.size();
    std::vector<int> buf_of(N, -1), depth(N, 0);
    std::vector<int> free_bufs;
    std::vector<int> live_vals;
    auto reset_bufs = [&]() {
      free_bufs.clear();
      for (int b = NB - 1; b >= 0; --b) free_bufs.push_back(b);
      live_vals.clear();
    };
    reset_bufs();
    auto emit = [&](Insn in, int val, int src) { pins.push_back({in, val, src}); };
    auto emit_store = [&](int v) {
      Insn s{}; s.op = I_STORE; s.a = (uint8_t)buf_of[v]; s.slot = -1;
      emit(s, v, -1);
      mat[v] = 1;
    };
    auto close_group = [&]() {
      if (pins.size() == g_first) return;
      // values still needed by later groups of this level and not yet in a
      // global slot are stored now (inputs loaded from earlier steps are not)
      for (int v : live_vals)
        if (pending[v] > 0 && !mat[v]) { emit_store(v); needs_store[v] = 1; }
      StepDesc s{}; s.kind = SK_GROUP;
      s.insn_off = (int)g_first;  // provisional: instruction index in pins
      s.insn_cnt = (int)(pins.size() - g_first);
      P.steps.push_back(s);
      for (size_t k = g_first; k < pins.size(); ++k) {
        if (pins[k].in.op == I_LOAD) note_read(pins[k].src, (int)P.steps.size() - 1);
        if (pins[k].in.op == I_STORE && def_step[pins[k].val] < 0)
          def_step[pins[k].val] = (int)P.steps.size() - 1;
      }
      g_first = pins.size();
      for (int v : live_vals) buf_of[v] = -1;
      reset_bufs();
    };
    for (int n : nodes) {
      const ENode& e = X[n];
      int ops[2] = {-1, -1};
      int na = arity(e.op);
      if (na >= 1) ops[0] = e.a;
      if (na == 2) ops[1] = e.b;
      auto in_group = [&](int v) { return v >= 0 && buf_of[v] >= 0; };
      int loads = 0, d = 0;
      for (int k = 0; k < na; ++k) {
        if (!in_group(ops[k]) && !(k == 1 && ops[1] == ops[0])) loads++;
        else if (in_group(ops[k])) d = std::max(d, depth[ops[k]]);
      }
      if (e.op == E_NEAR) d += 1;
      if ((int)free_bufs.size() < loads + 1 || d > pp.hmax) {
        close_group();
        loads = 0;
        for (int k = 0; k < na; ++k)
          if (!(k == 1 && ops[1] == ops[0])) loads++;
        d = e.op == E_NEAR ? 1 : 0;
      }
      if ((int)free_bufs.size() < loads + 1) { *err = "internal: group buffers exhausted"; return VL_ERR_INTERNAL; }
      for (int k = 0; k < na; ++k) {
        int v = ops[k];
        if (in_group(v)) continue;
        if (!mat[v]) { *err = "internal: operand not materialised"; return VL_ERR_INTERNAL; }
        int b = free_bufs.back(); free_bufs.pop_back();
        buf_of[v] = b; depth[v] = 0; live_vals.push_back(v);
        Insn l{}; l.op = I_LOAD; l.dst = (uint8_t)b; l.slot = -1;
        emit(l, v, v);
      }
      int b = free_bufs.back(); free_bufs.pop_back();
      Insn in{}; in.dst = (uint8_t)b; in.slot = -1;
      switch (e.op) {
        case E_TRUE: in.op = I_CONST; in.b = 1; break;
        case E_FALSE: in.op = I_CONST; in.b = 0; break;
        case E_THR: in.op = I_THR; in.b = (uint8_t)e.lt; in.img = (int16_t)e.img; in.ch = (int16_t)e.ch; in.t = e.t; break;
        case E_PCT: in.op = I_THR; in.b = (uint8_t)e.lt; in.img = (int16_t)e.img; in.ch = (int16_t)e.ch; in.slot = (int16_t)e.pct_slot; break;
        case E_NOT: in.op = I_NOT; in.a = (uint8_t)buf_of[e.a]; break;
        case E_NEAR: in.op = I_NEAR; in.a = (uint8_t)buf_of[e.a]; break;
        case E_AND: in.op = I_AND; in.a = (uint8_t)buf_of[e.a]; in.b = (uint8_t)buf_of[e.b]; break;
        case E_OR: in.op = I_OR; in.a = (uint8_t)buf_of[e.a]; in.b = (uint8_t)buf_of[e.b]; break;
        case E_ANDNOT: in.op = I_ANDNOT; in.a = (uint8_t)buf_of[e.a]; in.b = (uint8_t)buf_of[e.b]; break;
        case E_COPY: in.op = I_OR; in.a = (uint8_t)buf_of[e.a]; in.b = (uint8_t)buf_of[e.a]; break;
        default: *err = "internal: bad group op"; return VL_ERR_INTERNAL;
      }
      emit(in, n, -1);
      buf_of[n] = b; depth[n] = d; live_vals.push_back(n);
      if (needs_store[n]) emit_store(n);
      // release operands with no more uses in this level
      for (int k = 0; k < na; ++k) {
        int v = ops[k];
        if (k == 1 && v == ops[0]) continue;
        pending[v]--;
        if (pending[v] <= 0 && buf_of[v] >= 0) {
          free_bufs.push_back(buf_of[v]); buf_of[v] = -1;
          live_vals.erase(std::find(live_vals.begin(), live_vals.end(), v));
        }
      }
      if (pending[n] <= 0) {
        free_bufs.push_back(buf_of[n]); buf_of[n] = -1;
        live_vals.erase(std::find(live_vals.begin(), live_vals.end(), n));
      }
    }
    close_group();
    // ---- component selects of the next level, in batches
    std::vector<int> rzs;
    for (int i = 0; i < N; ++i)
      if (X[i].op == E_RZ && L[i] == level + 1) rzs.push_back(i);
    for (size_t k0 = 0; k0 < rzs.size(); k0 += MAX_RZ_BATCH) {
      // (selects of a batch take consecutive sets of the pool, round robin)
      int cnt = (int)std::min<size_t>(MAX_RZ_BATCH, rzs.size() - k0);
      int base_step = (int)P.steps.size();
      int rz_off = (int)P.rz.size();
      for (int j = 0; j < cnt; ++j) {
        int z = rzs[k0 + j];
        RzDesc r{}; r.phi1_slot = (int16_t)X[z].a; r.phi2_slot = (int16_t)X[z].b;  // value ids for now
        r.z_slot = (int16_t)z; r.scratch = (int16_t)((next_set + j) % pp.scratch_sets);
        P.rz.push_back(r);
        if (!mat[X[z].a] || !mat[X[z].b]) { *err = "internal: select operand not materialised"; return VL_ERR_INTERNAL; }
        note_read(X[z].a, base_step + 2);
        note_read(X[z].b, base_step + 2);
        mat[z] = 1;
        def_step[z] = base_step + 2;
      }
      // three phases: tile labelling, border merge, select (the seed flags
      // travel with the union-find keys, so no phase gathers them)
      for (int kind : {SK_RZ_LOCAL, SK_RZ_MERGE, SK_RZ_FINAL}) {
        StepDesc s{}; s.kind = kind; s.rz_off = rz_off; s.rz_cnt = cnt;
        P.steps.push_back(s);
      }
      next_set = (next_set + cnt) % pp.scratch_sets;
      n_selects_total += cnt;
      P.n_scratch_sets = std::min(pp.scratch_sets, n_selects_total);
    }
  }
  // roots must be materialised
  for (int r : P.exec_roots)
    if (!mat[r]) { *err = "internal: root not materialised"; return VL_ERR_INTERNAL; }

  // ---- 4. slots.  Roots: one dedicated slot per distinct root value; masks:
  // fixed slots; the rest: greedy interval colouring over steps.
  std::map<int, int> root_slot_of;
  std::vector<int> order;
  for (int v = 0; v < N; ++v)
    if (mat[v] && X[v].op != E_MASK && !is_root[v]) order.push_back(v);
  std::sort(order.begin(), order.end(), [&](int a, int b) { return def_step[a] < def_step[b]; });
  std::vector<int> slot_free_after;  // last step that reads the slot's current value
  for (int v : order) {
    int s = -1;
    for (size_t k = 0; k < slot_free_after.size(); ++k)
      if (slot_free_after[k] + pp.reuse_distance < def_step[v]) { s = (int)k; break; }
    if (s < 0) { s = (int)slot_free_after.size(); slot_free_after.push_back(0); }
    slot_free_after[s] = std::max(last_step[v], def_step[v]);
    slot_of[v] = s;
  }
  P.n_inter_slots = (int)slot_free_after.size();
  for (int r : P.exec_roots)
    if (!root_slot_of.count(r)) {
      int s = P.n_inter_slots + (int)root_slot_of.size();
      root_slot_of[r] = s;
      slot_of[r] = s;
    }
  P.n_root_slots = (int)root_slot_of.size();
  for (int r : P.exec_roots) P.root_slot.push_back(root_slot_of[r]);
  const int mask_base = P.n_inter_slots + P.n_root_slots;
  for (int v = 0; v < N; ++v)
    if (X[v].op == E_MASK) slot_of[v] = mask_base + mask_slot_idx[X[v].img];
  P.n_mask_slots = (int)mask_slot_idx.size();
  for (int v = 0; v < N; ++v)
    if (mat[v] && slot_of[v] < 0) { *err = "internal: slot missing"; return VL_ERR_INTERNAL; }
  if (mask_base + P.n_mask_slots > 32767) { *err = "formula needs too many mask slots"; return VL_ERR_FORMULA; }

  // resolve instructions, halos
  for (StepDesc& s : P.steps) {
    if (s.kind != SK_GROUP) continue;
    const int off = s.insn_off, cnt = s.insn_cnt;
    std::map<int, int> h;  // value -> halo
    for (int k = off + cnt - 1; k >= off; --k) {
      PendingInsn& p = pins[k];
      if (p.in.op == I_STORE) { h[p.val] = std::max(h[p.val], 0); continue; }
      int hv = h.count(p.val) ? h[p.val] : 0;
      p.in.h = (int16_t)hv;
      const ENode& e = X[p.val];
      if (p.in.op == I_LOAD || p.in.op == I_THR || p.in.op == I_CONST) continue;
      int inc = p.in.op == I_NEAR ? 1 : 0;
      if (arity(e.op) >= 1) h[e.a] = std::max(h.count(e.a) ? h[e.a] : 0, hv + inc);
      if (arity(e.op) == 2) h[e.b] = std::max(h.count(e.b) ? h[e.b] : 0, hv + inc);
    }
    int halo = 0;
    for (int k = off; k < off + cnt; ++k) {
      PendingInsn& p = pins[k];
      if (p.in.op == I_LOAD) { p.in.h = (int16_t)(h.count(p.val) ? h[p.val] : 0); p.in.slot = (int16_t)slot_of[p.src]; }
      if (p.in.op == I_STORE) { p.in.slot = (int16_t)slot_of[p.val]; p.in.h = 0; }
      halo = std::max(halo, (int)p.in.h);
    }
    if (halo > pp.hmax) { *err = "internal: halo above budget"; return VL_ERR_INTERNAL; }
    s.halo = halo;
    s.insn_off = (int)P.insns.size();
    for (int k = off; k < off + cnt; ++k) P.insns.push_back(pins[k].in);
    P.max_group_halo = std::max(P.max_group_halo, halo);
  }
  // ---- 5. rank codes.  A channel read by many constant thresholds gets a
  // table of its distinct thresholds; its thresholds become comparisons of
  // the pixels' rank codes (one pass over the floats per formula instead of
  // one per threshold and tile).  Thresholds from percentiles stay direct.
  {
    std::map<std::pair<int, int>, std::vector<float>> by_ch;
    for (const Insn& in : P.insns)
      if (in.op == I_THR && in.slot < 0 && !std::isnan(in.t)) by_ch[{in.img, in.ch}].push_back(in.t);
    std::map<std::pair<int, int>, int> tab_of;
    for (auto& kv : by_ch) {
      if ((int)kv.second.size() < kRankMinThresholds || (int)P.rtab.size() >= kRankMaxTables) continue;
      std::vector<float> v = kv.second;
      std::sort(v.begin(), v.end());
      v.erase(std::unique(v.begin(), v.end(), [](float x, float y) { return x == y; }), v.end());
      if ((int)v.size() > kRankMaxValues) continue;
      RankTab t{};
      t.img = kv.first.first;
      t.ch = kv.first.second;
      t.m = (int)v.size();
      t.nbits = 0;
      for (unsigned c = 2u * (unsigned)t.m + 1u; c; c >>= 1) t.nbits++;
      t.val_off = (int)P.rvals.size();
      t.plane0 = P.n_planes;
      P.n_planes += t.nbits + 1;
      P.rvals.insert(P.rvals.end(), v.begin(), v.end());
      tab_of[kv.first] = (int)P.rtab.size();
      P.rtab.push_back(t);
    }
    for (StepDesc& s : P.steps) {
      if (s.kind != SK_GROUP) continue;
      for (int k = s.insn_off; k < s.insn_off + s.insn_cnt; ++k) {
        Insn& in = P.insns[k];
        if (in.op != I_THR || in.slot >= 0 || std::isnan(in.t)) continue;
        auto it = tab_of.find({in.img, in.ch});
        if (it == tab_of.end()) continue;
        const RankTab& t = P.rtab[it->second];
        const float* v = P.rvals.data() + t.val_off;
        const int pos = (int)(std::lower_bound(v, v + t.m, in.t) - v);  // v[pos] == t
        const int kk = pos + 1;
        const bool lt = in.b & 1;
        in.op = I_RTHR;
        in.a = (uint8_t)it->second;
        in.img = (int16_t)(lt ? 2 * kk - 1 : 2 * kk);
        in.ch = (int16_t)t.nbits;
        in.slot = (int16_t)t.plane0;
        s.rank_mask |= 1 << it->second;
        s.rank_halo = std::max(s.rank_halo, (int)in.h);
      }
    }
    if (!P.rtab.empty()) {
      StepDesc r{};
      r.kind = SK_RANK;
      P.steps.insert(P.steps.begin(), r);
    }
  }
  // tile buffers each group uses (buffers are taken lowest first): the
  // executor places the stage of rank planes right after them
  for (StepDesc& s : P.steps) {
    if (s.kind != SK_GROUP) continue;
    int hi = 0;
    for (int k = s.insn_off; k < s.insn_off + s.insn_cnt; ++k) {
      const Insn& in = P.insns[k];
      const int op = insn_op(in);
      if (op != I_STORE) hi = std::max(hi, in.dst + 1);
      if (op == I_NOT || op == I_NEAR || op == I_AND || op == I_OR || op == I_ANDNOT ||
          op == I_STORE)
        hi = std::max(hi, in.a + 1);
      if (op == I_AND || op == I_OR || op == I_ANDNOT) hi = std::max(hi, in.b + 1);
    }
    s.n_bufs = hi;
  }
  // ---- 5b. block barriers inside groups.  Every instruction but the float
  // threshold writes (and a store reads) each buffer word from the thread
  // that owns it -- one fixed owner per buffer word -- so a value read at
  // its own word right after it was written needs no barrier.  A barrier
  // (bit I_SYNC of the opcode) goes before an instruction only where a
  // thread could touch a word another thread touched since the last one:
  // N reads the neighbours of its operand's words, and the float threshold
  // writes its words from the lanes that assembled them.  Tracked per
  // buffer since the last barrier: own-mapped writes, threshold writes,
  // own-word reads and neighbour reads.
  for (StepDesc& s : P.steps) {
    if (s.kind != SK_GROUP) continue;
    uint64_t w_own = 0, w_thr = 0, r_own = 0, r_nbr = 0;  // <= 64 buffers
    for (int k = s.insn_off; k < s.insn_off + s.insn_cnt; ++k) {
      Insn& in = P.insns[k];
      const uint64_t A = in.op == I_NOT || in.op == I_NEAR || in.op == I_STORE ? 1ull << in.a
                         : (in.op == I_AND || in.op == I_OR || in.op == I_ANDNOT)
                             ? (1ull << in.a) | (1ull << in.b)
                             : 0ull;
      const uint64_t D = in.op == I_STORE ? 0ull : 1ull << in.dst;
      bool need;
      if (in.op == I_NEAR) {
        if (in.a == in.dst) { *err = "internal: N in place"; return VL_ERR_INTERNAL; }
        need = (A & (w_own | w_thr)) || (D & (r_nbr | w_thr));
      } else if (in.op == I_THR) {
        need = D & (w_own | w_thr | r_own | r_nbr);
      } else {
        need = (A & w_thr) || (D & (r_nbr | w_thr));
      }
      if (need) {
        in.op |= I_SYNC;
        w_own = w_thr = r_own = r_nbr = 0;
      }
      if ((in.op & ~I_SYNC) == I_NEAR) r_nbr |= A;
      else r_own |= A;
      if ((in.op & ~I_SYNC) == I_THR) w_thr |= D;
      else w_own |= D;
    }
  }
  // ---- 6. number terms run first: everything that compares them waits
  if (!P.arith.empty()) {
    StepDesc a{};
    a.kind = SK_ARITH;
    a.insn_cnt = (int)P.arith.size();
    P.steps.insert(P.steps.begin(), a);
  }
  for (RzDesc& r : P.rz) {
    r.phi1_slot = (int16_t)slot_of[r.phi1_slot];
    r.phi2_slot = (int16_t)slot_of[r.phi2_slot];
    r.z_slot = (int16_t)slot_of[r.z_slot];
  }
  // ---- 7. step dependencies.  Slots are reused by liveness, so besides
  // reads after writes a step must also follow the readers and the writer of
  // the previous value of every slot it writes.  Pseudo slots stand for the
  // rank planes, the percentile values and each select scratch set.
  {
    const int n = (int)P.steps.size();
    const int n_real = P.n_inter_slots + P.n_root_slots + P.n_mask_slots;
    const int ps_rank = n_real, ps_pct = n_real + 1, ps_num = n_real + 2, ps_scr = n_real + 3;
    const int first_num = (int)P.img_kind.size();
    std::vector<std::vector<int>> R(n), Wr(n);
    for (int i = 0; i < n; ++i) {
      const StepDesc& s = P.steps[i];
      switch (s.kind) {
        case SK_GROUP:
          for (int k = s.insn_off; k < s.insn_off + s.insn_cnt; ++k) {
            const Insn& in = P.insns[k];
            const int op = insn_op(in);
            if (op == I_LOAD) R[i].push_back(in.slot);
            if (op == I_STORE) Wr[i].push_back(in.slot);
            if (op == I_RTHR) R[i].push_back(ps_rank);
            if (op == I_THR && in.slot >= 0) R[i].push_back(ps_pct);
            if (op == I_THR && in.img >= first_num) R[i].push_back(ps_num);
          }
          break;
        case SK_PCT:
          Wr[i].push_back(ps_pct);
          for (const PctDesc& d : P.pct)
            if (d.img >= first_num) R[i].push_back(ps_num);
          break;
        case SK_RANK:
          Wr[i].push_back(ps_rank);
          for (const RankTab& t : P.rtab)
            if (t.img >= first_num) R[i].push_back(ps_num);
          break;
        case SK_ARITH: Wr[i].push_back(ps_num); break;
        default:
          for (int j = 0; j < s.rz_cnt; ++j) {
            const RzDesc& r = P.rz[s.rz_off + j];
            if (s.kind == SK_RZ_LOCAL || s.kind == SK_RZ_FINAL) {
              R[i].push_back(r.phi1_slot);
              R[i].push_back(r.phi2_slot);
            }
            if (s.kind == SK_RZ_LOCAL) Wr[i].push_back(ps_scr + r.scratch);
            else R[i].push_back(ps_scr + r.scratch);
            if (s.kind == SK_RZ_FINAL) Wr[i].push_back(r.z_slot);
          }
          break;
      }
    }
    std::map<int, int> last_w;
    std::map<int, std::vector<int>> readers;
    P.dep_off.assign(1, 0);
    P.deps.clear();
    for (int i = 0; i < n; ++i) {
      std::vector<int> d;
      const int kind = P.steps[i].kind;
      if (kind == SK_RZ_MERGE || kind == SK_RZ_FINAL) d.push_back(i - 1);
      for (int sl : R[i]) {
        auto it = last_w.find(sl);
        if (it != last_w.end()) d.push_back(it->second);
      }
      for (int sl : Wr[i]) {
        for (int rd : readers[sl])
          if (rd != i) d.push_back(rd);
        auto it = last_w.find(sl);
        if (it != last_w.end()) d.push_back(it->second);
      }
      for (int sl : Wr[i]) { readers[sl].clear(); last_w[sl] = i; }
      for (int sl : R[i]) readers[sl].push_back(i);
      std::sort(d.begin(), d.end());
      d.erase(std::unique(d.begin(), d.end()), d.end());
      for (int x : d)
        if (x < i) P.deps.push_back(x);
      P.dep_off.push_back((int32_t)P.deps.size());
    }
  }
  *out = std::move(P);
  return VL_OK;
}

}  // namespace vl
