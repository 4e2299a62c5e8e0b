// TEST INFRASTRUCTURE ONLY.  Scalar types the checker's model is
// instantiated on:
//   * double  : the plain FP64 reference;
//   * Var     : FP64 reverse mode by a Wengert tape (one tape per thread);
//   * Cnt     : FP64 that counts the non-trivial floating operations it does.
// Nothing here is shared with, or imported by, the CUDA library.
#pragma once
#include <cmath>
#include <cstdint>
#include <vector>

namespace orc {

// ---------------------------------------------------------------------------
// Reverse mode.  Every operation on Var appends one node holding the local
// partials with respect to its (at most two) operands.  A Var with idx < 0 is
// a constant.  The subgradient conventions of the piecewise operations are
// those of the rollout's reading: clamp passes the gradient where
// lo <= x <= hi (bounds included), sqrt(0) has derivative 0, and comparisons
// (branch choices, sign flips) are treated as constants.
// ---------------------------------------------------------------------------
struct Node {
  int32_t a, b;
  double da, db;
};

struct Tape {
  std::vector<Node> nodes;
  int32_t push(int32_t a, double da, int32_t b, double db) {
    nodes.push_back(Node{a, b, da, db});
    return (int32_t)nodes.size() - 1;
  }
  void clear() { nodes.clear(); }
  // adj must be sized nodes.size(); seeds already placed.  Sweeps backwards.
  void backprop(std::vector<double>& adj) const {
    for (int64_t i = (int64_t)nodes.size() - 1; i >= 0; --i) {
      const double g = adj[i];
      if (g == 0.0) continue;
      const Node& n = nodes[i];
      if (n.a >= 0) adj[n.a] += n.da * g;
      if (n.b >= 0) adj[n.b] += n.db * g;
    }
  }
};

extern thread_local Tape* g_tape;

struct Var {
  double v;
  int32_t idx;
  Var() : v(0.0), idx(-1) {}
  Var(double x) : v(x), idx(-1) {}  // constants carry no gradient
  static Var leaf(double x) {
    Var r;
    r.v = x;
    r.idx = g_tape->push(-1, 0.0, -1, 0.0);
    return r;
  }
};

inline Var mk(double v, int32_t a, double da, int32_t b, double db) {
  Var r;
  r.v = v;
  if (a < 0 && b < 0) {
    r.idx = -1;
  } else {
    r.idx = g_tape->push(a, da, b, db);
  }
  return r;
}
inline Var operator+(Var x, Var y) { return mk(x.v + y.v, x.idx, 1.0, y.idx, 1.0); }
inline Var operator-(Var x, Var y) { return mk(x.v - y.v, x.idx, 1.0, y.idx, -1.0); }
inline Var operator*(Var x, Var y) { return mk(x.v * y.v, x.idx, y.v, y.idx, x.v); }
inline Var operator/(Var x, Var y) {
  const double q = x.v / y.v;
  return mk(q, x.idx, 1.0 / y.v, y.idx, -q / y.v);
}
inline Var operator-(Var x) { return mk(-x.v, x.idx, -1.0, -1, 0.0); }
inline Var& operator+=(Var& x, Var y) { x = x + y; return x; }
inline Var& operator-=(Var& x, Var y) { x = x - y; return x; }
inline Var& operator*=(Var& x, Var y) { x = x * y; return x; }
inline Var sqrt(Var x) {
  const double s = std::sqrt(x.v);
  return mk(s, x.idx, s > 0.0 ? 0.5 / s : 0.0, -1, 0.0);
}
inline Var cos(Var x) { return mk(std::cos(x.v), x.idx, -std::sin(x.v), -1, 0.0); }
inline Var sin(Var x) { return mk(std::sin(x.v), x.idx, std::cos(x.v), -1, 0.0); }
inline double val(Var x) { return x.v; }

// ---------------------------------------------------------------------------
// Operation counter.  Counts adds/subs, muls, divs and sqrts whose result is
// not trivially given by an operand (x*1, x*0, x+0 and negation are free), so
// the count reflects the arithmetic the step needs, not how it is spelled.
// ---------------------------------------------------------------------------
struct OpCount {
  int64_t add = 0, mul = 0, div = 0, sqrt = 0, trig = 0, cmp = 0;
};
extern thread_local OpCount g_count;

struct Cnt {
  double v;
  Cnt() : v(0.0) {}
  Cnt(double x) : v(x) {}
};
inline Cnt operator+(Cnt x, Cnt y) {
  if (x.v != 0.0 && y.v != 0.0) g_count.add++;
  return Cnt(x.v + y.v);
}
inline Cnt operator-(Cnt x, Cnt y) {
  if (x.v != 0.0 && y.v != 0.0) g_count.add++;
  return Cnt(x.v - y.v);
}
inline Cnt operator*(Cnt x, Cnt y) {
  const bool triv = x.v == 0.0 || y.v == 0.0 || x.v == 1.0 || y.v == 1.0 || x.v == -1.0 || y.v == -1.0;
  if (!triv) g_count.mul++;
  return Cnt(x.v * y.v);
}
inline Cnt operator/(Cnt x, Cnt y) {
  if (!(y.v == 1.0 || x.v == 0.0)) g_count.div++;
  return Cnt(x.v / y.v);
}
inline Cnt operator-(Cnt x) { return Cnt(-x.v); }
inline Cnt& operator+=(Cnt& x, Cnt y) { x = x + y; return x; }
inline Cnt& operator-=(Cnt& x, Cnt y) { x = x - y; return x; }
inline Cnt& operator*=(Cnt& x, Cnt y) { x = x * y; return x; }
inline Cnt sqrt(Cnt x) { g_count.sqrt++; return Cnt(std::sqrt(x.v)); }
inline Cnt cos(Cnt x) { g_count.trig++; return Cnt(std::cos(x.v)); }
inline Cnt sin(Cnt x) { g_count.trig++; return Cnt(std::sin(x.v)); }
inline Cnt tan(Cnt x) { g_count.trig++; return Cnt(std::tan(x.v)); }
inline Cnt atan2(Cnt y, Cnt x) { g_count.trig++; return Cnt(std::atan2(y.v, x.v)); }
inline double val(Cnt x) { g_count.cmp++; return x.v; }

inline double val(double x) { return x; }
inline double sqrt(double x) { return std::sqrt(x); }
inline double tan(double x) { return std::tan(x); }
inline double atan2(double y, double x) { return std::atan2(y, x); }

}  // namespace orc
