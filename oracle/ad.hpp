// Differentiation types for the oracle's adjoint pins. TEST INFRASTRUCTURE
// ONLY (see amr_oracle.cpp).
//
// Rev: reverse mode. Every arithmetic result with an active operand appends a
// node (two parents, two partial derivatives) to one global tape; sweeping the
// tape backwards from seeded final values gives the exact transpose of the
// linearised forward map, operation by operation.
// Tan: forward mode with one tangent direction (the same derivatives pushed
// forwards), for the dot-product test of the reverse sweep.
//
// Branches (comparisons, minmod, HLLD cases, upwinding) follow the values, so
// the derivative is the one of the branch the forward took; |x| has
// derivative sign(x) (0 at 0).
#pragma once
#include <cmath>
#include <cstdint>
#include <vector>

namespace oracle {

struct Tape {
  std::vector<int32_t> pa, pb;
  std::vector<double> da, db;
  int32_t push(int32_t a, double x, int32_t b, double y) {
    pa.push_back(a);
    da.push_back(x);
    pb.push_back(b);
    db.push_back(y);
    return (int32_t)(pa.size() - 1);
  }
  int32_t input() { return push(-1, 0.0, -1, 0.0); }
  void clear() { pa.clear(); pb.clear(); da.clear(); db.clear(); }
  size_t size() const { return pa.size(); }
  // adj holds seeded adjoints of every node; accumulates into the parents
  void sweep(std::vector<double>& adj) const {
    for (size_t n = pa.size(); n-- > 0;) {
      const double g = adj[n];
      if (g == 0.0) continue;
      if (pa[n] >= 0) adj[pa[n]] += da[n] * g;
      if (pb[n] >= 0) adj[pb[n]] += db[n] * g;
    }
  }
};

inline Tape& tape() {
  static Tape t;
  return t;
}

struct Rev {
  double v;
  int32_t i;
  Rev() : v(0.0), i(-1) {}
  Rev(double x) : v(x), i(-1) {}
};
inline Rev rnode(double v, int32_t a, double da, int32_t b, double db) {
  Rev r(v);
  if (a >= 0 || b >= 0) r.i = tape().push(a, da, b, db);
  return r;
}
inline Rev operator+(Rev x, Rev y) { return rnode(x.v + y.v, x.i, 1.0, y.i, 1.0); }
inline Rev operator-(Rev x, Rev y) { return rnode(x.v - y.v, x.i, 1.0, y.i, -1.0); }
inline Rev operator*(Rev x, Rev y) { return rnode(x.v * y.v, x.i, y.v, y.i, x.v); }
inline Rev operator/(Rev x, Rev y) {
  const double q = x.v / y.v;
  return rnode(q, x.i, 1.0 / y.v, y.i, -q / y.v);
}
inline Rev operator-(Rev x) { return rnode(-x.v, x.i, -1.0, -1, 0.0); }
inline Rev& operator+=(Rev& x, Rev y) { x = x + y; return x; }
inline Rev& operator-=(Rev& x, Rev y) { x = x - y; return x; }
inline bool operator>(Rev x, Rev y) { return x.v > y.v; }
inline bool operator<(Rev x, Rev y) { return x.v < y.v; }
inline bool operator>=(Rev x, Rev y) { return x.v >= y.v; }
inline bool operator<=(Rev x, Rev y) { return x.v <= y.v; }
inline bool operator==(Rev x, Rev y) { return x.v == y.v; }
inline bool operator!=(Rev x, Rev y) { return x.v != y.v; }
inline Rev sqrt(Rev x) {
  const double r = std::sqrt(x.v);
  return rnode(r, x.i, 0.5 / r, -1, 0.0);
}
inline Rev fabs(Rev x) { return rnode(std::fabs(x.v), x.i, x.v > 0 ? 1.0 : (x.v < 0 ? -1.0 : 0.0), -1, 0.0); }

struct Tan {
  double v, d;
  Tan() : v(0.0), d(0.0) {}
  Tan(double x) : v(x), d(0.0) {}
  Tan(double x, double t) : v(x), d(t) {}
};
inline Tan operator+(Tan x, Tan y) { return Tan(x.v + y.v, x.d + y.d); }
inline Tan operator-(Tan x, Tan y) { return Tan(x.v - y.v, x.d - y.d); }
inline Tan operator*(Tan x, Tan y) { return Tan(x.v * y.v, x.d * y.v + x.v * y.d); }
inline Tan operator/(Tan x, Tan y) {
  const double q = x.v / y.v;
  return Tan(q, (x.d - q * y.d) / y.v);
}
inline Tan operator-(Tan x) { return Tan(-x.v, -x.d); }
inline Tan& operator+=(Tan& x, Tan y) { x = x + y; return x; }
inline Tan& operator-=(Tan& x, Tan y) { x = x - y; return x; }
inline bool operator>(Tan x, Tan y) { return x.v > y.v; }
inline bool operator<(Tan x, Tan y) { return x.v < y.v; }
inline bool operator>=(Tan x, Tan y) { return x.v >= y.v; }
inline bool operator<=(Tan x, Tan y) { return x.v <= y.v; }
inline bool operator==(Tan x, Tan y) { return x.v == y.v; }
inline bool operator!=(Tan x, Tan y) { return x.v != y.v; }
inline Tan sqrt(Tan x) {
  const double r = std::sqrt(x.v);
  return Tan(r, 0.5 * x.d / r);
}
inline Tan fabs(Tan x) { return Tan(std::fabs(x.v), x.v > 0 ? x.d : (x.v < 0 ? -x.d : 0.0)); }

}  // namespace oracle
