// Counting-scalar build of the oracle -- test infrastructure only.
//
// The oracle's own C source (z4c_oracle.c, unchanged) compiled as C++ with its
// floating-point type replaced by a scalar that performs the same IEEE double
// operation and counts it: the results are the oracle's to the bit (same
// operations in the same order, no contraction), and the counts are the FP64
// operations of the method as the oracle evaluates it, point by point.
//
//   flop_count <nx> <ny> <nz> <dx> <input.bin> <output.bin>
//
// input.bin: the patch array (25 x (nz+6) x (ny+6) x (nx+6) doubles); the
// program writes the Z4c right-hand side (sources + advection + dissipation,
// the paper's default parameters) to output.bin and prints one JSON line of
// operation counts per active point: the whole right-hand side, its three
// parts, and one RK4 stage of the 5-pass kind (right-hand side, update,
// algebraic constraints; stage 2).
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <vector>

namespace cnt {
struct Counts {
  long long add = 0, mul = 0, div = 0, sqrt = 0, other = 0;
};
Counts C;
}  // namespace cnt

struct Real {
  double v;
  Real() = default;
  Real(double x) : v(x) {}
  Real(int x) : v((double)x) {}
  Real(long x) : v((double)x) {}
  Real(long long x) : v((double)x) {}
  Real(unsigned x) : v((double)x) {}
  Real(unsigned long x) : v((double)x) {}
  explicit operator double() const { return v; }
  explicit operator int() const { return (int)v; }
  explicit operator long() const { return (long)v; }
  explicit operator long long() const { return (long long)v; }
  Real& operator+=(Real b) {
    ++cnt::C.add;
    v += b.v;
    return *this;
  }
  Real& operator-=(Real b) {
    ++cnt::C.add;
    v -= b.v;
    return *this;
  }
  Real& operator*=(Real b) {
    ++cnt::C.mul;
    v *= b.v;
    return *this;
  }
  Real& operator/=(Real b) {
    ++cnt::C.div;
    v /= b.v;
    return *this;
  }
};
inline Real operator+(Real a, Real b) {
  ++cnt::C.add;
  return Real(a.v + b.v);
}
inline Real operator-(Real a, Real b) {
  ++cnt::C.add;
  return Real(a.v - b.v);
}
inline Real operator*(Real a, Real b) {
  ++cnt::C.mul;
  return Real(a.v * b.v);
}
inline Real operator/(Real a, Real b) {
  ++cnt::C.div;
  return Real(a.v / b.v);
}
inline Real operator-(Real a) { return Real(-a.v); }
inline Real operator+(Real a) { return a; }
inline bool operator<(Real a, Real b) { return a.v < b.v; }
inline bool operator>(Real a, Real b) { return a.v > b.v; }
inline bool operator<=(Real a, Real b) { return a.v <= b.v; }
inline bool operator>=(Real a, Real b) { return a.v >= b.v; }
inline bool operator==(Real a, Real b) { return a.v == b.v; }
inline bool operator!=(Real a, Real b) { return a.v != b.v; }
inline Real sqrt(Real a) {
  ++cnt::C.sqrt;
  return Real(std::sqrt(a.v));
}
inline Real cbrt(Real a) {
  ++cnt::C.other;
  return Real(std::cbrt(a.v));
}
inline Real pow(Real a, Real b) {
  ++cnt::C.other;
  return Real(std::pow(a.v, b.v));
}
inline Real exp(Real a) {
  ++cnt::C.other;
  return Real(std::exp(a.v));
}
inline Real log(Real a) {
  ++cnt::C.other;
  return Real(std::log(a.v));
}
inline Real sin(Real a) {
  ++cnt::C.other;
  return Real(std::sin(a.v));
}
inline Real cos(Real a) {
  ++cnt::C.other;
  return Real(std::cos(a.v));
}
inline Real acos(Real a) {
  ++cnt::C.other;
  return Real(std::acos(a.v));
}
inline Real atan2(Real a, Real b) {
  ++cnt::C.other;
  return Real(std::atan2(a.v, b.v));
}
inline Real fabs(Real a) { return Real(std::fabs(a.v)); }
inline Real floor(Real a) { return Real(std::floor(a.v)); }
inline Real fmax(Real a, Real b) { return Real(std::fmax(a.v, b.v)); }
inline Real fmin(Real a, Real b) { return Real(std::fmin(a.v, b.v)); }
inline bool isfinite(Real a) { return std::isfinite(a.v); }

#define double Real
#include "z4c_oracle.c"
#undef double

static double per_point(cnt::Counts a, cnt::Counts b, long long n, const char* name, bool last) {
  const double add = (double)(b.add - a.add) / n, mul = (double)(b.mul - a.mul) / n,
               dv = (double)(b.div - a.div) / n, sq = (double)(b.sqrt - a.sqrt) / n,
               ot = (double)(b.other - a.other) / n;
  printf("\"%s\": {\"add\": %.2f, \"mul\": %.2f, \"div\": %.2f, \"sqrt\": %.2f, \"other\": %.2f, \"flops\": %.2f}%s",
         name, add, mul, dv, sq, ot, add + mul + dv + sq + ot, last ? "" : ", ");
  return add + mul + dv + sq + ot;
}

int main(int argc, char** argv) {
  if (argc != 7) {
    fprintf(stderr, "usage: flop_count nx ny nz dx input.bin output.bin\n");
    return 2;
  }
  orc_patch p;
  p.n[0] = atoi(argv[1]);
  p.n[1] = atoi(argv[2]);
  p.n[2] = atoi(argv[3]);
  p.g = 3;
  p.dx = Real(atof(argv[4]));
  p.origin[0] = Real(-0.5 * p.n[0] * atof(argv[4]));
  p.origin[1] = Real(-0.5 * p.n[1] * atof(argv[4]));
  p.origin[2] = Real(-0.5 * p.n[2] * atof(argv[4]));
  const size_t np = (size_t)NF * (p.n[0] + 6) * (p.n[1] + 6) * (p.n[2] + 6);
  std::vector<double> in(np), out(np);
  FILE* f = fopen(argv[5], "rb");
  if (!f || fread(in.data(), sizeof(double), np, f) != np) return 3;
  fclose(f);
  std::vector<Real> u(np), r(np), y(np), s2(np);
  for (size_t i = 0; i < np; ++i) u[i] = Real(in[i]);
  orc_params prm;
  prm.kappa1 = Real(0.005);
  prm.kappa2 = Real(0.0);
  prm.eta = Real(0.36);
  prm.sigma_ko = Real(0.5);
  prm.w_floor = Real(1e-10);
  prm.lapse = 0;
  prm.shift = 0;
  prm.lapse_uses_khat = 0;
  const long long npts = (long long)p.n[0] * p.n[1] * p.n[2];
  cnt::Counts c0 = cnt::C;
  orc_z4c_rhs_terms(&p, &prm, u.data(), r.data(), 7);
  cnt::Counts c1 = cnt::C;
  for (size_t i = 0; i < np; ++i) out[i] = r[i].v;
  std::vector<Real> tmp(np);
  orc_z4c_rhs_terms(&p, &prm, u.data(), tmp.data(), 1);
  cnt::Counts c2 = cnt::C;
  orc_z4c_rhs_terms(&p, &prm, u.data(), tmp.data(), 2);
  cnt::Counts c3 = cnt::C;
  orc_z4c_rhs_terms(&p, &prm, u.data(), tmp.data(), 4);
  cnt::Counts c4 = cnt::C;
  for (size_t i = 0; i < np; ++i) y[i] = u[i];
  orc_rk4_stage(&p, &prm, 2, Real(0.1), 0, u.data(), u.data(), y.data(), s2.data());
  cnt::Counts c5 = cnt::C;
  printf("{\"points\": %lld, ", npts);
  per_point(c0, c1, npts, "rhs", false);
  per_point(c1, c2, npts, "sources", false);
  per_point(c2, c3, npts, "advection", false);
  per_point(c3, c4, npts, "dissipation", false);
  per_point(c4, c5, npts, "rk4_stage_2", true);
  printf("}\n");
  f = fopen(argv[6], "wb");
  if (!f || fwrite(out.data(), sizeof(double), np, f) != np) return 4;
  fclose(f);
  return 0;
}
