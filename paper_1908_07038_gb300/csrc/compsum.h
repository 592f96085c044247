// Compensated (Dot2-style) accumulation for the host geometry builders:
// error-free transformations of Ogita, Rump and Oishi (2005), TwoSum and
// TwoProduct through fma, accumulated as a sum plus a running correction.
#pragma once

#include <cmath>

namespace atlasgb {

inline void tsum(double a, double b, double& s, double& e) {
  s = a + b;
  double z = s - a;
  e = (a - (s - z)) + (b - z);
}
inline void tprod(double a, double b, double& p, double& e) {
  p = a * b;
  e = std::fma(a, b, -p);
}
struct Comp {
  double s = 0, c = 0;
  void add(double x) {
    double t, e;
    tsum(s, x, t, e);
    s = t;
    c += e;
  }
  void add_prod(double x, double y) {
    double p, e;
    tprod(x, y, p, e);
    add(p);
    c += e;
  }
  double value() const { return s + c; }
};

}  // namespace atlasgb
