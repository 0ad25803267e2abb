// Host check of the double-float primitives in csrc/df.cuh: sums of products
// accumulated with df_acc_prod against the exact value computed in long double
// (x86) or double-double-free rational bounds.  Prints the worst relative
// error; the pytest wrapper asserts it.  Build: g++ -O2 -ffp-contract=off.
#include <cstdio>
#include <cstdlib>
#include <random>
#include "../../paper_2603_25691_gb300/csrc/df.cuh"

using cphifi::df;

int main(int argc, char** argv) {
  std::mt19937_64 rng(12345);
  std::normal_distribution<double> N(0.0, 1.0);
  double worst_dot = 0.0, worst_prod = 0.0, worst_split = 0.0;
  for (int trial = 0; trial < 2000; ++trial) {
    const int k = 1 + (int)(rng() % 2000);
    df acc{0.f, 0.f};
    // reference: exact-ish sum with long double and Kahan (the inputs are
    // double-float values, so each product is exact in 53+ bits? no: 48x48
    // bits; long double on x86 has 64, elsewhere we rely on the bound check)
    long double ref = 0.0L, mag = 0.0L;
    for (int i = 0; i < k; ++i) {
      const df x = cphifi::df_from_double(N(rng));
      const df y = cphifi::df_from_double(N(rng) * 3.0);
      cphifi::df_acc_prod(acc, x, y);
      const long double xv = (long double)x.hi + (long double)x.lo;
      const long double yv = (long double)y.hi + (long double)y.lo;
      ref += xv * yv;
      mag += (xv * yv < 0 ? -xv * yv : xv * yv);
    }
    const df s = cphifi::df_norm(acc);
    const long double got = (long double)s.hi + (long double)s.lo;
    const double err = (double)((got - ref) / mag);
    if (std::abs(err) > worst_dot) worst_dot = std::abs(err);
    const double a = N(rng), b = N(rng);
    const df pa = cphifi::df_from_double(a), pb = cphifi::df_from_double(b);
    const df pr = cphifi::df_mul(pa, pb);
    const long double exact = ((long double)pa.hi + pa.lo) * ((long double)pb.hi + pb.lo);
    const double perr = (double)((((long double)pr.hi + pr.lo) - exact) / exact);
    if (std::abs(perr) > worst_prod) worst_prod = std::abs(perr);
    const double serr = std::abs((cphifi::df_to_double(pa) - a) / a);
    if (serr > worst_split) worst_split = serr;
  }
  std::printf("%.3e %.3e %.3e\n", worst_dot, worst_prod, worst_split);
  return 0;
}
