// Host check of the vertex-partial identities of heget.cuh: every amplitude
// vertex equals the contraction of any one of its wavefunctions with the
// partial built from the others (vvvxxx, ggggxx, iovxx0 of arXiv:0909.5257,
// Sec. 4), on random complex wavefunctions and momenta in double precision.
// Prints the largest relative deviation; exit status 0.
#define MEA_HD inline
#include <cmath>
#include <cstdio>
#include <initializer_list>
#include <random>

#include "heget.cuh"

typedef cx<double> C;
typedef W4<double> V;

static std::mt19937_64 rng(0x09095257);
static double u() { return std::uniform_real_distribution<double>(-1.0, 1.0)(rng); }
static V rv() {
  V v;
  for (int k = 0; k < 4; ++k) v.c[k] = C{u(), u()};
  return v;
}
static double worst = 0.0;
static void cmp(C a, C b, double scale) {
  double d = std::hypot(a.r - b.r, a.i - b.i) / scale;
  if (d > worst) worst = d;
}
// product of the 1-norms of the wavefunctions: bounds every term of a vertex
static double mag(std::initializer_list<const V*> vs) {
  double s = 1.0;
  for (const V* v : vs) {
    double m = 0;
    for (int k = 0; k < 4; ++k) m += std::hypot(v->c[k].r, v->c[k].i);
    s *= m;
  }
  return s;
}

int main() {
  const double g = 1.2177, gg = g * g;
  for (int trial = 0; trial < 2000; ++trial) {
    V a = rv(), b = rv(), c = rv(), d = rv();
    double pa[4], pb[4], pc[4];
    for (int m = 0; m < 4; ++m) { pb[m] = u(); pc[m] = u(); pa[m] = -(pb[m] + pc[m]); }
    const double s3 = mag({&a, &b, &c}) * 8;
    // vvvxxx with each argument free (cyclic shift)
    C ref = vvv_amp(a, b, c, pa, pb, pc, g);
    cmp(part_contract(a, vvv_part(b, c, pa, pb, pc, g), false, false), ref, s3);
    cmp(part_contract(b, vvv_part(c, a, pb, pc, pa, g), false, false), ref, s3);
    cmp(part_contract(c, vvv_part(a, b, pc, pa, pb, g), false, false), ref, s3);
    // ggggxx: a.G(b,c,d) = b.G(a,d,c) = c.G(d,a,b) = d.G(c,b,a), G(x,y,z) = -G(x,z,y)
    const double s4 = mag({&a, &b, &c, &d}) * gg;
    ref = gggg_amp(a, b, c, d, gg);
    cmp(part_contract(a, gggg_part(b, c, d, gg), false, false), ref, s4);
    cmp(part_contract(b, gggg_part(a, d, c, gg), false, false), ref, s4);
    cmp(part_contract(c, gggg_part(d, a, b, gg), false, false), ref, s4);
    cmp(part_contract(d, gggg_part(c, b, a, gg), false, false), ref, s4);
    cmp(part_contract(a, gggg_part(b, d, c, gg), false, true), ref, s4);
    // iovxx0(fi, fo, V) with fi, fo or V free
    ref = iov_amp(a, b, c, g);
    cmp(part_contract(a, iov_part_i(b, c, g), true, false), ref, s3);
    cmp(part_contract(b, iov_part_o(a, c, g), true, false), ref, s3);
    cmp(part_contract(c, iov_part_v(a, b, g), false, false), ref, s3);
  }
  std::printf("%.3e\n", worst);
  return 0;
}
