// Host check of the gluon vertex functions of heget.cuh and of the
// vertex-partial identities, on random complex wavefunctions and momenta in
// double precision:
//  * vvvxxx and jvvxx0 against the three-gluon Feynman rule of Sec. 4.1,
//    Gamma^{mu nu rho} = g^{mu nu}(k1-k2)^rho + g^{nu rho}(k2-k3)^mu +
//    g^{rho mu}(k3-k1)^nu, built here as an explicit rank-3 tensor and
//    contracted index by index with the metric diag(1,-1,-1,-1);
//  * ggggxx and jgggx0 against the quartic structure of Sec. 4.2,
//    g^{mu sigma} g^{nu rho} - g^{mu rho} g^{nu sigma}, as an explicit rank-4
//    tensor;
//  * every amplitude vertex (vvvxxx, ggggxx, iovxx0) equals the contraction of
//    any one of its wavefunctions with the partial built from the others.
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

static const double kEta[4] = {1.0, -1.0, -1.0, -1.0};

// Gamma^{mu nu rho}(k1, k2, k3) with all indices up, as an explicit array
static void ggg_tensor(const double* k1, const double* k2, const double* k3, double T[4][4][4]) {
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu)
      for (int rho = 0; rho < 4; ++rho) {
        double v = 0.0;
        if (mu == nu) v += kEta[mu] * (k1[rho] - k2[rho]);
        if (nu == rho) v += kEta[nu] * (k2[mu] - k3[mu]);
        if (rho == mu) v += kEta[rho] * (k3[nu] - k1[nu]);
        T[mu][nu][rho] = v;
      }
}
// -g Gamma_{mu nu rho} x^mu y^nu z^rho (every index lowered with the metric)
static C ggg_full(const V& x, const V& y, const V& z, const double* k1, const double* k2, const double* k3,
                  double g) {
  double T[4][4][4];
  ggg_tensor(k1, k2, k3, T);
  C s{0.0, 0.0};
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu)
      for (int rho = 0; rho < 4; ++rho)
        s = s + (T[mu][nu][rho] * kEta[mu] * kEta[nu] * kEta[rho]) * (x.c[mu] * y.c[nu] * z.c[rho]);
  return (-g) * s;
}
// current (-g / q^2) Gamma^{mu}_{nu rho}(-(kx+ky), kx, ky) x^nu y^rho
static V ggg_current(const V& x, const V& y, const double* kx, const double* ky, double inv_q2, double g) {
  double k1[4], T[4][4][4];
  for (int m = 0; m < 4; ++m) k1[m] = -(kx[m] + ky[m]);
  ggg_tensor(k1, kx, ky, T);
  V j;
  for (int mu = 0; mu < 4; ++mu) {
    C s{0.0, 0.0};
    for (int nu = 0; nu < 4; ++nu)
      for (int rho = 0; rho < 4; ++rho) s = s + (T[mu][nu][rho] * kEta[nu] * kEta[rho]) * (x.c[nu] * y.c[rho]);
    j.c[mu] = (-g * inv_q2) * s;
  }
  return j;
}
// quartic structure Q_{mu nu rho sigma} = g_{mu sigma} g_{nu rho} - g_{mu rho} g_{nu sigma}
static double quartic(int mu, int nu, int rho, int sg) {
  return (mu == sg && nu == rho ? kEta[mu] * kEta[nu] : 0.0) - (mu == rho && nu == sg ? kEta[mu] * kEta[nu] : 0.0);
}
static C gggg_full(const V& a, const V& b, const V& c, const V& d, double gg) {
  C s{0.0, 0.0};
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu)
      for (int rho = 0; rho < 4; ++rho)
        for (int sg = 0; sg < 4; ++sg) {
          const double q = quartic(mu, nu, rho, sg);
          if (q != 0.0) s = s + q * (a.c[mu] * b.c[nu] * c.c[rho] * d.c[sg]);
        }
  return gg * s;
}
// current of one structure: the open slot first, (gg / q^2) Q^{mu}_{nu rho sigma} a^nu b^rho c^sigma
static V gggg_current(const V& a, const V& b, const V& c, double inv_q2, double gg) {
  V j;
  for (int mu = 0; mu < 4; ++mu) {
    C s{0.0, 0.0};
    for (int nu = 0; nu < 4; ++nu)
      for (int rho = 0; rho < 4; ++rho)
        for (int sg = 0; sg < 4; ++sg) {
          const double q = quartic(mu, nu, rho, sg) * kEta[mu];  // raise the open index
          if (q != 0.0) s = s + q * (a.c[nu] * b.c[rho] * c.c[sg]);
        }
    j.c[mu] = (gg * inv_q2) * s;
  }
  return j;
}
static void cmpv(const V& a, const V& b, double scale) {
  for (int m = 0; m < 4; ++m) cmp(a.c[m], b.c[m], scale);
}

int main() {
  const double g = 1.2177, gg = g * g;
  for (int trial = 0; trial < 2000; ++trial) {
    V a = rv(), b = rv(), c = rv(), d = rv();
    double pa[4], pb[4], pc[4];
    for (int m = 0; m < 4; ++m) { pb[m] = u(); pc[m] = u(); pa[m] = -(pb[m] + pc[m]); }
    const double inv_q2 = 1.0 / (0.3 + u() * u());
    // the gluon vertex functions against the Feynman rules written out index by index
    cmp(vvv_amp(a, b, c, pa, pb, pc, g), ggg_full(a, b, c, pa, pb, pc, g), mag({&a, &b, &c}) * 8);
    cmpv(jvv(a, b, pb, pc, inv_q2, g), ggg_current(a, b, pb, pc, inv_q2, g), mag({&a, &b}) * 8 * inv_q2);
    cmp(gggg_amp(a, b, c, d, gg), gggg_full(a, b, c, d, gg), mag({&a, &b, &c, &d}) * gg);
    // jgggx0(a, b, c) is the open first slot of ggggxx(open, c, b, a)
    cmpv(jggg(a, b, c, inv_q2, gg), gggg_current(c, b, a, inv_q2, gg), mag({&a, &b, &c}) * gg * inv_q2);
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
