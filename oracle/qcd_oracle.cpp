// FP64 CPU ORACLE -- TEST INFRASTRUCTURE ONLY.
//
// Plain, slow, obviously-correct evaluation of helicity-summed, colour-summed
// tree-level squared matrix elements for massless QCD, written from
// Hagiwara et al., "Calculation of HELAS amplitudes for QCD processes using
// GPU" (arXiv:0909.5257).  Only tests/, the smoke check and the CPU-baseline
// leg of the benchmark may load this library.  It shares no code with the
// CUDA path.
//
// What it computes (Sec. 2.1):
//   M^{c}_{lambda} = sum over Feynman diagrams l of (M_lambda)_l^c   Eq. (matrix-element)
//   M = sum_alpha T_alpha^{c} J_alpha                                 Eq. (color-amplitude)
//   N_ab = 1/(n_a n_b) sum_c T_a^c (T_b^c)^*                          Eq. (color-matrix)
//   |M|^2 = 1/4 sum_lambda sum_ab J_a N_ab J_b^*                     Eq. (color-averaged-amplitude)
//                                                                     and the helicity average below it.
// Steps, in the paper's order:
//   1. enumerate every tree diagram from the qqg, ggg and gggg vertices
//      (Sec. 4; the gggg vertex is split into its three colour structures, so
//      that each structure is one diagram, as Table 1 counts them);
//   2. external states of helicity +-1 (Sec. 2.1) for every one of the
//      2^{n_ext} helicity combinations;
//   3. each diagram's Lorentz value by explicit contraction, with the vertex
//      rules derived by summing over all field assignments of the paper's
//      Lagrangian terms (Eq. (qqg-lagrangian), Eq. (vvv-lagrangian) and the
//      gggg Lagrangian of Sec. 4.2), Feynman-gauge propagators (Sec. 4.1.2);
//   4. each diagram's colour factor expanded onto a colour basis by exact
//      colour algebra (f^{abc} = -2i Tr(T^a[T^b,T^c]), the SU(N) completeness
//      relation, N = 3), giving J_alpha = sum_d c_{d alpha} A_d;
//   5. the colour matrix of Eq. (color-matrix) by the same exact algebra;
//   6. the quadratic form and the helicity sum with compensated summation.
// The colour basis is whatever set of independent colour structures the
// reduction produces: single traces for gluons (Eq. (color-basis)), open
// strings for one quark line, products of two strings for two quark lines.
// |M|^2 does not depend on that choice.
//
// Conventions: metric (+,-,-,-); momenta (E,px,py,pz); legs 0,1 incoming,
// 2.. outgoing; helicity combination h has lambda_i = +1 when bit
// (n_ext-1-i) of h is set, else -1.  Chiral (Weyl) gamma matrices.
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

// Test hook: a nonzero OQ_MUTATION plants one deliberate, plausible mistake
// (a dropped vertex term, a flipped sign, a slipped index, a wrong colour
// average, a forgotten crossing sign) so that tests/test_oracle_mutations.py
// can show that the pins catch it.  Only that test sets it, in a separate build;
// the oracle's own build never does.
#ifndef OQ_MUTATION
#define OQ_MUTATION 0
#endif

namespace oq {

constexpr int kMutation = OQ_MUTATION;

typedef std::complex<double> cd;
typedef long long i64;
typedef __int128 i128;

// ---------------------------------------------------------------- rationals
static i128 gcd128(i128 a, i128 b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b) { i128 t = a % b; a = b; b = t; }
  return a;
}
struct Q {
  i64 n = 0, d = 1;
};
static Q qmk(i128 n, i128 d) {
  if (d == 0) throw std::runtime_error("rational: zero denominator");
  if (d < 0) { n = -n; d = -d; }
  i128 g = gcd128(n, d);
  if (g > 1) { n /= g; d /= g; }
  if (n == 0) d = 1;
  const i128 lim = ((i128)1) << 62;
  if (n > lim || n < -lim || d > lim) throw std::runtime_error("rational overflow");
  Q r; r.n = (i64)n; r.d = (i64)d; return r;
}
static Q operator+(Q a, Q b) { return qmk((i128)a.n * b.d + (i128)b.n * a.d, (i128)a.d * b.d); }
static Q operator-(Q a, Q b) { return qmk((i128)a.n * b.d - (i128)b.n * a.d, (i128)a.d * b.d); }
static Q operator*(Q a, Q b) { return qmk((i128)a.n * b.n, (i128)a.d * b.d); }
static Q qneg(Q a) { a.n = -a.n; return a; }
static bool qzero(Q a) { return a.n == 0; }
static Q qint(i64 v) { Q r; r.n = v; r.d = 1; return r; }

struct CQ {  // exact complex rational
  Q re, im;
};
static CQ operator+(CQ a, CQ b) { return CQ{a.re + b.re, a.im + b.im}; }
static CQ operator*(CQ a, CQ b) {
  return CQ{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
static CQ operator*(CQ a, Q s) { return CQ{a.re * s, a.im * s}; }
static CQ cqconj(CQ a) { return CQ{a.re, qneg(a.im)}; }
static bool cqzero(CQ a) { return qzero(a.re) && qzero(a.im); }
static cd cqval(CQ a) {
  return cd((double)a.re.n / (double)a.re.d, (double)a.im.n / (double)a.im.d);
}

// ----------------------------------------------------------- colour algebra
// A colour term is a coefficient times a product of chains.  An open chain is
// (T^{g_1} ... T^{g_k})_{row,col}; a closed chain is Tr(T^{g_1} ... T^{g_k}).
// Labels below kInternal are external legs; labels at or above it are summed.
static const int kNc = 3;
static const int kInternal = 1000;

struct Chain {
  std::vector<int> g;
  int row = -1, col = -1;
  bool closed = false;
};
struct CTerm {
  CQ c;
  std::vector<Chain> ch;
};

static std::vector<int> cat(const std::vector<int>& a, const std::vector<int>& b) {
  std::vector<int> r(a);
  r.insert(r.end(), b.begin(), b.end());
  return r;
}
static std::vector<int> sub(const std::vector<int>& v, size_t b, size_t e) {
  return std::vector<int>(v.begin() + b, v.begin() + e);
}

// Join chains through summed quark indices; evaluate Tr(1) = N and
// Tr(T^a) = 0.  Returns false when the term vanishes.
static bool normalise(CTerm& t) {
  bool changed = true;
  while (changed) {
    changed = false;
    for (size_t i = 0; i < t.ch.size() && !changed; ++i) {
      Chain& A = t.ch[i];
      if (A.closed || A.col < kInternal) continue;
      if (A.row == A.col) {  // (X)_{xx} summed over x: a trace
        A.closed = true; A.row = A.col = -1; changed = true; break;
      }
      for (size_t j = 0; j < t.ch.size(); ++j) {
        if (j == i || t.ch[j].closed || t.ch[j].row != A.col) continue;
        Chain m;
        m.g = cat(A.g, t.ch[j].g);
        m.row = A.row;
        m.col = t.ch[j].col;
        size_t hi = std::max(i, j), lo = std::min(i, j);
        t.ch.erase(t.ch.begin() + hi);
        t.ch.erase(t.ch.begin() + lo);
        t.ch.push_back(m);
        changed = true;
        break;
      }
    }
  }
  for (size_t i = 0; i < t.ch.size();) {
    if (t.ch[i].closed && t.ch[i].g.empty()) {
      t.c = t.c * qint(kNc);
      t.ch.erase(t.ch.begin() + i);
    } else if (t.ch[i].closed && t.ch[i].g.size() == 1) {
      return false;
    } else {
      ++i;
    }
  }
  return !cqzero(t.c);
}

// Canonical key of a term whose labels are all external.
static std::vector<int> term_key(const CTerm& t) {
  std::vector<std::vector<int>> parts;
  for (const Chain& c : t.ch) {
    std::vector<int> p;
    if (c.closed) {
      std::vector<int> g = c.g;
      auto it = std::min_element(g.begin(), g.end());
      std::rotate(g.begin(), it, g.end());
      p.push_back(1);           // closed marker
      p.push_back(-1);
      p.push_back(-1);
      p.insert(p.end(), g.begin(), g.end());
    } else {
      p.push_back(0);
      p.push_back(c.row);
      p.push_back(c.col);
      p.insert(p.end(), c.g.begin(), c.g.end());
    }
    parts.push_back(p);
  }
  std::sort(parts.begin(), parts.end());
  std::vector<int> key;
  for (auto& p : parts) {
    key.push_back((int)p.size());
    key.insert(key.end(), p.begin(), p.end());
  }
  return key;
}

// Fully reduce: every summed gluon is removed with
//   sum_x T^x_{ab} T^x_{cd} = 1/2 (d_ad d_cb - 1/N d_ab d_cd).
static std::map<std::vector<int>, CQ> reduce(std::vector<CTerm> work) {
  const Q half = qmk(1, 2);
  const Q m1_2n = qmk(-1, 2 * kNc);
  std::map<std::vector<int>, CQ> out;
  while (!work.empty()) {
    CTerm t = std::move(work.back());
    work.pop_back();
    if (!normalise(t)) continue;
    int ci = -1, pi = -1, cj = -1, pj = -1;
    for (size_t i = 0; i < t.ch.size() && cj < 0; ++i)
      for (size_t p = 0; p < t.ch[i].g.size() && cj < 0; ++p) {
        int x = t.ch[i].g[p];
        if (x < kInternal) continue;
        ci = (int)i; pi = (int)p;
        for (size_t j = 0; j < t.ch.size() && cj < 0; ++j)
          for (size_t q = 0; q < t.ch[j].g.size(); ++q) {
            if ((j == i && q == p) || t.ch[j].g[q] != x) continue;
            cj = (int)j; pj = (int)q; break;
          }
        if (cj < 0) throw std::runtime_error("colour: unpaired summed gluon");
      }
    if (ci < 0) {  // nothing left to sum
      std::vector<int> k = term_key(t);
      auto it = out.find(k);
      if (it == out.end()) out.emplace(k, t.c);
      else it->second = it->second + t.c;
      continue;
    }
    CTerm t1, t2;
    t1.c = t.c * half;
    t2.c = t.c * m1_2n;
    std::vector<Chain> rest;
    for (size_t k = 0; k < t.ch.size(); ++k)
      if ((int)k != ci && (int)k != cj) rest.push_back(t.ch[k]);
    t1.ch = rest;
    t2.ch = rest;
    if (ci == cj) {
      const Chain& A = t.ch[ci];
      int p = std::min(pi, pj), q = std::max(pi, pj);
      std::vector<int> P = sub(A.g, 0, p), Qm = sub(A.g, p + 1, q),
                       R = sub(A.g, q + 1, A.g.size());
      Chain trQ; trQ.closed = true; trQ.g = Qm;
      if (!A.closed) {  // (P x Q x R) -> 1/2 (P R) Tr(Q) - 1/2N (P Q R)
        Chain a; a.row = A.row; a.col = A.col; a.g = cat(P, R);
        Chain b; b.row = A.row; b.col = A.col; b.g = cat(cat(P, Qm), R);
        t1.ch.push_back(a); t1.ch.push_back(trQ);
        t2.ch.push_back(b);
      } else {  // Tr(P x Q x R) -> 1/2 Tr(R P) Tr(Q) - 1/2N Tr(R P Q)
        Chain a; a.closed = true; a.g = cat(R, P);
        Chain b; b.closed = true; b.g = cat(cat(R, P), Qm);
        t1.ch.push_back(a); t1.ch.push_back(trQ);
        t2.ch.push_back(b);
      }
    } else {
      Chain A = t.ch[ci], B = t.ch[cj];
      int pa = pi, pb = pj;
      if (A.closed && !B.closed) { std::swap(A, B); std::swap(pa, pb); }
      if (!A.closed && !B.closed) {
        // (P x Q)_{r1 c1} (R x S)_{r2 c2} -> 1/2 (P S)_{r1 c2} (R Q)_{r2 c1}
        //                                   - 1/2N (P Q)_{r1 c1} (R S)_{r2 c2}
        std::vector<int> P = sub(A.g, 0, pa), Qm = sub(A.g, pa + 1, A.g.size());
        std::vector<int> R = sub(B.g, 0, pb), S = sub(B.g, pb + 1, B.g.size());
        Chain a; a.row = A.row; a.col = B.col; a.g = cat(P, S);
        Chain b; b.row = B.row; b.col = A.col; b.g = cat(R, Qm);
        Chain c; c.row = A.row; c.col = A.col; c.g = cat(P, Qm);
        Chain d; d.row = B.row; d.col = B.col; d.g = cat(R, S);
        t1.ch.push_back(a); t1.ch.push_back(b);
        t2.ch.push_back(c); t2.ch.push_back(d);
      } else if (!A.closed && B.closed) {
        // (P x Q)_{rc} Tr(W x) -> 1/2 (P W Q)_{rc} - 1/2N (P Q)_{rc} Tr(W)
        std::vector<int> P = sub(A.g, 0, pa), Qm = sub(A.g, pa + 1, A.g.size());
        std::vector<int> W = cat(sub(B.g, pb + 1, B.g.size()), sub(B.g, 0, pb));
        Chain a; a.row = A.row; a.col = A.col; a.g = cat(cat(P, W), Qm);
        Chain b; b.row = A.row; b.col = A.col; b.g = cat(P, Qm);
        Chain trW; trW.closed = true; trW.g = W;
        t1.ch.push_back(a);
        t2.ch.push_back(b); t2.ch.push_back(trW);
      } else {
        // Tr(U x) Tr(W x) -> 1/2 Tr(U W) - 1/2N Tr(U) Tr(W)
        std::vector<int> U = cat(sub(A.g, pa + 1, A.g.size()), sub(A.g, 0, pa));
        std::vector<int> W = cat(sub(B.g, pb + 1, B.g.size()), sub(B.g, 0, pb));
        Chain a; a.closed = true; a.g = cat(U, W);
        Chain u; u.closed = true; u.g = U;
        Chain w; w.closed = true; w.g = W;
        t1.ch.push_back(a);
        t2.ch.push_back(u); t2.ch.push_back(w);
      }
    }
    work.push_back(std::move(t1));
    work.push_back(std::move(t2));
  }
  for (auto it = out.begin(); it != out.end();) {
    if (cqzero(it->second)) it = out.erase(it);
    else ++it;
  }
  return out;
}

// f^{abc} = -2i [ Tr(T^a T^b T^c) - Tr(T^c T^b T^a) ]  (from [T^a,T^b] = i f^{abc} T^c
// and Tr(T^a T^b) = delta^{ab}/2).  Multiplies every term of `e` by it.
static std::vector<CTerm> times_f(const std::vector<CTerm>& e, int a, int b, int c) {
  std::vector<CTerm> r;
  r.reserve(e.size() * 2);
  CQ m2i{qint(0), qint(-2)}, p2i{qint(0), qint(2)};
  for (const CTerm& t : e) {
    CTerm u = t, v = t;
    Chain x; x.closed = true; x.g = {a, b, c};
    Chain y; y.closed = true; y.g = {c, b, a};
    u.c = t.c * m2i; u.ch.push_back(x);
    v.c = t.c * p2i; v.ch.push_back(y);
    r.push_back(u);
    r.push_back(v);
  }
  return r;
}
static std::vector<CTerm> times_T(const std::vector<CTerm>& e, int gl, int row, int col) {
  std::vector<CTerm> r = e;
  for (CTerm& t : r) {
    Chain x; x.g = {gl}; x.row = row; x.col = col;
    t.ch.push_back(x);
  }
  return r;
}

// Rename every external label to a summed one (shift by `off`).
static Chain internalise(const Chain& c, int off) {
  Chain r = c;
  for (int& x : r.g) if (x < kInternal) x += off;
  if (r.row >= 0 && r.row < kInternal) r.row += off;
  if (r.col >= 0 && r.col < kInternal) r.col += off;
  return r;
}
// Complex conjugate of a chain: (T^{g1}..T^{gk})_{ij}^* = (T^{gk}..T^{g1})_{ji}.
static Chain conj_chain(const Chain& c) {
  Chain r = c;
  std::reverse(r.g.begin(), r.g.end());
  if (!c.closed) std::swap(r.row, r.col);
  return r;
}

// Decode a basis key back into chains.
static std::vector<Chain> key_chains(const std::vector<int>& key) {
  std::vector<Chain> out;
  size_t i = 0;
  while (i < key.size()) {
    int len = key[i++];
    Chain c;
    c.closed = key[i] == 1;
    c.row = key[i + 1];
    c.col = key[i + 2];
    c.g.assign(key.begin() + i + 3, key.begin() + i + len);
    if (c.closed) { c.row = c.col = -1; }
    out.push_back(c);
    i += len;
  }
  return out;
}

// ------------------------------------------------------------ Lorentz basics
typedef std::array<cd, 4> V4;  // four-vector (index position stated at use)
static const double kMetric[4] = {1.0, -1.0, -1.0, -1.0};

static cd dot_ll(const V4& a, const V4& b) {  // a_mu b_nu g^{mu nu}
  return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}
static cd dot_ul(const double* k, const V4& w) {  // k^mu w_mu
  return k[0] * w[0] + k[1] * w[1] + k[2] * w[2] + k[3] * w[3];
}

// Chiral-representation gamma matrices gamma^mu (upper index).
struct Gam {
  cd m[4][4][4];
  Gam() {
    const cd I(0, 1);
    std::memset((void*)m, 0, sizeof(m));
    // gamma^0 = [[0,1],[1,0]]
    m[0][0][2] = m[0][1][3] = m[0][2][0] = m[0][3][1] = 1.0;
    // gamma^k = [[0, sigma^k], [-sigma^k, 0]]
    cd s[3][2][2] = {{{0, 1}, {1, 0}}, {{0, -I}, {I, 0}}, {{1, 0}, {0, -1}}};
    for (int k = 0; k < 3; ++k)
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          m[k + 1][a][b + 2] = s[k][a][b];
          m[k + 1][a + 2][b] = -s[k][a][b];
        }
  }
};
static const Gam kG;

typedef std::array<cd, 4> Sp;  // Dirac spinor (column) or barred spinor (row)

// slash(w) = gamma^mu w_mu for a lower-index vector w.
static void slash_lower(const V4& w, cd out[4][4]) {
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      cd s = 0;
      for (int mu = 0; mu < 4; ++mu) s += kG.m[mu][a][b] * w[mu];
      out[a][b] = s;
    }
}
// slash(k) = gamma^mu k_mu for a real upper-index vector k.
static void slash_upper(const double* k, cd out[4][4]) {
  V4 w;
  for (int mu = 0; mu < 4; ++mu) w[mu] = kMetric[mu] * k[mu];
  slash_lower(w, out);
}
static Sp mat_col(const cd m[4][4], const Sp& v) {
  Sp r;
  for (int a = 0; a < 4; ++a) {
    cd s = 0;
    for (int b = 0; b < 4; ++b) s += m[a][b] * v[b];
    r[a] = s;
  }
  return r;
}
static Sp row_mat(const Sp& v, const cd m[4][4]) {
  Sp r;
  for (int b = 0; b < 4; ++b) {
    cd s = 0;
    for (int a = 0; a < 4; ++a) s += v[a] * m[a][b];
    r[b] = s;
  }
  return r;
}
static cd row_col(const Sp& r, const Sp& c) {
  cd s = 0;
  for (int a = 0; a < 4; ++a) s += r[a] * c[a];
  return s;
}

// ------------------------------------------------------- external states
// Two-component helicity eigenstates chi_lambda(p) with sigma.p_hat chi = lambda chi.
static void chi(const double* p, int lam, cd out[2]) {
  double pp = std::sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
  double a = pp + p[3];
  if (a <= 1e-300 * (pp + 1.0) || a <= 0.0) {  // along -z: theta = pi, phi = 0
    if (lam > 0) { out[0] = 0.0; out[1] = 1.0; }
    else { out[0] = -1.0; out[1] = 0.0; }
    return;
  }
  double nrm = 1.0 / std::sqrt(2.0 * pp * a);
  if (lam > 0) { out[0] = a * nrm; out[1] = cd(p[1], p[2]) * nrm; }
  else { out[0] = cd(-p[1], p[2]) * nrm; out[1] = a * nrm; }
}
// u(p,lambda): massless, right-handed components in the lower half.
static Sp spinor_u(const double* p, int lam) {
  cd c[2]; chi(p, lam, c);
  double r = std::sqrt(2.0 * p[0]);
  Sp s{0.0, 0.0, 0.0, 0.0};
  if (lam > 0) { s[2] = r * c[0]; s[3] = r * c[1]; }
  else { s[0] = r * c[0]; s[1] = r * c[1]; }
  return s;
}
// v(p,lambda) for an antiquark of helicity lambda (spin state chi_{-lambda}).
static Sp spinor_v(const double* p, int lam) {
  cd c[2]; chi(p, -lam, c);
  double r = std::sqrt(2.0 * p[0]);
  Sp s{0.0, 0.0, 0.0, 0.0};
  if (lam > 0) { s[0] = r * c[0]; s[1] = r * c[1]; }
  else { s[2] = -r * c[0]; s[3] = -r * c[1]; }
  return s;
}
static Sp bar(const Sp& s) {  // psi^dagger gamma^0
  return Sp{std::conj(s[2]), std::conj(s[3]), std::conj(s[0]), std::conj(s[1])};
}
// Polarisation vector eps^mu(k,lambda) (upper index).
static V4 polvec(const double* k, int lam) {
  double kk = std::sqrt(k[1] * k[1] + k[2] * k[2] + k[3] * k[3]);
  double kt = std::sqrt(k[1] * k[1] + k[2] * k[2]);
  double ct = k[3] / kk, st = kt / kk, cp, sp;
  if (kt > 0.0) { cp = k[1] / kt; sp = k[2] / kt; }
  else { cp = 1.0; sp = 0.0; if (k[3] < 0) { ct = -1.0; } else { ct = 1.0; } st = 0.0; }
  double e1[3] = {ct * cp, ct * sp, -st};
  double e2[3] = {-sp, cp, 0.0};
  const double r = 1.0 / std::sqrt(2.0);
  V4 e;
  e[0] = 0.0;
  for (int i = 0; i < 3; ++i) {
    // eps(+) = -(e1 + i e2)/sqrt2,  eps(-) = (e1 - i e2)/sqrt2
    if (lam > 0) e[i + 1] = -r * cd(e1[i], e2[i]);
    else e[i + 1] = r * cd(e1[i], -e2[i]);
  }
  return e;
}
static V4 lower(const V4& u) {
  V4 l;
  for (int mu = 0; mu < 4; ++mu) l[mu] = kMetric[mu] * u[mu];
  return l;
}

// ------------------------------------------------------------------ process
enum Kind { KG = 0, KPSI = 1, KPSIBAR = 2 };  // how a line looks from inside

struct Node {
  int type;                 // 0 ext, 1 ggg, 2 gggg, 3 qqg->g, 4 qqg->psi, 5 qqg->psibar
  int kind;                 // line kind it produces: KG, KPSI, KPSIBAR
  int flav;                 // quark flavour for KPSI/KPSIBAR lines
  uint32_t mask;            // external legs below this line
  int leg;                  // for ext
  int structure;            // for gggg: 0,1,2
  std::vector<const Node*> kids;
};

struct Diagram {
  int root_type;            // vertex type at the root (1 ggg, 2 gggg, 3/4/5 qqg)
  int structure;
  std::vector<const Node*> kids;
  int fermion_sign;
};

struct Process {
  int n_ext = 0;
  std::vector<int> pdg;
  std::vector<int> kind, flav;   // per leg
  int root = 0;
  double gs = 0;
  int n_a = 1, n_b = 1;
  std::vector<std::unique_ptr<Node>> pool;
  std::map<std::pair<uint32_t, int>, std::vector<const Node*>> memo;
  std::vector<Diagram> diagrams;
  int n_topologies = 0;
  // colour
  std::vector<std::vector<int>> basis;                          // keys
  std::vector<std::vector<std::pair<int, CQ>>> coef;            // per diagram
  std::vector<std::vector<std::pair<int, cd>>> coefd;
  std::vector<CQ> cmat_exact;                                    // m*m
  std::vector<double> cmat;                                      // m*m (real part)
};

static int line_code(int kind, int flav) { return kind * 64 + flav; }

static const Node* mknode(Process& P, Node n) {
  P.pool.emplace_back(new Node(n));
  return P.pool.back().get();
}

static const std::vector<const Node*>& currents(Process& P, uint32_t S, int kind, int flav);

// Vertex structures producing a line of (kind, flav) from the legs in S.
// Each returned Node is one way; gggg vertices are split into their three
// colour structures (Sec. 4.2, Eq. (gggg-functions-calls)).
static std::vector<Node> vertex_splits(Process& P, uint32_t S, int kind, int flav) {
  std::vector<Node> out;
  auto add2 = [&](int type, uint32_t A, int ka, int fa, uint32_t B, int kb, int fb) {
    const auto& la = currents(P, A, ka, fa);
    const auto& lb = currents(P, B, kb, fb);
    for (const Node* x : la)
      for (const Node* y : lb) {
        Node n; n.type = type; n.kind = kind; n.flav = flav; n.mask = S; n.leg = -1;
        n.structure = 0; n.kids = {x, y};
        out.push_back(n);
      }
  };
  uint32_t low = S & (~S + 1u);
  if (kind == KG) {
    // two blocks: A holds the lowest leg
    for (uint32_t A = (S - 1) & S; A; A = (A - 1) & S) {
      if (!(A & low)) continue;
      uint32_t B = S & ~A;
      add2(1, A, KG, 0, B, KG, 0);                       // ggg
      for (int f = 1; f <= 6; ++f) {                     // qqg: (psi, psibar)
        add2(3, A, KPSI, f, B, KPSIBAR, f);
        add2(3, B, KPSI, f, A, KPSIBAR, f);
      }
    }
    // three blocks for gggg
    for (uint32_t A = (S - 1) & S; A; A = (A - 1) & S) {
      if (!(A & low)) continue;
      uint32_t R = S & ~A;
      uint32_t lowR = R & (~R + 1u);
      for (uint32_t B = (R - 1) & R; B; B = (B - 1) & R) {
        if (!(B & lowR)) continue;
        uint32_t C = R & ~B;
        const auto& la = currents(P, A, KG, 0);
        const auto& lb = currents(P, B, KG, 0);
        const auto& lc = currents(P, C, KG, 0);
        for (const Node* x : la)
          for (const Node* y : lb)
            for (const Node* z : lc)
              for (int s = 0; s < 3; ++s) {
                Node n; n.type = 2; n.kind = KG; n.flav = 0; n.mask = S; n.leg = -1;
                n.structure = s; n.kids = {x, y, z};
                out.push_back(n);
              }
      }
    }
  } else {
    // psi (psibar) line continues from a psi (psibar) line in X after absorbing a gluon line from Y
    int type = (kind == KPSI) ? 4 : 5;
    for (uint32_t X = (S - 1) & S; X; X = (X - 1) & S) {
      uint32_t Y = S & ~X;
      add2(type, X, kind, flav, Y, KG, 0);
    }
  }
  return out;
}

static const std::vector<const Node*>& currents(Process& P, uint32_t S, int kind, int flav) {
  auto key = std::make_pair(S, line_code(kind, flav));
  auto it = P.memo.find(key);
  if (it != P.memo.end()) return it->second;
  std::vector<const Node*> res;
  if (__builtin_popcount(S) == 1) {
    int leg = __builtin_ctz(S);
    if (P.kind[leg] == kind && (kind == KG || P.flav[leg] == flav)) {
      Node n; n.type = 0; n.kind = kind; n.flav = flav; n.mask = S; n.leg = leg;
      n.structure = 0;
      res.push_back(mknode(P, n));
    }
  } else {
    // quick reject: fermion content must match the line kind
    int npsi[7] = {0}, nbar[7] = {0};
    for (int l = 0; l < P.n_ext; ++l)
      if (S >> l & 1u) {
        if (P.kind[l] == KPSI) npsi[P.flav[l]]++;
        if (P.kind[l] == KPSIBAR) nbar[P.flav[l]]++;
      }
    bool ok = true;
    for (int f = 1; f <= 6; ++f) {
      int want = 0;
      if (kind == KPSI && f == flav) want = 1;
      if (kind == KPSIBAR && f == flav) want = -1;
      if (npsi[f] - nbar[f] != want) ok = false;
    }
    if (ok)
      for (Node& n : vertex_splits(P, S, kind, flav)) res.push_back(mknode(P, n));
  }
  return P.memo.emplace(key, res).first->second;
}

// Fermion lines of a diagram: pairs (psi leg, psibar leg).
static void collect_lines(const Node* n, int* open_psi, int* open_bar,
                          std::vector<std::pair<int, int>>& pairs);
static void collect_lines(const Node* n, int* open_psi, int* open_bar,
                          std::vector<std::pair<int, int>>& pairs) {
  // returns through open_psi/open_bar the external leg at the open end of a
  // psi / psibar line produced by n
  *open_psi = -1; *open_bar = -1;
  if (n->type == 0) {
    if (n->kind == KPSI) *open_psi = n->leg;
    if (n->kind == KPSIBAR) *open_bar = n->leg;
    return;
  }
  std::vector<int> ps, bs;
  for (const Node* k : n->kids) {
    int a, b;
    collect_lines(k, &a, &b, pairs);
    if (a >= 0) ps.push_back(a);
    if (b >= 0) bs.push_back(b);
  }
  if (n->type == 3) pairs.push_back({ps.at(0), bs.at(0)});
  if (n->type == 4) *open_psi = ps.at(0);
  if (n->type == 5) *open_bar = bs.at(0);
}

static int permutation_sign(std::vector<int> v) {
  int s = 1;
  for (size_t i = 0; i < v.size(); ++i)
    for (size_t j = i + 1; j < v.size(); ++j)
      if (v[i] > v[j]) s = -s;
  return s;
}

static void count_topologies(Process& P) {
  int t = 0;
  for (const Diagram& d : P.diagrams) {
    // one topology per gggg colour-structure triple: count only structure 0
    bool first = (d.root_type != 2 || d.structure == 0);
    std::vector<const Node*> st(d.kids.begin(), d.kids.end());
    while (first && !st.empty()) {
      const Node* n = st.back(); st.pop_back();
      if (n->type == 2 && n->structure != 0) first = false;
      for (const Node* k : n->kids) st.push_back(k);
    }
    if (first) ++t;
  }
  P.n_topologies = t;
}

static void enumerate(Process& P) {
  int r = P.root;
  uint32_t all = (1u << P.n_ext) - 1u;
  uint32_t R = all & ~(1u << r);
  int kr = P.kind[r], fr = P.flav[r];
  std::vector<Node> tops;
  if (kr == KG) tops = vertex_splits(P, R, KG, 0);
  else if (kr == KPSIBAR) tops = vertex_splits(P, R, KPSI, fr);   // psi line ends on the root
  else tops = vertex_splits(P, R, KPSIBAR, fr);
  for (const Node& t : tops) {
    Diagram d;
    d.root_type = t.type;
    d.structure = t.structure;
    d.kids = t.kids;
    std::vector<std::pair<int, int>> pairs;
    int op[3], ob[3];
    for (size_t i = 0; i < t.kids.size(); ++i) collect_lines(t.kids[i], &op[i], &ob[i], pairs);
    if (t.type == 3) pairs.push_back({op[0], ob[1]});
    if (t.type == 4) pairs.push_back({op[0], r});      // root is psibar-type
    if (t.type == 5) pairs.push_back({r, ob[0]});      // root is psi-type
    // sign of the pairing: psibar legs in increasing order, their psi partners
    std::sort(pairs.begin(), pairs.end(),
              [](const std::pair<int, int>& a, const std::pair<int, int>& b) { return a.second < b.second; });
    std::vector<int> psis;
    for (auto& pr : pairs) psis.push_back(pr.first);
    d.fermion_sign = permutation_sign(psis);
    P.diagrams.push_back(d);
  }
  count_topologies(P);
}

// ------------------------------------------------------------ colour factors
struct LabelGen { int next = kInternal; };

static int line_label(const Node* n, LabelGen& lg, std::map<const Node*, int>& lab) {
  if (n->type == 0) return n->leg;
  auto it = lab.find(n);
  if (it != lab.end()) return it->second;
  int v = lg.next++;
  lab[n] = v;
  return v;
}

// gggg colour structures with legs (a,b,c,d): f^{abe}f^{cde}, f^{ace}f^{dbe}, f^{ade}f^{bce}.
static const int kQuarticPerm[3][4] = {{0, 1, 2, 3}, {0, 2, 3, 1}, {0, 3, 1, 2}};

static std::vector<CTerm> vertex_colour(std::vector<CTerm> e, int type, int structure,
                                         const int* lab, int out_label, LabelGen& lg) {
  // lab: labels of the kids in order; out_label: label of the produced line
  if (type == 1) return times_f(e, lab[0], lab[1], out_label);
  if (type == 2) {
    int L[4] = {lab[0], lab[1], lab[2], out_label};
    const int* p = kQuarticPerm[structure];
    int ex = lg.next++;
    e = times_f(e, L[p[0]], L[p[1]], ex);
    return times_f(e, L[p[2]], L[p[3]], ex);
  }
  if (type == 3) return times_T(e, out_label, lab[1], lab[0]);   // psibar T psi
  if (type == 4) return times_T(e, lab[1], out_label, lab[0]);   // psi_out = T psi_in
  return times_T(e, lab[1], lab[0], out_label);                  // psibar_out = psibar_in T
}

static std::vector<CTerm> node_colour(const Node* n, std::vector<CTerm> e, LabelGen& lg,
                                      std::map<const Node*, int>& lab) {
  if (n->type == 0) return e;
  int kl[3];
  for (size_t i = 0; i < n->kids.size(); ++i) {
    e = node_colour(n->kids[i], e, lg, lab);
    kl[i] = line_label(n->kids[i], lg, lab);
  }
  int me = line_label(n, lg, lab);
  return vertex_colour(e, n->type, n->structure, kl, me, lg);
}

static void build_colour(Process& P) {
  std::map<std::vector<int>, int> index;
  std::vector<std::map<std::vector<int>, CQ>> per;
  for (const Diagram& d : P.diagrams) {
    LabelGen lg;
    std::map<const Node*, int> lab;
    CTerm one; one.c = CQ{qint(1), qint(0)};
    std::vector<CTerm> e{one};
    int kl[3];
    for (size_t i = 0; i < d.kids.size(); ++i) {
      e = node_colour(d.kids[i], e, lg, lab);
      kl[i] = line_label(d.kids[i], lg, lab);
    }
    e = vertex_colour(e, d.root_type, d.structure, kl, P.root, lg);
    per.push_back(reduce(e));
    for (auto& kv : per.back())
      if (!index.count(kv.first)) index[kv.first] = 0;
  }
  int m = 0;
  for (auto& kv : index) { kv.second = m++; P.basis.push_back(kv.first); }
  for (auto& mp : per) {
    std::vector<std::pair<int, CQ>> v;
    std::vector<std::pair<int, cd>> vd;
    for (auto& kv : mp) {
      v.push_back({index[kv.first], kv.second});
      vd.push_back({index[kv.first], cqval(kv.second)});
    }
    P.coef.push_back(v);
    P.coefd.push_back(vd);
  }
  // Eq. (color-matrix): N_ab = 1/(n_a n_b) sum_c T_a^c (T_b^c)^*
  P.cmat_exact.assign((size_t)m * m, CQ{qint(0), qint(0)});
  P.cmat.assign((size_t)m * m, 0.0);
  Q avg = qmk(1, kMutation == 5 ? (i128)64 : (i128)P.n_a * P.n_b);  // mutation 5: gluon averaging for quarks
  std::vector<std::vector<Chain>> bc(m);
  for (int a = 0; a < m; ++a) bc[a] = key_chains(P.basis[a]);
  std::vector<std::pair<int, int>> jobs;
  for (int a = 0; a < m; ++a)
    for (int b = a; b < m; ++b) jobs.push_back({a, b});
  std::string err;
#pragma omp parallel for schedule(dynamic, 64)
  for (long j = 0; j < (long)jobs.size(); ++j) {
    int a = jobs[j].first, b = jobs[j].second;
    try {
      CTerm t; t.c = CQ{qint(1), qint(0)};
      for (const Chain& c : bc[a]) t.ch.push_back(internalise(c, kInternal));
      for (const Chain& c : bc[b]) t.ch.push_back(internalise(conj_chain(c), kInternal));
      auto r = reduce({t});
      CQ v{qint(0), qint(0)};
      for (auto& kv : r) {
        if (!kv.first.empty()) throw std::runtime_error("colour matrix: open labels left");
        v = v + kv.second;
      }
      v = v * avg;
      P.cmat_exact[(size_t)a * m + b] = v;
      P.cmat_exact[(size_t)b * m + a] = cqconj(v);
    } catch (std::exception& ex) {
#pragma omp critical
      err = ex.what();
    }
  }
  if (!err.empty()) throw std::runtime_error(err);
  for (size_t i = 0; i < P.cmat_exact.size(); ++i) P.cmat[i] = cqval(P.cmat_exact[i]).real();
}

// ------------------------------------------------------------ Lorentz values
// Everything a diagram needs for one event and one helicity combination.
struct EvalCtx {
  const Process* P;
  double k[16][4];      // incoming momenta k_i (p_i for incoming legs, -p_i for outgoing)
  V4 wv[16];            // lower-index external gluon wavefunctions
  Sp sp[16];            // external spinors (column for psi legs, row for psibar legs)
  double gs;
};

struct Wave {
  V4 v;                 // lower-index gluon current (propagator included)
  Sp s;                 // spinor current (propagator included)
};

static void mask_momentum(const EvalCtx& C, uint32_t m, double* K) {
  K[0] = K[1] = K[2] = K[3] = 0.0;
  for (int l = 0; l < C.P->n_ext; ++l)
    if (m >> l & 1u)
      for (int mu = 0; mu < 4; ++mu)  // mutation 7: the crossing sign of outgoing legs forgotten
        K[mu] += (kMutation == 7 && l >= 2) ? -C.k[l][mu] : C.k[l][mu];
}
static double msq(const double* K) {
  return K[0] * K[0] - K[1] * K[1] - K[2] * K[2] - K[3] * K[3];
}

// Cubic vertex from L_ggg = g f^{abc} (d^mu A^{a nu}) A^b_mu A^c_nu, Eq. (vvv-lagrangian):
// summing i * L over the 3! assignments of legs to fields (d -> -i k_in) gives, as the
// coefficient of f^{a1 a2 a3}, the contraction
//   g * sum_sigma sgn(sigma) (k_{s1}.W_{s2}) (W_{s1}.W_{s3}).
static cd ggg_contract(double gs, const double* k[3], const V4* W[3]) {
  static const int perm[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {0, 2, 1}, {2, 1, 0}, {1, 0, 2}};
  static const int sgn[6] = {1, 1, 1, -1, -1, -1};
  cd s = 0;
  for (int p = 0; p < 6; ++p) {
    if (kMutation == 1 && p == 5) continue;  // mutation: a dropped vertex term
    int a = perm[p][0], b = perm[p][1], c = perm[p][2];
    s += (double)sgn[p] * dot_ul(k[a], *W[b]) * dot_ll(*W[a], *W[c]);
  }
  return gs * s;
}

// Quartic vertex from L_gggg = -(g^2/4) f^{abe} f^{cde} A^{a mu} A^{b nu} A^c_mu A^d_nu
// (Sec. 4.2): i * L summed over the 4! assignments; each assignment's colour factor is
// +-1 times one of the three structures of kQuarticPerm.  Returns the Lorentz factor
// multiplying structure `st`.
static int quartic_structure(const int* x, int* sign) {
  // colour of an assignment: f^{x0 x1 e} f^{x2 x3 e}
  for (int s = 0; s < 3; ++s) {
    const int* p = kQuarticPerm[s];
    for (int swap = 0; swap < 2; ++swap) {
      int a0 = swap ? x[2] : x[0], a1 = swap ? x[3] : x[1];
      int b0 = swap ? x[0] : x[2], b1 = swap ? x[1] : x[3];
      int sa = 0, sb = 0;
      if (a0 == p[0] && a1 == p[1]) sa = 1;
      if (a0 == p[1] && a1 == p[0]) sa = -1;
      if (b0 == p[2] && b1 == p[3]) sb = 1;
      if (b0 == p[3] && b1 == p[2]) sb = -1;
      if (sa && sb) { *sign = sa * sb; return s; }
    }
  }
  throw std::runtime_error("quartic colour structure not found");
}
static cd gggg_contract(double gs, int st, const V4* W[4]) {
  int x[4] = {0, 1, 2, 3};
  cd s = 0;
  do {
    int sign;
    if (quartic_structure(x, &sign) != st) continue;
    s += (double)sign * dot_ll(*W[x[0]], *W[x[2]]) * dot_ll(*W[x[1]], *W[x[3]]);
  } while (std::next_permutation(x, x + 4));
  if (kMutation == 2 && st == 1) s = -s;  // mutation: a flipped sign
  return cd(0, 1) * (-(gs * gs) / 4.0) * s;
}

static V4 unit_lower(int mu) {
  V4 e{0.0, 0.0, 0.0, 0.0};
  e[mu] = 1.0;
  return e;
}

static Wave eval_node(const EvalCtx& C, const Node* n);

// Vertex with one open leg (the produced line) -> upper-index vector out^mu.
static V4 open_gluon_vertex(const EvalCtx& C, const Node* n, const std::vector<Wave>& kw) {
  V4 out;
  double K[3][4];
  const double* kp[3];
  for (size_t i = 0; i < n->kids.size(); ++i) { mask_momentum(C, n->kids[i]->mask, K[i]); kp[i] = K[i]; }
  double Kout[4];
  mask_momentum(C, n->mask, Kout);
  for (int mu = 0; mu < 4; ++mu) Kout[mu] = -Kout[mu];  // incoming momentum at the parent leg
  if (n->type == 1) {
    kp[2] = Kout;
    for (int mu = 0; mu < 4; ++mu) {
      V4 e = unit_lower(mu);
      const V4* W[3] = {&kw[0].v, &kw[1].v, &e};
      out[mu] = ggg_contract(C.gs, kp, W);
    }
  } else if (n->type == 2) {
    for (int mu = 0; mu < 4; ++mu) {
      V4 e = unit_lower(mu);
      const V4* W[4] = {&kw[0].v, &kw[1].v, &kw[2].v, &e};
      out[mu] = gggg_contract(C.gs, n->structure, W);
    }
  } else {  // type 3: psibar (-i g gamma^mu) psi
    for (int mu = 0; mu < 4; ++mu) {
      cd g[4][4];
      for (int a = 0; a < 4; ++a) for (int b = 0; b < 4; ++b) g[a][b] = kG.m[mu][a][b];
      out[mu] = cd(0, kMutation == 6 ? C.gs : -C.gs) * row_col(kw[1].s, mat_col(g, kw[0].s));  // mutation 6
    }
  }
  return out;
}

static Wave eval_node(const EvalCtx& C, const Node* n) {
  Wave w;
  if (n->type == 0) {
    if (n->kind == KG) w.v = C.wv[n->leg];
    else w.s = C.sp[n->leg];
    return w;
  }
  std::vector<Wave> kw;
  for (const Node* k : n->kids) kw.push_back(eval_node(C, k));
  double K[4];
  mask_momentum(C, n->mask, K);
  double K2 = msq(K);
  if (n->kind == KG) {
    // gluon propagator -i g_{mu nu} / K^2
    V4 up = open_gluon_vertex(C, n, kw);
    for (int mu = 0; mu < 4; ++mu)
      w.v[mu] = cd(0, -1) * (kMutation == 3 ? 1.0 : kMetric[mu]) * up[mu] / K2;  // mutation 3: index slip
    return w;
  }
  // qqg vertex -i g gamma^mu T^a (Eq. (qqg-lagrangian)); quark propagator i pslash / p^2
  cd vs[4][4], ps[4][4];
  slash_lower(kw[1].v, vs);
  if (n->kind == KPSI) {
    // momentum along the fermion arrow = K (flows out of the subset)
    slash_upper(K, ps);
    Sp t = mat_col(vs, kw[0].s);
    for (int a = 0; a < 4; ++a) t[a] *= cd(0, -C.gs);
    Sp u = mat_col(ps, t);
    for (int a = 0; a < 4; ++a) w.s[a] = cd(0, 1) * u[a] / K2;
  } else {
    // momentum along the arrow (into the subset) = -K
    const double sK = kMutation == 4 ? 1.0 : -1.0;  // mutation 4: wrong momentum direction
    double mK[4] = {sK * K[0], sK * K[1], sK * K[2], sK * K[3]};
    slash_upper(mK, ps);
    Sp t = row_mat(kw[0].s, vs);
    for (int a = 0; a < 4; ++a) t[a] *= cd(0, -C.gs);
    Sp u = row_mat(t, ps);
    for (int a = 0; a < 4; ++a) w.s[a] = cd(0, 1) * u[a] / K2;
  }
  return w;
}

static cd eval_diagram(const EvalCtx& C, const Diagram& d) {
  const Process& P = *C.P;
  int r = P.root;
  std::vector<Wave> kw;
  for (const Node* k : d.kids) kw.push_back(eval_node(C, k));
  cd A;
  if (d.root_type == 1) {
    double K[2][4];
    mask_momentum(C, d.kids[0]->mask, K[0]);
    mask_momentum(C, d.kids[1]->mask, K[1]);
    const double* kp[3] = {K[0], K[1], C.k[r]};
    const V4* W[3] = {&kw[0].v, &kw[1].v, &C.wv[r]};
    A = ggg_contract(C.gs, kp, W);
  } else if (d.root_type == 2) {
    const V4* W[4] = {&kw[0].v, &kw[1].v, &kw[2].v, &C.wv[r]};
    A = gggg_contract(C.gs, d.structure, W);
  } else if (d.root_type == 3) {
    cd vs[4][4];
    slash_lower(C.wv[r], vs);
    A = cd(0, -C.gs) * row_col(kw[1].s, mat_col(vs, kw[0].s));
  } else if (d.root_type == 4) {  // root psibar-type leg closes a psi line
    cd vs[4][4];
    slash_lower(kw[1].v, vs);
    A = cd(0, -C.gs) * row_col(C.sp[r], mat_col(vs, kw[0].s));
  } else {                        // root psi-type leg closes a psibar line
    cd vs[4][4];
    slash_lower(kw[1].v, vs);
    A = cd(0, -C.gs) * row_col(kw[0].s, mat_col(vs, C.sp[r]));
  }
  return (double)d.fermion_sign * A;
}

// Neumaier compensated sum.
struct KSum {
  double s = 0, c = 0;
  void add(double x) {
    double t = s + x;
    if (std::fabs(s) >= std::fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
  }
  double val() const { return s + c; }
};

static void setup_ctx(const Process& P, const double* mom, int hel, int ward_leg, EvalCtx& C) {
  C.P = &P;
  C.gs = P.gs;
  for (int l = 0; l < P.n_ext; ++l) {
    const double* p = mom + 4 * l;
    bool in = l < 2;
    int lam = (hel >> (P.n_ext - 1 - l) & 1) ? 1 : -1;
    for (int mu = 0; mu < 4; ++mu) C.k[l][mu] = in ? p[mu] : -p[mu];
    if (P.kind[l] == KG) {
      V4 e = polvec(p, lam);
      if (!in) for (int mu = 0; mu < 4; ++mu) e[mu] = std::conj(e[mu]);
      if (l == ward_leg)  // Ward test: eps -> k / E
        for (int mu = 0; mu < 4; ++mu) e[mu] = p[mu] / p[0];
      C.wv[l] = lower(e);
    } else {
      bool quark = P.pdg[l] > 0;
      if (in && quark) C.sp[l] = spinor_u(p, lam);               // psi: u
      else if (!in && !quark) C.sp[l] = spinor_v(p, lam);        // psi: v
      else if (!in && quark) C.sp[l] = bar(spinor_u(p, lam));    // psibar: ubar
      else C.sp[l] = bar(spinor_v(p, lam));                      // psibar: vbar
    }
  }
}

static void jamp_one(const Process& P, const double* mom, int hel, int ward_leg, std::vector<cd>& J) {
  EvalCtx C;
  setup_ctx(P, mom, hel, ward_leg, C);
  size_t m = P.basis.size();
  std::vector<KSum> re(m), im(m);
  for (size_t d = 0; d < P.diagrams.size(); ++d) {
    cd A = eval_diagram(C, P.diagrams[d]);
    for (auto& cv : P.coefd[d]) {
      cd x = cv.second * A;
      re[cv.first].add(x.real());
      im[cv.first].add(x.imag());
    }
  }
  J.resize(m);
  for (size_t a = 0; a < m; ++a) J[a] = cd(re[a].val(), im[a].val());
}

static double quad_form(const Process& P, const std::vector<cd>& J) {
  size_t m = J.size();
  KSum s;
  for (size_t a = 0; a < m; ++a)
    for (size_t b = 0; b < m; ++b) {
      double n = P.cmat[a * m + b];
      if (n == 0.0) continue;
      s.add(n * (J[a].real() * J[b].real() + J[a].imag() * J[b].imag()));
    }
  return s.val();
}

static Process* create(const int* pdg, int n_ext, double alpha_s) {
  if (n_ext < 4 || n_ext > 9) throw std::runtime_error("n_ext must be 4..9");
  std::unique_ptr<Process> P(new Process());
  P->n_ext = n_ext;
  P->pdg.assign(pdg, pdg + n_ext);
  P->kind.resize(n_ext);
  P->flav.resize(n_ext);
  for (int l = 0; l < n_ext; ++l) {
    int c = pdg[l];
    bool in = l < 2;
    if (c == 21) { P->kind[l] = KG; P->flav[l] = 0; }
    else if (c >= 1 && c <= 6) { P->kind[l] = in ? KPSI : KPSIBAR; P->flav[l] = c; }
    else if (c <= -1 && c >= -6) { P->kind[l] = in ? KPSIBAR : KPSI; P->flav[l] = -c; }
    else throw std::runtime_error("unsupported pdg code");
  }
  P->n_a = pdg[0] == 21 ? 8 : 3;
  P->n_b = pdg[1] == 21 ? 8 : 3;
  P->gs = std::sqrt(4.0 * M_PI * alpha_s);
  P->root = n_ext - 1;
  enumerate(*P);
  if (P->diagrams.empty()) throw std::runtime_error("process has no tree diagrams");
  build_colour(*P);
  return P.release();
}

}  // namespace oq

// ------------------------------------------------------------------- C API
extern "C" {

static thread_local std::string g_err;

const char* oq_last_error() { return g_err.c_str(); }

void* oq_create(const int* pdg, int n_ext, double alpha_s) {
  try {
    return oq::create(pdg, n_ext, alpha_s);
  } catch (std::exception& e) {
    g_err = e.what();
    return nullptr;
  }
}

void oq_destroy(void* h) { delete (oq::Process*)h; }

int oq_info(void* h, int* n_diag, int* n_colour, int* n_topo) {
  oq::Process* P = (oq::Process*)h;
  if (!P) return -1;
  if (n_diag) *n_diag = (int)P->diagrams.size();
  if (n_colour) *n_colour = (int)P->basis.size();
  if (n_topo) *n_topo = P->n_topologies;
  return 0;
}

int oq_max_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// me2[n]: 1/4 sum_h sum_ab J N J*.  me2_hel (nullable): [n][2^n_ext] per
// helicity combination, colour-summed-and-averaged, before the 1/4.
int oq_me2(void* h, const double* mom, long long n, double* me2, double* me2_hel, int nthreads) {
  oq::Process* P = (oq::Process*)h;
  if (!P || !mom || !me2 || n < 0) return -1;
  int nh = 1 << P->n_ext;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  std::string err;
#pragma omp parallel for schedule(dynamic, 1)
  for (long long e = 0; e < n; ++e) {
    try {
      const double* p = mom + (size_t)e * P->n_ext * 4;
      oq::KSum tot;
      std::vector<oq::cd> J;
      for (int hel = 0; hel < nh; ++hel) {
        oq::jamp_one(*P, p, hel, -1, J);
        double v = oq::quad_form(*P, J);
        if (me2_hel) me2_hel[(size_t)e * nh + hel] = v;
        tot.add(v);
      }
      me2[e] = 0.25 * tot.val();
    } catch (std::exception& ex) {
#pragma omp critical
      err = ex.what();
    }
  }
  if (!err.empty()) { g_err = err; return -1; }
  return 0;
}

// Colour amplitudes J_alpha for one event and one helicity combination.
// ward_leg >= 0 replaces that gluon's polarisation by k/E.  jamp: [2*m] (re, im).
int oq_jamp(void* h, const double* mom, int hel, int ward_leg, double* jamp) {
  oq::Process* P = (oq::Process*)h;
  if (!P || !mom || !jamp) return -1;
  try {
    std::vector<oq::cd> J;
    oq::jamp_one(*P, mom, hel, ward_leg, J);
    for (size_t a = 0; a < J.size(); ++a) { jamp[2 * a] = J[a].real(); jamp[2 * a + 1] = J[a].imag(); }
  } catch (std::exception& ex) {
    g_err = ex.what();
    return -1;
  }
  return 0;
}

// Colour matrix (real parts, including 1/(n_a n_b)), [m*m].
int oq_colour_matrix(void* h, double* out) {
  oq::Process* P = (oq::Process*)h;
  if (!P || !out) return -1;
  std::copy(P->cmat.begin(), P->cmat.end(), out);
  return 0;
}

// Exact colour matrix as rationals: num_re, den_re, num_im, den_im, each [m*m].
int oq_colour_matrix_exact(void* h, long long* nre, long long* dre, long long* nim, long long* dim) {
  oq::Process* P = (oq::Process*)h;
  if (!P) return -1;
  for (size_t i = 0; i < P->cmat_exact.size(); ++i) {
    nre[i] = P->cmat_exact[i].re.n; dre[i] = P->cmat_exact[i].re.d;
    nim[i] = P->cmat_exact[i].im.n; dim[i] = P->cmat_exact[i].im.d;
  }
  return 0;
}

// Basis element alpha as a flat int list: repeated [len, closed, row, col, gluons...].
int oq_basis(void* h, int alpha, int* buf, int buflen) {
  oq::Process* P = (oq::Process*)h;
  if (!P || alpha < 0 || alpha >= (int)P->basis.size()) return -1;
  const auto& k = P->basis[alpha];
  if ((int)k.size() > buflen) return -2;
  for (size_t i = 0; i < k.size(); ++i) buf[i] = k[i];
  return (int)k.size();
}

// Colour coefficients of diagram d: writes up to cap (alpha, re, im) triples.
int oq_diagram_colour(void* h, int d, int* alpha, double* re, double* im, int cap) {
  oq::Process* P = (oq::Process*)h;
  if (!P || d < 0 || d >= (int)P->diagrams.size()) return -1;
  const auto& v = P->coefd[d];
  int n = 0;
  for (auto& x : v) {
    if (n >= cap) break;
    alpha[n] = x.first; re[n] = x.second.real(); im[n] = x.second.imag();
    ++n;
  }
  return (int)v.size();
}

}  // extern "C"
