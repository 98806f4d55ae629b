// Device library of wavefunction, vertex and off-shell-current functions
// (the HEGET set of arXiv:0909.5257, Sec. 4 and Appendix A), written for
// sm_103a and templated on the real type (float for the mixed path, double
// for the FP64 path).
//
// Conventions (HELAS): every vector wavefunction is a contravariant complex
// 4-vector, dot products carry the metric (+,-,-,-), and the momentum attached
// to a wavefunction is the flowing-OUT momentum of the partons below it.
// Spinors use the chiral representation, upper two components left-handed.
//
// Colour factors that go with each function (applied by the generator):
//   vvv_amp, jvv          : i f^{abc}                         (Sec. 4.1)
//   gggg_amp, jggg calls  : f^{abe}f^{cde}, f^{ace}f^{dbe},
//                           f^{ade}f^{bce} for the three calls  (Sec. 4.2)
//   iov_amp               : -T^a_{ij}                          (Eq. (qqg-amplitude))
//   fvi, fvo, jio         : T^a
// With these, every current equals the Feynman-rule current and every
// amplitude equals -i times the Feynman-rule vertex, so that each diagram
// yields M with one common phase.
#pragma once

#ifndef MEA_HD
#define MEA_HD __host__ __device__ __forceinline__
#endif

template <typename R>
struct cx {
  R r, i;
};

template <typename R>
MEA_HD cx<R> mk(R r, R i) { return cx<R>{r, i}; }
template <typename R>
MEA_HD cx<R> operator+(cx<R> a, cx<R> b) { return {a.r + b.r, a.i + b.i}; }
template <typename R>
MEA_HD cx<R> operator-(cx<R> a, cx<R> b) { return {a.r - b.r, a.i - b.i}; }
template <typename R>
MEA_HD cx<R> operator-(cx<R> a) { return {-a.r, -a.i}; }
template <typename R>
MEA_HD cx<R> operator*(cx<R> a, cx<R> b) {
  return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r};
}
template <typename R>
MEA_HD cx<R> operator*(R s, cx<R> a) { return {s * a.r, s * a.i}; }
template <typename R>
MEA_HD cx<R> conj(cx<R> a) { return {a.r, -a.i}; }
template <typename R>
MEA_HD cx<R> times_i(cx<R> a) { return {-a.i, a.r}; }

// Four complex components: a vector (contravariant) or a Dirac spinor.
template <typename R>
struct W4 {
  cx<R> c[4];
};

// a.b = a0 b0 - a1 b1 - a2 b2 - a3 b3 for complex vectors
template <typename R>
MEA_HD cx<R> dot(const W4<R>& a, const W4<R>& b) {
  return a.c[0] * b.c[0] - a.c[1] * b.c[1] - a.c[2] * b.c[2] - a.c[3] * b.c[3];
}
// p.a for a real vector p
template <typename R>
MEA_HD cx<R> dot(const R* p, const W4<R>& a) {
  return p[0] * a.c[0] - p[1] * a.c[1] - p[2] * a.c[2] - p[3] * a.c[3];
}

// ---------------------------------------------------------------- ggg vertex
// Feynman rule of the three-gluon term of the Lagrangian (Sec. 4.1) with the
// colour factor i f^{abc} taken off and all three momenta k1, k2, k3 flowing
// into the vertex:
//   Gamma^{mu nu rho}(k1, k2, k3) = g^{mu nu} (k1 - k2)^rho + g^{nu rho} (k2 - k3)^mu
//                                 + g^{rho mu} (k3 - k1)^nu,
// unchanged by a cyclic shift of its (index, momentum) pairs.  Contracting the
// nu and rho slots with wavefunctions y and z leaves a vector in mu:
//   O^mu(y, z) = y^mu (k1 - k2).z + (k2 - k3)^mu (y.z) + z^mu (k3 - k1).y .
// HEGET normalisation (Sec. 4.1): an amplitude is -g times the full
// contraction, an off-shell current -g O / q^2.  Everything below is built on
// the one open contraction, so vertex, current and vertex partial share it.

// -g O^mu(y, z): the ggg vertex with the slot of momentum k1 left open (also
// the vertex partial of a diagram whose free wavefunction sits in that slot)
template <typename R>
MEA_HD W4<R> vvv_part(const W4<R>& y, const W4<R>& z, const R* k1, const R* k2, const R* k3, R g) {
  R d12[4], d23[4], d31[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    d12[m] = k1[m] - k2[m];
    d23[m] = k2[m] - k3[m];
    d31[m] = k3[m] - k1[m];
  }
  const R ng = -g;
  const cx<R> along_y = ng * dot(d12, z);
  const cx<R> along_z = ng * dot(d31, y);
  const cx<R> along_d = ng * dot(y, z);
  W4<R> o;
#pragma unroll
  for (int m = 0; m < 4; ++m) o.c[m] = along_y * y.c[m] + along_z * z.c[m] + d23[m] * along_d;
  return o;
}

// Amplitude of three gluon wavefunctions x, y, z with momenta kx, ky, kz into
// the vertex (vvvxxx): the open slot of -g O(y, z) closed with x.
template <typename R>
MEA_HD cx<R> vvv_amp(const W4<R>& x, const W4<R>& y, const W4<R>& z, const R* kx, const R* ky, const R* kz, R g) {
  return dot(x, vvv_part(y, z, kx, ky, kz, g));
}

// Off-shell gluon from two gluon wavefunctions (jvvxx0, listed as jggxxx):
// the open slot carries the current's momentum into the vertex, -(kx + ky),
// times the Feynman-gauge propagator factor 1/q^2 (inv_q2, from the prep).
template <typename R>
MEA_HD W4<R> jvv(const W4<R>& x, const W4<R>& y, const R* kx, const R* ky, R inv_q2, R g) {
  R k_open[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) k_open[m] = -(kx[m] + ky[m]);
  W4<R> o = vvv_part(x, y, k_open, kx, ky, g);
#pragma unroll
  for (int m = 0; m < 4; ++m) o.c[m] = inv_q2 * o.c[m];
  return o;
}

// ---------------------------------------------------------------- gggg vertex
// One colour structure of the four-gluon term (Sec. 4.2; the three structures
// f^{abe}f^{cde}, f^{ace}f^{dbe}, f^{ade}f^{bce} are three calls with the
// wavefunctions permuted), coupling gg = g_s^2.  With one slot open the
// structure is the vector
//   G(x, y, z) = gg [ z (x.y) - y (x.z) ]   (so G(x, y, z) = -G(x, z, y)),
// and the amplitude of four wavefunctions is
//   a . G(b, c, d) = gg [ (a.d)(b.c) - (a.c)(b.d) ] = b.G(a, d, c) = c.G(d, a, b) = d.G(c, b, a).
template <typename R>
MEA_HD W4<R> gggg_part(const W4<R>& x, const W4<R>& y, const W4<R>& z, R gg) {
  const cx<R> xy = gg * dot(x, y), xz = gg * dot(x, z);
  W4<R> o;
#pragma unroll
  for (int m = 0; m < 4; ++m) o.c[m] = xy * z.c[m] - xz * y.c[m];
  return o;
}

// Amplitude of one gggg colour structure (ggggxx).
template <typename R>
MEA_HD cx<R> gggg_amp(const W4<R>& a, const W4<R>& b, const W4<R>& c, const W4<R>& d, R gg) {
  return dot(a, gggg_part(b, c, d, gg));
}

// Off-shell gluon of one gggg colour structure (jgggx0): the open first slot
// of ggggxx(open, c, b, a), G(c, b, a) = gg [ a (c.b) - b (c.a) ], times 1/q^2.
template <typename R>
MEA_HD W4<R> jggg(const W4<R>& a, const W4<R>& b, const W4<R>& c, R inv_q2, R gg) {
  W4<R> o = gggg_part(c, b, a, gg);
#pragma unroll
  for (int m = 0; m < 4; ++m) o.c[m] = inv_q2 * o.c[m];
  return o;
}

// ---------------------------------------------------------------- qqg
// slash(V) psi for a column spinor, V contravariant complex.
template <typename R>
MEA_HD W4<R> slash_col(const W4<R>& V, const W4<R>& s) {
  cx<R> vp = V.c[0] + V.c[3], vm = V.c[0] - V.c[3];
  cx<R> v12m = V.c[1] - times_i(V.c[2]);  // V1 - i V2
  cx<R> v12p = V.c[1] + times_i(V.c[2]);  // V1 + i V2
  W4<R> o;
  o.c[0] = vm * s.c[2] - v12m * s.c[3];
  o.c[1] = vp * s.c[3] - v12p * s.c[2];
  o.c[2] = vp * s.c[0] + v12m * s.c[1];
  o.c[3] = v12p * s.c[0] + vm * s.c[1];
  return o;
}
// barred spinor (row) times slash(V)
template <typename R>
MEA_HD W4<R> row_slash(const W4<R>& s, const W4<R>& V) {
  cx<R> vp = V.c[0] + V.c[3], vm = V.c[0] - V.c[3];
  cx<R> v12m = V.c[1] - times_i(V.c[2]);
  cx<R> v12p = V.c[1] + times_i(V.c[2]);
  W4<R> o;
  o.c[0] = s.c[2] * vp + s.c[3] * v12p;
  o.c[1] = s.c[2] * v12m + s.c[3] * vm;
  o.c[2] = s.c[0] * vm - s.c[1] * v12p;
  o.c[3] = s.c[1] * vp - s.c[0] * v12m;
  return o;
}
// slash(P) for a real momentum
template <typename R>
MEA_HD W4<R> slash_real_col(const R* P, const W4<R>& s) {
  R vp = P[0] + P[3], vm = P[0] - P[3];
  cx<R> v12m = mk<R>(P[1], -P[2]);
  cx<R> v12p = mk<R>(P[1], P[2]);
  W4<R> o;
  o.c[0] = vm * s.c[2] - v12m * s.c[3];
  o.c[1] = vp * s.c[3] - v12p * s.c[2];
  o.c[2] = vp * s.c[0] + v12m * s.c[1];
  o.c[3] = v12p * s.c[0] + vm * s.c[1];
  return o;
}
template <typename R>
MEA_HD W4<R> row_slash_real(const W4<R>& s, const R* P) {
  R vp = P[0] + P[3], vm = P[0] - P[3];
  cx<R> v12m = mk<R>(P[1], -P[2]);
  cx<R> v12p = mk<R>(P[1], P[2]);
  W4<R> o;
  o.c[0] = vp * s.c[2] + s.c[3] * v12p;
  o.c[1] = s.c[2] * v12m + vm * s.c[3];
  o.c[2] = vm * s.c[0] - s.c[1] * v12p;
  o.c[3] = vp * s.c[1] - s.c[0] * v12m;
  return o;
}

// iovxx0: amplitude  g * fo slash(V) fi  (colour -T^a, Eq. (qqg-amplitude))
template <typename R>
MEA_HD cx<R> iov_amp(const W4<R>& fi, const W4<R>& fo, const W4<R>& v, R g) {
  W4<R> t = slash_col(v, fi);
  cx<R> s = fo.c[0] * t.c[0] + fo.c[1] * t.c[1] + fo.c[2] * t.c[2] + fo.c[3] * t.c[3];
  return g * s;
}

// Off-shell quark from fi and a gluon: Feynman current (i Q/Q^2)(-i g V) fi with
// Q = -P the momentum along the fermion arrow, P the flowing-out momentum:
//   -(g/P^2) slash(P) slash(V) fi
template <typename R>
MEA_HD W4<R> fvi(const W4<R>& fi, const W4<R>& v, const R* P, R inv_p2, R g) {
  W4<R> t = slash_col(v, fi);
  W4<R> u = slash_real_col(P, t);
  R f = -g * inv_p2;
#pragma unroll
  for (int m = 0; m < 4; ++m) u.c[m] = f * u.c[m];
  return u;
}
// Off-shell barred quark: fo (-i g V)(i P / P^2) = (g/P^2) fo slash(V) slash(P)
template <typename R>
MEA_HD W4<R> fvo(const W4<R>& fo, const W4<R>& v, const R* P, R inv_p2, R g) {
  W4<R> t = row_slash(fo, v);
  W4<R> u = row_slash_real(t, P);
  R f = g * inv_p2;
#pragma unroll
  for (int m = 0; m < 4; ++m) u.c[m] = f * u.c[m];
  return u;
}
// Off-shell gluon from a quark pair: J^mu = -(g/q^2) fo gamma^mu fi
template <typename R>
MEA_HD W4<R> jio(const W4<R>& fi, const W4<R>& fo, R inv_q2, R g) {
  const W4<R>& a = fo;
  const W4<R>& b = fi;
  cx<R> j0 = a.c[0] * b.c[2] + a.c[1] * b.c[3] + a.c[2] * b.c[0] + a.c[3] * b.c[1];
  cx<R> j1 = a.c[0] * b.c[3] + a.c[1] * b.c[2] - a.c[2] * b.c[1] - a.c[3] * b.c[0];
  cx<R> j2 = times_i(a.c[1] * b.c[2] - a.c[0] * b.c[3] + a.c[2] * b.c[1] - a.c[3] * b.c[0]);
  cx<R> j3 = a.c[0] * b.c[2] - a.c[1] * b.c[3] - a.c[2] * b.c[0] + a.c[3] * b.c[1];
  R f = -g * inv_q2;
  W4<R> j;
  j.c[0] = f * j0; j.c[1] = f * j1; j.c[2] = f * j2; j.c[3] = f * j3;
  return j;
}

// ------------------------------------------------------- vertex partials
// Every amplitude vertex is linear in each of its wavefunctions.  Diagrams
// whose amplitude vertex shares all but one input (the "free" one) share the
// vertex with that input taken out -- a complex 4-vector, the partial -- and
// each diagram amplitude is then the contraction of its free wavefunction
// with the partial.  The amplitude of every diagram is still formed and
// summed into the colour amplitudes on its own; only the common factor of the
// vertex is computed once.

// vvv_part and gggg_part above are the partials of vvvxxx and ggggxx: any
// slot of either can be the free one (cyclic shift of vvvxxx; the four slot
// orders of ggggxx listed with G).

// iovxx0 = g fo slash(V) fi with V free: the vector g fo gamma^mu fi, so that
// iov_amp = V . P (metric contraction).
template <typename R>
MEA_HD W4<R> iov_part_v(const W4<R>& fi, const W4<R>& fo, R g) {
  const W4<R>& a = fo;
  const W4<R>& b = fi;
  W4<R> j;
  j.c[0] = g * (a.c[0] * b.c[2] + a.c[1] * b.c[3] + a.c[2] * b.c[0] + a.c[3] * b.c[1]);
  j.c[1] = g * (a.c[0] * b.c[3] + a.c[1] * b.c[2] - a.c[2] * b.c[1] - a.c[3] * b.c[0]);
  j.c[2] = g * times_i(a.c[1] * b.c[2] - a.c[0] * b.c[3] + a.c[2] * b.c[1] - a.c[3] * b.c[0]);
  j.c[3] = g * (a.c[0] * b.c[2] - a.c[1] * b.c[3] - a.c[2] * b.c[0] + a.c[3] * b.c[1]);
  return j;
}
// ... with fi free: the row spinor g fo slash(V), iov_amp = sum_k P_k fi_k.
template <typename R>
MEA_HD W4<R> iov_part_i(const W4<R>& fo, const W4<R>& v, R g) {
  W4<R> t = row_slash(fo, v);
#pragma unroll
  for (int m = 0; m < 4; ++m) t.c[m] = g * t.c[m];
  return t;
}
// ... with fo free: the column spinor g slash(V) fi, iov_amp = sum_k fo_k P_k.
template <typename R>
MEA_HD W4<R> iov_part_o(const W4<R>& fi, const W4<R>& v, R g) {
  W4<R> t = slash_col(v, fi);
#pragma unroll
  for (int m = 0; m < 4; ++m) t.c[m] = g * t.c[m];
  return t;
}

// Contraction of a free wavefunction with a partial: metric (vector partials)
// or plain (spinor partials), negated when neg is set.
template <typename R>
MEA_HD cx<R> part_contract(const W4<R>& w, const W4<R>& p, bool plain, bool neg) {
  cx<R> s = w.c[0] * p.c[0];
  if (plain) s = s + w.c[1] * p.c[1] + w.c[2] * p.c[2] + w.c[3] * p.c[3];
  else s = s - w.c[1] * p.c[1] - w.c[2] * p.c[2] - w.c[3] * p.c[3];
  return neg ? -s : s;
}

// ------------------------------------------------------- external states
// Gluon of helicity lam with transverse unit vectors e1, e2 (e1 x e2 = p_hat):
// eps = (-lam e1 - i e2)/sqrt2, conjugated for an outgoing gluon.
template <typename R>
MEA_HD W4<R> ext_gluon(const R* e1, const R* e2, int lam, bool outgoing) {
  const R r = R(0.70710678118654752440);
  R sgn = outgoing ? R(1) : R(-1);
  W4<R> w;
  w.c[0] = mk<R>(R(0), R(0));
#pragma unroll
  for (int k = 0; k < 3; ++k) w.c[k + 1] = mk<R>(-R(lam) * e1[k] * r, sgn * e2[k] * r);
  return w;
}

// Massless spinors from r = sqrt(2E) and chi_+ = (a, b) (a real),
// chi_- = (-b*, a).  kind: 0 u, 1 v, 2 ubar, 3 vbar.
template <typename R>
MEA_HD W4<R> ext_spinor(R r, R a, cx<R> b, int lam, int kind) {
  W4<R> s;
  cx<R> z = mk<R>(R(0), R(0));
  cx<R> ra = mk<R>(r * a, R(0));
  cx<R> rb = r * b;
  cx<R> rbc = conj(rb);
  bool plus = lam > 0;
  if (kind == 0 || kind == 2) {          // u
    if (plus) { s.c[0] = z; s.c[1] = z; s.c[2] = ra; s.c[3] = rb; }
    else { s.c[0] = -rbc; s.c[1] = ra; s.c[2] = z; s.c[3] = z; }
  } else {                               // v
    if (plus) { s.c[0] = -rbc; s.c[1] = ra; s.c[2] = z; s.c[3] = z; }
    else { s.c[0] = z; s.c[1] = z; s.c[2] = -ra; s.c[3] = -rb; }
  }
  if (kind >= 2) {                       // bar: psi^dagger gamma^0
    W4<R> t;
    t.c[0] = conj(s.c[2]); t.c[1] = conj(s.c[3]); t.c[2] = conj(s.c[0]); t.c[3] = conj(s.c[1]);
    return t;
  }
  return s;
}
