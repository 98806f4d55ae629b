"""Independent reference formulas used to pin the oracle (test side only).

Nothing here is shared with the oracle or with the CUDA path; each function is
a textbook result restated from its published form:

* 2 -> 2 colour/spin-averaged |M|^2 (Combridge, Kripfganz, Ranft 1977; the
  forms quoted in Ellis-Stirling-Webber, "QCD and collider physics", Table 7.1),
* Parke-Taylor MHV amplitudes and the n <= 5 colour sum,
* the Berends-Giele recursion with colour-ordered Feynman rules (Berends and
  Giele, Nucl. Phys. B306 (1988) 759; rules as in Dixon, TASI 1995 lectures),
* explicit Gell-Mann generators T = lambda/2 for brute-force colour sums,
* rotations and z-boosts for Lorentz-invariance checks.
"""
from __future__ import annotations

import itertools
import math
from functools import lru_cache

import numpy as np

METRIC = np.array([1.0, -1.0, -1.0, -1.0])


def mdot(a, b):
    return a[..., 0] * b[..., 0] - (a[..., 1:] * b[..., 1:]).sum(-1)


def g_s(alpha_s=0.118):
    return math.sqrt(4.0 * math.pi * alpha_s)


# --------------------------------------------------------------- 2 -> 2 forms
def mandelstam(mom):
    pa, pb, p1, p2 = (mom[:, i] for i in range(4))
    return mdot(pa + pb, pa + pb), mdot(pa - p1, pa - p1), mdot(pa - p2, pa - p2)


def me2_gg_gg(mom, alpha_s=0.118):
    s, t, u = mandelstam(mom)
    g4 = g_s(alpha_s) ** 4
    return 4.5 * g4 * (3.0 - t * u / s**2 - s * u / t**2 - s * t / u**2)


def me2_uubar_gg(mom, alpha_s=0.118):
    s, t, u = mandelstam(mom)
    g4 = g_s(alpha_s) ** 4
    return g4 * ((32.0 / 27.0) * (t * t + u * u) / (t * u) - (8.0 / 3.0) * (t * t + u * u) / s**2)


def me2_uu_uu(mom, alpha_s=0.118):
    s, t, u = mandelstam(mom)
    g4 = g_s(alpha_s) ** 4
    return g4 * ((4.0 / 9.0) * ((s * s + u * u) / t**2 + (s * s + t * t) / u**2)
                 - (8.0 / 27.0) * s * s / (t * u))


# ------------------------------------------------------------ all-outgoing
def all_outgoing(mom_one):
    """Momenta with incoming legs (0, 1) negated."""
    k = np.array(mom_one, dtype=np.float64).copy()
    k[:2] *= -1.0
    return k


def helicities(hel_index, n_ext):
    """Physical helicities of combination hel_index (bit n_ext-1-i -> leg i)."""
    return [1 if (hel_index >> (n_ext - 1 - i)) & 1 else -1 for i in range(n_ext)]


def outgoing_helicities(hel_index, n_ext):
    """Helicities in the all-outgoing convention (incoming ones flip)."""
    h = helicities(hel_index, n_ext)
    return [-h[0], -h[1]] + h[2:]


# ------------------------------------------------------------- Parke-Taylor
def quark_line_mhv_sq(k, order, q_minus, q_plus, g_minus):
    """|A(order)|^2 of the colour-ordered MHV amplitude with one quark line:
    all-outgoing antiquark/quark legs q_minus (helicity -) and q_plus (+), one
    negative-helicity gluon g_minus, the rest positive:
    |s_{q- g-}|^3 |s_{q+ g-}| / |s_12 s_23 ... s_n1| over the cyclic order
    (quark pair adjacent), normalisation Tr(T^a T^b) = delta^{ab}."""
    def s(a, b):
        return abs(mdot(k[a] + k[b], k[a] + k[b]))
    den = 1.0
    n = len(order)
    for a in range(n):
        den *= s(order[a], order[(a + 1) % n])
    return s(q_minus, g_minus) ** 3 * s(q_plus, g_minus) / den


def parke_taylor_sq(k, order, neg):
    """|A(order)|^2 for the MHV configuration whose two negative-helicity legs
    (all-outgoing convention) are `neg`: s_ij^4 / |s_12 s_23 ... s_n1|,
    normalisation Tr(T^a T^b) = delta^{ab}."""
    i, j = neg
    sij = mdot(k[i] + k[j], k[i] + k[j])
    den = 1.0
    n = len(order)
    for a in range(n):
        x, y = order[a], order[(a + 1) % n]
        den *= mdot(k[x] + k[y], k[x] + k[y])
    return sij**4 / abs(den)


def gluon_me2_leading_colour_exact(mom_one, alpha_s=0.118, nc=3):
    """gg -> (n-2) g for n = 4, 5: all non-vanishing helicity amplitudes are MHV
    or anti-MHV and the leading-colour sum is exact there, so
    sum |M|^2 = g^{2n-4} N^{n-2} (N^2-1) sum_{sigma in S_{n-1}} sum_hel |A(1,sigma)|^2,
    averaged by 1/4 * 1/64."""
    k = all_outgoing(mom_one)
    n = k.shape[0]
    assert n in (4, 5)
    tot = 0.0
    for rest in itertools.permutations(range(1, n)):
        order = (0,) + rest
        s = 0.0
        for neg in itertools.combinations(range(n), 2):
            s += parke_taylor_sq(k, order, neg)
        if n == 5:
            s *= 2.0  # anti-MHV configurations (two positive helicities)
        tot += s
    g = g_s(alpha_s)
    return g ** (2 * n - 4) * nc ** (n - 2) * (nc * nc - 1) * tot / 256.0


# ------------------------------------------------------- polarisation vectors
def transverse_pair(kvec):
    """Right-handed orthonormal (e1, e2) with e1 x e2 = k_hat, built from a
    fixed reference axis (a different gauge from the oracle's)."""
    kh = kvec / np.linalg.norm(kvec)
    ref = np.array([0.3, 0.5, 0.8]) / np.linalg.norm([0.3, 0.5, 0.8])
    e1 = np.cross(ref, kh)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(kh, e1)
    return e1, e2


def polarisation(p, lam, outgoing):
    """eps^mu(p, lam) (upper index); conjugated for an outgoing gluon."""
    e1, e2 = transverse_pair(p[1:])
    v = (e1 + 1j * lam * e2) / math.sqrt(2.0)
    eps = np.concatenate([[0.0 + 0j], v])
    return np.conj(eps) if outgoing else eps


# ------------------------------------------------------------ Berends-Giele
def _v3(P, Q, a, b):
    """Colour-ordered three-vertex contracted with upper-index currents a (momentum
    P outgoing into it) and b (momentum Q), giving an upper-index vector:
    V3 = (i/sqrt2) [ g^{nu rho}(P-Q)^mu + 2 g^{rho mu} Q^nu - 2 g^{mu nu} P^rho ]."""
    ab = mdot(a, b)
    return (1j / math.sqrt(2.0)) * (ab * (P - Q) + 2.0 * mdot(Q, a) * b - 2.0 * mdot(P, b) * a)


def _v4(a, b, c):
    """Colour-ordered four-vertex: (i/2)[2 g^{mu rho} g^{nu sigma} - g^{mu nu} g^{rho sigma}
    - g^{mu sigma} g^{nu rho}] contracted with a (nu), b (rho), c (sigma)."""
    return (1j / 2.0) * (2.0 * mdot(a, c) * b - mdot(b, c) * a - mdot(a, b) * c)


def bg_amplitude(k, eps, order):
    """Colour-ordered amplitude A(order) by the Berends-Giele recursion.

    k: all-outgoing momenta [n, 4]; eps: external upper-index polarisation
    vectors [n, 4]; order: tuple of leg indices.  Normalisation Tr(T T) = delta.
    """
    n = len(order)
    seq = order[:-1]

    def vertices(i, j):
        """Sum of vertices joining sub-currents of seq[i..j] (no propagator)."""
        acc = np.zeros(4, dtype=complex)
        for m in range(i, j):
            Pa = sum(k[seq[x]] for x in range(i, m + 1))
            Pb = sum(k[seq[x]] for x in range(m + 1, j + 1))
            acc = acc + _v3(Pa, Pb, J(i, m), J(m + 1, j))
        for m in range(i, j):
            for l in range(m + 1, j):
                acc = acc + _v4(J(i, m), J(m + 1, l), J(l + 1, j))
        return acc

    @lru_cache(maxsize=None)
    def J(i, j):
        if i == j:
            return eps[seq[i]]
        P = sum(k[seq[x]] for x in range(i, j + 1))
        return (-1j / mdot(P, P)) * vertices(i, j)

    # the last current is on shell: contract its vertex sum (amputated) with eps_n
    return mdot(vertices(0, n - 2), eps[order[-1]])


# -------------------------------------------- Berends-Giele, one quark line
# Dirac matrices in the chiral representation (upper two components
# left-handed), built here independently of the oracle.
_SIG = [np.array([[0, 1], [1, 0]], dtype=complex), np.array([[0, -1j], [1j, 0]], dtype=complex),
        np.array([[1, 0], [0, -1]], dtype=complex)]
_Z2 = np.zeros((2, 2), dtype=complex)
_GAMMA = [np.block([[_Z2, np.eye(2)], [np.eye(2), _Z2]]).astype(complex)] + \
         [np.block([[_Z2, s], [-s, _Z2]]) for s in _SIG]


def slash(v):
    """gamma^mu v_mu for an upper-index (complex) 4-vector v."""
    return _GAMMA[0] * v[0] - _GAMMA[1] * v[1] - _GAMMA[2] * v[2] - _GAMMA[3] * v[3]


def _helicity_spinor(pvec, lam):
    """Two-component helicity eigenstate of sigma.p_hat with eigenvalue lam."""
    p = np.linalg.norm(pvec)
    th = math.acos(max(-1.0, min(1.0, pvec[2] / p)))
    ph = math.atan2(pvec[1], pvec[0])
    if lam > 0:
        return np.array([math.cos(th / 2), np.exp(1j * ph) * math.sin(th / 2)])
    return np.array([-np.exp(-1j * ph) * math.sin(th / 2), math.cos(th / 2)])


def u_spinor(p, lam):
    """Massless Dirac spinor u(p, lam): left-handed (upper) for lam = -1."""
    r = math.sqrt(2.0 * p[0])
    c = _helicity_spinor(p[1:], lam)
    return r * np.concatenate([c, [0, 0]]) if lam < 0 else r * np.concatenate([[0, 0], c])


def vbar_spinor(p, lam):
    """v-bar(p, lam) = v^dagger gamma^0 with v(p, lam) = u(p, -lam) up to a phase."""
    return u_spinor(p, -lam).conj() @ _GAMMA[0]


def bg_quark_line_amplitude(mom, eps, gluons, ubar_left, u_right):
    """Colour-ordered amplitude of one quark line with gluons attached in the
    order `gluons` (the order of the generators in the colour string, read from
    the barred end), by the Berends-Giele recursion with colour-ordered rules:
    qqg vertex (i/sqrt2) gamma^mu, quark propagator i P-slash / P^2, the gluon
    sub-currents of consecutive gluons as in bg_amplitude.  mom: physical
    momenta [n, 4] (leg 0 the incoming quark, gluons outgoing); eps: outgoing
    gluon polarisation vectors by leg; ubar_left / u_right: the external
    spinors at the two ends of the line.  Normalisation Tr(T T) = delta."""
    kg = len(gluons)

    @lru_cache(maxsize=None)
    def J(i, j):
        if i == j:
            return eps[gluons[i]]
        P = sum(mom[gluons[x]] for x in range(i, j + 1))
        acc = np.zeros(4, dtype=complex)
        for m in range(i, j):
            Pa = sum(mom[gluons[x]] for x in range(i, m + 1))
            Pb = sum(mom[gluons[x]] for x in range(m + 1, j + 1))
            acc = acc + _v3(Pa, Pb, J(i, m), J(m + 1, j))
        for m in range(i, j):
            for l in range(m + 1, j):
                acc = acc + _v4(J(i, m), J(m + 1, l), J(l + 1, j))
        return (-1j / mdot(P, P)) * acc

    @lru_cache(maxsize=None)
    def R(j):
        """Column spinor of the line from gluon j to the unbarred end."""
        if j == kg:
            return u_right
        acc = np.zeros(4, dtype=complex)
        for m in range(j, kg):
            rest = R(m + 1)
            if m + 1 < kg:  # quark propagator between this block and the next
                Pq = mom[0] - sum(mom[gluons[x]] for x in range(m + 1, kg))
                rest = (1j * slash(Pq) / mdot(Pq, Pq)) @ rest
            acc = acc + (1j / math.sqrt(2.0)) * (slash(J(j, m)) @ rest)
        return acc

    return ubar_left @ R(0)


# ------------------------------- two quark lines by explicit Feynman diagrams
def _ubar(p, lam):
    return u_spinor(p, lam).conj() @ _GAMMA[0]


_METRIC = np.diag([1.0, -1.0, -1.0, -1.0])


def _mu_vec(bar, ket, mid=None):
    """bar gamma^mu [mid] ket for mu = 0..3 (upper index)."""
    m = np.eye(4) if mid is None else mid
    return np.array([bar @ _GAMMA[k] @ m @ ket for k in range(4)])


def quark_quark_gluon_diagrams(m, lam, g, ward=False):
    """Lorentz values (couplings, propagators and i's included) of the five
    tree diagrams of q(p0) Q(p1) -> q(p2) Q(p3) g(p4) for distinct quark
    lines q and Q, from the textbook Feynman-gauge rules (Peskin-Schroeder
    conventions: qqg vertex i g gamma^mu t^a, three-gluon vertex
    g f^{abc}[g^{mu nu}(k-p)^rho + g^{nu rho}(p-q)^mu + g^{rho mu}(q-k)^nu]
    with incoming momenta, gluon propagator -i g_{mu nu}/k^2, quark
    propagator i k-slash/k^2), in the order: gluon from incoming q, outgoing q,
    incoming Q, outgoing Q, and from the exchanged gluon.  ward=True replaces
    the gluon's polarisation by its momentum."""
    p0, p1, p2, p3, p4 = m
    u0, u1 = u_spinor(p0, lam[0]), u_spinor(p1, lam[1])
    b2, b3 = _ubar(p2, lam[2]), _ubar(p3, lam[3])
    eps = p4.astype(complex) if ward else polarisation(p4, lam[4], outgoing=True)
    es = slash(eps)
    ig = 1j * g
    J1, J2 = _mu_vec(b2, u0), _mu_vec(b3, u1)
    q1, q2 = p0 - p2, p1 - p3

    def prop_q(k):
        return 1j * slash(k) / mdot(k, k)

    def dot(a, b):
        return a @ _METRIC @ b

    L = np.zeros(5, dtype=complex)
    for d, (bar, ket, k, outgoing, other, q) in enumerate(
            ((b2, u0, p0 - p4, False, J2, q2), (b2, u0, p2 + p4, True, J2, q2),
             (b3, u1, p1 - p4, False, J1, q1), (b3, u1, p3 + p4, True, J1, q1))):
        S = prop_q(k)
        if outgoing:  # gluon off the outgoing quark: next to the barred spinor
            A = np.array([bar @ es @ S @ _GAMMA[mu] @ ket for mu in range(4)])
        else:         # gluon off the incoming quark
            A = np.array([bar @ _GAMMA[mu] @ S @ es @ ket for mu in range(4)])
        L[d] = ig ** 3 * (-1j / mdot(q, q)) * dot(A, other)
    X1 = ig * J1 * (-1j / mdot(q1, q1))
    X2 = ig * J2 * (-1j / mdot(q2, q2))
    k4 = -p4
    L[4] = g * (dot(eps, X1) * dot(k4 - q1, X2) + dot(X1, X2) * dot(q1 - q2, eps) + dot(X2, eps) * dot(q2 - k4, X1))
    return L


def quark_quark_gluon_colours():
    """Colour tensors C_d[i_out q, i_in q, j_out Q, j_in Q, a] of the five
    diagrams, explicit SU(3) generators t = lambda/2 and
    f^{abc} = -2i Tr([t^a, t^b] t^c)."""
    T = gell_mann_T()
    f = np.zeros((8, 8, 8))
    for a in range(8):
        for b in range(8):
            comm = T[a] @ T[b] - T[b] @ T[a]
            for c in range(8):
                f[a, b, c] = np.real(-2j * np.trace(comm @ T[c]))
    C = np.zeros((5, 3, 3, 3, 3, 8), dtype=complex)
    C[0] = np.einsum("bxy,ayz,bwv->xzwva", T, T, T)
    C[1] = np.einsum("axy,byz,bwv->xzwva", T, T, T)
    C[2] = np.einsum("bxz,bwy,ayv->xzwva", T, T, T)
    C[3] = np.einsum("bxz,awy,byv->xzwva", T, T, T)
    C[4] = np.einsum("abc,bxz,cwv->xzwva", f, T, T)
    return C


# --------------------------------------------------------------- Gell-Mann
def gell_mann_T():
    l = np.zeros((8, 3, 3), dtype=complex)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1] = -1j; l[1][1, 0] = 1j
    l[2][0, 0] = 1; l[2][1, 1] = -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2] = -1j; l[4][2, 0] = 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2] = -1j; l[6][2, 1] = 1j
    l[7] = np.diag([1, 1, -2]) / math.sqrt(3.0)
    return l / 2.0


def colour_tensor(chains, legs_kind):
    """Numerical colour tensor of a product of chains over all external colour
    indices.  chains: list of (closed, row, col, gluon_legs); legs_kind: 'g' or
    'q' per leg.  Returns an array with one axis per leg (8 for a gluon, 3 for a
    quark), built by explicit index contraction with Gell-Mann generators."""
    T = gell_mann_T()
    letters = iter("abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ")
    leg_letter = {i: next(letters) for i in range(len(legs_kind))}
    operands, subs = [], []
    for closed, row, col, gl in chains:
        if not gl:
            operands.append(np.eye(3))
            subs.append(leg_letter[row] + leg_letter[col])
            continue
        inner = [next(letters) for _ in range(len(gl) + 1)]
        if closed:
            inner[-1] = inner[0]
        else:
            inner[0] = leg_letter[row]
            inner[-1] = leg_letter[col]
        for pos, g in enumerate(gl):
            operands.append(T)
            subs.append(leg_letter[g] + inner[pos] + inner[pos + 1])
    out = "".join(leg_letter[i] for i in range(len(legs_kind)))
    res = np.einsum(",".join(subs) + "->" + out, *operands, optimize=True)
    return res


# ------------------------------------------------------- Lorentz transforms
def random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([
        [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
        [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
        [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


def transform(mom, R=None, beta_z=0.0):
    out = np.array(mom, dtype=np.float64).copy()
    if R is not None:
        out[..., 1:] = out[..., 1:] @ R.T
    if beta_z:
        g = 1.0 / math.sqrt(1.0 - beta_z * beta_z)
        e, z = out[..., 0].copy(), out[..., 3].copy()
        out[..., 0] = g * (e + beta_z * z)
        out[..., 3] = g * (z + beta_z * e)
    return out
