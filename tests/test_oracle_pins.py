"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test targets a different way the oracle could be wrong: a dropped
diagram (Table 1 counts, closed forms), a wrong vertex sign or factor
(closed forms, Parke-Taylor, Ward identities, Berends-Giele in
test_oracle_bg.py), a wrong colour factor (Table 5, Gell-Mann brute force,
closed forms), a wrong external state (helicity zeros, Lorentz invariance),
a wrong fermion sign (uu -> uu closed form, Bose symmetry).
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_0909_5257_gb300 import phasespace as ps
from tests import physics_ref as ref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


def _table1():
    out = {}
    for r in _read_golden("table1_counts.txt"):
        name, pdg, nd, nc = r[0], [int(x) for x in r[1:-2]], int(r[-2]), int(r[-1])
        out[name] = (pdg, nd, nc)
    return out


TABLE1 = _table1()
_cache = {}


def proc(pdg):
    key = tuple(pdg)
    if key not in _cache:
        _cache[key] = oracle.OracleProcess(list(pdg))
    return _cache[key]


def events(n_final, n, lo=200.0, hi=2000.0, seed=ps.SEED_BASE):
    return ps.generate(ps.PhaseSpaceConfig(n_final, rs_lo=lo, rs_hi=hi, seed=seed), n)


# ------------------------------------------------------------------ Table 1
@pytest.mark.parametrize("name", [k for k in TABLE1 if k != "gg>ggggg"])
def test_table1_diagram_counts(name):
    pdg, nd, nc = TABLE1[name]
    P = proc(pdg)
    assert P.n_diagrams == nd
    if not name.startswith("uu>"):
        # gluon traces and single-line strings are the paper's bases (Eq. (color-basis));
        # for two quark lines the oracle reduces to a different, fully Fierzed basis.
        assert P.n_colour == nc


@pytest.mark.slow
def test_table1_gg5g():
    pdg, nd, nc = TABLE1["gg>ggggg"]
    P = proc(pdg)
    assert (P.n_diagrams, P.n_colour) == (nd, nc)


# ------------------------------------------------------------------ Table 5
def _unique_upper(P):
    re, im = P.colour_matrix_exact()
    m = P.n_colour
    vals = set()
    for i in range(m):
        for j in range(i, m):
            assert im[i][j] == 0
            if re[i][j] != 0:
                vals.add(re[i][j])
    return len(vals)


@pytest.mark.parametrize("jets", [2, 3, 4, 5])
@pytest.mark.parametrize("family", ["gg", "uu~"])
def test_table5_unique_values(family, jets):
    rows = {int(r[0]): (int(r[1]), int(r[2]), int(r[3])) for r in _read_golden("table5_unique.txt")}
    if family == "gg":
        pdg, want = [21] * (2 + jets), rows[jets][0]
    else:
        pdg, want = [2, -2] + [21] * jets, rows[jets][1]
    if family == "gg" and jets == 5:
        pytest.importorskip("numpy")
    assert _unique_upper(proc(pdg)) == want


# ------------------------------------------------- colour matrix brute force
@pytest.mark.parametrize("pdg", [[21] * 4, [21] * 5, [2, -2, 21, 21], [2, -2, 21, 21, 21],
                                 [2, 2, 2, 2], [2, 2, 2, 2, 21], [2, 2, 2, 2, 21, 21]])
def test_colour_matrix_gell_mann_brute_force(pdg):
    """N_ab = 1/(n_a n_b) sum_c T_a^c (T_b^c)^* summed numerically over every
    explicit colour index with Gell-Mann generators (Eq. (color-matrix))."""
    P = proc(pdg)
    kinds = ["g" if c == 21 else "q" for c in pdg]
    tens = [ref.colour_tensor(P.basis(a), kinds).ravel() for a in range(P.n_colour)]
    B = np.array(tens)
    na = 8 if pdg[0] == 21 else 3
    nb = 8 if pdg[1] == 21 else 3
    N_bf = (B @ B.conj().T) / (na * nb)
    assert np.allclose(N_bf.imag, 0.0, atol=1e-12)
    assert np.allclose(N_bf.real, P.colour_matrix(), rtol=1e-12, atol=1e-12)


def test_mc_colour_statistics_gg4g():
    """Sec. 3.3: fraction of non-zero (configuration, basis vector) pairs and of
    all-zero configurations for the 120 traces of gg -> 4g."""
    want = {r[0]: float(r[1]) for r in _read_golden("mc_colour_gg4g.txt")}
    T = ref.gell_mann_T()
    X = np.einsum("aij,bjk,ckl,dlm,emn,fni->abcdef", T, T, T, T, T, T, optimize=True)
    P = proc([21] * 6)
    nz_pairs = 0
    any_nz = np.zeros((8,) * 6, dtype=bool)
    for a in range(P.n_colour):
        (closed, _, _, gl), = P.basis(a)
        assert closed and gl[0] == 0
        # X is indexed by trace position; bring it to leg order
        Y = np.moveaxis(X, list(range(6)), gl)
        nz = np.abs(Y) > 1e-12
        nz_pairs += int(nz.sum())
        any_nz |= nz
    frac_pairs = nz_pairs / (120 * 8 ** 6)
    frac_zero = 1.0 - any_nz.mean()
    assert abs(frac_pairs - want["nonzero_pair_fraction"]) < 0.01
    assert abs(frac_zero - want["all_zero_config_fraction"]) < 0.01


def test_mc_colour_variance_inflation_gg3g():
    """Sec. 3.3's alternative -- one uniformly drawn colour assignment per event
    instead of the colour sum -- measured: for gg -> ggg the estimator
    8^5 sum_h |sum_alpha J_h,alpha Tr_alpha(c)|^2 has, per event, a colour
    variance about 40 times the square of the exact sum, so it needs tens of
    times more events than the exact colour sum for the same precision; the
    colour sum it would save is a fraction of the per-event cost.  (Its mean
    over all assignments is the exact colour sum: checked.)"""
    n = 5
    T = ref.gell_mann_T()
    letters, inner = "abcde", "ijklm"
    subs = ",".join(letters[k] + inner[k] + inner[(k + 1) % n] for k in range(n))
    X = np.einsum(subs + "->" + letters, *([T] * n), optimize=True)
    P = proc([21] * n)
    Y = np.array([np.moveaxis(X, list(range(n)), P.basis(a)[0][3]).reshape(-1) for a in range(P.n_colour)])
    N = P.colour_matrix()
    mom = events(n - 2, 60, lo=300.0, hi=3000.0, seed=ps.SEED_BASE + 31)
    exact, var_c = [], []
    for m in mom:
        S = np.zeros(Y.shape[1])
        tot = 0.0
        for h in range(1 << n):
            J = P.jamp(m, h)
            if not np.any(J):
                continue
            S += np.abs(J @ Y) ** 2
            tot += float(np.real(np.conj(J) @ N @ J)) * 64.0  # N carries 1/(n_a n_b)
        assert abs(S.sum() / tot - 1.0) < 1e-10  # the mean over assignments is the colour sum
        exact.append(S.sum())
        var_c.append(np.mean((8.0 ** n * S) ** 2) - S.sum() ** 2)
    exact, var_c = np.array(exact), np.array(var_c)
    per_event = float(np.mean(var_c / exact ** 2))
    inflation = 1.0 + var_c.mean() / exact.var()
    assert 20.0 < per_event < 80.0
    assert inflation > 10.0


# ------------------------------------------------------------ closed forms
@pytest.mark.parametrize("pdg,fn", [([21] * 4, ref.me2_gg_gg),
                                    ([2, -2, 21, 21], ref.me2_uubar_gg),
                                    ([2, 2, 2, 2], ref.me2_uu_uu)])
def test_two_to_two_closed_forms(pdg, fn):
    mom = events(2, 256)
    got = proc(pdg).me2(mom)
    want = fn(mom)
    assert np.max(np.abs(got / want - 1.0)) < 1e-13


def test_parke_taylor_five_gluons():
    mom = events(3, 64)
    got = proc([21] * 5).me2(mom)
    want = np.array([ref.gluon_me2_leading_colour_exact(m) for m in mom])
    assert np.max(np.abs(got / want - 1.0)) < 1e-12


def test_parke_taylor_four_gluons_equals_closed_form():
    mom = events(2, 32)
    a = np.array([ref.gluon_me2_leading_colour_exact(m) for m in mom])
    assert np.max(np.abs(a / ref.me2_gg_gg(mom) - 1.0)) < 1e-11


@pytest.mark.parametrize("n_ext", [5, 6])
def test_mhv_partial_amplitudes(n_ext):
    """|J_alpha|^2 = g^{2n-4} 2^n s_ij^4/|s_12...s_n1| for every ordering alpha
    of every MHV helicity configuration (trace basis, Tr(t t) = 1/2)."""
    P = proc([21] * n_ext)
    mom = events(n_ext - 2, 2, lo=300.0, hi=3000.0)
    g = ref.g_s()
    orders = [P.basis(a)[0][3] for a in range(P.n_colour)]
    for m in mom:
        k = ref.all_outgoing(m)
        for hel in range(1 << n_ext):
            ho = ref.outgoing_helicities(hel, n_ext)
            neg = [i for i in range(n_ext) if ho[i] < 0]
            if len(neg) != 2:
                continue
            J = P.jamp(m, hel)
            for a, order in enumerate(orders):
                pt = ref.parke_taylor_sq(k, order, tuple(neg))
                assert abs(abs(J[a]) ** 2 / (g ** (2 * n_ext - 4) * 2 ** n_ext * pt) - 1.0) < 1e-10


@pytest.mark.parametrize("n_ext", [5, 6, 7])
def test_quark_line_mhv_partial_amplitudes(n_ext):
    """u u~ -> (n-2) g: for every string-basis ordering (T^{a_s1}...T^{a_sk})
    and every MHV helicity configuration with the negative helicities on one
    quark and one gluon, |J_alpha|^2 = g^{2n-4} 2^{n-2} |A|^2 with A the
    colour-ordered one-quark-line MHV amplitude in the cyclic order
    (leg 0, leg 1, s1, ..., sk) of the crossed momenta (textbook closed form;
    2^{n-2} from Tr(T^a T^b) = delta/2 on the n-2 gluon generators).  Pins
    the qqg vertex, the spinors and quark propagators, and the colour strings,
    for every diagram of the process."""
    pdg = [2, -2] + [21] * (n_ext - 2)
    P = proc(pdg)
    mom = events(n_ext - 2, 2 if n_ext < 7 else 1, lo=300.0, hi=3000.0, seed=ps.SEED_BASE + 5)
    g = ref.g_s()
    orders = [P.basis(a)[0][3] for a in range(P.n_colour)]
    checked = 0
    for m in mom:
        k = ref.all_outgoing(m)
        for hel in range(1 << n_ext):
            ho = ref.outgoing_helicities(hel, n_ext)
            neg = [i for i in range(n_ext) if ho[i] < 0]
            if len(neg) != 2 or ho[0] == ho[1]:
                continue
            q_minus = 0 if ho[0] < 0 else 1
            g_minus = [i for i in neg if i >= 2][0]
            J = P.jamp(m, hel)
            for a, gl in enumerate(orders):
                a2 = ref.quark_line_mhv_sq(k, [0, 1] + gl, q_minus, 1 - q_minus, g_minus)
                assert abs(abs(J[a]) ** 2 / (g ** (2 * n_ext - 4) * 2 ** (n_ext - 2) * a2) - 1.0) < 1e-10
                checked += 1
    assert checked >= P.n_colour * 2 * (n_ext - 2)


# ------------------------------------------------------------ helicity zeros
def _allowed(pdg, hel):
    n = len(pdg)
    h = ref.helicities(hel, n)
    ho = ref.outgoing_helicities(hel, n)
    gl = [i for i in range(n) if pdg[i] == 21]
    if len(gl) == n:
        npos = sum(1 for x in ho if x > 0)
        return 2 <= npos <= n - 2
    if pdg[:2] == [2, -2]:
        if h[0] != -h[1]:
            return False
        hg = [ho[i] for i in gl]
        return not (all(x > 0 for x in hg) or all(x < 0 for x in hg))
    # uu -> uu + gluons: {lambda_1, lambda_2} a permutation of {lambda_a, lambda_b}
    return sorted([h[0], h[1]]) == sorted([h[2], h[3]])


@pytest.mark.parametrize("pdg", [[21] * 4, [21] * 5, [21] * 6, [2, -2, 21, 21], [2, -2, 21, 21, 21],
                                 [2, -2, 21, 21, 21, 21], [2, 2, 2, 2], [2, 2, 2, 2, 21],
                                 [2, 2, 2, 2, 21, 21]])
def test_helicity_selection_rules(pdg):
    """Massless tree amplitudes vanish for all-equal / one-different gluon helicities
    and conserve helicity along quark lines; the oracle evaluates all 2^n and the
    vanishing ones must come out at rounding level."""
    n = len(pdg)
    mom = events(n - 2, 4, lo=300.0, hi=3000.0)
    _, hel = proc(pdg).me2(mom, per_helicity=True)
    for e in range(mom.shape[0]):
        scale = hel[e].max()
        for h in range(1 << n):
            if _allowed(pdg, h):
                assert hel[e, h] > 1e-14 * scale
            else:
                assert hel[e, h] < 1e-22 * scale


# ------------------------------------------------------------ Ward identities
@pytest.mark.parametrize("pdg", [[21] * 4, [21] * 5, [21] * 6, [2, -2, 21, 21], [2, -2, 21, 21, 21],
                                 [2, 2, 2, 2, 21], [2, 2, 2, 2, 21, 21]])
def test_ward_identity(pdg):
    """A gluon polarisation replaced by its momentum gives a vanishing amplitude
    in every colour component and in the colour sum."""
    P = proc(pdg)
    n = len(pdg)
    mom = events(n - 2, 2, lo=300.0, hi=3000.0)
    N = P.colour_matrix()
    for m in mom:
        hels = list(range(0, 1 << n, 3))
        Js = {h: P.jamp(m, h) for h in hels}
        scale = max(float(np.real(J.conj() @ N @ J)) for J in Js.values())
        norm = max(float(np.sum(np.abs(J) ** 2)) for J in Js.values())
        for leg in [i for i in range(n) if pdg[i] == 21]:
            for hel in hels:
                W = P.jamp(m, hel, ward_leg=leg)
                assert np.real(W.conj() @ N @ W) < 1e-20 * scale
                assert np.sum(np.abs(W) ** 2) < 1e-20 * norm


# ------------------------------------------------------------ symmetries
@pytest.mark.parametrize("pdg", [[21] * 5, [21] * 6, [2, -2, 21, 21, 21], [2, 2, 2, 2, 21, 21]])
def test_bose_symmetry(pdg):
    n = len(pdg)
    mom = events(n - 2, 8, lo=300.0, hi=3000.0)
    P = proc(pdg)
    base = P.me2(mom)
    gl_out = [i for i in range(2, n) if pdg[i] == 21]
    rng = np.random.default_rng(7)
    perm = list(range(n))
    shuffled = list(gl_out)
    while shuffled == gl_out:
        shuffled = list(rng.permutation(gl_out))
    for a, b in zip(gl_out, shuffled):
        perm[a] = b
    assert np.allclose(P.me2(mom[:, perm]), base, rtol=1e-12, atol=0)
    if pdg[0] == pdg[1]:  # identical incoming partons
        sw = [1, 0] + list(range(2, n))
        assert np.allclose(P.me2(mom[:, sw]), base, rtol=1e-12, atol=0)
    if pdg[:4] == [2, 2, 2, 2]:  # identical outgoing quarks
        sw = [0, 1, 3, 2] + list(range(4, n))
        assert np.allclose(P.me2(mom[:, sw]), base, rtol=1e-12, atol=0)


@pytest.mark.parametrize("pdg", [[21] * 5, [2, -2, 21, 21, 21], [2, 2, 2, 2, 21], [21] * 6])
def test_lorentz_invariance(pdg):
    n = len(pdg)
    mom = events(n - 2, 8, lo=300.0, hi=3000.0)
    P = proc(pdg)
    base = P.me2(mom)
    rng = np.random.default_rng(11)
    moved = ref.transform(mom, R=ref.random_rotation(rng), beta_z=0.37)
    assert np.max(np.abs(P.me2(moved) / base - 1.0)) < 1e-11


@pytest.mark.parametrize("pdg", [[21] * 4, [21] * 5, [2, -2, 21, 21, 21], [2, 2, 2, 2, 21]])
def test_exact_power_scaling(pdg):
    """|M|^2 has mass dimension 8 - 2 n_ext; scaling every momentum by 4 scales
    spinors by exactly 2 and propagators by exactly 1/16, so the result is exact."""
    n = len(pdg)
    mom = events(n - 2, 16)
    P = proc(pdg)
    a = P.me2(mom)
    b = P.me2(4.0 * mom)
    assert np.array_equal(b, a * 4.0 ** (8 - 2 * n))
