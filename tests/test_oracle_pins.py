"""Pins of the FP64 oracle to facts other than itself.

Each check is chosen so that a plausible slip in the oracle (a dropped
factor 3, a wrong sign, the wrong vertex's cosine, i counted among j,k, a
transposed operand) fails at least one of them:
  * closed forms of phi (tests/golden, Sec. 1 formula);
  * a 50-digit decimal brute force that forms the cosines by the law of
    cosines (a different route from the oracle's dot products);
  * sum_i Phi_i = 3E with E from a separate enumeration (Eq. 1, footnote);
  * permutation, translation and rotation invariance; exact 2^-9 scaling;
  * gradient vs central differences of E, momentum, torque and virial
    identities (degree -9 homogeneity), VJP identities.
"""
import decimal
import os

import numpy as np
import pytest

from paper_1105_2769_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_fixture(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([c.strip() for c in line.split("|")])
    return rows


def test_closed_forms(oracle_lib):
    rows = _read_fixture("closed_forms.txt")
    assert len(rows) >= 8
    for name, pts, expected, _why in rows:
        P = np.array([[float(v) for v in p.split()] for p in pts.split(";")])
        expected = float(expected)
        got = oracle_lib.at_phi(P[0], P[1], P[2])
        assert got == pytest.approx(expected, rel=1e-13, abs=0), name
        # N = 3: every particle's Phi is the single triple's phi
        Phi = oracle_lib.phi(P)
        np.testing.assert_allclose(Phi, expected, rtol=1e-13, err_msg=name)


def test_tetrahedron(oracle_lib):
    X = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
    rows = _read_fixture("tetrahedron.txt")
    expected = np.array([float(r[1]) for r in rows])
    np.testing.assert_allclose(oracle_lib.phi(X), expected, rtol=1e-13)
    # E = 4 faces * 1.375 / d^9; sum_i Phi_i = 3E
    E = oracle_lib.energy(X)
    assert E == pytest.approx(4 * 1.375 / 2 ** 13.5, rel=1e-13)


def _decimal_phi_all(X, digits=50):
    """Phi_i by brute force over ordered (j, k), halved, in `digits`-digit
    decimal arithmetic; cosines from the law of cosines on squared lengths."""
    ctx = decimal.Context(prec=digits)
    D = decimal.Decimal
    P = [[D(repr(float(v))) for v in row] for row in X]
    n = len(P)
    r2 = [[None] * n for _ in range(n)]
    for a in range(n):
        for b in range(n):
            if a != b:
                s = D(0)
                for d in range(3):
                    t = ctx.subtract(P[a][d], P[b][d])
                    s = ctx.add(s, ctx.multiply(t, t))
                r2[a][b] = s
    r = [[ctx.sqrt(r2[a][b]) if a != b else None for b in range(n)] for a in range(n)]

    def cosine(at, p, q):  # angle at vertex `at` of triangle (at, p, q)
        num = ctx.subtract(ctx.add(r2[at][p], r2[at][q]), r2[p][q])
        return ctx.divide(num, ctx.multiply(D(2), ctx.multiply(r[at][p], r[at][q])))

    out = []
    for i in range(n):
        tot = D(0)
        for j in range(n):
            for k in range(n):
                if len({i, j, k}) < 3:
                    continue
                cp = ctx.multiply(ctx.multiply(cosine(i, j, k), cosine(j, i, k)), cosine(k, i, j))
                num = ctx.add(D(1), ctx.multiply(D(3), cp))
                den = ctx.power(ctx.multiply(ctx.multiply(r[i][j], r[i][k]), r[j][k]), 3)
                tot = ctx.add(tot, ctx.divide(num, den))
        out.append(float(ctx.divide(tot, D(2))))
    return np.array(out)


@pytest.mark.parametrize("n,seed", [(4, 11), (9, 12), (14, 13)])
def test_decimal_brute_force(oracle_lib, n, seed):
    X = inputs.uniform_cube(n, 1.0, 0.05, seed)
    ref = _decimal_phi_all(X)
    got = oracle_lib.phi(X)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)


def test_sum_is_three_energy(oracle_lib):
    X = inputs.uniform_cube(60, 2.0, 0.05, 21)
    Phi = oracle_lib.phi(X)
    E = oracle_lib.energy(X)
    assert Phi.sum() == pytest.approx(3.0 * E, rel=1e-12)


def test_permutation_translation_rotation(oracle_lib):
    X = inputs.uniform_cube(40, 1.5, 0.05, 31)
    Phi = oracle_lib.phi(X)
    perm = np.random.default_rng(0).permutation(len(X))
    np.testing.assert_allclose(oracle_lib.phi(X[perm]), Phi[perm], rtol=1e-13)
    np.testing.assert_allclose(oracle_lib.phi(X + np.array([3.25, -7.5, 11.0])), Phi, rtol=1e-10)
    # rotation by a random orthogonal matrix
    q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((3, 3)))
    np.testing.assert_allclose(oracle_lib.phi(X @ q.T), Phi, rtol=1e-10)


def test_scaling_exact(oracle_lib):
    """phi(lambda x) = lambda^-9 phi(x); lambda = 2 is exact in FP64."""
    X = inputs.uniform_cube(30, 1.0, 0.05, 41)
    a = oracle_lib.phi(X)
    b = oracle_lib.phi(2.0 * X)
    assert np.array_equal(b * 512.0, a)
    assert oracle_lib.energy(2.0 * X) * 512.0 == oracle_lib.energy(X)


def test_gradient_central_differences(oracle_lib):
    X = inputs.uniform_cube(12, 1.0, 0.1, 51)
    G = oracle_lib.grad(X)
    h = 1e-5
    fd = np.zeros_like(X)
    for i in range(len(X)):
        for d in range(3):
            Xp = X.copy(); Xp[i, d] += h
            Xm = X.copy(); Xm[i, d] -= h
            fd[i, d] = (oracle_lib.energy(Xp) - oracle_lib.energy(Xm)) / (2 * h)
    scale = np.abs(G).max()
    np.testing.assert_allclose(G, fd, rtol=1e-6, atol=1e-7 * scale)


def test_force_identities(oracle_lib):
    X = inputs.uniform_cube(50, 2.0, 0.1, 61)
    F = oracle_lib.forces(X)
    E = oracle_lib.energy(X)
    fs = np.abs(F).sum()
    # momentum: sum_i F_i = 0 (translation invariance)
    assert np.abs(F.sum(axis=0)).max() <= 1e-11 * fs
    # torque: sum_i x_i x F_i = 0 (rotation invariance)
    tq = np.cross(X, F).sum(axis=0)
    assert np.abs(tq).max() <= 1e-11 * np.abs(np.cross(X, F)).sum()
    # virial: sum_i x_i . F_i = 9E (homogeneity of degree -9)
    vir = (X * F).sum()
    assert vir == pytest.approx(9.0 * E, rel=1e-10)


def test_vjp_identities(oracle_lib):
    X = inputs.uniform_cube(16, 1.0, 0.1, 71)
    n = len(X)
    ones = np.ones(n)
    # sum_l Phi_l = 3E, so the VJP with g = 1 is 3 dE/dx
    np.testing.assert_allclose(oracle_lib.vjp(X, ones), 3.0 * oracle_lib.grad(X), rtol=1e-12)
    # random g: compare with central differences of sum_l g_l Phi_l
    g = inputs.random_weights(n, 72)
    V = oracle_lib.vjp(X, g)
    h = 1e-5
    fd = np.zeros_like(X)
    for m in range(n):
        for d in range(3):
            Xp = X.copy(); Xp[m, d] += h
            Xm = X.copy(); Xm[m, d] -= h
            fd[m, d] = (g @ oracle_lib.phi(Xp) - g @ oracle_lib.phi(Xm)) / (2 * h)
    np.testing.assert_allclose(V, fd, rtol=1e-6, atol=1e-7 * np.abs(V).max())


def test_subset_matches_full(oracle_lib):
    X = inputs.uniform_cube(80, 2.0, 0.05, 81)
    full = oracle_lib.phi(X)
    idx = np.array([0, 5, 79, 40])
    np.testing.assert_array_equal(oracle_lib.phi(X, idx), full[idx])


# ---------------------------------------------------------------------------
# Planted mistakes: each mutant below is a copy of the oracle's phi source
# with one plausible slip, compiled on its own; the pins above must reject
# every one of them (and accept the unmodified copy).
# ---------------------------------------------------------------------------
_MUTANTS = {
    "control": None,
    "sign of the cosine term": ("return (1.0 + 3.0 * ci * cj * ck) / den;",
                                "return (1.0 - 3.0 * ci * cj * ck) / den;"),
    "dropped factor 3": ("return (1.0 + 3.0 * ci * cj * ck) / den;",
                         "return (1.0 + ci * cj * ck) / den;"),
    "wrong power of r_ij": ("double den = rij * rij * rij * rik",
                            "double den = rij * rij * rik"),
    "wrong vertex vector for cos t_j": ("double cj = dot3(eji, ejk) / (rij * rjk);",
                                        "double cj = dot3(eij, ejk) / (rij * rjk);"),
    "transposed length in cos t_k": ("double ck = dot3(eki, ekj) / (rik * rjk);",
                                     "double ck = dot3(eki, ekj) / (rik * rij);"),
    "ordered pairs counted twice": ("for (int64_t k = j + 1; k < N; ++k) {\n                if (k == i) continue;\n                double p = oracle_at_phi",
                                    "for (int64_t k = 0; k < N; ++k) {\n                if (k == i || k == j) continue;\n                double p = oracle_at_phi"),
}


def _build_mutant(tmp_path, name, edit):
    import ctypes
    import subprocess
    src = open(os.path.join(os.path.dirname(GOLDEN), "..", "oracle", "at_oracle.c")).read()
    if edit is not None:
        assert src.count(edit[0]) == 1, name
        src = src.replace(edit[0], edit[1])
    c = tmp_path / f"m{abs(hash(name))}.c"
    so = tmp_path / f"m{abs(hash(name))}.so"
    c.write_text(src)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                    "-o", str(so), str(c), "-lm"], check=True)
    L = ctypes.CDLL(str(so))
    dp, i64, ip = (ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                   ctypes.POINTER(ctypes.c_int64))
    L.oracle_at_phi.restype = ctypes.c_double
    L.oracle_at_phi.argtypes = [dp, dp, dp]
    L.oracle_phi.argtypes = [dp, i64, ip, i64, dp, dp, ctypes.c_int]

    def at_phi(a, b, c3):
        a, b, c3 = (np.ascontiguousarray(v, dtype=np.float64) for v in (a, b, c3))
        return L.oracle_at_phi(*(v.ctypes.data_as(dp) for v in (a, b, c3)))

    def phi(X):
        X = np.ascontiguousarray(X, dtype=np.float64)
        idx = np.arange(len(X), dtype=np.int64)
        out = np.zeros(len(X))
        assert L.oracle_phi(X.ctypes.data_as(dp), len(X), idx.ctypes.data_as(ip), len(X),
                            out.ctypes.data_as(dp), None, 1) == 0
        return out

    return at_phi, phi


def _pins_hold(at_phi, phi):
    """The closed forms, the tetrahedron and the decimal brute force, as booleans."""
    def close(a, b):
        a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
        return bool(np.all(np.isfinite(a)) and np.allclose(a, b, rtol=1e-12, atol=0))
    for _name, pts, expected, _why in _read_fixture("closed_forms.txt"):
        P = np.array([[float(v) for v in p.split()] for p in pts.split(";")])
        if not (close(at_phi(P[0], P[1], P[2]), float(expected)) and
                close(phi(P), float(expected))):
            return False
    T = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
    if not close(phi(T), [float(r[1]) for r in _read_fixture("tetrahedron.txt")]):
        return False
    X = inputs.uniform_cube(6, 1.0, 0.05, 31)
    return close(phi(X), _decimal_phi_all(X))


@pytest.mark.parametrize("name", list(_MUTANTS))
def test_pins_reject_planted_mistakes(tmp_path, name):
    at_phi, phi = _build_mutant(tmp_path, name, _MUTANTS[name])
    if name == "control":
        assert _pins_hold(at_phi, phi)
    else:
        assert not _pins_hold(at_phi, phi), f"the pins did not catch: {name}"


def test_phi_parts_closed_forms(oracle_lib):
    """The rounding scale sum_t (1 + 3|cos cos cos|)/(r r r)^3 of each term:
    equal to |phi| where the cosine product is >= 0 (equilateral: 1/8; right
    angle: 0), larger where it is negative: collinear, cosine product -1,
    (1 + 3)/(1 * 8 * 1) = 0.5 (|phi| = 0.25); 120-degree isosceles, product
    -0.375, (1 + 1.125)/3^1.5 (|phi| = 0.125/3^1.5)."""
    for name, pts, expected, _why in _read_fixture("closed_forms.txt"):
        P = np.array([[float(v) for v in p.split()] for p in pts.split(";")])
        parts = oracle_lib.phi_parts(P)
        assert np.all(parts >= np.abs(float(expected)) * (1 - 1e-13)), name
        if name.startswith(("equilateral", "right_angle")):
            np.testing.assert_allclose(parts, abs(float(expected)), rtol=1e-13, err_msg=name)
    col = np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0]], dtype=np.float64)
    np.testing.assert_allclose(oracle_lib.phi_parts(col), 0.5, rtol=1e-13)
    iso = np.array([[0, 0, 0], [1, 0, 0], [-0.5, np.sqrt(3) / 2, 0]])
    np.testing.assert_allclose(oracle_lib.phi_parts(iso)[0], 2.125 / 3 ** 1.5, rtol=1e-12)
