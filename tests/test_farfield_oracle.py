"""Pins of the far-field expansion oracle (oracle/farfield_oracle.c), §3.2.

What fixes the expansion independently of the oracle's own loops:
  * the product-term form of Axilrod-Teller (law of cosines) reproduces phi
    from its cosine definition on random triangles;
  * derivatives of (v.v)^s equal sympy's symbolic derivatives;
  * moments obey the binomial shift identity between two centres;
  * p = 0 is the monopole n2 n3 phi(x, c2, c3) of the paper's p = 0 rule (§4);
  * single-point source sets are exact at every order (no higher moments);
  * a product of non-negative integer powers of squared lengths is a
    polynomial of degree 2 (s12 + s13 + s23) in the source offsets, so its
    expansion is exact from that order on, on any geometry, and not below;
  * for Axilrod-Teller, the expansion equals the sum over source pairs of the
    degree-p Taylor polynomial of t -> phi(x, c2 + t(y2 - c2), c3 + t(y3 - c3))
    at t = 1, computed here with univariate power series of (abc)^s;
  * on separated clusters the error falls with the order.
Each planted slip in a copy of the oracle fails at least one of these.
"""
import ctypes
import math
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import farfield as ff


def _clusters(seed, sep=5.0, rad=0.3, n2=12, n3=15, nq=5):
    rng = np.random.default_rng(seed)
    Y2 = rng.normal(size=(n2, 3)) * rad + np.array([sep, 0.0, 0.0])
    Y3 = rng.normal(size=(n3, 3)) * rad + np.array([0.2 * sep, sep, 0.1 * sep])
    Xq = rng.normal(size=(nq, 3)) * rad
    return Xq, Y2, Y3


# ---------------------------------------------------------------- pin checks
# Each returns True when the pin holds; the planted-mistake test runs them all
# on a mutant library.

def pin_at_terms(L=None):
    rng = np.random.default_rng(3)
    terms = ff.at_product_terms(L)
    for _ in range(20):
        x, y2, y3 = rng.normal(size=(3, 3))
        ref = oracle.at_phi(x, y2, y3)
        got = ff.pairset_sum(x[None], y2[None], y3[None], terms, L=L)[0]
        parts = sum(abs(w) * np.dot(x - y2, x - y2) ** a * np.dot(x - y3, x - y3) ** b
                    * np.dot(y2 - y3, y2 - y3) ** c for a, b, c, w in zip(*terms))
        if not abs(got - ref) <= 1e-13 * parts:
            return False
    return len(terms[0]) == 11


def _sympy_derivs(v0, s, alphas):
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    g = (x * x + y * y + z * z) ** sp.Rational(s).limit_denominator(8)
    vals = []
    for a in alphas:
        d = sp.diff(g, x, int(a[0]), y, int(a[1]), z, int(a[2]))
        vals.append(float(d.subs({x: sp.Rational(v0[0]), y: sp.Rational(v0[1]),
                                  z: sp.Rational(v0[2])}).evalf(30)))
    return np.array(vals)


def pin_derivs(L=None):
    v0 = (Fraction(3, 4), Fraction(-5, 4), Fraction(1, 2))
    vf = np.array([float(c) for c in v0])
    al = ff.multi_indices(5, L)
    for s in (0.5, -0.5, -1.5, -2.5, 2.0):
        got = ff.derivs(vf, s, 5, L)
        ref = _sympy_derivs(v0, s, al)
        if not np.all(np.abs(got - ref) <= 1e-12 * np.maximum(1.0, np.abs(ref))):
            return False
    return True


def pin_moment_shift(L=None):
    rng = np.random.default_rng(5)
    Y = rng.normal(size=(30, 3))
    c, c1 = np.array([0.1, -0.2, 0.3]), np.array([-0.4, 0.5, 0.2])
    p = 5
    al = ff.multi_indices(p, L)
    M, M1 = ff.moments(Y, p, c, L), ff.moments(Y, p, c1, L)
    idx = {tuple(a): t for t, a in enumerate(al)}
    # (y - c1)^g / g! = sum_{a <= g} (y - c)^a / a! (c - c1)^(g - a) / (g - a)!; with the
    # (-1)^|g| of the moments this is M_g(c1) = sum_a M_a(c) (c1 - c)^(g - a) / (g - a)!
    d = c1 - c
    for g in al:
        acc = 0.0
        for a in al:
            if np.all(a <= g):
                e = g - a
                acc += M[idx[tuple(a)]] * np.prod(d ** e) / np.prod([math.factorial(k) for k in e])
        if not abs(acc - M1[idx[tuple(g)]]) <= 1e-12 * max(1.0, np.abs(M1).max()):
            return False
    # first moments vanish about the centre of mass; M_0 = n
    Mc = ff.moments(Y, 1, None, L)
    return abs(Mc[0] - 30) <= 1e-12 and np.all(np.abs(Mc[1:4]) <= 1e-12)


def pin_monopole(L=None):
    Xq, Y2, Y3 = _clusters(7, sep=2.0, rad=0.5)
    c2, c3 = Y2.mean(0), Y3.mean(0)
    got = ff.farfield3(Xq, Y2, Y3, 0, L=L)
    ref = np.array([len(Y2) * len(Y3) * oracle.at_phi(x, c2, c3) for x in Xq])
    return bool(np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref)))


def pin_single_points(L=None):
    rng = np.random.default_rng(9)
    Xq = rng.normal(size=(4, 3))
    y2, y3 = rng.normal(size=(1, 3)) + 3.0, rng.normal(size=(1, 3)) - 3.0
    ref = ff.pairset_sum(Xq, y2, y3, L=L)
    return all(np.all(np.abs(ff.farfield3(Xq, y2, y3, p, L=L) - ref) <= 1e-13 * np.abs(ref))
               for p in (0, 3, 6))


POLY_TERMS = (np.array([1.0, 2.0, 0.0, 0.0]), np.array([1.0, 0.0, 1.0, 0.0]),
              np.array([1.0, 1.0, 2.0, 1.0]), np.array([0.7, -1.3, 0.4, 2.1]))


def pin_polynomial_exact(L=None):
    rng = np.random.default_rng(11)
    Y2, Y3, Xq = rng.normal(size=(7, 3)), rng.normal(size=(9, 3)) + 0.5, rng.normal(size=(5, 3))
    c2, c3 = np.array([0.3, -0.1, 0.2]), np.array([-0.2, 0.4, 0.1])  # not the centres of mass
    ref = ff.pairset_sum(Xq, Y2, Y3, POLY_TERMS, L=L)
    scale = ff.pairset_sum(Xq, Y2, Y3, (*POLY_TERMS[:3], np.abs(POLY_TERMS[3])), L=L)
    ok = True
    for p in range(0, 9):
        e = np.abs(ff.farfield3(Xq, Y2, Y3, p, POLY_TERMS, c2, c3, L=L) - ref)
        exact = np.all(e <= 1e-12 * np.abs(scale))
        ok &= exact if p >= 6 else not exact  # degree 2 * (1 + 1 + 1) = 6
    return bool(ok)


def _series_pow(h, s, p):
    """Taylor coefficients (degree <= p) of h(t)^s for a polynomial h, h[0] > 0."""
    h = np.asarray(h, dtype=np.float64)
    q = np.zeros(p + 1)
    q[:min(len(h), p + 1)] = h[:p + 1] / h[0]
    q[0] = 0.0
    out, qk, c = np.zeros(p + 1), np.zeros(p + 1), 1.0
    qk[0] = 1.0
    for k in range(p + 1):
        out += c * qk
        qk = np.convolve(qk, q)[:p + 1]
        c *= (s - k) / (k + 1)
    return h[0] ** s * out


def _taylor_at_phi(x, c2, c3, y2, y3, p):
    """Sum of the degree <= p Taylor coefficients in t of
    phi(x, c2 + t (y2 - c2), c3 + t (y3 - c3)), phi by the law of cosines."""
    d2, d3 = y2 - c2, y3 - c3
    u, v, w = x - c2, x - c3, c2 - c3

    def sq(a0, a1):  # |a0 + t a1|^2 as coefficients in t
        return np.array([a0 @ a0, 2 * a0 @ a1, a1 @ a1])

    a, b, c = sq(u, -d2), sq(v, -d3), sq(w, d2 - d3)
    abc = np.convolve(np.convolve(a, b), c)
    cub = np.convolve(np.convolve(b + c - a, a + c - b), a + b - c)
    f = _series_pow(abc, -1.5, p) + 0.375 * np.convolve(cub, _series_pow(abc, -2.5, p))[:p + 1]
    return f[:p + 1].sum()


def pin_univariate_taylor(L=None):
    Xq, Y2, Y3 = _clusters(13, sep=3.0, rad=0.4, n2=6, n3=7, nq=3)
    c2, c3 = Y2.mean(0), Y3.mean(0)
    for p in (1, 2, 3, 5):
        got = ff.farfield3(Xq, Y2, Y3, p, L=L)
        for q, x in enumerate(Xq):
            ref = sum(_taylor_at_phi(x, c2, c3, y2, y3, p) for y2 in Y2 for y3 in Y3)
            scale = sum(abs(oracle.at_phi(x, y2, y3)) for y2 in Y2 for y3 in Y3)
            if not abs(got[q] - ref) <= 1e-11 * scale:
                return False
    return True


def pin_convergence(L=None):
    Xq, Y2, Y3 = _clusters(1, sep=5.0, rad=0.3, n2=20, n3=25, nq=6)
    ex = ff.pairset_sum(Xq, Y2, Y3, L=L)
    err = [np.abs(ff.farfield3(Xq, Y2, Y3, p, L=L) - ex).max() / np.abs(ex).max() for p in range(9)]
    return all(err[p + 2] < err[p] for p in range(7)) and err[8] < 1e-5 * err[0] and err[0] > 1e-3


PINS = [pin_at_terms, pin_derivs, pin_moment_shift, pin_monopole, pin_single_points,
        pin_polynomial_exact, pin_univariate_taylor, pin_convergence]


@pytest.mark.parametrize("pin", PINS, ids=[f.__name__ for f in PINS])
def test_farfield_pin(pin):
    assert pin()


def test_farfield_rejects_bad_order():
    Xq, Y2, Y3 = _clusters(2)
    with pytest.raises(ValueError):
        ff.farfield3(Xq, Y2, Y3, 9)
    with pytest.raises(ValueError):
        ff.farfield3(Xq, Y2, Y3, -1)


# ---------------------------------------------------------------- planted slips

MUTANTS = {
    "control": None,
    "no (-1)^|b| in the P2 x P3 coupling": ("const double sign = ((ib + jb + kb) % 2) ? -1.0 : 1.0;",
                                           "const double sign = 1.0;"),
    "second binomial dropped": ("mbinom(g2, a12) * mbinom(g3, a13) *", "mbinom(g2, a12) *"),
    "moments without their sign": (
        "const double sign = ((a[0] + a[1] + a[2]) % 2) ? -1.0 : 1.0;\n        const double inv",
        "const double sign = 1.0;\n        const double inv"),
    "P3 moment at the P2 index": ("M3[I.idx[g3[0]][g3[1]][g3[2]]]", "M3[I.idx[g2[0]][g2[1]][g2[2]]]"),
    "series linear term halved": ("= 2.0 * v0[d] / r2;", "= v0[d] / r2;"),
    "cosine product weight 3/4": ("w[n] = 0.375 * cub[i][j][k];", "w[n] = 0.75 * cub[i][j][k];"),
    "g23 expanded at c3 - c2": ("wv[d] = c2[d] - c3[d];", "wv[d] = c3[d] - c2[d];"),
    "g13 expanded about c2": ("v[d] = x[d] - c3[d];", "v[d] = x[d] - c2[d];"),
}


def _mutant(tmp_path, name, edit):
    here = os.path.dirname(oracle.__file__)
    src = open(os.path.join(here, "farfield_oracle.c")).read()
    if edit is not None:
        assert src.count(edit[0]) == 1, name
        src = src.replace(edit[0], edit[1])
    tag = "ff" + "".join(ch if ch.isalnum() else "_" for ch in name)
    c, so = tmp_path / f"{tag}.c", tmp_path / f"{tag}.so"
    c.write_text(src)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                    "-o", str(so), str(c), os.path.join(here, "at_oracle.c"), "-lm"], check=True)
    return ctypes.CDLL(str(so))


@pytest.mark.parametrize("name", list(MUTANTS))
def test_farfield_pins_reject_planted_mistakes(tmp_path, name):
    L = _mutant(tmp_path, name, MUTANTS[name])
    holds = [bool(pin(L)) for pin in PINS]
    print(name, holds)
    if name == "control":
        assert all(holds)
    else:
        assert not all(holds), f"the far-field pins did not catch: {name}"
