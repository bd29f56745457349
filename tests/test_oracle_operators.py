"""Pins of the FP64 oracle's special functions and single operators.

Each check compares against something other than the oracle's own formula: a
library routine (scipy), a textbook closed form, an exactness invariant of the
translation theorems, finite differences, or the O(N^2) direct sum.
"""
import numpy as np
import pytest
import scipy.special as sp

import oracle as O
from paper_1010_1482_gb300 import inputs

RNG = np.random.default_rng(1234)


# --- Eq. 7-9: associated Legendre, Eq. 6: spherical harmonics ------------------------------

@pytest.mark.parametrize("x", [-1.0, -0.73, 0.0, 0.31, 0.999, 1.0])
def test_legendre_matches_scipy_lpmv(x):
    # scipy.special.lpmv includes the Condon-Shortley phase, as Eq. 8 (read with (2m-1)!!) does
    nmax = 20
    P = O.legendre(nmax, x)
    for n in range(nmax):
        for m in range(n + 1):
            ref = sp.lpmv(m, n, x)
            assert P[O.tri(n, m)] == pytest.approx(ref, rel=1e-12, abs=1e-12 * max(1.0, abs(ref)))


def test_ynm_matches_scipy_sph_harm():
    # Eq. 6 normalisation = sqrt(4 pi / (2n+1)) x scipy's orthonormal harmonic
    for _ in range(5):
        a, b = RNG.uniform(0, np.pi), RNG.uniform(-np.pi, np.pi)
        Y = O.ynm(16, a, b)
        for n in range(16):
            for m in range(n + 1):
                ref = np.sqrt(4 * np.pi / (2 * n + 1)) * sp.sph_harm_y(n, m, a, b)
                assert abs(Y[O.tri(n, m)] - ref) < 1e-12 * max(1.0, abs(ref))


def test_addition_theorem():
    # sum_m Y_n^{-m}(a) Y_n^m(b) = P_n(cos gamma): the identity behind Eq. 2 and 3
    a1, b1, a2, b2 = 0.4, 1.3, 2.1, -0.5
    Y1, Y2 = O.ynm(12, a1, b1), O.ynm(12, a2, b2)
    u1 = np.array([np.sin(a1) * np.cos(b1), np.sin(a1) * np.sin(b1), np.cos(a1)])
    u2 = np.array([np.sin(a2) * np.cos(b2), np.sin(a2) * np.sin(b2), np.cos(a2)])
    cg = float(u1 @ u2)
    for n in range(12):
        s = Y1[O.tri(n, 0)].conjugate() * Y2[O.tri(n, 0)]
        for m in range(1, n + 1):
            s += 2 * np.real(Y1[O.tri(n, m)].conjugate() * Y2[O.tri(n, m)])
        assert np.real(s) == pytest.approx(sp.eval_legendre(n, cg), abs=1e-12)


# --- Eq. 2: P2M and M2P -------------------------------------------------------------------

def test_single_charge_at_centre_is_exact():
    c = np.array([0.1, -0.2, 0.3])
    q = 0.7
    M = O.p2m(8, c, np.array([[*c, q]]))
    assert M[0] == pytest.approx(q, abs=0)
    assert np.max(np.abs(M[1:])) == 0.0
    x = np.array([1.3, 0.4, -0.9])
    d = x - c
    r = np.linalg.norm(d)
    out = O.m2p(8, c, M, x)
    assert out[0] == pytest.approx(q / r, rel=1e-15)
    assert np.allclose(out[1:], -q * d / r**3, rtol=1e-14, atol=0)


def test_charge_on_axis_matches_legendre_series():
    # M_n^0 = q d^n, M_n^{m!=0} = 0, and M2P = sum_n q d^n P_n(cos g) / r^{n+1}
    p, q, d = 10, 1.3, 0.35
    c = np.zeros(3)
    M = O.p2m(p, c, np.array([[0.0, 0.0, d, q]]))
    for n in range(p):
        assert M[O.tri(n, 0)] == pytest.approx(q * d**n, rel=1e-13)
        for m in range(1, n + 1):
            assert abs(M[O.tri(n, m)]) < 1e-14
    for _ in range(5):
        x = RNG.normal(size=3)
        x *= 2.0 / np.linalg.norm(x)
        r = np.linalg.norm(x)
        cg = x[2] / r
        ref = sum(q * d**n * sp.eval_legendre(n, cg) / r ** (n + 1) for n in range(p))
        assert O.m2p(p, c, M, x)[0] == pytest.approx(ref, rel=1e-13)


def _cluster(n, centre, half, seed):
    u = inputs.uniform01(seed, 4 * n).reshape(n, 4)
    x = np.empty((n, 4))
    x[:, :3] = centre + (2 * u[:, :3] - 1) * half
    x[:, 3] = u[:, 3] - 0.3  # mixed signs
    return x


def test_p2m_m2p_converges_to_direct():
    c = np.array([0.5, 0.5, 0.5])
    src = _cluster(40, c, 0.5, 11)
    tgt = np.array([[3.1, 0.2, -1.0], [0.5, 0.5, 3.0], [-2.0, -2.0, 2.0]])
    ref = O.direct(np.vstack([src, np.c_[tgt, np.zeros(3)]]), targets=np.arange(40, 43))
    errs = []
    for p in (2, 4, 6, 8, 10, 12):
        M = O.p2m(p, c, src)
        got = np.array([O.m2p(p, c, M, t) for t in tgt])
        errs.append(O.rel_l2(got, ref))
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-6


# --- gradients: analytic vs central differences, on and off the z axis --------------------

@pytest.mark.parametrize("local", [False, True])
def test_series_gradient_matches_finite_differences(local):
    p = 9
    c = np.array([0.2, -0.1, 0.4])
    C = RNG.normal(size=O.ntri(p)) + 1j * RNG.normal(size=O.ntri(p))
    for n in range(p):
        C[O.tri(n, 0)] = C[O.tri(n, 0)].real
    ev = O.l2p if local else O.m2p
    r0 = 0.3 if local else 2.0
    pts = [c + r0 * np.array(v) for v in ([0.3, -0.5, 0.8], [0, 0, 1], [0, 0, -1], [0.6, 0.1, -0.2])]
    h = 1e-5
    for x in pts:
        g = ev(p, c, C, x)[1:]
        fd = np.zeros(3)
        for d in range(3):
            e = np.zeros(3)
            e[d] = h
            fd[d] = (ev(p, c, C, x + e)[0] - ev(p, c, C, x - e)[0]) / (2 * h)
        assert np.allclose(g, fd, rtol=1e-6, atol=1e-6 * np.max(np.abs(fd)))


# --- M2M and L2L: exact at fixed truncation --------------------------------------------------

def test_m2m_is_exact():
    # P2M about the parent == M2M of P2M about each child (all degrees < p)
    p = 10
    parent = np.array([0.0, 0.0, 0.0])
    h = 0.5
    total = np.zeros(O.ntri(p), dtype=complex)
    allp = []
    for cidx in range(8):
        off = np.array([cidx & 1, (cidx >> 1) & 1, (cidx >> 2) & 1]) - 0.5
        cc = parent + off * h
        src = _cluster(15, cc, h / 2, 100 + cidx)
        allp.append(src)
        total += O.m2m(p, cc, parent, O.p2m(p, cc, src))
    direct_M = O.p2m(p, parent, np.vstack(allp))
    assert np.max(np.abs(total - direct_M)) < 1e-13 * np.max(np.abs(direct_M))


def test_l2l_is_exact():
    # a truncated local expansion is a harmonic polynomial: L2P(L2L(L)) == L2P(L)
    p = 10
    pc = np.array([0.1, 0.2, 0.3])
    C = RNG.normal(size=O.ntri(p)) + 1j * RNG.normal(size=O.ntri(p))
    for n in range(p):
        C[O.tri(n, 0)] = C[O.tri(n, 0)].real
    for cidx in (0, 3, 7):
        cc = pc + (np.array([cidx & 1, (cidx >> 1) & 1, (cidx >> 2) & 1]) - 0.5) * 0.25
        Lc = O.l2l(p, pc, cc, C)
        for _ in range(3):
            x = cc + RNG.uniform(-0.1, 0.1, size=3)
            a, b = O.l2p(p, cc, Lc, x), O.l2p(p, pc, C, x)
            assert np.allclose(a, b, rtol=1e-12, atol=1e-12 * np.max(np.abs(b)))


# --- Eq. 4: M2L ------------------------------------------------------------------------------

def test_m2l_then_l2p_converges_to_m2p():
    # source and target cells of side 1 at offset (2, 1, -1): L2P(M2L(M)) -> M2P(M) with p
    sc = np.array([0.5, 0.5, 0.5])
    tc = sc + np.array([2.0, 1.0, -1.0])
    src = _cluster(30, sc, 0.5, 7)
    tgt = tc + RNG.uniform(-0.5, 0.5, size=(6, 3))
    ref = O.direct(np.vstack([src, np.c_[tgt, np.zeros(6)]]), targets=np.arange(30, 36))
    errs = []
    for p in (2, 4, 6, 8, 10, 12, 14):
        L = O.m2l(p, sc, tc, O.p2m(p, sc, src))
        got = np.array([O.l2p(p, tc, L, t) for t in tgt])
        errs.append(O.rel_l2(got, ref))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-5


def test_m2l_direction_reading_planted_mistake():
    # Eq. 4 with v = source - target (the other reading) must not converge at odd degrees
    sc = np.array([0.5, 0.5, 0.5])
    tc = sc + np.array([3.0, 0.0, 0.0])
    src = _cluster(20, sc, 0.5, 3)
    x = tc + np.array([0.1, -0.2, 0.15])
    ref = O.direct(np.vstack([src, [[*x, 0.0]]]), targets=[20])[0]
    p = 10
    good = O.l2p(p, tc, O.m2l(p, sc, tc, O.p2m(p, sc, src)), x)
    # swapping the centres evaluates the reflected field about the midpoint
    bad = O.l2p(p, tc, O.m2l(p, tc, sc, O.p2m(p, sc, src)), x)
    assert O.rel_l2(good, ref) < 1e-5
    assert O.rel_l2(bad, ref) > 1e-2
