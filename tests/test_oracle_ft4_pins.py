"""Pins of the oracle's finite-T model with a 4D regulator on a k-scaled
frequency domain (Sec. 5.3.2 "Quadraturex0" with 4-dimensional regulators;
App. G external fermion legs at p0f = pi T exp(-k/(pi T))), no GPU.

Each branch is tied to an independent evaluation of the same integral:
the Matsubara sum branch to mpmath radial integrals frequency by frequency,
the quadrature branch to a 2-D mpmath integral over (q0, |q|); the two
branches to each other as T -> 0 (the sum becomes the integral); the
quadrature branch to the O(4) invariance of the continuum integral (the
result depends on the external 4-momentum only through |P|); the fermion
leg's frequency shift to a direct sum with p0f written here.
"""
import math

import numpy as np
import pytest

import ffrg_inputs as fi
import oracle

mpmath = pytest.importorskip("mpmath")


def _exp_r(x):
    return mpmath.mpf(1) if x == 0 else x / mpmath.expm1(x)


def _exp_rdot(x):
    if x == 0:
        return mpmath.mpf(2)
    em = mpmath.expm1(-x)
    return 2 * x * x * mpmath.exp(-x) / (em * em)


def _problem(N, T, n_x0, fermionic=False, n_rad=96, n_ang=4, n_ext_m=1, w=0.5):
    return fi.Problem(model=fi.MODEL_FINITE_T_4D, n_rad=n_rad, n_ang1=n_ang, n_ext_p=1, n_ext_ang=n_ext_m,
                      n_matsubara=N, regulator=fi.REG_EXP, m2_over_k2=w, T=T, n_tables=2, n_pts=8, n_stack=1,
                      p_min=1e-200, p_max=1e-200, statistics=fi.STAT_FERMI if fermionic else fi.STAT_BOSE,
                      n_x0=n_x0)


def _G(Q2, k, m2):
    return 1 / (Q2 + k * k * _exp_r(Q2 / (k * k)) + m2)


def test_frequency_sets_follow_the_domain_rule():
    """Bosonic 2 pi T n with |n| <= floor(L0/(2 pi T)); fermionic (2n+1) pi T
    inside |nu| <= L0; beyond the cap the Gauss-Legendre nodes on [-L0, L0]."""
    T, k = 0.2, 1.0
    L0 = 4.0 * k
    w, wt = oracle.ft4_frequencies(_problem(8, T, 12), k)
    Nk = int(math.floor(L0 / (2 * math.pi * T)))
    assert np.allclose(w, 2 * math.pi * T * np.arange(-Nk, Nk + 1), rtol=0, atol=1e-15) and np.all(wt == T)
    w, wt = oracle.ft4_frequencies(_problem(8, T, 12, fermionic=True), k)
    n = np.arange(-100, 100)
    nu = (2 * n + 1) * math.pi * T
    assert np.allclose(w, np.sort(nu[np.abs(nu) <= L0]), rtol=0, atol=1e-15)
    w, wt = oracle.ft4_frequencies(_problem(1, T, 12), k)     # 7 frequencies > cap 3
    x, ww = np.polynomial.legendre.leggauss(12)
    assert np.allclose(w, L0 * x, atol=1e-14) and np.allclose(wt, L0 * ww / (2 * math.pi), atol=1e-15)


@pytest.mark.parametrize("fermionic", [False, True])
def test_matsubara_branch_at_p0_vs_radial_integrals(fermionic):
    """Z = lam = 1, p -> 0, m = 0: T sum_n (1/2 pi^2) int_0^{4k} q^2 dR(Q) G(Q)^2
    G(Q + P) dq with Q^2 = w_n^2 + q^2 and the external frequency P0 = 0
    (bosonic) or p0f = pi T exp(-k/(pi T)) (the fermion leg)."""
    k, T, w = 1.3, 0.15, 0.4
    pb = _problem(40, T, 8, fermionic=fermionic, w=w)
    tabs = fi.constant_tables(pb, [1.0, 1.0])
    got = oracle.rhs(pb, tabs, k)[0]
    L0 = 4 * k
    with mpmath.workdps(30):
        kk, TT, m2 = mpmath.mpf(k), mpmath.mpf(T), mpmath.mpf(w) * k * k
        if fermionic:
            P0 = mpmath.pi * TT * mpmath.exp(-kk / (mpmath.pi * TT))
            freqs = [(2 * n + 1) * mpmath.pi * TT for n in range(-60, 60)]
        else:
            P0 = mpmath.mpf(0)
            freqs = [2 * mpmath.pi * TT * n for n in range(-60, 61)]
        freqs = [f for f in freqs if abs(f) <= L0]
        tot = mpmath.mpf(0)
        for f in freqs:
            def integrand(q):
                Q2 = f * f + q * q
                QP2 = (f + P0) ** 2 + q * q
                return q * q * kk * kk * _exp_rdot(Q2 / (kk * kk)) * _G(Q2, kk, m2) ** 2 * _G(QP2, kk, m2)
            tot += mpmath.quad(integrand, [0, kk, 2 * kk, 4 * kk])
        want = float(TT * tot / (2 * mpmath.pi ** 2))
    assert abs(got - want) / want < 1e-12, (got, want)


def test_quadrature_branch_at_p0_vs_two_dimensional_integral():
    """Beyond the cap: (1/2 pi) int_{-4k}^{4k} dq0 (1/2 pi^2) int_0^{4k} q^2 f(q0^2 + q^2) dq."""
    k, T, w = 0.9, 0.01, 0.6
    pb = _problem(2, T, 96, w=w)
    tabs = fi.constant_tables(pb, [1.0, 1.0])
    got = oracle.rhs(pb, tabs, k)[0]
    with mpmath.workdps(20):
        kk, m2 = mpmath.mpf(k), mpmath.mpf(w) * k * k

        def f(q0, q):
            Q2 = q0 * q0 + q * q
            return q * q * kk * kk * _exp_rdot(Q2 / (kk * kk)) * _G(Q2, kk, m2) ** 3
        L0 = 4 * kk
        want = float(mpmath.quad(f, [-L0, -kk, 0, kk, L0], [0, kk, 2 * kk, L0]) / (4 * mpmath.pi ** 3))
    assert abs(got - want) / want < 1e-11, (got, want)


def test_sum_tends_to_the_quadrature_as_T_goes_to_zero():
    """With 2 pi T = 0.2 k the Matsubara sum over |w_n| <= 6k (61 terms) and the
    frequency quadrature over [-6k, 6k] agree: with constant dressings the
    integrand is analytic in q0 (the sum's aliasing error falls like
    exp(-1/T); seeded tables have kinks at their nodes and ln|Q| a branch
    point at Q = 0, which both discretisations resolve only algebraically)
    and negligible at the domain edge (x^2 exp(-x) at x = 36); both branches
    use the same radial and angle rules, and the 4D regulator enters both
    lines at the shifted external frequencies."""
    k = 1.0
    T = 0.2 * k / (2 * math.pi)
    wl = fi.make_finite_t_4d(seed=31, N=40, T=T, n_pts=24, n_ext_p=5, n_ext_m=3, n_rad=64, n_ang=16, n_x0=160)
    pb = wl.problem
    pb.qmax_over_k = 6.0
    tabs = fi.constant_tables(pb, [1.1, 0.8])
    s = oracle.rhs(pb, tabs, k)
    assert oracle.ft4_frequencies(pb, k)[0].size == 61
    pb.n_matsubara = 2                   # cap 5 < 61: the quadrature branch
    qd = oracle.rhs(pb, tabs, k)
    assert np.max(np.abs(s - qd) / np.abs(qd)) < 1e-13


def test_quadrature_branch_is_o4_invariant():
    """The continuum integral depends on P only through |P|: the external point
    (w_m, p) equals (0, sqrt(w_m^2 + p^2)) up to the domain edge, with
    non-constant dressings (linear in ln|Q|, exact under the lookup)."""
    k, T = 1.0, 0.06
    pb = fi.Problem(model=fi.MODEL_FINITE_T_4D, n_rad=96, n_ang1=48, n_ext_p=1, n_ext_ang=3, n_matsubara=1,
                    regulator=fi.REG_EXP, m2_over_k2=0.5, T=T, n_tables=2, n_pts=32, n_stack=1, p_min=0.3,
                    p_max=0.3, n_x0=96)
    lg = np.log(fi.log_grid(pb.n_pts, pb.x_min, pb.x_max) / pb.x_min)
    tabs = np.stack([1.0 + 0.02 * lg, 0.9 + 0.03 * lg]).reshape(2, 1, -1)
    got = oracle.rhs(pb, tabs, k)           # m = 0, 1, 2 at p = 0.3
    for m in (1, 2):
        P = math.hypot(0.3, 2 * math.pi * T * m)
        pm = fi.Problem(**{**pb.__dict__, "n_ext_ang": 1, "p_min": P, "p_max": P})
        ref = oracle.rhs(pm, tabs, k)[0]
        assert abs(got[m] - ref) / abs(ref) < 1e-6, (m, got[m], ref)
    assert abs(got[1] - got[0]) / abs(got[0]) > 1e-4     # the frequency shift does enter
