"""Pins of the CPU oracle against mathematics (no GPU).

Each test ties one part of the oracle to something other than itself: a
library routine (numpy/scipy quadrature rules, scipy's adaptive integrators),
a closed form (flat-regulator threshold integrals, Matsubara sums, Beta
functions), an invariant (rotations of the external momenta) or brute force
(Monte Carlo in the loop-momentum ball).  Citations give the paper section
that defines the piece being pinned.
"""
import dataclasses
import math

import numpy as np
import pytest

import ffrg_inputs as fi
import oracle

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 40


def vd(d):
    """v_d = 1/(2^{d+1} pi^{d/2} Gamma(d/2)) (threshold-function normalisation)."""
    return 1.0 / (2 ** (d + 1) * math.pi ** (d / 2) * math.gamma(d / 2))


def litim_threshold(d, k, w, n):
    """int d^dq/(2pi)^d  k d_k R  G^n for the flat regulator, Z = 1, p = 0
    (all momenta below k): 4 v_d k^{d+2-2n} (2/d) / (1+w)^n."""
    return 4 * vd(d) * k ** (d + 2 - 2 * n) * (2.0 / d) / (1 + w) ** n


# --------------------------------------------------------------------------
# quadrature rules (Sec. 5.3.2 "quadrature rules of arbitrary order")
# --------------------------------------------------------------------------
def _gl_mpmath(n):
    """40-digit Gauss-Legendre rule: Newton on mpmath's Legendre polynomials
    from numpy's nodes (numpy's own endpoint weights carry ~1e-12 error)."""
    xr, _ = np.polynomial.legendre.leggauss(n)
    xs, ws = [], []
    for z0 in xr:
        z = mpmath.mpf(z0)
        for _ in range(6):
            pn, pm = mpmath.legendre(n, z), mpmath.legendre(n - 1, z)
            dp = n * (z * pn - pm) / (z * z - 1) if n > 1 else mpmath.mpf(1)
            z -= pn / dp
        pn, pm = mpmath.legendre(n, z), mpmath.legendre(n - 1, z)
        dp = n * (z * pn - pm) / (z * z - 1) if n > 1 else mpmath.mpf(1)
        xs.append(float(z))
        ws.append(float(2 / ((1 - z * z) * dp * dp)))
    return np.array(xs), np.array(ws)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 16, 32, 48, 64, 96])
def test_gauss_legendre_matches_high_precision(n):
    x, w = oracle.gauss_legendre(n)
    xr, wr = _gl_mpmath(n)
    assert np.max(np.abs(x - xr)) < 4e-15
    assert np.max(np.abs(w - wr) / wr) < 2e-13
    assert abs(np.sum(w) - 2.0) < 1e-14


@pytest.mark.parametrize("n", [4, 17, 64])
def test_gauss_legendre_exact_moments_on_interval(n):
    a, b = 0.0, 40.0
    x, w = oracle.gauss_legendre(n, a, b)
    for m in (0, 1, 5, 2 * n - 1):
        exact = (b ** (m + 1) - a ** (m + 1)) / (m + 1)
        got = np.sum(w * (x / b) ** m) * b ** m
        assert abs(got - exact) / exact < 1e-12, m
    assert np.allclose(x[::-1] - (a + b) / 2, -(x - (a + b) / 2), atol=1e-12)


@pytest.mark.parametrize("n", [1, 5, 16, 64])
def test_gauss_chebyshev2(n):
    from scipy.special import roots_chebyu
    x, w = oracle.gauss_chebyshev2(n)
    xr, wr = roots_chebyu(n)
    o = np.argsort(x)
    assert np.max(np.abs(x[o] - xr)) < 1e-14
    assert np.max(np.abs(w[o] - wr)) < 1e-14
    # int sqrt(1-x^2) x^{2m} = Beta(m+1/2, 3/2), exact for 2m <= 2n-1
    for m in range(0, n):
        exact = math.gamma(m + 0.5) * math.gamma(1.5) / math.gamma(m + 2)
        assert abs(np.sum(w * x ** (2 * m)) - exact) < 1e-14 * 10, m
    assert abs(np.sum(w) - math.pi / 2) < 1e-14


# --------------------------------------------------------------------------
# regulators (Sec. 5.3.1, RB / RBdot; flat regulator of Fig. polyExpReg)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("x", [1e-12, 1e-6, 1e-3, 0.1, 0.5, 1.0, 3.0, 16.0, 80.0, 300.0, 690.0])
def test_exp_regulator_shape_and_scale_derivative(x):
    X = mpmath.mpf(x)
    r_exact = X / mpmath.expm1(X)
    assert abs(oracle.reg_r(fi.REG_EXP, x) - float(r_exact)) <= 2e-16 * float(r_exact)

    # k d_k [k^2 r(q^2/k^2)] / k^2 at fixed q, by high-precision differentiation in k
    def R(kk):
        return kk ** 2 * (mpmath.mpf(x) / kk ** 2) / mpmath.expm1(mpmath.mpf(x) / kk ** 2)
    dk = mpmath.diff(R, mpmath.mpf(1))   # q^2 = x at k = 1
    assert abs(oracle.reg_rdot(fi.REG_EXP, x) - float(dk)) <= 1e-14 * abs(float(dk)) + 1e-300


def test_regulator_limits_and_cutoffs():
    assert oracle.reg_r(fi.REG_EXP, 0.0) == 1.0
    assert oracle.reg_rdot(fi.REG_EXP, 0.0) == 2.0
    assert oracle.reg_r(fi.REG_EXP, 701.0) == 0.0
    assert oracle.reg_rdot(fi.REG_EXP, 701.0) == 0.0
    for x in (0.0, 0.3, 0.999):
        assert oracle.reg_r(fi.REG_LITIM, x) == 1.0 - x
        assert oracle.reg_rdot(fi.REG_LITIM, x) == 2.0
    assert oracle.reg_r(fi.REG_LITIM, 1.0) == 0.0 and oracle.reg_rdot(fi.REG_LITIM, 1.0) == 0.0


def test_litim_scale_derivative_by_differentiation():
    # flat regulator k^2 (1 - q^2/k^2) Theta: k d_k = 2 k^2 below the cut
    for q2 in (0.1, 0.5, 0.9):
        def R(kk):
            return kk ** 2 - q2
        assert abs(oracle.reg_rdot(fi.REG_LITIM, q2) - float(mpmath.diff(R, 1))) < 1e-14


# --------------------------------------------------------------------------
# logarithmic-grid interpolation (App. F, LogarithmicCoordinates1D)
# --------------------------------------------------------------------------
def test_log_interpolation():
    n, lo, hi = 17, 1e-3, 10.0
    xs = fi.log_grid(n, lo, hi)
    T = np.cos(np.arange(n) * 0.7) + 2.0
    for j in range(n):
        assert abs(oracle.lerp_log(T, lo, hi, xs[j]) - T[j]) < 1e-13
    # linear in ln s between nodes: geometric midpoint -> arithmetic mean
    for j in range(n - 1):
        sm = math.sqrt(xs[j] * xs[j + 1])
        assert abs(oracle.lerp_log(T, lo, hi, sm) - 0.5 * (T[j] + T[j + 1])) < 1e-13
        s1 = xs[j] * (xs[j + 1] / xs[j]) ** 0.25
        assert abs(oracle.lerp_log(T, lo, hi, s1) - (0.75 * T[j] + 0.25 * T[j + 1])) < 1e-13
    # clamps at both ends
    assert oracle.lerp_log(T, lo, hi, 0.0) == T[0]
    assert oracle.lerp_log(T, lo, hi, 1e-9) == T[0]
    assert abs(oracle.lerp_log(T, lo, hi, 1e6) - T[-1]) < 1e-15
    # a table linear in ln s is reproduced exactly everywhere inside
    L = 0.3 + 0.05 * np.log(xs / lo)
    for s in (2e-3, 0.017, 0.5, 3.3, 9.9):
        assert abs(oracle.lerp_log(L, lo, hi, s) - (0.3 + 0.05 * math.log(s / lo))) < 1e-13


# --------------------------------------------------------------------------
# closed forms with the flat regulator (threshold functions, Sec. 2 / ref. in
# Sec. 4 "threshold functions for the flat or Litim regulator")
# --------------------------------------------------------------------------
def _d3_litim(k=1.7, w=0.5, n_rad=16, n_ang=4):
    pb = fi.Problem(model=fi.MODEL_D3, n_rad=n_rad, n_ang1=n_ang, n_ext_p=1, include_p0=1,
                    regulator=fi.REG_LITIM, m2_over_k2=w, qmax_over_k=1.0)
    return pb


@pytest.mark.parametrize("k,w", [(1.7, 0.5), (0.3, 0.0), (5.0, 2.5), (1.0, -0.4)])
def test_d3_litim_closed_form(k, w):
    pb = _d3_litim(k, w)
    out = oracle.rhs(pb, fi.constant_tables(pb, [1.0]), k)
    exact = litim_threshold(3, k, w, 3)            # dR G(q)^2 G(q) at p = 0
    assert abs(out[-1] - exact) / exact < 1e-14
    pb.lam = 0.7
    pb.prefactor = -2.0
    out = oracle.rhs(pb, fi.constant_tables(pb, [1.0]), k)
    assert abs(out[-1] - (-2.0 * 0.49 * exact)) / exact < 1e-14


def test_d3_litim_threshold_to_double_precision():
    """Flat regulator, Z = 1, p = 0, q < k: G = 1/(k^2 (1 + w)), dR = 2 k^2, so
    I(0) = (1/2 pi^2) (k^3/3) 2 k^2 G^3 = 1/(3 pi^2 k (1 + w)^3); at k = 1.7,
    w = 0.5 in 30-digit arithmetic, the oracle agrees to a few ulp."""
    mpmath = pytest.importorskip("mpmath")
    with mpmath.workdps(30):
        k, w = mpmath.mpf("1.7"), mpmath.mpf("0.5")
        exact = float(1 / (3 * mpmath.pi ** 2 * k * (1 + w) ** 3))
    pb = _d3_litim()
    out = oracle.rhs(pb, fi.constant_tables(pb, [1.0]), 1.7)
    assert abs(out[-1] - exact) < 3e-18


def test_d3_litim_with_running_Z_log_linear():
    """Z(q) = alpha + beta ln(q/x_min) is reproduced exactly by the log-grid
    lerp; flat regulator, p = 0: G = 1/(Z k^2 + m^2), dR = 2 Z k^2 for q < k,
    so I(0) = 1/(2 pi^2) int_0^k q^2 2 Z k^2 / (Z k^2 + m^2)^3 dq (mpmath)."""
    k, w = 2.0, 0.5
    pb = _d3_litim(k, w, n_rad=96)
    xs = fi.log_grid(pb.n_pts, pb.x_min, pb.x_max)
    al, be = 1.0, 0.02
    tab = (al + be * np.log(xs / pb.x_min)).reshape(1, 1, -1)
    out = oracle.rhs(pb, tab, k)

    def Z(q):
        return al + be * mpmath.log(max(q, pb.x_min) / pb.x_min)
    m2 = w * k * k
    f = lambda q: q ** 2 * 2 * Z(q) * k * k / (Z(q) * k * k + m2) ** 3 / (2 * mpmath.pi ** 2)
    exact = float(mpmath.quad(f, [0, pb.x_min, k]))
    assert abs(out[-1] - exact) / exact < 1e-10


@pytest.mark.parametrize("k,M2", [(1.0, 0.0), (2.0, 1.0)])
def test_d4_litim_closed_forms(k, M2):
    """d=4 measure with the Gauss-Chebyshev-II angle: at p = 0 with constant
    vertices the three diagram classes reduce to flat-regulator threshold
    integrals with n = 2, 3, 4 propagator powers."""
    pb = fi.Problem(model=fi.MODEL_D4_VERTEX, n_rad=8, n_ang1=4, n_ang2=3, n_ext_p=2, n_ext_ang=3,
                    regulator=fi.REG_LITIM, m2_over_k2=0.5, m2_shift=M2, qmax_over_k=1.0,
                    n_tables=3, n_pts=16, p_min=1e-200, p_max=2e-200, x_min=1e-3, x_max=10.0)
    w = 0.5 + M2 / k ** 2
    np_ = pb.n_ext_p
    # Z-diagram, lambda3 = 1, lambda4 = 0:  dR G^3
    out = oracle.rhs(pb, fi.constant_tables(pb, [1.0, 1.0, 0.0]), k)
    ex3 = litim_threshold(4, k, w, 3)
    assert abs(out[np_] - ex3) / ex3 < 1e-13           # the p = 0 point
    assert abs(out[0] - ex3) / ex3 < 1e-13             # p = 1e-200
    # Z-diagram, lambda3 = 0, lambda4 = -2: dR G^2
    out = oracle.rhs(pb, fi.constant_tables(pb, [1.0, 0.0, -2.0]), k)
    ex2 = litim_threshold(4, k, w, 2)
    assert abs(out[np_] - ex2) / ex2 < 1e-13
    # lambda3-diagram, lambda3 = c: 3 c^3 dR G^4 ; lambda4-diagram: 3/2 c4^2 dR G^3
    c3, c4 = 0.8, 1.3
    out = oracle.rhs(pb, fi.constant_tables(pb, [1.0, c3, c4]), k)
    ex4 = litim_threshold(4, k, w, 4)
    blk3 = out[np_ + 1: np_ + 1 + np_ * pb.n_ext_ang]
    blk4 = out[np_ + 1 + np_ * pb.n_ext_ang:]
    assert np.max(np.abs(blk3 - 3 * c3 ** 3 * ex4)) / ex4 < 1e-13
    assert np.max(np.abs(blk4 - 1.5 * c4 ** 2 * ex3)) / ex3 < 1e-13


def test_d4_average_momentum_arguments_at_p0():
    """Vertex tables linear in ln S pin the average-momentum arguments at p=0
    (Sec. 3.3 average-momentum parametrisation): S0 of (q,-q,0,0) is
    q/sqrt(2) and S0 of (q,-q,0) is q sqrt(2/3)."""
    k, M2 = 1.5, 0.5
    pb = fi.Problem(model=fi.MODEL_D4_VERTEX, n_rad=96, n_ang1=2, n_ang2=2, n_ext_p=1, n_ext_ang=2,
                    regulator=fi.REG_LITIM, m2_over_k2=0.5, m2_shift=M2, qmax_over_k=1.0,
                    n_tables=3, n_pts=32, p_min=1e-200, p_max=1e-200)
    xs = fi.log_grid(pb.n_pts, pb.x_min, pb.x_max)
    a3, b3, a4, b4 = 1.1, 0.03, 0.7, -0.02
    tab = np.stack([np.ones(pb.n_pts), a3 + b3 * np.log(xs / pb.x_min),
                    a4 + b4 * np.log(xs / pb.x_min)]).reshape(3, 1, -1)
    out = oracle.rhs(pb, tab, k)
    m2 = 0.5 * k * k + M2
    G = 1 / (k * k + m2)
    xm = pb.x_min

    def lam(a, b, s):
        return a + b * mpmath.log(max(s, xm) / xm)
    meas = lambda q: q ** 3 / (8 * mpmath.pi ** 3) * (mpmath.pi / 2) * 2   # angles: pi/2 * 2
    c23, c12 = mpmath.sqrt(mpmath.mpf(2) / 3), 1 / mpmath.sqrt(2)
    fz = lambda q: meas(q) * 2 * k * k * G ** 2 * (-0.5 * lam(a4, b4, q * c12) + lam(a3, b3, q * c23) ** 2 * G)
    f3 = lambda q: meas(q) * 3 * 2 * k * k * G ** 4 * lam(a3, b3, q * c23) ** 3
    f4 = lambda q: meas(q) * 1.5 * 2 * k * k * G ** 3 * lam(a4, b4, q * c12) ** 2
    pts = [0, xm, xm * math.sqrt(2), xm * math.sqrt(1.5), k]
    ez, e3, e4 = (float(mpmath.quad(f, sorted(pts))) for f in (fz, f3, f4))
    assert abs(out[1] - ez) / abs(ez) < 1e-9          # p = 0 point of the Z block
    assert abs(out[2] - e3) / abs(e3) < 1e-9
    assert abs(out[-1] - e4) / abs(e4) < 1e-9


def _matsubara_litim_sum(T, N, E2, m):
    """T sum_{|n|<=N} 1/((w_n^2+E^2)^2 (w_{n+m}^2+E^2)), w_n = 2 pi T n (mpmath)."""
    T = mpmath.mpf(T)
    s = mpmath.mpf(0)
    for n in range(-N, N + 1):
        wn = 2 * mpmath.pi * T * n
        wm = 2 * mpmath.pi * T * (n + m)
        s += 1 / ((wn ** 2 + E2) ** 2 * (wm ** 2 + E2))
    return T * s


@pytest.mark.parametrize("T,N", [(0.05, 4), (0.3, 16), (1.0, 2)])
def test_finite_t_litim_truncated_matsubara(T, N):
    """Quadratureq0 (Sec. 5.3.2) with the spatial flat regulator, Z = lam = 1,
    p -> 0: the spatial integral is (k^3/(6 pi^2)) 2 k^2 and the frequency sum
    is a rational-function sum computed independently."""
    k, w = 1.3, 0.5
    pb = fi.Problem(model=fi.MODEL_FINITE_T, n_rad=8, n_ang1=3, n_ext_p=1, n_ext_ang=3, n_matsubara=N,
                    regulator=fi.REG_LITIM, m2_over_k2=w, T=T, qmax_over_k=1.0, n_tables=2, n_pts=8,
                    n_stack=N + 3, p_min=1e-200, p_max=1e-200)
    out = oracle.rhs(pb, fi.constant_tables(pb, [1.0, 1.0]), k)
    E2 = k * k * (1 + w)
    for m in range(3):
        exact = float(k ** 3 / (6 * mpmath.pi ** 2) * 2 * k * k * _matsubara_litim_sum(T, N, E2, m))
        assert abs(out[m] - exact) / exact < 1e-13, m


def test_finite_t_litim_infinite_sum_limit():
    """N -> infinity: T sum_n (w_n^2+E^2)^-3 = (1/2) d^2/d(E^2)^2 [coth(E/2T)/(2E)]."""
    k, w, T, N = 1.0, 0.5, 0.4, 400
    pb = fi.Problem(model=fi.MODEL_FINITE_T, n_rad=4, n_ang1=2, n_ext_p=1, n_ext_ang=1, n_matsubara=N,
                    regulator=fi.REG_LITIM, m2_over_k2=w, T=T, qmax_over_k=1.0, n_tables=2, n_pts=4,
                    n_stack=N + 1, p_min=1e-200, p_max=1e-200)
    out = oracle.rhs(pb, fi.constant_tables(pb, [1.0, 1.0]), k)
    S1 = lambda e2: mpmath.coth(mpmath.sqrt(e2) / (2 * T)) / (2 * mpmath.sqrt(e2))
    E2 = mpmath.mpf(k * k * (1 + w))
    S3 = mpmath.diff(S1, E2, 2) / 2
    exact = float(k ** 3 / (6 * mpmath.pi ** 2) * 2 * k * k * S3)
    # truncation tail ~ sum_{|n|>N} (2 pi T n)^-6 -> ~1e-15 relative here
    assert abs(out[0] - exact) / exact < 1e-11


# --------------------------------------------------------------------------
# exponential regulator, Z = 1, p = 0: 1D high-precision quadrature
# --------------------------------------------------------------------------
@pytest.mark.parametrize("k", [10.0, 0.37])
def test_d3_exp_regulator_vs_mpmath_quadrature(k):
    w = 0.5
    pb = fi.Problem(model=fi.MODEL_D3, n_rad=64, n_ang1=4, n_ext_p=1, include_p0=1, m2_over_k2=w)
    out = oracle.rhs(pb, fi.constant_tables(pb, [1.0]), k)

    def f(q):
        x = q * q / (k * k)
        r = x / mpmath.expm1(x) if x > 0 else mpmath.mpf(1)
        rd = 2 * x * x * mpmath.exp(-x) / mpmath.expm1(-x) ** 2 if x > 0 else mpmath.mpf(2)
        G = 1 / (q * q + w * k * k + k * k * r)
        return q * q * k * k * rd * G ** 3 / (2 * mpmath.pi ** 2)
    exact = float(mpmath.quad(f, [0, k, 2 * k, 4 * k]))
    assert abs(out[-1] - exact) / exact < 1e-13


def test_d3_geometric_convergence_in_nodes():
    """With a smooth integrand (exponential regulator, constant Z) the product
    GL rule converges geometrically in (n_rad, n_ang); with piecewise-linear
    tables the lerp kinks make it algebraic, so the pin uses Z = 1."""
    wl = fi.make_d3(seed=11, n_ext_p=8)
    pb = wl.problem
    tab = fi.constant_tables(pb, [1.0])
    vals = []
    for nr, na in [(8, 4), (16, 8), (32, 16), (64, 32), (128, 64)]:
        pb.n_rad, pb.n_ang1 = nr, na
        vals.append(oracle.rhs(pb, tab, 1.0))
    d = [np.max(np.abs(vals[i + 1] - vals[i]) / np.abs(vals[-1])) for i in range(4)]
    assert d[0] > d[1] > d[2] and d[2] < 1e-9 and d[3] < 1e-13, d


# --------------------------------------------------------------------------
# rotational invariance: one-angle reduction vs a full 3D product rule with
# the external momentum in an arbitrary direction (Sec. 5.3.2 / App. F angles)
# --------------------------------------------------------------------------
def _loglinear(pb, coeffs):
    """tables a + b ln(s/x_min): the log-grid lerp reproduces them exactly, so
    the integrand stays smooth and product rules converge geometrically."""
    xs = fi.log_grid(pb.n_pts, pb.x_min, pb.x_max)
    rows = [a + b * np.log(xs / pb.x_min) for a, b in coeffs]
    return np.stack(rows).reshape(pb.n_tables, pb.n_stack, pb.n_pts)


def test_d3_rotational_invariance():
    wl = fi.make_d3(seed=5, n_ext_p=64)
    pb = wl.problem
    k = 1.0
    pb.n_rad, pb.n_ang1 = 48, 48
    wl.tables = _loglinear(pb, [(1.0, 0.015)])
    ref = oracle.rhs(pb, wl.tables, k)
    xr, wr = oracle.gauss_legendre(pb.n_rad, 0.0, pb.qmax_over_k * k)
    xc, wc = np.polynomial.legendre.leggauss(48)
    nphi = 48
    phi = 2 * np.pi * np.arange(nphi) / nphi
    rng = np.random.default_rng(3)
    for e in (20, 40, 55):
        p = pb.p_min * (pb.p_max / pb.p_min) ** (e / (pb.n_ext_p - 1))
        u = rng.normal(size=3)
        pv = p * u / np.linalg.norm(u)
        Q, C, P = np.meshgrid(xr, xc, phi, indexing="ij")
        S = np.sqrt(1 - C ** 2)
        qv = np.stack([Q * S * np.cos(P), Q * S * np.sin(P), Q * C], axis=-1)
        s2 = np.sum((qv + pv) ** 2, axis=-1)
        f = oracle.d3_summand_batch(pb, wl.tables, k, (Q ** 2).ravel(), s2.ravel()).reshape(Q.shape)
        W = (wr[:, None, None] * wc[None, :, None] * (2 * np.pi / nphi) * Q ** 2)
        val = np.sum(W * f) / (8 * np.pi ** 3)
        assert abs(val - ref[e]) / abs(ref[e]) < 1e-8, (e, val, ref[e])


def _rot4(rng):
    q, _ = np.linalg.qr(rng.normal(size=(4, 4)))
    return q


def test_d4_rotational_invariance():
    """Two-angle reduction (c1 Gauss-Chebyshev-II, c2 GL) vs a three-angle
    hyperspherical product rule with p1, p2 rotated by a random O(4) matrix."""
    wl = fi.make_d4(seed=9, n_pts=32, n_ext_ang=3, n_rad=24, n_ang1=40, n_ang2=40)
    pb = wl.problem
    k = 1.0
    wl.tables = _loglinear(pb, [(1.0, 0.015), (1.2, -0.03), (0.8, 0.02)])
    ref = oracle.rhs(pb, wl.tables, k)
    xr, wr = oracle.gauss_legendre(pb.n_rad, 0.0, pb.qmax_over_k * k)
    x1, w1 = oracle.gauss_chebyshev2(40)
    x2, w2 = np.polynomial.legendre.leggauss(40)
    nphi = 40
    ph = 2 * np.pi * np.arange(nphi) / nphi
    cpsi, _ = np.polynomial.legendre.leggauss(pb.n_ext_ang)
    rng = np.random.default_rng(7)
    Q, C1, C2, PH = np.meshgrid(xr, x1, x2, ph, indexing="ij")
    S1, S2 = np.sqrt(1 - C1 ** 2), np.sqrt(1 - C2 ** 2)
    qv = np.stack([Q * C1, Q * S1 * C2, Q * S1 * S2 * np.cos(PH), Q * S1 * S2 * np.sin(PH)], -1)
    W = (wr[:, None, None, None] * w1[None, :, None, None] * w2[None, None, :, None]
         * (2 * np.pi / nphi) * Q ** 3) / (2 * np.pi) ** 4
    np_ = pb.n_ext_p
    for ip, j in [(18, 0), (25, 2)]:
        p = pb.p_min * (pb.p_max / pb.p_min) ** (ip / (np_ - 1))
        Rm = _rot4(rng)
        p1 = Rm @ np.array([p, 0, 0, 0])
        p2 = Rm @ np.array([p * cpsi[j], p * math.sqrt(1 - cpsi[j] ** 2), 0, 0])
        A2 = np.sum((qv + p1) ** 2, -1).ravel()
        B2 = np.sum((qv - p2) ** 2, -1).ravel()
        C2 = float(np.sum((p1 + p2) ** 2))
        q2 = (Q ** 2).ravel()
        for block, idx in [(0, ip), (1, np_ + 1 + ip * pb.n_ext_ang + j), (2, np_ + 1 + np_ * pb.n_ext_ang + ip)]:
            f = oracle.d4_summand_batch(block, pb, wl.tables, k, q2, p * p, A2, B2, C2).reshape(Q.shape)
            val = np.sum(W * f)
            assert abs(val - ref[idx]) / abs(ref[idx]) < 2e-8, (block, ip, val, ref[idx])


# --------------------------------------------------------------------------
# brute force: Monte Carlo in the ball |q| < q_max (d = 3)
# --------------------------------------------------------------------------
def test_d3_monte_carlo():
    wl = fi.make_d3(seed=13, n_ext_p=64)
    pb = wl.problem
    k = 1.0
    ref = oracle.rhs(pb, wl.tables, k)
    rng = np.random.default_rng(2024)
    n = 2_000_000
    qmax = pb.qmax_over_k * k
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    r = qmax * rng.uniform(size=n) ** (1 / 3)
    qv = v * r[:, None]
    vol = 4 / 3 * np.pi * qmax ** 3 / (2 * np.pi) ** 3
    for e in (10, 45, 60):
        p = pb.p_min * (pb.p_max / pb.p_min) ** (e / (pb.n_ext_p - 1))
        s2 = np.sum((qv + np.array([0.3, -0.5, 0.81]) / np.linalg.norm([0.3, -0.5, 0.81]) * p) ** 2, 1)
        f = oracle.d3_summand_batch(pb, wl.tables, k, r ** 2, s2)
        mean, sd = vol * f.mean(), vol * f.std() / math.sqrt(n)
        assert abs(mean - ref[e]) < 4 * sd, (e, mean, ref[e], sd)


# --------------------------------------------------------------------------
# RG-time flow (Sec. 2.1 t_+ convention, Sec. 5.2.2 Eq. assVar / flowVar,
# Sec. 5.2.1 RK45 stepper, App. C step parameters)
# --------------------------------------------------------------------------
def test_frozen_flow_endpoint_vs_adaptive_quadrature():
    """Frozen background: y(t) = y(0) - int_0^t I(k(t')) dt', k = Lambda e^{-t'}."""
    from scipy.integrate import quad_vec
    wl = fi.make_d3(seed=21, n_ext_p=16, n_rad=32, n_ang=16)
    pb = wl.problem
    t1 = math.log(wl.Lambda / wl.k_end)
    y, st = oracle.flow(pb, wl.tables, wl.y0, wl.Lambda, t1, rtol=1e-12, atol=1e-15)
    integ, _ = quad_vec(lambda t: oracle.rhs(pb, wl.tables, wl.Lambda * math.exp(-t)), 0.0, t1,
                        epsabs=1e-15, epsrel=1e-13, limit=2000)
    exact = wl.y0 - integ
    assert np.max(np.abs(y - exact) / np.abs(exact)) < 1e-10
    assert st["steps"] > 3


def test_flow_litim_exact_in_t():
    """Flat regulator, Z = 1, p -> 0, w fixed: I = k^{-1}/(3 pi^2 (1+w)^3), so
    y(t) = y0 - (e^t - 1)/(3 pi^2 (1+w)^3 Lambda)."""
    w, Lam = 0.5, 10.0
    pb = fi.Problem(model=fi.MODEL_D3, n_rad=4, n_ang1=2, n_ext_p=1, regulator=fi.REG_LITIM, m2_over_k2=w,
                    qmax_over_k=1.0, p_min=1e-200, p_max=1e-200)
    t1 = math.log(1000.0)
    y, _ = oracle.flow(pb, fi.constant_tables(pb, [1.0]), np.array([3.0]), Lam, t1, rtol=1e-13, atol=1e-16)
    exact = 3.0 - (math.exp(t1) - 1) / (3 * math.pi ** 2 * (1 + w) ** 3 * Lam)
    assert abs(y[0] - exact) / abs(exact) < 1e-11


def test_feedback_flow_vs_scipy_dop853():
    """State-dependent flow (d=3 feedback: m^2 and Z_i flow): the oracle's
    DP5(4) against scipy's independent DOP853 at tight tolerance.  The grid
    starts at 0.05: d_t Z_i = -(I(p_i)-I(0))/p_i^2 amplifies rounding noise by
    1/p_i^2, which at p = 1e-3 would dominate the comparison."""
    from scipy.integrate import solve_ivp
    wl = fi.make_d3(seed=4, n_pts=12, n_ext_p=12, n_rad=24, n_ang=12, feedback=1, x_min=0.05)
    pb = wl.problem
    t1 = 2.0
    y, st = oracle.flow(pb, wl.tables, wl.y0, wl.Lambda, t1, feedback=1, rtol=1e-11, atol=1e-14)
    sol = solve_ivp(lambda t, yy: oracle.flow_deriv(pb, wl.tables, 1, wl.Lambda, t, yy), (0.0, t1), wl.y0,
                    method="DOP853", rtol=1e-13, atol=1e-15)
    ref = sol.y[:, -1]
    assert np.max(np.abs(y - ref) / (np.abs(ref) + 1e-3)) < 1e-9
    assert st["rejects"] >= 0 and st["steps"] > 2


@pytest.mark.parametrize("which", [0, 1, 2])
def test_dp45_fifth_order_on_textbook_odes(which):
    """Fixed steps (dt_min = dt_max = h, tolerance inert): the global error of
    the Dormand-Prince tableau falls like h^5 against the closed forms."""
    t1 = 2.0
    y0 = [1.0, 0.0] if which == 2 else [1.0]
    exact = {0: [math.exp(math.sin(t1))], 1: [1.0 / (1.0 + t1 ** 2)],
             2: [math.cos(t1), -math.sin(t1)]}[which]
    errs = []
    for h in (0.2, 0.1, 0.05, 0.025):
        y, st = oracle.dp45_textbook(which, y0, t1, dt0=h, dt_min=h, dt_max=h, rtol=1e6, atol=1e6)
        assert st["status"] == 0 and st["rejects"] == 0
        errs.append(np.max(np.abs(y - exact)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert all(4.6 < o < 5.6 for o in orders[1:]), (errs, orders)


@pytest.mark.parametrize("rtol", [1e-6, 1e-9, 1e-12])
def test_dp45_adaptive_error_tracks_tolerance(rtol):
    """The embedded fourth-order estimate controls the step: the global error
    stays within a modest multiple of the requested tolerance."""
    y, st = oracle.dp45_textbook(0, [1.0], 10.0, dt0=0.01, rtol=rtol, atol=0.0)
    assert st["status"] == 0
    err = abs(y[0] - math.exp(math.sin(10.0))) / math.exp(math.sin(10.0))
    assert err < 50 * rtol
    y2, st2 = oracle.dp45_textbook(0, [1.0], 10.0, dt0=0.01, rtol=rtol * 1e-2, atol=0.0)
    assert st2["steps"] > st["steps"]


def test_flow_underflow_and_maxsteps_status():
    wl = fi.make_d3(seed=1, n_ext_p=4, n_rad=8, n_ang=4)
    pb = wl.problem
    t1 = math.log(1000.0)
    _, st = oracle.flow(pb, wl.tables, wl.y0, wl.Lambda, t1, dt0=0.5, dt_min=0.5, dt_max=0.5,
                        rtol=1e-16, atol=1e-300, raise_on_error=False)
    assert st["status"] == oracle.ESTEP_UNDERFLOW
    _, st = oracle.flow(pb, wl.tables, wl.y0, wl.Lambda, t1, max_steps=3, raise_on_error=False)
    assert st["status"] == oracle.EMAXSTEPS


# --------------------------------------------------------------------------
# forward-mode derivatives (Sec. 5.2.2 "AD" Jacobians) vs finite differences
# --------------------------------------------------------------------------
@pytest.mark.parametrize("model", [fi.MODEL_D3, fi.MODEL_D4_VERTEX])
def test_jvp_matches_central_differences(model):
    if model == fi.MODEL_D3:
        wl = fi.make_d3(seed=8, n_pts=16, n_ext_p=6, n_rad=16, n_ang=8)
    else:
        wl = fi.make_d4(seed=8, n_pts=12, n_ext_ang=2, n_rad=12, n_ang1=6, n_ang2=4)
    pb = wl.problem
    k = 1.3
    rng = np.random.default_rng(1)
    dT = rng.normal(size=wl.tables.shape)
    val, der = oracle.rhs_jvp(pb, wl.tables, dT, k)
    base = oracle.rhs(pb, wl.tables, k)
    assert np.max(np.abs(val - base) / np.abs(base)) < 1e-14
    h = 1e-6
    fd = (oracle.rhs(pb, wl.tables + h * dT, k) - oracle.rhs(pb, wl.tables - h * dT, k)) / (2 * h)
    scale = np.max(np.abs(der))
    assert np.max(np.abs(fd - der)) / scale < 1e-7


def test_jacobian_columns_are_jvps():
    wl = fi.make_d3(seed=8, n_pts=8, n_ext_p=4, n_rad=8, n_ang=4)
    pb = wl.problem
    J = oracle.rhs_jacobian(pb, wl.tables, 0.9)
    rng = np.random.default_rng(2)
    v = rng.normal(size=wl.tables.size)
    _, d = oracle.rhs_jvp(pb, wl.tables, v.reshape(wl.tables.shape), 0.9)
    assert np.max(np.abs(J @ v - d)) / np.max(np.abs(d)) < 1e-13
    # linear in the table: integrand is rational in Z -> no, but the lambda-free
    # d=3 RHS depends on Z only through lerps: columns far from all lookups vanish
    assert J.shape == (pb.n_ext(), wl.tables.size)


# --------------------------------------------------------------------------
# linearly implicit ROS2 (Rosenbrock) driver and the d=4 feedback flow
# --------------------------------------------------------------------------
@pytest.mark.parametrize("which", [0, 2, 4])
def test_ros2_second_order(which):
    """ROS2 (Verwer, Spee, Blom, Hundsdorfer 1999) is second order, also with a
    zero matrix in place of the Jacobian (which 4: W-method property)."""
    t1 = 2.0
    y0 = [1.0, 0.0] if which in (2, 4) else [1.0]
    exact = [math.exp(math.sin(t1))] if which == 0 else [math.cos(t1), -math.sin(t1)]
    errs = []
    for h in (0.1, 0.05, 0.025, 0.0125):
        y, st = oracle.ros2_textbook(which, y0, t1, dt0=h, dt_min=h, dt_max=h, rtol=1e6, atol=1e6)
        assert st["status"] == 0
        errs.append(np.max(np.abs(y - exact)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert all(1.8 < o < 2.3 for o in orders[1:]), orders


def test_ros2_stiff_problem_is_stable_at_large_steps():
    """Prothero-Robinson, lambda = 1e4: fixed steps with lambda h = 1000 stay
    bounded and first-order accurate (the known stiff order reduction of
    Rosenbrock methods on non-autonomous problems without a time-derivative
    term); an explicit method would be unstable at these steps."""
    errs = []
    for h in (0.2, 0.1, 0.05):
        y, st = oracle.ros2_textbook(3, [1.0], 2.0, dt0=h, dt_min=h, dt_max=h, rtol=1e6, atol=1e6)
        errs.append(abs(y[0] - math.cos(2.0)))
        assert errs[-1] < h
    assert 0.8 < math.log2(errs[1] / errs[2]) < 1.3


def test_ros2_d4_feedback_flow_matches_dp45():
    wl = fi.make_d4(seed=6, n_pts=8, n_ext_ang=2, n_rad=8, n_ang1=4, n_ang2=3)
    pb = wl.problem
    pb.p_min = pb.x_min = 0.05
    t1 = 2.0
    ref, _ = oracle.flow(pb, wl.tables, wl.y0, wl.Lambda, t1, feedback=1, rtol=1e-12, atol=1e-14)
    y, st = oracle.ros2_flow(pb, wl.y0, wl.Lambda, t1, rtol=1e-8, atol=1e-12)
    assert np.max(np.abs(y - ref) / np.abs(ref)) < 2e-6, np.max(np.abs(y - ref) / np.abs(ref))
    assert st["steps"] > 3


# --------------------------------------------------------------------------
# fermionic loop frequencies nu_n = (2n+1) pi T (App. F fermionic stacks)
# --------------------------------------------------------------------------
def _fermionic_litim_sum(T, N, E2, m):
    """T sum_{n=-N-1}^{N} 1/((nu_n^2+E^2)^2 (nu_{n+m}^2+E^2)), nu_n = (2n+1) pi T (mpmath)."""
    T = mpmath.mpf(T)
    s = mpmath.mpf(0)
    for n in range(-N - 1, N + 1):
        vn = (2 * n + 1) * mpmath.pi * T
        vm = (2 * (n + m) + 1) * mpmath.pi * T
        s += 1 / ((vn ** 2 + E2) ** 2 * (vm ** 2 + E2))
    return T * s


def _fermionic_litim_problem(T, N, n_ext_m, k_pts=8):
    return fi.Problem(model=fi.MODEL_FINITE_T, n_rad=k_pts, n_ang1=3, n_ext_p=1, n_ext_ang=n_ext_m,
                      n_matsubara=N, regulator=fi.REG_LITIM, m2_over_k2=0.5, T=T, qmax_over_k=1.0,
                      n_tables=2, n_pts=8, n_stack=N + n_ext_m + 1, p_min=1e-200, p_max=1e-200,
                      statistics=fi.STAT_FERMI)


@pytest.mark.parametrize("T,N", [(0.05, 4), (0.3, 16), (1.0, 2)])
def test_finite_t_fermionic_litim_truncated_matsubara(T, N):
    """Fermionic loop, spatial flat regulator, Z = lam = 1, p -> 0: the 2N+2
    frequencies nu_n, n = -N-1..N, against an independent rational sum."""
    k, w = 1.3, 0.5
    pb = _fermionic_litim_problem(T, N, 3)
    out = oracle.rhs(pb, fi.constant_tables(pb, [1.0, 1.0]), k)
    E2 = k * k * (1 + w)
    for m in range(3):
        exact = float(k ** 3 / (6 * mpmath.pi ** 2) * 2 * k * k * _fermionic_litim_sum(T, N, E2, m))
        assert abs(out[m] - exact) / exact < 1e-13, m


def test_finite_t_fermionic_infinite_sum_limit():
    """N -> infinity: T sum_n (nu_n^2+E^2)^-3 = (1/2) d^2/d(E^2)^2 [tanh(E/2T)/(2E)]."""
    k, w, T, N = 1.0, 0.5, 0.4, 400
    pb = _fermionic_litim_problem(T, N, 1, k_pts=4)
    out = oracle.rhs(pb, fi.constant_tables(pb, [1.0, 1.0]), k)
    S1 = lambda e2: mpmath.tanh(mpmath.sqrt(e2) / (2 * T)) / (2 * mpmath.sqrt(e2))
    E2 = mpmath.mpf(k * k * (1 + w))
    exact = float(k ** 3 / (6 * mpmath.pi ** 2) * 2 * k * k * mpmath.diff(S1, E2, 2) / 2)
    assert abs(out[0] - exact) / exact < 1e-11


def test_finite_t_fermionic_stack_index_and_low_T_limit():
    """Row j of a fermionic stack holds nu_j = (2j+1) pi T and serves n = j and
    n = -j-1: with Z rows that grow in j the sum is even under n -> -n-1 only if
    both members of a pair read the same row.  At T -> 0 both statistics approach
    the continuum frequency integral int dnu/(2 pi) (nu^2+E^2)^-3 = 3/(16 E^5)."""
    k, w, T, N = 1.0, 0.5, 0.3, 6
    pb = _fermionic_litim_problem(T, N, 1)
    tab = fi.constant_tables(pb, [1.0, 1.0])
    tab[0] = (1.0 + 0.1 * np.arange(pb.n_stack))[:, None]      # Z_j = 1 + j/10
    out = oracle.rhs(pb, tab, k)[0]
    E2 = k * k * (1 + w)
    s = mpmath.mpf(0)
    for n in range(-N - 1, N + 1):
        j = n if n >= 0 else -n - 1
        Z = 1 + mpmath.mpf(j) / 10
        vn2 = ((2 * n + 1) * mpmath.pi * T) ** 2
        den = Z * (vn2 + k * k) + k * k * w            # flat regulator: q^2 + R = k^2 for q < k
        s += Z * 2 * k * k / den ** 3                  # dR = Z 2 k^2
    exact = float(k ** 3 / (6 * mpmath.pi ** 2) * T * s)
    assert abs(out - exact) / exact < 1e-13
    # low temperature: bosonic and fermionic sums both -> the continuum integral
    Tl, Nl = 0.002, 4000
    for stat in (fi.STAT_BOSE, fi.STAT_FERMI):
        pl = fi.Problem(model=fi.MODEL_FINITE_T, n_rad=2, n_ang1=1, n_ext_p=1, n_ext_ang=1, n_matsubara=Nl,
                        regulator=fi.REG_LITIM, m2_over_k2=w, T=Tl, qmax_over_k=1.0, n_tables=2, n_pts=4,
                        n_stack=2, p_min=1e-200, p_max=1e-200, statistics=stat)
        o = oracle.rhs(pl, fi.constant_tables(pl, [1.0, 1.0]), k)[0]
        cont = k ** 3 / (6 * math.pi ** 2) * 2 * k * k * 3 / (16 * E2 ** 2.5)
        assert abs(o - cont) / cont < 1e-6, stat


# --------------------------------------------------------------------------
# Adams-Bashforth-Moulton (PECE, fixed step, RK4 start)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("order", [2, 3, 4, 5])
def test_abm_order_of_convergence(order):
    """Global error ~ h^order: error ratio 2^order per halving of h on the
    harmonic oscillator and (orders 3-5) on y' = y cos t (y = exp(sin t)); for
    order 2 the latter's error changes sign near t = 3, so it gives no rate."""
    cases = [(2, [1.0, 0.0], lambda t: [math.cos(t), -math.sin(t)], (80, 160, 320))]
    if order >= 3:
        cases.append((0, [1.0], lambda t: [math.exp(math.sin(t))], (160, 320, 640)))
    for which, y0, exact, ns in cases:
        t1 = 3.0
        errs = []
        for n in ns:
            y, ev = oracle.abm_textbook(which, order, y0, t1, n)
            errs.append(np.max(np.abs(y - np.array(exact(t1)))))
            assert ev == 1 + 4 * (order - 1) + 2 * (n - order + 1)
        rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
        assert all(order - 0.35 < r < order + 0.6 for r in rates), (which, order, rates)


def test_abm4_exact_for_cubic_derivative():
    """y' = 4 t^3: Simpson-exact RK4 start and AB4/AM4 exact for cubic f."""
    y, _ = oracle.abm_textbook(3, 4, [0.5], 2.0, 13, t0=0.25)
    assert abs(y[0] - (0.5 + 2.0 ** 4 - 0.25 ** 4)) < 1e-13


def test_abm_flow_matches_dp45_flow():
    """The ABM flow of a frozen d=3 RHS against a tight DP5(4) flow."""
    wl = fi.make_d3(seed=3, n_pts=16, n_ext_p=8, n_rad=10, n_ang=6)
    t1 = math.log(wl.Lambda / wl.k_end)
    ref, _ = oracle.flow(wl.problem, wl.tables, wl.y0, wl.Lambda, t1, rtol=1e-12, atol=1e-15)
    errs = []
    for n in (100, 200):
        y, st = oracle.abm_flow(wl.problem, wl.tables, wl.y0, wl.Lambda, t1, n, order=4)
        errs.append(np.max(np.abs(y - ref) / np.abs(ref)))
        assert st["rhs_evals"] == 1 + 4 * 3 + 2 * (n - 3)
    assert errs[1] < 1e-6 and errs[0] / errs[1] > 8      # fourth order


# --------------------------------------------------------------------------
# d=4 with the three-point vertex on (S0, a, b) ("Full" vertex dependence)
# --------------------------------------------------------------------------
def test_d4_full_reduces_to_d4_vertex_for_angle_independent_vertex():
    """With lambda3 rows equal in (a, b) the full model is the vertex model."""
    wl = fi.make_d4(seed=31, n_pts=12, n_ext_ang=3, n_rad=7, n_ang1=5, n_ang2=4)
    ref = oracle.rhs(wl.problem, wl.tables, 0.9)
    na, nb = 3, 4
    pf = dataclasses.replace(wl.problem, model=fi.MODEL_D4_FULL, n_stack=na * nb, n_va=na, n_vb=nb)
    tf = np.zeros((3, na * nb, pf.n_pts))
    tf[0, 0], tf[2, 0] = wl.tables[0, 0], wl.tables[2, 0]
    tf[1, :] = wl.tables[1, 0]
    out = oracle.rhs(pf, tf, 0.9)
    assert np.max(np.abs(out - ref) / np.abs(ref)) < 1e-13


def test_d4_full_trilinear_lookup_is_exact_on_trilinear_tables():
    """Tables of f = c0 + c1 ln S + c2 a + c3 b + c4 a b + c5 a ln S are
    reproduced exactly by the lookup (linear in ln S, a and b between nodes)."""
    na, nb, n = 5, 4, 9
    pb = fi.Problem(model=fi.MODEL_D4_FULL, n_rad=2, n_ang1=2, n_ang2=2, n_ext_p=n, n_ext_ang=1, n_tables=3,
                    n_pts=n, n_stack=na * nb, n_va=na, n_vb=nb)
    c = [0.7, 0.3, -0.2, 0.15, 0.05, 0.1]
    f = lambda S, a, b: c[0] + c[1] * math.log(S) + c[2] * a + c[3] * b + c[4] * a * b + c[5] * a * math.log(S)
    xs = fi.log_grid(n, pb.x_min, pb.x_max)
    av, bv = np.linspace(-1, 1, na), np.linspace(-1, 1, nb)
    tab = np.zeros((3, na * nb, n))
    for ia in range(na):
        for ib in range(nb):
            tab[1, ia * nb + ib] = [f(x, av[ia], bv[ib]) for x in xs]
    rng = np.random.default_rng(3)
    for _ in range(200):
        s1, s2, s3 = rng.uniform(0.01, 30.0, 3)
        S = math.sqrt((s1 + s2 + s3) / 3)
        if not (pb.x_min <= S <= pb.x_max):
            continue
        a, b = oracle.d4_shape(s1, s2, s3)
        assert abs(oracle.lam3_full(pb, tab, s1, s2, s3) - f(S, a, b)) < 1e-13


def test_d4_full_shape_variables_from_vectors():
    """a is the cosine between legs 1 and 2, b = (k1^2 - k2^2)/(k1^2 + k2^2),
    for random 4-vectors with k3 = -k1 - k2 (clamped to [-1, 1])."""
    rng = np.random.default_rng(7)
    for _ in range(100):
        k1, k2 = rng.normal(size=4), rng.normal(size=4)
        k3 = -k1 - k2
        a, b = oracle.d4_shape(k1 @ k1, k2 @ k2, k3 @ k3)
        assert abs(a - k1 @ k2 / math.sqrt((k1 @ k1) * (k2 @ k2))) < 1e-12
        assert abs(b - (k1 @ k1 - k2 @ k2) / (k1 @ k1 + k2 @ k2)) < 1e-13
    assert oracle.d4_shape(1.0, 1.0, 9.0)[0] == 1.0 and oracle.d4_shape(1.0, 1.0, -5.0)[0] == -1.0


# --------------------------------------------------------------------------
# Non-constant tables away from p = 0, against an independent route to the
# same continuum integral.  With s^2 = |q + p|^2 = q^2 + p^2 + 2 q p c the
# angular integral of a function of |q + p| becomes a 1-D integral in s:
#   int_{-1}^{1} f(|q+p|) dc = (1/qp) int_{|q-p|}^{q+p} s f(s) ds
# (d=4, Gauss-Chebyshev-II weight: the same with sqrt(1 - c(s)^2) inside).
# Nested adaptive quadrature of that form (scipy) against the oracle's
# Gauss product rule.  Tables linear in ln s, which the log-grid lookup
# reproduces exactly; smooth exponential regulator.
# --------------------------------------------------------------------------
def _exp_r(x):
    return 1.0 if x < 1e-12 else x / math.expm1(x)


def _exp_rdot(x):
    if x < 1e-12:
        return 2.0
    em = math.expm1(-x)
    return 2.0 * x * x * math.exp(-x) / (em * em)


def _loglin(pb, a, b):
    """lookup of a + b ln(s / x_min), clamped like the table lookup"""
    def f(s):
        return a + b * math.log(min(max(s, pb.x_min), pb.x_max) / pb.x_min)
    return f


def _ang(q, p, f, gc2=False):
    from scipy import integrate

    def g(s):
        if not gc2:
            return s * f(s)
        c = (s * s - q * q - p * p) / (2 * q * p)
        return s * math.sqrt(max(0.0, 1.0 - c * c)) * f(s)
    v, _ = integrate.quad(g, abs(q - p), q + p, epsabs=0, epsrel=1e-13, limit=200)
    return v / (q * p)


def _radial(f, qmax):
    from scipy import integrate
    v, _ = integrate.quad(f, 0.0, qmax, epsabs=0, epsrel=1e-12, limit=200)
    return v


def test_d3_nonconstant_table_at_finite_p_vs_angle_substitution():
    pytest.importorskip("scipy")
    k, w, a, b = 1.0, 0.5, 1.0, 0.04
    wl = fi.make_d3(seed=5, n_pts=48, n_ext_p=16, n_rad=128, n_ang=128)
    pb = wl.problem
    pb.m2_over_k2, pb.m2_shift = w, 0.0
    xs = fi.log_grid(pb.n_pts, pb.x_min, pb.x_max)
    ref = oracle.rhs(pb, (a + b * np.log(xs / pb.x_min)).reshape(1, 1, -1), k)
    Z, m2 = _loglin(pb, a, b), w * k * k

    def G(s):
        return 1.0 / (Z(s) * (s * s + k * k * _exp_r(s * s / (k * k))) + m2)
    ps = [pb.p_min * (pb.p_max / pb.p_min) ** (e / (pb.n_ext_p - 1)) for e in range(pb.n_ext_p)]
    for e in (4, 8, 11, 13):
        p = ps[e]
        val = _radial(lambda q: q * q * Z(q) * k * k * _exp_rdot(q * q / (k * k)) * G(q) ** 2 * _ang(q, p, G),
                      pb.qmax_over_k * k) / (4 * math.pi ** 2)
        # the lookup clamp at s -> 0 (q = p, c = -1) limits the product rule
        # to algebraic convergence: 3e-8 at 128 x 128 nodes
        assert abs(val - ref[e]) / abs(ref[e]) < 2e-7, (e, val, ref[e])


@pytest.mark.parametrize("fermionic", [False, True])
def test_finite_t_row_dependent_tables_at_finite_p_and_m_vs_angle_substitution(fermionic):
    """Z and lambda linear in ln s with coefficients that depend on the stack
    row: pins the frequency of every line, the row of n and n + m, and both
    vertex factors of the finite-T loop."""
    pytest.importorskip("scipy")
    k, w, T, N, M = 1.0, 0.5, 0.3, 2, 2
    wl = fi.make_finite_t(seed=8 if fermionic else 7, N=N, T=T, n_pts=40, n_ext_p=6, n_ext_m=M, n_rad=128,
                          n_ang=128, fermionic=fermionic)
    pb = wl.problem
    pb.m2_over_k2, pb.m2_shift = w, 0.0
    ns = pb.n_stack
    za = [1.0 + 0.05 * j for j in range(ns)]
    zb = [0.03 - 0.004 * j for j in range(ns)]
    la = [0.9 - 0.03 * j for j in range(ns)]
    lb = [0.02 + 0.003 * j for j in range(ns)]
    lg = np.log(fi.log_grid(pb.n_pts, pb.x_min, pb.x_max) / pb.x_min)
    tab = np.stack([np.stack([za[j] + zb[j] * lg for j in range(ns)]),
                    np.stack([la[j] + lb[j] * lg for j in range(ns)])])
    ref = oracle.rhs(pb, tab, k)
    m2 = w * k * k

    def row(n):          # bosonic omega_n: |n|; fermionic nu_n = (2n+1) pi T: n or -n-1
        return min(abs(n) if not fermionic else (n if n >= 0 else -n - 1), ns - 1)

    def freq2(n):
        return ((2 * n + 1) * math.pi * T) ** 2 if fermionic else (2 * math.pi * T * n) ** 2

    def Z(n, s):
        return _loglin(pb, za[row(n)], zb[row(n)])(s)

    def lam(n, s):
        return _loglin(pb, la[row(n)], lb[row(n)])(s)

    def G(n, s):
        return 1.0 / (Z(n, s) * (freq2(n) + s * s + k * k * _exp_r(s * s / (k * k))) + m2)
    ps = [pb.p_min * (pb.p_max / pb.p_min) ** (e / (pb.n_ext_p - 1)) for e in range(pb.n_ext_p)]
    loop = range(-N - 1, N + 1) if fermionic else range(-N, N + 1)
    for ip in (2, 4):
        for m in range(M):
            p = ps[ip]
            tot = sum(_radial(lambda q: q * q * Z(n, q) * k * k * _exp_rdot(q * q / (k * k)) * G(n, q) ** 2
                              * lam(n, q) * _ang(q, p, lambda s: lam(n + m, s) * G(n + m, s)), pb.qmax_over_k * k)
                      for n in loop) * T / (4 * math.pi ** 2)
            e = ip * M + m
            assert abs(tot - ref[e]) / abs(ref[e]) < 5e-9, (ip, m, tot, ref[e])


def test_d4_two_point_blocks_at_finite_p_vs_angle_substitution():
    """The propagator block D2(p) = int dR G^2 [-lam4/2 + lam3^2 G(|q+p|)] and
    the four-point block 3/2 int dR G^2 G(|q+p|) lam4^2 with all three tables
    linear in ln s; the second angle integrates to 2."""
    pytest.importorskip("scipy")
    k = 1.0
    wl = fi.make_d4(seed=9, n_pts=40, n_ext_ang=2, n_rad=128, n_ang1=128, n_ang2=2)
    pb = wl.problem
    co = [(1.0, 0.03), (1.1, -0.02), (0.8, 0.025)]
    lg = np.log(fi.log_grid(pb.n_pts, pb.x_min, pb.x_max) / pb.x_min)
    ref = oracle.rhs(pb, np.stack([(a + b * lg).reshape(1, -1) for a, b in co]), k)
    Z, l3, l4 = (_loglin(pb, a, b) for a, b in co)
    m2 = pb.m2_over_k2 * k * k + pb.m2_shift

    def G(s):
        return 1.0 / (Z(s) * (s * s + k * k * _exp_r(s * s / (k * k))) + m2)

    def base(q):
        return q ** 3 * Z(q) * k * k * _exp_rdot(q * q / (k * k)) * G(q) ** 2 * 2.0
    np_, npsi = pb.n_ext_p, pb.n_ext_ang
    ps = [pb.p_min * (pb.p_max / pb.p_min) ** (e / (np_ - 1)) for e in range(np_)]
    norm = 8 * math.pi ** 3
    for ip in (np_ // 2, (3 * np_) // 4, np_ - 3):
        p = ps[ip]
        zb = _radial(lambda q: base(q) * (-0.5 * l4(math.sqrt((q * q + p * p) / 2)) * math.pi / 2
                                          + _ang(q, p, lambda s: l3(math.sqrt((q * q + s * s + p * p) / 3)) ** 2
                                                 * G(s), gc2=True)), pb.qmax_over_k * k) / norm
        f4 = _radial(lambda q: 1.5 * base(q) * _ang(q, p, lambda s: G(s) * l4(math.sqrt((q * q + s * s + 2 * p * p)
                                                                                      / 4)) ** 2, gc2=True),
                     pb.qmax_over_k * k) / norm
        for val, e in ((zb, ip), (f4, np_ + 1 + np_ * npsi + ip)):
            assert abs(val - ref[e]) / abs(ref[e]) < 2e-9, (ip, e, val, ref[e])


def test_d4_three_point_block_summand_written_from_the_model():
    """The three-point block 3 int dR G(q)^2 G(|q+p1|) G(|q-p2|) lam3 lam3 lam3,
    with the three vertices at S0 of their legs (q, q+p1, p1), (q, q-p2, p2),
    (q+p1, q-p2, p1+p2), written here from the model definition and summed
    over explicit 4-vectors (three-angle product rule, p1 and p2 under a random
    O(4) rotation) -- independent of the oracle's summand, its two-angle
    reduction and its angle variables.  Tables linear in ln s."""
    wl = fi.make_d4(seed=9, n_pts=32, n_ext_ang=3, n_rad=24, n_ang1=40, n_ang2=40)
    pb = wl.problem
    k = 1.0
    co = [(1.0, 0.015), (1.2, -0.03), (0.8, 0.02)]
    lg = np.log(fi.log_grid(pb.n_pts, pb.x_min, pb.x_max) / pb.x_min)
    ref = oracle.rhs(pb, np.stack([(a + b * lg).reshape(1, -1) for a, b in co]), k)

    def look(i, s):
        a, b = co[i]
        return a + b * np.log(np.clip(s, pb.x_min, pb.x_max) / pb.x_min)

    def r(x):
        out = np.ones_like(x)
        m = x > 1e-12
        out[m] = x[m] / np.expm1(x[m])
        return out

    def rdot(x):
        out = np.full_like(x, 2.0)
        m = x > 1e-12
        em = np.expm1(-x[m])
        out[m] = 2 * x[m] ** 2 * np.exp(-x[m]) / em ** 2
        return out
    m2 = pb.m2_over_k2 * k * k + pb.m2_shift

    def G(s2):
        return 1.0 / (look(0, np.sqrt(np.maximum(s2, 0.0))) * (s2 + k * k * r(s2 / (k * k))) + m2)
    xr, wr = oracle.gauss_legendre(pb.n_rad, 0.0, pb.qmax_over_k * k)
    x1, w1 = oracle.gauss_chebyshev2(40)
    x2, w2 = np.polynomial.legendre.leggauss(40)
    nphi = 40
    ph = 2 * np.pi * np.arange(nphi) / nphi
    cpsi, _ = np.polynomial.legendre.leggauss(pb.n_ext_ang)
    Q, C1, C2, PH = np.meshgrid(xr, x1, x2, ph, indexing="ij")
    S1, S2 = np.sqrt(1 - C1 ** 2), np.sqrt(1 - C2 ** 2)
    qv = np.stack([Q * C1, Q * S1 * C2, Q * S1 * S2 * np.cos(PH), Q * S1 * S2 * np.sin(PH)], -1)
    W = (wr[:, None, None, None] * w1[None, :, None, None] * w2[None, None, :, None]
         * (2 * np.pi / nphi) * Q ** 3) / (2 * np.pi) ** 4
    q2 = Q ** 2
    base = 3 * look(0, Q) * k * k * rdot(q2 / (k * k)) * G(q2) ** 2
    rng = np.random.default_rng(7)
    np_ = pb.n_ext_p
    for ip, j in [(18, 0), (25, 2), (29, 1)]:
        p = pb.p_min * (pb.p_max / pb.p_min) ** (ip / (np_ - 1))
        Rm = _rot4(rng)
        p1 = Rm @ np.array([p, 0, 0, 0])
        p2 = Rm @ np.array([p * cpsi[j], p * math.sqrt(1 - cpsi[j] ** 2), 0, 0])
        A2 = np.sum((qv + p1) ** 2, -1)
        B2 = np.sum((qv - p2) ** 2, -1)
        Cc = float(np.sum((p1 + p2) ** 2))
        f = (base * G(A2) * G(B2) * look(1, np.sqrt((q2 + A2 + p * p) / 3))
             * look(1, np.sqrt((q2 + B2 + p * p) / 3)) * look(1, np.sqrt((A2 + B2 + Cc) / 3)))
        val = float(np.sum(W * f))
        e = np_ + 1 + ip * pb.n_ext_ang + j
        assert abs(val - ref[e]) / abs(ref[e]) < 2e-8, (ip, j, val, ref[e])


def test_d4_full_vertex_blocks_with_shape_variables_from_leg_vectors():
    """Full vertex: lambda3 multilinear in (ln S0, a, b) (reproduced exactly by
    the trilinear lookup), its a = cos(k1, k2) and b = (|k1|^2 - |k2|^2) /
    (|k1|^2 + |k2|^2) taken here from dot products of the explicit leg
    4-vectors; the propagator block and the three-point block summed over the
    three-angle product rule with p1, p2 under a random O(4) rotation (and the
    four-point block, whose table sits at another row offset here).  The
    difference is the two rules' discretisation (2.9e-7 here, 1.9e-8 with 64^2
    and 64^2 x 48 nodes); a wrong leg or leg order changes a or b at O(1)."""
    na, nb = 4, 3
    wl = fi.make_d4_full(seed=11, n_pts=32, n_va=na, n_vb=nb, n_ext_ang=3, n_rad=24, n_ang1=40, n_ang2=40)
    pb = wl.problem
    k = 1.0
    lg = np.log(fi.log_grid(pb.n_pts, pb.x_min, pb.x_max) / pb.x_min)
    zc, l4c = (1.0, 0.015), (0.8, 0.02)
    g = (1.1, -0.02, 0.15, -0.1, 0.05)      # lam3 = g0 + g1 ln(S0/x_min) + g2 a + g3 b + g4 a b
    av, bv = np.linspace(-1, 1, na), np.linspace(-1, 1, nb)
    tab = np.zeros((3, na * nb, pb.n_pts))
    tab[0, 0] = zc[0] + zc[1] * lg
    tab[2, 0] = l4c[0] + l4c[1] * lg
    for ia in range(na):
        for ib in range(nb):
            tab[1, ia * nb + ib] = g[0] + g[1] * lg + g[2] * av[ia] + g[3] * bv[ib] + g[4] * av[ia] * bv[ib]

    def ell(s):
        return np.log(np.clip(s, pb.x_min, pb.x_max) / pb.x_min)

    def lam3(k1, k2):     # vertex with legs k1, k2, -(k1 + k2)
        s1, s2 = np.sum(k1 * k1, -1), np.sum(k2 * k2, -1)
        s3 = np.sum((k1 + k2) ** 2, -1)
        with np.errstate(invalid="ignore", divide="ignore"):
            a = np.sum(k1 * k2, -1) / np.sqrt(s1 * s2)
            b = (s1 - s2) / (s1 + s2)
        a = np.nan_to_num(np.clip(a, -1, 1), nan=-1.0)
        b = np.nan_to_num(np.clip(b, -1, 1), nan=-1.0)
        return g[0] + g[1] * ell(np.sqrt((s1 + s2 + s3) / 3)) + g[2] * a + g[3] * b + g[4] * a * b

    def r(x):
        out = np.ones_like(x)
        m = x > 1e-12
        out[m] = x[m] / np.expm1(x[m])
        return out

    def rdot(x):
        out = np.full_like(x, 2.0)
        m = x > 1e-12
        em = np.expm1(-x[m])
        out[m] = 2 * x[m] ** 2 * np.exp(-x[m]) / em ** 2
        return out
    m2 = pb.m2_over_k2 * k * k + pb.m2_shift

    def G(s2):
        return 1.0 / ((zc[0] + zc[1] * ell(np.sqrt(np.maximum(s2, 0.0)))) * (s2 + k * k * r(s2 / (k * k))) + m2)
    xr, wr = oracle.gauss_legendre(pb.n_rad, 0.0, pb.qmax_over_k * k)
    x1, w1 = oracle.gauss_chebyshev2(40)
    x2, w2 = np.polynomial.legendre.leggauss(40)
    nphi = 40
    ph = 2 * np.pi * np.arange(nphi) / nphi
    cpsi, _ = np.polynomial.legendre.leggauss(pb.n_ext_ang)
    Q, C1, C2, PH = np.meshgrid(xr, x1, x2, ph, indexing="ij")
    S1, S2 = np.sqrt(1 - C1 ** 2), np.sqrt(1 - C2 ** 2)
    qv = np.stack([Q * C1, Q * S1 * C2, Q * S1 * S2 * np.cos(PH), Q * S1 * S2 * np.sin(PH)], -1)
    W = (wr[:, None, None, None] * w1[None, :, None, None] * w2[None, None, :, None]
         * (2 * np.pi / nphi) * Q ** 3) / (2 * np.pi) ** 4
    q2 = Q ** 2
    base = (zc[0] + zc[1] * ell(Q)) * k * k * rdot(q2 / (k * k)) * G(q2) ** 2
    rng = np.random.default_rng(5)
    np_ = pb.n_ext_p
    sel, vals = [], []
    for ip, j in [(12, 0), (20, 2), (26, 1)]:
        p = pb.p_min * (pb.p_max / pb.p_min) ** (ip / (np_ - 1))
        Rm = _rot4(rng)
        p1 = Rm @ np.array([p, 0, 0, 0])
        p2 = Rm @ np.array([p * cpsi[j], p * math.sqrt(1 - cpsi[j] ** 2), 0, 0])
        A2 = np.sum((qv + p1) ** 2, -1)
        B2 = np.sum((qv - p2) ** 2, -1)
        l4 = l4c[0] + l4c[1] * ell(np.sqrt((2 * q2 + 2 * p * p) / 4))
        zblock = base * (-0.5 * l4 + lam3(qv, -(qv + p1)) ** 2 * G(A2))
        three = 3 * base * G(A2) * G(B2) * lam3(qv, -(qv + p1)) * lam3(qv, -(qv - p2)) * lam3(qv + p1, -(qv - p2))
        four = 1.5 * base * G(A2) * (l4c[0] + l4c[1] * ell(np.sqrt((q2 + A2 + 2 * p * p) / 4))) ** 2
        sel += [ip, np_ + 1 + ip * pb.n_ext_ang + j, np_ + 1 + np_ * pb.n_ext_ang + ip]
        vals += [float(np.sum(W * zblock)), float(np.sum(W * three)), float(np.sum(W * four))]
    ref = oracle.rhs_subset(pb, tab, k, sel)
    for e, v, rf in zip(sel, vals, ref):
        assert abs(v - rf) / abs(rf) < 1e-6, (e, v, rf)
