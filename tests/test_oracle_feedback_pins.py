"""Pins of the oracle's feedback maps against mathematics (no GPU).

In a feedback flow the state is the truncation itself and its RG-time
derivative is a fixed linear map of the raw loop integrals (Sec. 2.1 t_+
convention, d_t y = -Flow; Sec. 5.2.2 Eqs. assVar / flowVar):
  d=3:  d_t m^2 = -I(0),           d_t Z_i = -(I(p_i) - I(0)) / p_i^2
  d=4:  d_t Z_i = -(D2(p_i) - D2(0)) / p_i^2,
        d_t lambda3_i = -sum_psi (w_psi / 2) Flow3(p_i, psi)  (angle average),
        d_t lambda4_i = -Flow4(p_i).
These tests tie each component to quantities computed without the oracle's
summands: flat-regulator closed forms, the p -> 0 limit of the difference
quotients (d/d(p^2) of the angle average, taken by mpmath), the angle
substitution s = |q + p| with adaptive quadrature, and summands written here
over explicit 4-vectors.  The d=4 state Jacobian used by the implicit stepper
is then tied to this map by central differences.  A sign slip, a missing 1/2
on the psi weights, the p = 0 value read from another slot, or the state's
m^2 / Z not reaching the loop each fail one of them.
"""
import math

import numpy as np
import pytest

import ffrg_inputs as fi
import oracle

mpmath = pytest.importorskip("mpmath")


def _rdot(x):
    if x < 1e-12:
        return 2.0
    em = math.expm1(-x)
    return 2.0 * x * x * math.exp(-x) / (em * em)


def _r(x):
    return 1.0 if x < 1e-12 else x / math.expm1(x)


def _mp_r(x):
    return mpmath.mpf(1) if x == 0 else x / mpmath.expm1(x)


def _mp_rdot(x):
    if x == 0:
        return mpmath.mpf(2)
    em = mpmath.expm1(-x)
    return 2 * x * x * mpmath.exp(-x) / (em * em)


def _loglin(pb, a, b):
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


def _t_of_k(Lambda, k):
    return math.log(Lambda / k)


# --------------------------------------------------------------------------
# d = 3 feedback: state (m^2, Z_0 .. Z_{n-1})
# --------------------------------------------------------------------------
@pytest.mark.parametrize("k,w,c", [(1.7, 0.5, 1.3), (0.4, -0.2, 1.0), (3.0, 2.0, 0.8)])
def test_d3_feedback_mass_component_flat_regulator_closed_form(k, w, c):
    """Flat regulator, Z state = c, m^2 state = w k^2, q < k: G = 1/(c k^2 + m^2)
    and dR = 2 c k^2, so I(0) = (1/2pi^2)(k^3/3) 2 c k^2 G^3 =
    c / (3 pi^2 k (c + w)^3) and d_t m^2 = -I(0).  The problem's own mass
    parameters are set to other values: only the state's m^2 may enter."""
    n = 8
    Lam = 10.0
    pb = fi.Problem(model=fi.MODEL_D3, n_rad=16, n_ang1=4, n_ext_p=n, regulator=fi.REG_LITIM,
                    m2_over_k2=0.7, m2_shift=5.0, qmax_over_k=1.0, n_tables=1, n_pts=n, n_stack=1,
                    include_p0=1, p_min=1e-3, p_max=10.0, x_min=1e-3, x_max=10.0)
    y = np.concatenate([[w * k * k], np.full(n, c)])
    dy = oracle.flow_deriv(pb, fi.constant_tables(pb, [1.0]), 1, Lam, _t_of_k(Lam, k), y)
    exact = c / (3 * math.pi ** 2 * k * (c + w) ** 3)
    assert abs(dy[0] + exact) / exact < 1e-13, (dy[0], -exact)


def test_d3_feedback_Z_components_at_small_p_vs_derivative_of_angle_average():
    """Exponential regulator, Z state constant (g smooth in u = |q+p|^2):
    int_{-1}^{1} dc g(q^2 + p^2 + 2 q p c) = 2 g(q^2) + p^2 (2 g'(q^2) +
    (4/3) q^2 g''(q^2)) + O(p^4), so at p_0 = 1e-3 the first Z component is
    -dI/d(p^2) at p = 0 up to O(p_0^2); the derivatives are taken by mpmath
    and the radial integral by mpmath.quad."""
    k, Lam, w, c, n = 1.0, 10.0, 0.4, 1.1, 12
    pb = fi.Problem(model=fi.MODEL_D3, n_rad=96, n_ang1=16, n_ext_p=n, regulator=fi.REG_EXP,
                    m2_over_k2=0.9, m2_shift=-0.3, qmax_over_k=4.0, n_tables=1, n_pts=n, n_stack=1,
                    include_p0=1, p_min=1e-3, p_max=10.0, x_min=1e-3, x_max=10.0)
    y = np.concatenate([[w * k * k], np.full(n, c)])
    dy = oracle.flow_deriv(pb, fi.constant_tables(pb, [1.0]), 1, Lam, _t_of_k(Lam, k), y)
    with mpmath.workdps(30):
        kk, cc, m2 = mpmath.mpf(k), mpmath.mpf(c), mpmath.mpf(w) * k * k

        def g(u):
            return 1 / (cc * (u + kk * kk * _mp_r(u / (kk * kk))) + m2)

        def integrand(q):
            u = q * q
            f = cc * kk * kk * _mp_rdot(u / (kk * kk)) * g(u) ** 2
            return q * q * f * (2 * mpmath.diff(g, u, 1) + mpmath.mpf(4) / 3 * u * mpmath.diff(g, u, 2))
        dI = float(mpmath.quad(integrand, [0, kk, 2 * kk, 4 * kk]) / (4 * mpmath.pi ** 2))
        I0 = float(mpmath.quad(lambda q: q * q * cc * kk * kk * _mp_rdot(q * q / (kk * kk)) * g(q * q) ** 3 * 2,
                               [0, kk, 2 * kk, 4 * kk]) / (4 * mpmath.pi ** 2))
    assert abs(dy[0] + I0) / I0 < 1e-12, (dy[0], -I0)
    assert abs(dy[1] + dI) / abs(dI) < 1e-5, (dy[1], -dI)
    # the next grid points still follow the p^2 expansion (p_1 = 2.3e-3 here)
    assert abs(dy[2] + dI) / abs(dI) < 1e-4


def test_d3_feedback_Z_components_at_finite_p_vs_angle_substitution():
    """Z state linear in ln s (reproduced exactly by the lookup), m^2 state,
    exponential regulator: each Z component equals -(I(p_i) - I(0))/p_i^2 with
    I(p) from the substitution s = |q + p| and adaptive quadrature and I(0) a
    radial integral of dR G^3."""
    pytest.importorskip("scipy")
    k, Lam, w, a, b = 1.0, 10.0, 0.3, 1.05, 0.03
    n = 40
    pb = fi.Problem(model=fi.MODEL_D3, n_rad=128, n_ang1=128, n_ext_p=n, regulator=fi.REG_EXP,
                    m2_over_k2=0.0, m2_shift=0.0, qmax_over_k=4.0, n_tables=1, n_pts=n, n_stack=1,
                    include_p0=1, p_min=1e-3, p_max=10.0, x_min=1e-3, x_max=10.0)
    xs = fi.log_grid(n, pb.x_min, pb.x_max)
    y = np.concatenate([[w * k * k], a + b * np.log(xs / pb.x_min)])
    dy = oracle.flow_deriv(pb, fi.constant_tables(pb, [1.0]), 1, Lam, _t_of_k(Lam, k), y)
    Z, m2 = _loglin(pb, a, b), w * k * k

    def G(s):
        return 1.0 / (Z(s) * (s * s + k * k * _r(s * s / (k * k))) + m2)

    def base(q):
        return q * q * Z(q) * k * k * _rdot(q * q / (k * k)) * G(q) ** 2
    qmax = pb.qmax_over_k * k
    I0 = _radial(lambda q: base(q) * 2 * G(q), qmax) / (4 * math.pi ** 2)
    assert abs(dy[0] + I0) / I0 < 1e-9
    for i in (20, 24, 27, 30):
        p = xs[i]
        Ip = _radial(lambda q: base(q) * _ang(q, p, G), qmax) / (4 * math.pi ** 2)
        want = -(Ip - I0) / (p * p)
        assert abs(dy[1 + i] - want) / abs(want) < 3e-6, (i, p, dy[1 + i], want)


# --------------------------------------------------------------------------
# d = 4 feedback: state = the tables (Z, lambda3, lambda4)
# --------------------------------------------------------------------------
def _d4_feedback_problem(n, n_rad, n_ang1, n_ang2, n_ext_ang, M2=1.0):
    return fi.Problem(model=fi.MODEL_D4_VERTEX, n_rad=n_rad, n_ang1=n_ang1, n_ang2=n_ang2, n_ext_p=n,
                      n_ext_ang=n_ext_ang, regulator=fi.REG_EXP, m2_over_k2=0.5, m2_shift=M2,
                      n_tables=3, n_pts=n, n_stack=1, p_min=1e-3, p_max=10.0, x_min=1e-3, x_max=10.0)


def test_d4_feedback_components_at_small_p_vs_p0_limits():
    """Constant tables Z = cz, lambda3 = c3, lambda4 = c4, exponential
    regulator.  At p_0 = 1e-3 (up to O(p_0^2)):
      d_t lambda4 = -(3/2) c4^2 J3,   d_t lambda3 = -3 c3^3 J4  (every psi
      gives the p = 0 value and the weights w_psi/2 sum to 1),
      d_t Z = -c3^2 (1/8pi^2) int q^3 dR G^2 (g' + q^2 g''/2)  (the d = 4
      angle average of c^2 is 1/4; the lambda4 term does not depend on p),
    with J_n = (1/8pi^2) int q^3 dR G^n, all by mpmath."""
    n, k, Lam = 10, 1.0, 10.0
    cz, c3, c4 = 1.15, 0.85, 1.3
    pb = _d4_feedback_problem(n, n_rad=96, n_ang1=16, n_ang2=4, n_ext_ang=3)
    y = np.concatenate([np.full(n, cz), np.full(n, c3), np.full(n, c4)])
    dy = oracle.flow_deriv(pb, y.reshape(3, 1, n), 1, Lam, _t_of_k(Lam, k), y)
    with mpmath.workdps(30):
        kk = mpmath.mpf(k)
        m2 = mpmath.mpf("0.5") * kk * kk + mpmath.mpf(pb.m2_shift)
        czm = mpmath.mpf(cz)

        def g(u):
            return 1 / (czm * (u + kk * kk * _mp_r(u / (kk * kk))) + m2)

        def dR(u):
            return czm * kk * kk * _mp_rdot(u / (kk * kk))
        pts = [0, kk, 2 * kk, 4 * kk]
        nrm = 8 * mpmath.pi ** 2
        J3 = float(mpmath.quad(lambda q: q ** 3 * dR(q * q) * g(q * q) ** 3, pts) / nrm)
        J4 = float(mpmath.quad(lambda q: q ** 3 * dR(q * q) * g(q * q) ** 4, pts) / nrm)
        dz = float(mpmath.quad(lambda q: q ** 3 * dR(q * q) * g(q * q) ** 2
                               * (mpmath.diff(g, q * q, 1) + q * q / 2 * mpmath.diff(g, q * q, 2)), pts) / nrm)
    want_l4 = -1.5 * c4 ** 2 * J3
    want_l3 = -3.0 * c3 ** 3 * J4
    want_z = -c3 ** 2 * dz
    assert abs(dy[2 * n] - want_l4) / abs(want_l4) < 1e-5, (dy[2 * n], want_l4)
    assert abs(dy[n] - want_l3) / abs(want_l3) < 1e-5, (dy[n], want_l3)
    assert abs(dy[0] - want_z) / abs(want_z) < 1e-5, (dy[0], want_z)


def test_d4_feedback_two_point_components_at_finite_p_vs_angle_substitution():
    """Tables linear in ln s: the Z components are -(D2(p_i) - D2(0))/p_i^2 and
    the lambda4 components -Flow4(p_i), with D2 and Flow4 from the angle
    substitution (Gauss-Chebyshev-II weight sqrt(1 - c^2) inside; the second
    angle integrates to 2) and D2(0) a radial integral."""
    pytest.importorskip("scipy")
    n, k, Lam = 40, 1.0, 10.0
    pb = _d4_feedback_problem(n, n_rad=128, n_ang1=128, n_ang2=2, n_ext_ang=2)
    co = [(1.0, 0.03), (1.1, -0.02), (0.8, 0.025)]
    lg = np.log(fi.log_grid(n, pb.x_min, pb.x_max) / pb.x_min)
    y = np.concatenate([a + b * lg for a, b in co])
    dy = oracle.flow_deriv(pb, y.reshape(3, 1, n), 1, Lam, _t_of_k(Lam, k), y)
    Z, l3, l4 = (_loglin(pb, a, b) for a, b in co)
    m2 = pb.m2_over_k2 * k * k + pb.m2_shift

    def G(s):
        return 1.0 / (Z(s) * (s * s + k * k * _r(s * s / (k * k))) + m2)

    def base(q):
        return q ** 3 * Z(q) * k * k * _rdot(q * q / (k * k)) * G(q) ** 2 * 2.0
    norm = 8 * math.pi ** 3
    qmax = pb.qmax_over_k * k
    # p = 0: |q + p| = q, every S0 argument at p = 0; the c1 weight integrates to pi/2
    D0 = _radial(lambda q: base(q) * (math.pi / 2) * (-0.5 * l4(q / math.sqrt(2))
                                                       + l3(q * math.sqrt(2.0 / 3.0)) ** 2 * G(q)), qmax) / norm
    xs = fi.log_grid(n, pb.x_min, pb.x_max)
    for i in (22, 26, 30):
        p = xs[i]
        D2 = _radial(lambda q: base(q) * (-0.5 * l4(math.sqrt((q * q + p * p) / 2)) * math.pi / 2
                                          + _ang(q, p, lambda s: l3(math.sqrt((q * q + s * s + p * p) / 3)) ** 2
                                                 * G(s), gc2=True)), qmax) / norm
        F4 = _radial(lambda q: 1.5 * base(q) * _ang(q, p, lambda s: G(s) * l4(math.sqrt((q * q + s * s + 2 * p * p)
                                                                                       / 4)) ** 2, gc2=True),
                     qmax) / norm
        want_z = -(D2 - D0) / (p * p)
        assert abs(dy[i] - want_z) / abs(want_z) < 1e-7, (i, dy[i], want_z)
        assert abs(dy[2 * n + i] + F4) / abs(F4) < 2e-9, (i, dy[2 * n + i], -F4)


def _rot4(rng):
    m = rng.standard_normal((4, 4))
    qm, r = np.linalg.qr(m)
    return qm * np.sign(np.diag(r))


def test_d4_feedback_lambda3_component_is_the_psi_average_of_explicit_4vector_sums():
    """lambda3 components at finite p: the three-point block written here from
    the model (three vertices at the S0 of their legs, propagators of the two
    shifted lines) and summed over explicit 4-vectors with p1, p2 under a
    random O(4) rotation, for each external angle psi_j (numpy's Gauss-
    Legendre nodes in cos psi), then averaged with numpy's weights / 2."""
    n, k, Lam, npsi = 32, 1.0, 10.0, 3
    pb = _d4_feedback_problem(n, n_rad=24, n_ang1=40, n_ang2=40, n_ext_ang=npsi)
    co = [(1.0, 0.015), (1.2, -0.03), (0.8, 0.02)]
    lg = np.log(fi.log_grid(n, pb.x_min, pb.x_max) / pb.x_min)
    y = np.concatenate([a + b * lg for a, b in co])
    dy = oracle.flow_deriv(pb, y.reshape(3, 1, n), 1, Lam, _t_of_k(Lam, k), y)

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
    xr, wr = np.polynomial.legendre.leggauss(pb.n_rad)
    xr, wr = (xr + 1) * 0.5 * pb.qmax_over_k * k, wr * 0.5 * pb.qmax_over_k * k
    j1 = np.arange(1, 41)
    x1 = np.cos(j1 * np.pi / 41)
    w1 = np.pi / 41 * np.sin(j1 * np.pi / 41) ** 2
    x2, w2 = np.polynomial.legendre.leggauss(40)
    nphi = 40
    ph = 2 * np.pi * np.arange(nphi) / nphi
    cpsi, wpsi = np.polynomial.legendre.leggauss(npsi)
    Q, C1, C2, PH = np.meshgrid(xr, x1, x2, ph, indexing="ij")
    S1, S2 = np.sqrt(1 - C1 ** 2), np.sqrt(1 - C2 ** 2)
    qv = np.stack([Q * C1, Q * S1 * C2, Q * S1 * S2 * np.cos(PH), Q * S1 * S2 * np.sin(PH)], -1)
    W = (wr[:, None, None, None] * w1[None, :, None, None] * w2[None, None, :, None]
         * (2 * np.pi / nphi) * Q ** 3) / (2 * np.pi) ** 4
    q2 = Q ** 2
    base = 3 * look(0, Q) * k * k * rdot(q2 / (k * k)) * G(q2) ** 2
    rng = np.random.default_rng(17)
    xs = fi.log_grid(n, pb.x_min, pb.x_max)
    for i in (19, 25):
        p = xs[i]
        avg = 0.0
        for j in range(npsi):
            Rm = _rot4(rng)
            p1 = Rm @ np.array([p, 0, 0, 0])
            p2 = Rm @ np.array([p * cpsi[j], p * math.sqrt(1 - cpsi[j] ** 2), 0, 0])
            A2 = np.sum((qv + p1) ** 2, -1)
            B2 = np.sum((qv - p2) ** 2, -1)
            Cc = float(np.sum((p1 + p2) ** 2))
            f = (base * G(A2) * G(B2) * look(1, np.sqrt((q2 + A2 + p * p) / 3))
                 * look(1, np.sqrt((q2 + B2 + p * p) / 3)) * look(1, np.sqrt((A2 + B2 + Cc) / 3)))
            avg += 0.5 * wpsi[j] * float(np.sum(W * f))
        assert abs(dy[n + i] + avg) / abs(avg) < 2e-8, (i, dy[n + i], -avg)


def test_d4_state_jacobian_columns_vs_central_differences_of_the_flow_derivative():
    """The implicit stepper's state Jacobian d(d_t y)/dy (the raw Jacobian under
    the feedback map) against central differences of the flow derivative pinned
    above: individual columns from each table and a random direction.  The grid
    starts at 0.05: the Z rows divide a difference by p_i^2, which at 1e-3
    would lift rounding noise above the differences' truncation error."""
    wl = fi.make_d4(seed=31, n_pts=8, n_ext_ang=3, n_rad=24, n_ang1=12, n_ang2=4)
    pb = wl.problem
    pb.p_min = pb.x_min = 0.05
    Lam, t = wl.Lambda, 1.3
    y = wl.y0.copy()
    J = oracle.d4_state_jacobian(pb, Lam, t, y)
    ny = y.size
    assert J.shape == (ny, ny)

    def fd(v, h):
        return (oracle.flow_deriv(pb, wl.tables, 1, Lam, t, y + h * v)
                - oracle.flow_deriv(pb, wl.tables, 1, Lam, t, y - h * v)) / (2 * h)
    rows = np.max(np.abs(J), axis=1)        # each row on its own scale (the Z rows carry 1/p_i^2)
    for j in range(ny):
        e = np.zeros(ny)
        e[j] = 1.0
        assert np.max(np.abs(J[:, j] - fd(e, 1e-4)) / rows) < 1e-6, j
    v = np.random.default_rng(3).standard_normal(ny)
    assert np.max(np.abs(J @ v - fd(v, 1e-4)) / rows) < 1e-6
