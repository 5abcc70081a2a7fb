"""Pins of the oracle's finite-T sums over many loop-side states (no GPU).

The finite-T RHS factorises into a loop-side factor F(n, q) = dR G^2 L at
(loop frequency, radial node) and the shifted line L G at (n + m, |q + p|)
whose angle integral is the kernel K(p, q) of Sec. 5.3.2.  orc_ft_states
sums any number of states F_s against the same shifted line, by the plain
definition.  Pins: with the model's own loop factor it is the (pinned) RHS;
it is linear in F; with the flat regulator and constant tables at p -> 0 it
reduces to a closed form that fixes the frequency of the shifted line, the
radial and angle weights and the normalisation.
"""
import math

import numpy as np
import pytest

import ffrg_inputs as fi
import oracle


@pytest.mark.parametrize("fermionic", [False, True])
def test_model_loop_factor_gives_the_rhs(fermionic):
    wl = fi.make_finite_t(seed=91, N=3, T=0.05, n_pts=16, n_ext_p=5, n_ext_m=4, n_rad=14, n_ang=9,
                          fermionic=fermionic)
    pb = wl.problem
    for k in (1.3, 0.2):
        F = oracle.ft_loop_factors(pb, wl.tables, k)
        assert F.shape == (oracle.ft_nfreq(pb), pb.n_rad)
        got = oracle.ft_states(pb, wl.tables, k, F[None])[0]
        ref = oracle.rhs(pb, wl.tables, k)
        assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-13


def test_states_are_linear_in_the_loop_factor():
    wl = fi.make_finite_t(seed=92, N=2, T=0.1, n_pts=12, n_ext_p=4, n_ext_m=3, n_rad=10, n_ang=6)
    pb = wl.problem
    rng = np.random.default_rng(4)
    F = rng.normal(size=(3, oracle.ft_nfreq(pb), pb.n_rad))
    out = oracle.ft_states(pb, wl.tables, 0.7, F)
    comb = oracle.ft_states(pb, wl.tables, 0.7, (0.3 * F[0] - 1.7 * F[1] + F[2])[None])[0]
    want = 0.3 * out[0] - 1.7 * out[1] + out[2]
    assert np.max(np.abs(comb - want)) / np.max(np.abs(want)) < 1e-13


@pytest.mark.parametrize("fermionic", [False, True])
def test_flat_regulator_indicator_states_closed_form(fermionic):
    """Flat regulator, Z = L = 1, p -> 0, radial rule on [0, k]: the shifted
    line is 1/(k^2 (1 + w) + omega_{n+m}^2) for q < k and the angle weights sum
    to 2.  A state equal to q_i^2 at loop frequency row n0 (zero elsewhere)
    gives pref T/(4 pi^2) 2 (k^5/5) / (k^2 (1 + w) + omega_{n0+m}^2), with
    omega_n = 2 pi T n (bosonic) or (2n+1) pi T (fermionic)."""
    k, w, T, N, M = 1.1, 0.4, 0.2, 3, 3
    nst = N + M + 1
    pb = fi.Problem(model=fi.MODEL_FINITE_T, n_rad=6, n_ang1=3, n_ext_p=1, n_ext_ang=M, n_matsubara=N,
                    regulator=fi.REG_LITIM, m2_over_k2=w, T=T, qmax_over_k=1.0, n_tables=2, n_pts=8,
                    n_stack=nst, p_min=1e-200, p_max=1e-200, prefactor=1.7,
                    statistics=fi.STAT_FERMI if fermionic else fi.STAT_BOSE)
    tabs = fi.constant_tables(pb, [1.0, 1.0])
    xr, _ = np.polynomial.legendre.leggauss(pb.n_rad)
    q = (xr + 1) * 0.5 * k
    nfreq = oracle.ft_nfreq(pb)
    n_lo = -N - 1 if fermionic else -N
    F = np.zeros((nfreq, nfreq, pb.n_rad))
    for r in range(nfreq):
        F[r, r] = q ** 2
    out = oracle.ft_states(pb, tabs, k, F)

    def omega(n):
        return (2 * n + 1) * math.pi * T if fermionic else 2 * math.pi * T * n
    for r in range(nfreq):
        n0 = r + n_lo
        for m in range(M):
            want = 1.7 * T / (4 * math.pi ** 2) * 2 * k ** 5 / 5 / (k * k * (1 + w) + omega(n0 + m) ** 2)
            assert abs(out[r, m] - want) / want < 1e-13, (r, m)
