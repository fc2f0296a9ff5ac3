"""Pins of the oracle's Fock--Pekeris functions and transition function.

Checked against: the residue (creeping-mode) series, which is the closed form of
the same integral for xi > 0; continuity of the regular part across the two
contour families; the geometrical-optics limit R -> -1 (soft) / +1 (hard) of
the lit-region reflection coefficient; the Fresnel-integral definition of F(X)
(scipy) and its small- and large-X limits.  The UTD functions are those of the
references the paper cites for R and T (Sec. II.B, after Eq. 4)."""
import numpy as np
import pytest
from scipy.special import fresnel, wofz

from oracle import fock

C = fock.C_SING


def _phat_rule(xi, hard, bucket):
    tau, Ws, Wh = fock.contour_rule(bucket)
    W = Wh if hard else Ws
    return np.exp(-1j * np.pi / 4) / np.sqrt(np.pi) * np.sum(W * np.exp(-1j * xi * tau))


@pytest.mark.parametrize("hard", [False, True])
@pytest.mark.parametrize("xi", [0.8, 1.0, 1.25, 1.5])
def test_quadrature_matches_residue_series(xi, hard):
    q = fock.phat(xi, hard) - C / xi
    r = fock.P_residue(xi, hard)
    assert abs(q - r) <= 2e-10 * max(1.0, abs(r))


@pytest.mark.parametrize("hard", [False, True])
def test_regular_part_continuous_at_zero(hard):
    # xi = 0 through the negative-xi contour (bucket 1) and the positive one (bucket 0)
    a = _phat_rule(0.0, hard, 1)
    b = _phat_rule(0.0, hard, 0)
    assert abs(a - b) < 1e-12
    # and phat is smooth through 0: symmetric difference quotient finite and small
    h = 1e-4
    d = (fock.phat(h, hard) - fock.phat(-h, hard)) / (2 * h)
    assert np.isfinite(d) and abs(d) < 5.0


@pytest.mark.parametrize("hard", [False, True])
@pytest.mark.parametrize("n", range(1, 10))
def test_adjacent_buckets_agree(n, hard):
    xi = -float(n)
    assert abs(_phat_rule(xi, hard, n) - _phat_rule(xi, hard, n + 1)) < 1e-11


@pytest.mark.parametrize("xi", [-4.0, -6.0, -8.0, -10.0])
def test_go_limit_of_reflection_coefficient(xi):
    # R = -sqrt(-4/xi) e^{-j xi^3/12} P(xi) -> -1 (soft), +1 (hard) with an |xi|^-3 residual
    for hard, go in ((False, -1.0), (True, 1.0)):
        R = -np.sqrt(-4 / xi) * np.exp(-1j * xi ** 3 / 12) * fock.P(xi, hard)
        assert abs(R - go) <= 2.5 / abs(xi) ** 3
        assert abs(R - go) >= 0.5 / abs(xi) ** 3      # the residual is real, not rounding


def test_go_residual_decays_like_inverse_cube():
    r = []
    for xi in (-5.0, -10.0):
        R = -np.sqrt(-4 / xi) * np.exp(-1j * xi ** 3 / 12) * fock.P(xi, False)
        r.append(abs(R + 1.0))
    assert 6.0 < r[0] / r[1] < 10.0                   # (10/5)^3 = 8


def test_singular_parts_equal():
    # P_s - P_h is regular at 0 (both singular parts are -c/xi)
    for xi in (1e-3, -1e-3):
        d = fock.P(xi, False) - fock.P(xi, True)
        assert abs(d) < 1.0


def _F_fresnel(X):
    # F(X) = 2j sqrt(X) e^{jX} Int_{sqrt X}^inf e^{-j t^2} dt, Int_0^a e^{-jt^2} = sqrt(pi/2)(C - jS)(a sqrt(2/pi))
    a = np.sqrt(X)
    S, Cc = fresnel(a * np.sqrt(2 / np.pi))
    tail = np.sqrt(np.pi / 2) * ((0.5 - Cc) - 1j * (0.5 - S))
    return 2j * np.sqrt(X) * np.exp(1j * X) * tail


def test_transition_function_matches_fresnel_definition(oracle_mod):
    X = np.logspace(-6, 3, 80)
    F = oracle_mod.transition_F(X)
    ref = _F_fresnel(X)
    assert np.max(np.abs(F - ref) / np.abs(ref)) < 1e-9
    # and the Faddeeva form used by the CUDA side's derivation
    w = np.sqrt(np.pi * X) * np.exp(1j * np.pi / 4) * wofz(np.exp(3j * np.pi / 4) * np.sqrt(X))
    assert np.max(np.abs(F - w) / np.abs(w)) < 1e-9


def test_transition_function_limits(oracle_mod):
    Xs = np.array([1e-6])
    F = oracle_mod.transition_F(Xs)[0]
    assert abs(F / (np.sqrt(np.pi * Xs[0]) * np.exp(1j * np.pi / 4)) - 1) < 1e-2
    X = 200.0
    F = oracle_mod.transition_F([X])[0]
    assert abs(F - (1 + 1j / (2 * X) - 3 / (4 * X * X))) < 1e-6


def test_c_bracket_matches_python(oracle_mod):
    rng = np.random.default_rng(5)
    xi = np.concatenate([rng.uniform(-10, 8, 40), [1e-3, -1e-3, 1.5, 1.5000001, -10.0]])
    K = rng.uniform(0.2, 6.0, xi.size)
    Bs, Bh = oracle_mod.fock_bracket(xi, K)
    for i in range(xi.size):
        X = (K[i] * xi[i]) ** 2
        Fx = np.sqrt(np.pi * X) * np.exp(1j * np.pi / 4) * wofz(np.exp(3j * np.pi / 4) * np.sqrt(X))
        ps = fock.phat_any(xi[i], False)
        ph = fock.phat_any(xi[i], True)
        es = ps - C * Fx / xi[i]
        eh = ph - C * Fx / xi[i]
        assert abs(Bs[i] - es) < 1e-9 * max(1, abs(es)), (xi[i], Bs[i], es)
        assert abs(Bh[i] - eh) < 1e-9 * max(1, abs(eh)), (xi[i], Bh[i], eh)


def test_residue_series_converged():
    for xi in (1.5, 3.0):
        for hard in (False, True):
            a = fock.P_residue(xi, hard, 20)
            b = fock.P_residue(xi, hard, 40)
            assert abs(a - b) < 1e-12 * max(1, abs(b))
