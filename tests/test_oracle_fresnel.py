"""Pins of the oracle's reflection at a dielectric face (Fresnel coefficients,
the dielectric (Fresnel) walls of the paper's rooms, Sec. IV) against
textbook forms that share no arithmetic with it:

* Fresnel's angle forms for a real permittivity, with Snell's law
  sin(t) = sin(i) / sqrt(eps):
      G_perp = -sin(i - t) / sin(i + t),   G_par = tan(i - t) / tan(i + t)
  (the basis in which a PEC face gives -1 / +1);
* normal incidence: G_perp = (1 - sqrt(eps)) / (1 + sqrt(eps)) for any eps;
* Brewster's angle tan(i) = sqrt(eps): no parallel reflection;
* grazing incidence: both coefficients -> -1;
* a passive medium reflects at most what arrives (|G| <= 1);
* eps -> infinity: the PEC image mirror.
"""
import numpy as np
import pytest

from oracle import oracle


def _basis(i_deg, n=np.array([0.0, 0.0, 1.0])):
    """Incidence i from the normal, in the x-z plane: si, sr, e_perp, e_par_i, e_par_r."""
    i = np.radians(i_deg)
    si = np.array([np.sin(i), 0.0, -np.cos(i)])
    sr = si - 2 * np.dot(si, n) * n
    ep = np.cross(n, si)
    ep /= np.linalg.norm(ep)
    return si, sr, ep, np.cross(ep, si), np.cross(ep, sr)


def _coeffs(i_deg, eps):
    n = np.array([0.0, 0.0, 1.0])
    si, sr, ep, epi, epr = _basis(i_deg, n)
    gs = oracle.reflect(n, si, sr, ep.astype(complex), eps)
    gp = oracle.reflect(n, si, sr, epi.astype(complex), eps)
    # the reflected perpendicular part stays along e_perp, the parallel along e_par_r
    assert np.allclose(np.cross(gs, ep), 0, atol=1e-14) and np.allclose(np.cross(gp, epr), 0, atol=1e-14)
    return np.dot(gs, ep), np.dot(gp, epr)


@pytest.mark.parametrize("eps", [2.0, 5.3, 81.0])
def test_fresnel_angle_forms(eps):
    for i_deg in (5.0, 20.0, 45.0, 60.0, 80.0, 89.0):
        i = np.radians(i_deg)
        t = np.arcsin(np.sin(i) / np.sqrt(eps))
        gs, gp = _coeffs(i_deg, (eps, 0.0))
        assert abs(gs - (-np.sin(i - t) / np.sin(i + t))) < 1e-12
        assert abs(gp - np.tan(i - t) / np.tan(i + t)) < 1e-12


def test_normal_incidence_brewster_grazing():
    for eps in [(4.0, 0.0), (5.3, 0.4), (12.0, 3.0)]:
        e = eps[0] - 1j * eps[1]
        n = np.array([0.0, 0.0, 1.0])
        E = np.array([0.3 + 0.1j, -0.7, 0.0])
        r = oracle.reflect(n, -n, n, E, eps)
        assert np.allclose(r, E * (1 - np.sqrt(e)) / (1 + np.sqrt(e)), atol=1e-14)
        gs, gp = _coeffs(89.9999, eps)
        assert abs(gs + 1) < 1e-4 and abs(gp + 1) < 1e-4
    for eps in (2.5, 9.0):
        _, gp = _coeffs(np.degrees(np.arctan(np.sqrt(eps))), (eps, 0.0))
        assert abs(gp) < 1e-12


def test_passive_and_pec_limit():
    rng = np.random.default_rng(3)
    for _ in range(20):
        eps = (rng.uniform(1.5, 30), rng.uniform(0, 5))
        gs, gp = _coeffs(rng.uniform(0, 89.9), eps)
        assert abs(gs) <= 1 + 1e-12 and abs(gp) <= 1 + 1e-12
    for _ in range(10):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        si = rng.standard_normal(3)
        si /= np.linalg.norm(si)
        if np.dot(si, n) > 0:
            si = -si
        sr = si - 2 * np.dot(si, n) * n
        E = rng.standard_normal(3) + 1j * rng.standard_normal(3)
        E -= np.dot(E, si) * si
        pec = oracle.reflect(n, si, sr, E)
        assert np.allclose(pec, -E + 2 * np.dot(n, E) * n, atol=1e-14)
        assert np.allclose(oracle.reflect(n, si, sr, E, (1e14, 0.0)), pec, atol=1e-6)
