"""The oracle's Fock--Pekeris functions against an independent high-precision
evaluation (mpmath), over the whole table domain xi in [-10, 1.5].

tests/golden/pekeris_mp.txt holds phat_s, phat_h (the regular parts
P + c/xi that the reflection and transfer coefficients after Eq. 4 use) at
51 points, written by tests/golden/make_pekeris_mp.py from the integral
definition on contours, quadrature and Airy functions other than the
oracle's.  The oracle must agree to 1e-10 everywhere, including the range
xi < 0 where its own contour quadrature is pinned otherwise only by
continuity and the GO limit.  The fixture itself is checked against a fresh
mpmath evaluation at other settings (when mpmath is present), against the
residue series at the top of the domain, and two plausible mistakes planted
in the oracle's quadrature (a contour family used outside its range, a
conjugated prefactor) are shown to fail the comparison.
"""
import os

import numpy as np
import pytest

from oracle import fock

HERE = os.path.dirname(os.path.abspath(__file__))
FIXTURE = os.path.join(HERE, "golden", "pekeris_mp.txt")
TOL = 1e-10


def _fixture():
    a = np.loadtxt(FIXTURE)
    return a[:, 0], a[:, 1] + 1j * a[:, 2], a[:, 3] + 1j * a[:, 4]


def test_fixture_covers_the_table_domain():
    xi, s, h = _fixture()
    assert len(xi) >= 50 and xi.min() == fock.XI_LO and xi.max() == fock.XI_HI
    assert np.all(np.isfinite(s)) and np.all(np.isfinite(h))


def test_oracle_phat_matches_mpmath():
    xi, s, h = _fixture()
    es = np.array([abs(fock.phat_any(x, False) - v) for x, v in zip(xi, s)])
    eh = np.array([abs(fock.phat_any(x, True) - v) for x, v in zip(xi, h)])
    assert es.max() < TOL, (xi[np.argmax(es)], es.max())
    assert eh.max() < TOL, (xi[np.argmax(eh)], eh.max())


def test_fixture_against_fresh_mpmath():
    mp = pytest.importorskip("mpmath")
    import sys
    sys.path.insert(0, os.path.join(HERE, "golden"))
    import make_pekeris_mp as gen
    xi, s, h = _fixture()
    for k in (2, 40):                                 # xi = -9.5 and 0.5
        assert abs(gen.phat_mp(xi[k], False, dps=24) - s[k]) < 1e-12
        assert abs(gen.phat_mp(xi[k], True, dps=24) - h[k]) < 1e-12
    assert mp is not None


def test_fixture_meets_the_residue_series():
    """At the top of the domain the fixture equals the creeping-wave mode
    (residue) series, summed here from scipy's Airy zeros."""
    from scipy.special import ai_zeros
    a, ap, ai, aip = ai_zeros(60)
    al, be = -a, -ap
    xi, s, h = _fixture()
    e = np.exp(-1j * np.pi / 3)
    pref = -np.exp(-1j * np.pi / 12) / (2 * np.sqrt(np.pi))
    c = np.exp(-1j * np.pi / 4) / (2 * np.sqrt(np.pi))
    for k in np.nonzero(xi >= 1.2)[0]:
        ps = pref * np.sum(np.exp(-1j * xi[k] * al * e) / aip ** 2) + c / xi[k]
        ph = pref * np.sum(np.exp(-1j * xi[k] * be * e) / (be * ai ** 2)) + c / xi[k]
        assert abs(ps - s[k]) < 1e-8 and abs(ph - h[k]) < 1e-8


def _planted(xi, hard, rule_bucket=None, conj_pref=False):
    """The oracle's quadrature with a mistake planted: the contour rule of
    another bucket, or the conjugate prefactor e^{+j pi/4}."""
    b = fock.bucket_of(xi) if rule_bucket is None else rule_bucket
    tau, ws, wh = fock.contour_rule(b)
    pref = np.conj(fock._PREF) if conj_pref else fock._PREF
    return complex(pref * np.sum((wh if hard else ws) * np.exp(-1j * xi * tau)))


def test_planted_mistakes_fail_the_pin():
    xi, s, h = _fixture()
    neg = np.nonzero(xi <= -4.0)[0]
    # the xi >= 0 contour (the ray into the lower half plane) used for xi < 0:
    # the integrand grows there and the quadrature loses the result
    worst = max(abs(_planted(xi[k], False, rule_bucket=0) - s[k]) for k in neg)
    assert worst > 1e-3
    # a conjugated prefactor
    worst = max(abs(_planted(xi[k], True, conj_pref=True) - h[k]) for k in neg)
    assert worst > 1e-3
    # and the unplanted rule passes on the same points
    assert max(abs(_planted(xi[k], False) - s[k]) for k in neg) < TOL
