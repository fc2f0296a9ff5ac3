"""The oracle against exact solutions (the paper's own sphere check is against
the analytical solution, Sec. IV.A, Fig. 10).

* 2-D PEC cylinder, line source: the UTD field built from the oracle's Fock
  bracket (lit: direct + Fock reflection + encircling ray; shadow: two
  creeping rays) vs the Hankel-series solution.
* PEC sphere, a = 0.5 m, source at 3 m, ring of radius 2 m, 2.4 GHz (ka = 25):
  - z-polarised source: E_z vs the scalar Dirichlet series (soft creeping) and
    vs the vector Mie series of a z-directed electric dipole;
  - y-polarised source: |E| vs the vector Mie series of a z-directed magnetic
    dipole (in-plane E, hard creeping; same directions and magnitudes on every
    ray that reaches the ring).
  Shadow receivers near the back axis sit in the axial caustic of the creeping
  rays, where the two-ray field does not hold; the comparisons use the
  receivers at least 2, 3 and 6 wavelengths off that axis respectively (see
  the tolerance notes below).
"""
import numpy as np
import pytest

import exact_series as X
from oracle import fock
from paper_2310_10578_gb300 import scenes

K24 = 2 * np.pi * 2.4e9 / 299792458.0


def _alhazen2d(a, S, P):
    from scipy.optimize import brentq
    phi = np.arctan2(P[1], P[0])

    def L(psi):
        Q = a * np.array([np.cos(psi), np.sin(psi)])
        return np.linalg.norm(S - Q) + np.linalg.norm(P - Q)
    psi = brentq(lambda p: (L(p + 1e-7) - L(p - 1e-7)) / 2e-7, 1e-9, phi - 1e-9)
    return a * np.array([np.cos(psi), np.sin(psi)])


def utd2d(oracle_mod, k, a, rs, rr, phi, hard):
    """2-D UTD (line source, cylindrical incident wave) using the oracle's Fock bracket."""
    C0 = np.sqrt(2 / (np.pi * k)) * np.exp(1j * np.pi / 4)     # H0^(2)(kr) ~ C0 e^{-jkr}/sqrt(r)
    bs, bp = np.arccos(a / rs), np.arccos(a / rr)
    sp, s = np.sqrt(rs ** 2 - a ** 2), np.sqrt(rr ** 2 - a ** 2)
    m = (k * a / 2) ** (1 / 3)
    tot = 0
    for g in (phi, 2 * np.pi - phi):
        t = a * (g - bs - bp)
        if t <= 0:
            continue
        xi = m * t / a
        L = sp * s / (sp + s)
        Bs, Bh = oracle_mod.fock_bracket([xi], [np.sqrt(k * L / (2 * m * m))])
        B = (Bh if hard else Bs)[0]
        T = -m * np.sqrt(2 / k) * B * np.exp(-1j * k * t)
        tot += C0 * np.exp(-1j * k * sp) / np.sqrt(sp) * T / np.sqrt(s) * np.exp(-1j * k * s)
    if phi < bs + bp:
        S = np.array([rs, 0.0]); P = rr * np.array([np.cos(phi), np.sin(phi)])
        d = np.linalg.norm(P - S)
        tot += C0 * np.exp(-1j * k * d) / np.sqrt(d)
        Q = _alhazen2d(a, S, P)
        n = Q / a
        si, sr = np.linalg.norm(Q - S), np.linalg.norm(P - Q)
        cth = (S - Q) @ n / si
        xi = -2 * m * cth
        L = si * sr / (si + sr)
        Bs, Bh = oracle_mod.fock_bracket([xi], [np.sqrt(k * L / (2 * m * m))])
        B = (Bh if hard else Bs)[0]
        R = -np.sqrt(-4 / xi) * np.exp(-1j * xi ** 3 / 12) * B if xi >= fock.XI_LO else (1 if hard else -1)
        rho = 1 / (1 / si + 2 / (a * cth))
        tot += C0 * np.exp(-1j * k * si) / np.sqrt(si) * R * np.sqrt(rho / (rho + sr)) * np.exp(-1j * k * sr)
    return tot


@pytest.mark.parametrize("hard", [False, True])
def test_cylinder_2d_vs_hankel_series(oracle_mod, hard):
    a, rs, rr = 0.5, 3.0, 2.0
    sb = np.degrees(np.arccos(a / rs) + np.arccos(a / rr))
    lit = [30, 60, 100, 130, 150, 154, 155.5, 155.9]
    shadow = [155.95, 156.3, 158, 160, 165, 170, 175, 180]
    for deg in lit + shadow:
        phi = np.radians(deg)
        ex = X.cyl2d_total(K24, a, rs, rr, phi, hard)
        u = utd2d(oracle_mod, K24, a, rs, rr, phi, hard)
        ddb = abs(20 * np.log10(abs(u) / abs(ex)))
        dph = abs(np.angle(u / ex))
        if deg < sb:
            assert ddb < 0.1 and dph < 0.02, (deg, ddb, dph)
        else:
            assert ddb < 0.45 and dph < 0.04, (deg, ddb, dph)


@pytest.fixture(scope="module")
def ring_runs(oracle_mod):
    out = {}
    for pol in ("z", "y"):
        sc = scenes.sphere_ring(n_rx=4096, pol=(0, 0, 1.0) if pol == "z" else (0, 1.0, 0))
        out[pol] = (sc, oracle_mod.evaluate(sc, want_paths=False))
    return out


def _angles(sc):
    return np.degrees(np.arctan2(np.abs(sc.rx[:, 1].astype(np.float64)), sc.rx[:, 0].astype(np.float64)))


SB_DEG = np.degrees(np.arccos(0.5 / 3.0) + np.arccos(0.5 / 2.0))


def _kdperp(sc):
    return K24 * np.abs(sc.rx[:, 1].astype(np.float64))      # distance from the x axis (S-c axis)


def test_sphere_soft_vs_scalar_dirichlet(ring_runs):
    sc, r = ring_runs["z"]
    ang = _angles(sc)
    sel = np.where((ang > SB_DEG + 0.3) & (_kdperp(sc) >= 4 * np.pi))[0]
    assert len(sel) > 100
    sel = sel[::3]
    ex = np.array([X.sphere_scalar_total(K24, 0.5, 3.0, 2.0, np.radians(ang[i]), False) for i in sel])
    d = 20 * np.log10(np.abs(r.E[0, 2, sel]) / np.abs(ex))
    assert np.max(np.abs(d)) < 1.0, np.max(np.abs(d))
    lit = np.where(ang < SB_DEG - 2)[0][::16]
    ex = np.array([X.sphere_scalar_total(K24, 0.5, 3.0, 2.0, np.radians(ang[i]), False) for i in lit])
    d = 20 * np.log10(np.abs(r.E[0, 2, lit]) / np.abs(ex))
    assert np.max(np.abs(d)) < 0.4


@pytest.mark.parametrize("pol", ["z", "y"])
def test_sphere_vs_vector_mie(ring_runs, pol):
    sc, r = ring_runs[pol]
    M = X.MieDipole(K24, 0.5, 3.0, magnetic=(pol == "y"))
    ang = _angles(sc)
    kd = _kdperp(sc)
    pts = sc.rx.astype(np.float64)
    amp_o = np.linalg.norm(r.E[0], axis=0)
    lit = np.where(ang < SB_DEG - 1.0)[0]
    lit = lit[(ang[lit] > 1.0)][::4]
    em = np.linalg.norm(M.total(pts[lit]), axis=1)
    d = 20 * np.log10(amp_o[lit] / em)
    # deep lit region: GO + Fock reflection; the shadow-boundary transition zone
    # (within ~10 deg of the SB at ka = 25) carries the UTD's O(1) dB error
    assert np.max(np.abs(d[ang[lit] < 120])) < 0.12, np.max(np.abs(d[ang[lit] < 120]))
    assert np.max(np.abs(d)) < 1.0, np.max(np.abs(d))
    # shadow, outside the axial caustic zone of the creeping rays
    zone = 6 * np.pi if pol == "y" else 12 * np.pi
    sh = np.where((ang > SB_DEG + 0.3) & (kd >= zone))[0]
    assert len(sh) > 20
    em = np.linalg.norm(M.total(pts[sh]), axis=1)
    d = 20 * np.log10(amp_o[sh] / em)
    assert np.max(np.abs(d)) < (1.0 if pol == "y" else 1.1), np.max(np.abs(d))
