"""Pins of the adjoint tests' reference (tests/adjoint_ref.py) on the CPU.

With no bodies and no walls only the direct ray exists, so the per-path
central differences must equal the central differences of the oracle's
total field, and both the closed-form derivative of E = e(d) e^{-jkR} / R
(Eq. 1) with respect to the transmitter and the frequency.
"""
import numpy as np

import adjoint_ref
from oracle import oracle
from paper_2310_10578_gb300 import scenes

C0 = 299792458.0


def _free_space():
    rng = np.random.default_rng(5)
    rx = rng.uniform(-3, 3, (40, 3))
    return scenes.Scene(np.zeros((0, 3, 3)), np.zeros(0), np.zeros((0, 6)), (0.3, -0.2, 0.5), (0.2, 0.1, 1.0),
                        [2.4e9, 5.8e9], rx, "free space", max_order=0)


def _los(S, P, pol, f):
    """Closed form of the direct field (complex [3])."""
    d = P - S
    R = np.linalg.norm(d)
    u = d / R
    e = pol - np.dot(pol, u) * u
    e = e / np.linalg.norm(e)
    k = 2 * np.pi * f / C0
    return e * np.exp(-1j * k * R) / R


def test_reference_vjp_direct_ray_closed_form():
    sc = _free_space()
    r = oracle.evaluate(sc)
    lists = [list(p) for p in r.paths]
    assert all(len(p) == 1 for p in lists)
    rng = np.random.default_rng(6)
    g = rng.standard_normal((2, 3, sc.n_rx)) + 1j * rng.standard_normal((2, 3, sc.n_rx))
    ref = adjoint_ref.vjp(sc, lists, g, bodies=())
    S0 = sc.tx.astype(np.float64)
    pol = sc.pol.astype(np.float64)
    P = sc.rx.astype(np.float64)

    def vjp_closed(dS=np.zeros(3), dfreq=np.zeros(2), h=1e-6, hf=10.0):
        # derivative of the closed form by central differences at steps other
        # than the reference's (1e-6 m; 10 Hz, a phase step of ~1e-6 rad)
        tot = 0.0
        for i in range(sc.n_rx):
            for fi, f in enumerate(sc.freqs):
                ep = _los(S0 + h * dS, P[i], pol, f + hf * dfreq[fi])
                em = _los(S0 - h * dS, P[i], pol, f - hf * dfreq[fi])
                dE = (ep - em) / (2 * (h if np.any(dS) else hf))
                tot += np.sum(g[fi, :, i].real * dE.real + g[fi, :, i].imag * dE.imag)
        return tot

    for k in range(3):
        e = np.zeros(3)
        e[k] = 1.0
        want = vjp_closed(dS=e)
        assert abs(ref["tx"][k] - want) <= 1e-6 * ref["tx_abs"][k], (k, ref["tx"][k], want)
    for k in range(2):
        e = np.zeros(2)
        e[k] = 1.0
        want = vjp_closed(dfreq=e)
        assert abs(ref["f"][k] - want) <= 1e-6 * ref["f_abs"][k], (k, ref["f"][k], want)


def test_per_path_fields_sum_to_the_field():
    sc = scenes.room(n_cyl=6, nx=7, ny=5, seed=12)
    r = oracle.evaluate(sc, path_fields=True, cap=64)
    tot = np.transpose(r.path_E.sum(axis=1), (1, 2, 0))
    assert np.max(np.abs(tot - r.E)) <= 1e-12 * np.max(np.abs(r.E))
