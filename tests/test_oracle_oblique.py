"""The oracle on a PEC circular cylinder at oblique 3-D incidence against the
exact eigenfunction series.

A plane wave whose direction makes the angle beta with the cylinder's axis
splits into two decoupled scalar problems in the transverse plane, with the
transverse wavenumber k_t = k sin(beta): E_z obeys the Dirichlet condition
(TM, the z-polarised source: incident E along (-cos b, 0, sin b), H along y)
and H_z the Neumann condition (TE, the y-polarised source).  For a wave
arriving from +x,

    u(rho, phi, z) = u_0 e^{j k cos(b) z} sum_n j^n [J_n(k_t rho) - c_n H2_n(k_t rho)] e^{j n phi},
    c_n = J_n(k_t a) / H2_n(k_t a) (TM),  J_n'(k_t a) / H2_n'(k_t a) (TE).

The oracle's scene: the tall cylinder (1 km, centred on the receivers'
plane) and the source 10 km away in the incident direction, so that the
wave is plane to within 1e-2 rad over the receivers; its E_z is compared for
TM, and for TE its H_z = sum over paths of (s x E_path)_z / eta, s each
path's arrival direction (eta cancels against the series' normalisation).
The lit side (direct ray plus the Fock-uniform reflection, R after Eq. 4,
with the oblique plane of incidence's surface radius) and the shadow
(helical creeping rays, Eq. 4) at two oblique angles: the parts that the 2-D
series at normal incidence cannot reach.
"""
import numpy as np
import pytest
from scipy.special import h2vp, hankel2, jv, jvp

from paper_2310_10578_gb300 import scenes

C0 = 299792458.0
F = 2.4e9
K = 2 * np.pi * F / C0
A, RHO, D = 0.5, 2.0, 1e4
LIT = np.array([0.0, 30.0, 60.0, 90.0, 120.0, 150.0, 160.0, 164.0])
SHADOW = np.array([167.0, 170.0, 175.0, 180.0])       # shadow boundary at 180 - asin(a / rho) = 165.5 deg


def _series(beta, phi, hard):
    kt = K * np.sin(beta)
    n = np.arange(-int(kt * RHO + 40), int(kt * RHO + 40) + 1)
    c = jvp(n, kt * A) / h2vp(n, kt * A) if hard else jv(n, kt * A) / hankel2(n, kt * A)
    terms = (1j ** n)[:, None] * (jv(n, kt * RHO)[:, None] - c[:, None] * hankel2(n, kt * RHO)[:, None])
    u0 = (-1.0 if hard else 1.0) * np.sin(beta) * np.exp(-1j * K * D) / D
    return u0 * np.sum(terms * np.exp(1j * np.outer(n, phi)), axis=0)


def _oracle(oracle_mod, beta, phi, hard):
    rx = np.stack([RHO * np.cos(phi), RHO * np.sin(phi), np.zeros_like(phi)], axis=1)
    tx = D * np.array([np.sin(beta), 0.0, np.cos(beta)])
    body = np.array([scenes.BODY_CYLINDER, 0.0, 0.0, -500.0, A, 1000.0])
    sc = scenes.Scene(np.zeros((0, 3, 3)), np.zeros(0), body[None, :], tx, (0, 1, 0) if hard else (0, 0, 1), [F], rx,
                      "oblique cylinder", max_order=0)
    r = oracle_mod.evaluate(sc, path_fields=hard)
    if not hard:
        return r.E[0, 2, :], r.counts
    rx64 = sc.rx.astype(np.float64)
    tx64 = sc.tx.astype(np.float64)
    out = np.zeros(len(phi), dtype=complex)
    for i in range(len(phi)):
        P = rx64[i]
        for k in range(int(r.counts[i])):
            t, _, _ = oracle_mod.decode(r.codes[i, k])
            if t == oracle_mod.PT_LOS:
                src = tx64
            elif t == oracle_mod.PT_RB:
                src = oracle_mod.body_reflection(body, tx64, P)["Q"]
            else:
                src = oracle_mod.body_creeping(body, tx64, P, 0 if t == oracle_mod.PT_CP else 1)["Q2"]
            s = (P - src) / np.linalg.norm(P - src)
            out[i] += np.cross(s, r.path_E[i, k, 0])[2]
    return out, r.counts


@pytest.mark.parametrize("hard", [False, True], ids=["tm_Ez", "te_Hz"])
@pytest.mark.parametrize("beta_deg", [60.0, 35.0])
def test_cylinder_oblique_vs_exact_series(oracle_mod, beta_deg, hard):
    beta = np.radians(beta_deg)
    phi = np.radians(np.concatenate([LIT, SHADOW]))
    u, counts = _oracle(oracle_mod, beta, phi, hard)
    ex = _series(beta, phi, hard)
    ddb = np.abs(20 * np.log10(np.abs(u) / np.abs(ex)))
    dph = np.abs(np.angle(u / ex))
    nl = len(LIT)
    assert np.all(counts[:nl] == 3) and np.all(counts[nl:] == 2)      # direct + reflection; two creeping rays
    assert np.all(ddb[:nl] < 0.3) and np.all(dph[:nl] < 0.05), (ddb[:nl], dph[:nl])
    assert np.all(ddb[nl:] < 0.4) and np.all(dph[nl:] < 0.05), (ddb[nl:], dph[nl:])


def test_oblique_pin_sees_a_wrong_surface_radius(oracle_mod):
    """A plausible mistake -- the reflection's Fock parameter taken with the
    cylinder's radius a instead of the oblique plane of incidence's surface
    radius -- moves the lit field near the shadow boundary by more than the
    tolerance: the series pins that quantity.  Planted here by evaluating
    the bracket of R with both radii for the oracle's own reflection point."""
    beta = np.radians(35.0)
    body = np.array([scenes.BODY_CYLINDER, 0.0, 0.0, -500.0, A, 1000.0])
    tx = D * np.array([np.sin(beta), 0.0, np.cos(beta)])
    P = np.array([RHO * np.cos(np.radians(164.0)), RHO * np.sin(np.radians(164.0)), 0.0])
    g = oracle_mod.body_reflection(body, tx, P)
    n = g["n"]
    si = (g["Q"] - tx) / np.linalg.norm(g["Q"] - tx)
    cth = -si @ n
    kh = (K / 2.0) ** (1.0 / 3.0)
    xi_ok = -2.0 * kh * g["rho_g"] ** (1.0 / 3.0) * cth
    xi_bad = -2.0 * kh * A ** (1.0 / 3.0) * cth
    assert g["rho_g"] > 1.5 * A                  # the oblique plane of incidence sees a flatter surface
    Lp = 1.0                                      # (the distance parameter's size: only the Fock part differs)
    r_ok = -np.sqrt(-4 / xi_ok) * np.exp(-1j * xi_ok ** 3 / 12) * oracle_mod.fock_bracket(
        np.array([xi_ok]), np.array([np.sqrt(K * Lp / (2 * (kh * g["rho_g"] ** (1 / 3)) ** 2))]))[0][0]
    r_bad = -np.sqrt(-4 / xi_bad) * np.exp(-1j * xi_bad ** 3 / 12) * oracle_mod.fock_bracket(
        np.array([xi_bad]), np.array([np.sqrt(K * Lp / (2 * (kh * A ** (1 / 3)) ** 2))]))[0][0]
    assert abs(20 * np.log10(abs(r_bad) / abs(r_ok))) > 0.3 or abs(np.angle(r_bad / r_ok)) > 0.05
