"""Exact eigenfunction-series solutions used to pin the FP64 oracle.

These are independent of the ray method: separation-of-variables solutions of
the canonical problems (PEC circular cylinder with a line source, PEC sphere
with a point dipole), written with scipy's Bessel / Legendre functions.  The
paper validates its sphere results against the analytical solution (Sec. IV.A,
Fig. 10); these series play that role here.

Time convention e^{+j w t}; outgoing waves use H^(2) / h^(2).
"""
import numpy as np
from scipy.special import hankel2, jv, jvp, h2vp, spherical_jn, spherical_yn, lpmv


# ----------------------------------------------------------------- 2-D cylinder
def cyl2d_total(k, a, rs, rr, phi, hard, nmax=None):
    """Total field of a line source H0^(2)(k|rho - rho_s|) at (rs, 0) near a PEC
    cylinder of radius a, observed at (rr, phi) with a < rr < rs.
    soft: E_z (Dirichlet), hard: H_z (Neumann)."""
    if nmax is None:
        nmax = int(k * rs + 40)
    n = np.arange(-nmax, nmax + 1)
    inc = hankel2(0, k * np.sqrt(rs ** 2 + rr ** 2 - 2 * rs * rr * np.cos(phi)))
    if hard:
        coef = jvp(n, k * a) / h2vp(n, k * a)
    else:
        coef = jv(n, k * a) / hankel2(n, k * a)
    sc = -np.sum(coef * hankel2(n, k * rr) * hankel2(n, k * rs) * np.exp(1j * n * phi))
    return inc + sc


# --------------------------------------------------------------- sphere helpers
def _h2(n, x, d=False):
    return spherical_jn(n, x, d) - 1j * spherical_yn(n, x, d)


def _riccati_d(n, x, kind):
    """d/dx [x z_n(x)] for z = j (kind 'j') or h^(2) (kind 'h')."""
    if kind == "j":
        return spherical_jn(n, x) + x * spherical_jn(n, x, True)
    return _h2(n, x) + x * _h2(n, x, True)


def sphere_scalar_total(k, a, r0, r, theta, hard, nmax=None):
    """Point source e^{-jkR}/R at distance r0 from the centre of a sphere of
    radius a (Dirichlet if not hard, Neumann if hard); observation at radius
    r < r0 and angle theta from the source axis.  Uses
    e^{-jkR}/R = -jk sum (2n+1) j_n(k r<) h_n(k r>) P_n(cos gamma)."""
    if nmax is None:
        nmax = int(k * r0 + 60)
    n = np.arange(nmax + 1)
    if hard:
        c = spherical_jn(n, k * a, True) / _h2(n, k * a, True)
    else:
        c = spherical_jn(n, k * a) / _h2(n, k * a)
    Pn = np.array([lpmv(0, nn, np.cos(theta)) for nn in n])
    R = np.sqrt(r0 ** 2 + r ** 2 - 2 * r0 * r * np.cos(theta))
    inc = np.exp(-1j * k * R) / R
    sc = -1j * k * np.sum((2 * n + 1) * (-c) * _h2(n, k * r) * _h2(n, k * r0) * Pn)
    return inc + sc


# --------------------------------------------------------------- vector Mie
def dipole_fields(k, src, moment, pts, magnetic=False):
    """E, H (eta = 1 units) of a point electric (or magnetic) dipole with the
    full near-field terms, e^{+jwt}; far field |E| = |m x n| / R."""
    d = pts - src
    R = np.linalg.norm(d, axis=-1)[..., None]
    n = d / R
    kr = k * R
    g = np.exp(-1j * kr) / R
    p = np.broadcast_to(moment, d.shape)
    nxp = np.cross(n, p)
    near = 1.0 / kr ** 2 + 1j / kr
    F1 = (np.cross(nxp, n) + (3 * n * np.sum(n * p, -1, keepdims=True) - p) * near) * g
    F2 = nxp * (1 - 1j / kr) * g
    if magnetic:
        return -F2, F1
    return F1, F2


class MieDipole:
    """PEC sphere (radius a, centre at the origin) illuminated by a point
    dipole on the +x axis at distance r0, moment along +z (electric or
    magnetic).  Scattered field from Debye potentials
        E = curl curl (r Pe) - jk curl (r Pm),  H = jk curl (r Pe) + curl curl (r Pm)
    with Pe, Pm = sum_n z_n(kr) P_n^1(cos t) (c_n cos f + s_n sin f) in a frame
    whose polar axis points at the dipole.  Incident coefficients come from
    projecting r E_r and r H_r of the closed-form dipole field onto P_n^1 on
    three spheres a < r < r0 (least squares); the PEC conditions
    d(r z_n)/dr = 0 (TM) and z_n = 0 (TE) at r = a give the scattered ones.
    """

    def __init__(self, k, a, r0, magnetic=False, nmax=60, nq=400):
        self.k, self.a, self.r0, self.magnetic, self.nmax = k, a, r0, magnetic, nmax
        # primed frame: z' = +x (towards the source), x' = +z (dipole), y' = -y
        self.Rm = np.array([[0, 0, 1.0], [0, -1.0, 0], [1.0, 0, 0]])  # rows: x', y', z' in global coords
        src = np.array([r0, 0.0, 0.0])
        mom = np.array([0.0, 0.0, 1.0])
        n = np.arange(1, nmax + 1)
        x, w = np.polynomial.legendre.leggauss(nq)
        th = np.arccos(x)
        Pn1 = np.array([lpmv(1, nn, x) for nn in n])            # [n, q]
        norm = 2.0 * n * (n + 1) / (2 * n + 1)
        radii = np.array([a + 0.4 * (r0 - a), a + 0.6 * (r0 - a), a + 0.8 * (r0 - a)])
        coefs = {}
        for name in ("Ec", "Es", "Hc", "Hs"):
            coefs[name] = (np.zeros(nmax, complex), np.zeros(nmax))
        acc = {key: [np.zeros(nmax, complex), np.zeros(nmax)] for key in ("Ec", "Es", "Hc", "Hs")}
        for r1 in radii:
            jn = spherical_jn(n, k * r1)
            for phi, suf in ((0.0, "c"), (np.pi / 2, "s")):
                # points in the primed frame -> global
                pp = np.stack([r1 * np.sin(th) * np.cos(phi), r1 * np.sin(th) * np.sin(phi), r1 * np.cos(th)], -1)
                pg = pp @ self.Rm
                E, H = dipole_fields(k, src, mom, pg, magnetic)
                rhat = pg / r1
                rEr = r1 * np.sum(E * rhat, -1)
                rHr = r1 * np.sum(H * rhat, -1)
                for fld, key in ((rEr, "E" + suf), (rHr, "H" + suf)):
                    proj = Pn1 @ (w * fld) / norm            # = n(n+1) coef j_n(k r1)
                    acc[key][0] += proj * n * (n + 1) * jn
                    acc[key][1] += (n * (n + 1) * jn) ** 2
        self.inc = {key: acc[key][0] / acc[key][1] for key in acc}
        ka = k * a
        tm = -_riccati_d(n, ka, "j") / _riccati_d(n, ka, "h")
        te = -spherical_jn(n, ka) / _h2(n, ka)
        self.sc = {"Ec": self.inc["Ec"] * tm, "Es": self.inc["Es"] * tm,
                   "Hc": self.inc["Hc"] * te, "Hs": self.inc["Hs"] * te}
        self.src, self.mom = src, mom

    def scattered(self, pts, coeffs=None, kind="h"):
        """Scattered E (global Cartesian) at points [m, 3] (r > a)."""
        c = self.sc if coeffs is None else coeffs
        k = self.k
        n = np.arange(1, self.nmax + 1)[:, None]
        pp = pts @ self.Rm.T
        r = np.linalg.norm(pp, axis=-1)
        th = np.arccos(np.clip(pp[:, 2] / r, -1, 1))
        ph = np.arctan2(pp[:, 1], pp[:, 0])
        x = np.cos(th)
        st = np.sin(th)
        kr = k * r
        z = _h2(n, kr) if kind == "h" else spherical_jn(n, kr)
        D = _riccati_d(n, kr, kind) / r * (1.0)        # d/dr (r z_n(kr)) = (x z_n(x))'
        P = np.array([lpmv(1, nn, x) for nn in n[:, 0]])
        Pm1 = np.array([lpmv(1, nn - 1, x) for nn in n[:, 0]])
        dP = (n * x * P - (n + 1) * Pm1) / st          # dP_n^1(cos t)/dt
        ec, es = c["Ec"][:, None], c["Es"][:, None]
        hc, hs = c["Hc"][:, None], c["Hs"][:, None]
        cf, sf = np.cos(ph), np.sin(ph)
        Ae = ec * cf + es * sf          # angular factor of Pe
        dAe = -ec * sf + es * cf        # d/dphi
        Am = hc * cf + hs * sf
        dAm = -hc * sf + hs * cf
        Er = np.sum(n * (n + 1) * z / r * P * Ae, 0)
        Et = np.sum(D * dP * Ae - 1j * k * z * P / st * dAm, 0)
        Ep = np.sum(D * P / st * dAe + 1j * k * z * dP * Am, 0)
        # spherical -> primed Cartesian -> global
        rh = np.stack([st * np.cos(ph), st * np.sin(ph), x], -1)
        thh = np.stack([x * np.cos(ph), x * np.sin(ph), -st], -1)
        phh = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)], -1)
        Ep_ = Er[:, None] * rh + Et[:, None] * thh + Ep[:, None] * phh
        return Ep_ @ self.Rm

    def incident(self, pts):
        return dipole_fields(self.k, self.src, self.mom, pts, self.magnetic)[0]

    def total(self, pts):
        return self.incident(pts) + self.scattered(pts)
