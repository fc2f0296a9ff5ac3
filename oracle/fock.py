"""Fock--Pekeris functions for the smooth-surface UTD coefficients, in FP64.

TEST INFRASTRUCTURE (oracle): imported only by tests, the smoke check and the
CPU legs of bench.py.

The paper states the lit/shadow field equations (Eqs. 1-4, Sec. II.B) and
leaves the reflection coefficient R and the transfer function T to the
off-surface UTD literature it cites (Pathak; Johansen).  The functions below
are the soft (s) and hard (h) Fock--Pekeris integrals of that theory, with the
time convention e^{+j w t}:

    P_s(xi) = e^{-j pi/4}/sqrt(pi) * Int_{-inf}^{inf} V(tau)/W2(tau)  e^{-j xi tau} dtau
    P_h(xi) = e^{-j pi/4}/sqrt(pi) * Int_{-inf}^{inf} V'(tau)/W2'(tau) e^{-j xi tau} dtau

with the Fock--Airy functions V = sqrt(pi) Ai, W_{1,2} = sqrt(pi) (Bi +- j Ai).
Both carry the singular part -c/xi at xi -> 0, c = e^{-j pi/4}/(2 sqrt(pi));
the regular parts phat = P + c/xi are what the contour quadrature returns.

Evaluation (all FP64, Airy functions from scipy.special, a library primitive):
  * xi in [XI_LO, XI_HI]: contour quadrature of phat.  Using V = (W1-W2)/(2j),
    phat = e^{-j pi/4}/sqrt(pi) [ Int_{-inf}^{0} W1/(2j W2) e^{-j xi tau} dtau
                                  + Int_0^{inf} V/W2 e^{-j xi tau} dtau ]
    (primes on every Airy function for the hard case).  The second integral
    runs on the real axis (super-exponential decay).  The first is written in
    x = -tau and its path is deformed where the integrand decays: for xi >= 0
    along x = u e^{j pi/3}; for xi < 0 along the real axis past the
    stationary point x* = xi^2/4 and then into the upper half plane.
  * xi > XI_HI: the residue (creeping-wave mode) series over the Airy zeros,
    closed form of the same integral for xi > 0.
  * xi < XI_LO: not evaluated; the reflection coefficient takes its GO value
    (-1 soft, +1 hard) there.

The identities used to evaluate W1, W2 from Ai at rotated arguments are
DLMF 9.2.11: W2(z) = 2 sqrt(pi) e^{-j pi/6} Ai(z e^{-2 pi j/3}),
W1(z) = 2 sqrt(pi) e^{+j pi/6} Ai(z e^{+2 pi j/3}).
"""
import numpy as np
from scipy.special import airye, ai_zeros

XI_LO = -10.0      # below: GO reflection coefficient (R_s = -1, R_h = +1)
XI_HI = 1.5        # above: residue series
N_RESIDUE = 40     # residue terms used by the oracle (FP64 converged for xi >= XI_HI)
C_SING = np.exp(-1j * np.pi / 4) / (2.0 * np.sqrt(np.pi))   # c in -c/xi
_OMEGA = np.exp(2j * np.pi / 3)
_PREF = np.exp(-1j * np.pi / 4) / np.sqrt(np.pi)


def _ai(z, deriv):
    """Ai(z) (or Ai'(z)) as (scaled value, exponent) with Ai = value * exp(-zeta)."""
    z = np.asarray(z, dtype=complex)
    eai, eaip, _, _ = airye(z)
    zeta = (2.0 / 3.0) * z ** 1.5
    return (eaip if deriv else eai), zeta


def _ratio(z1, z2, deriv):
    """Ai^(d)(z1) / Ai^(d)(z2) without overflow."""
    v1, e1 = _ai(z1, deriv)
    v2, e2 = _ai(z2, deriv)
    return v1 / v2 * np.exp(-e1 + e2)


def integrand_pos(tau, hard):
    """V/W2 (soft) or V'/W2' (hard) at tau (used on tau >= 0)."""
    tau = np.asarray(tau, dtype=complex)
    if not hard:
        # V/W2 = sqrt(pi) Ai(tau) / (2 sqrt(pi) e^{-j pi/6} Ai(tau w^-1))
        return np.exp(1j * np.pi / 6) / 2.0 * _ratio(tau, tau * np.conj(_OMEGA), False)
    # W2'(tau) = 2 sqrt(pi) e^{-j 5pi/6} Ai'(tau w^-1)
    return np.exp(5j * np.pi / 6) / 2.0 * _ratio(tau, tau * np.conj(_OMEGA), True)


def integrand_neg(tau, hard):
    """W1/(2j W2) (soft) or W1'/(2j W2') (hard) at tau (used for tau <= 0)."""
    tau = np.asarray(tau, dtype=complex)
    if not hard:
        # W1/W2 = e^{j pi/3} Ai(tau w)/Ai(tau w^-1)
        return np.exp(1j * np.pi / 3) * _ratio(tau * _OMEGA, tau * np.conj(_OMEGA), False) / 2j
    # W1'/W2' = e^{-j pi/3} Ai'(tau w)/Ai'(tau w^-1)
    return np.exp(-1j * np.pi / 3) * _ratio(tau * _OMEGA, tau * np.conj(_OMEGA), True) / 2j


def _panels(a, b, width, n):
    """Composite Gauss-Legendre nodes/weights on the real interval [a, b]."""
    m = max(1, int(np.ceil((b - a) / width)))
    x, w = np.polynomial.legendre.leggauss(n)
    edges = np.linspace(a, b, m + 1)
    xs = [(edges[i] + edges[i + 1]) / 2 + (edges[i + 1] - edges[i]) / 2 * x for i in range(m)]
    ws = [(edges[i + 1] - edges[i]) / 2 * w for i in range(m)]
    return np.concatenate(xs), np.concatenate(ws)


# Quadrature buckets: bucket 0 serves xi in [0, XI_HI]; bucket n >= 1 serves
# xi in [-n, -n+1).  Each bucket has one fixed contour valid for all its xi.
N_BUCKETS = 1 + int(-XI_LO)


def bucket_of(xi):
    if xi >= 0.0:
        return 0
    return int(np.ceil(-xi))


def contour_rule(bucket, width=0.5, order=16, tau_max=8.0, ray_len=None):
    """Nodes tau_i (complex) and weights Ws_i, Wh_i such that

        phat_{s,h}(xi) = e^{-j pi/4}/sqrt(pi) * sum_i W_i exp(-j xi tau_i)

    for every xi in the bucket.  The weights already include the Airy-ratio
    integrand and the path Jacobian."""
    # Int_0^inf V/W2 e^{-j xi tau} dtau on the real axis
    tp, wp = _panels(0.0, tau_max, width, order)
    nodes = [tp.astype(complex)]
    ws = [wp * integrand_pos(tp, False)]
    wh = [wp * integrand_pos(tp, True)]
    # Int_0^inf h(-x) e^{+j xi x} dx on a deformed path in x (tau = -x)
    if bucket == 0:
        e = np.exp(1j * np.pi / 3)
        u, wu = _panels(0.0, tau_max if ray_len is None else ray_len, width, order)
        x = u * e
        dx = wu * e
    else:
        xi_min = -float(bucket)
        x1 = xi_min * xi_min / 4.0 + 1.0 + 0.5 * bucket
        xr, wr = _panels(0.0, x1, width, order)
        e = np.exp(1j * np.pi / 3)
        L = 14.0 if ray_len is None else ray_len
        u, wu = _panels(0.0, L, width, order)
        x = np.concatenate([xr.astype(complex), x1 + u * e])
        dx = np.concatenate([wr.astype(complex), wu * e])
    nodes.append(-x)
    ws.append(dx * integrand_neg(-x, False))
    wh.append(dx * integrand_neg(-x, True))
    return np.concatenate(nodes), np.concatenate(ws), np.concatenate(wh)


_RULES = {}


def _rule(bucket):
    if bucket not in _RULES:
        _RULES[bucket] = contour_rule(bucket)
    return _RULES[bucket]


def phat(xi, hard):
    """Regular part P + c/xi by contour quadrature, xi in [XI_LO, XI_HI]."""
    xi = float(xi)
    if not (XI_LO <= xi <= XI_HI):
        raise ValueError("phat quadrature domain is [XI_LO, XI_HI]")
    tau, Ws, Wh = _rule(bucket_of(xi))
    W = Wh if hard else Ws
    return complex(_PREF * np.sum(W * np.exp(-1j * xi * tau)))


_ZEROS = None


def airy_zero_data(n=N_RESIDUE):
    """alpha_n = -a_n, beta_n = -a'_n and Ai'(a_n), Ai(a'_n) (scipy)."""
    global _ZEROS
    if _ZEROS is None or len(_ZEROS[0]) < n:
        a, ap, ai, aip = ai_zeros(n)
        _ZEROS = (-a, -ap, aip, ai)
    al, be, aip, ai = _ZEROS
    return al[:n], be[:n], aip[:n], ai[:n]


def P_residue(xi, hard, nterms=N_RESIDUE):
    """Residue series of P_{s,h}(xi), valid for xi > 0 (converges fast for xi >~ 1).

    Poles of V/W2 are at tau_n = alpha_n e^{-j pi/3} (zeros of W2); the
    residues follow from the Airy Wronskians (DLMF 9.2.8-9.2.9):
      P_s = -e^{-j pi/12}/(2 sqrt(pi)) sum exp(-j xi alpha_n e^{-j pi/3}) / Ai'(-alpha_n)^2
      P_h = -e^{-j pi/12}/(2 sqrt(pi)) sum exp(-j xi beta_n e^{-j pi/3}) / (beta_n Ai(-beta_n)^2)
    """
    al, be, aip, ai = airy_zero_data(nterms)
    e = np.exp(-1j * np.pi / 3)
    if not hard:
        s = np.sum(np.exp(-1j * xi * al * e) / aip ** 2)
    else:
        s = np.sum(np.exp(-1j * xi * be * e) / (be * ai ** 2))
    return complex(-np.exp(-1j * np.pi / 12) / (2.0 * np.sqrt(np.pi)) * s)


def phat_any(xi, hard):
    """phat on xi >= XI_LO: quadrature inside the table domain, residue series above."""
    if xi > XI_HI:
        return P_residue(xi, hard) + C_SING / xi
    return phat(xi, hard)


def P(xi, hard):
    """Full Fock--Pekeris function P_{s,h}(xi) (singular at xi = 0)."""
    return phat_any(xi, hard) - C_SING / xi


def c_tables():
    """Flattened arrays handed to the C oracle: per bucket the node/weight
    rule, plus the residue-series constants."""
    taus, Wss, Whs, offs = [], [], [], [0]
    for b in range(N_BUCKETS):
        t, s, h = _rule(b)
        taus.append(t); Wss.append(s); Whs.append(h); offs.append(offs[-1] + len(t))
    al, be, aip, ai = airy_zero_data(N_RESIDUE)
    return dict(
        tau=np.concatenate(taus), Ws=np.concatenate(Wss), Wh=np.concatenate(Whs),
        offsets=np.asarray(offs, dtype=np.int32),
        res_alpha=al.astype(np.float64), res_cs=(1.0 / aip ** 2).astype(np.float64),
        res_beta=be.astype(np.float64), res_ch=(1.0 / (be * ai ** 2)).astype(np.float64))
