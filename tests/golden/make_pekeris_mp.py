"""Writes tests/golden/pekeris_mp.txt: high-precision values of the regular
parts of the soft and hard Fock--Pekeris functions at 51 points of
xi in [-10, 1.5], computed with mpmath from their integral definition alone
(nothing of oracle/ or of the CUDA library is used).

Definition (the off-surface UTD functions the paper defers to its
references for T and R after Eq. 4; time convention e^{+j w t}):

    P_s(xi) = e^{-j pi/4}/sqrt(pi) Int V(tau)/W2(tau) e^{-j xi tau} dtau,
    P_h(xi) = the same with V', W2',
    V = sqrt(pi) Ai,  W_{1,2} = sqrt(pi) (Bi +- j Ai),

whose singular part is -c/xi, c = e^{-j pi/4}/(2 sqrt(pi)).  With
V = (W1 - W2)/(2j) the integrand on tau < 0 is W1/(2j W2) + j/2; the
constant j/2 integrates to exactly -c/xi, so the regular part phat = P + c/xi
is

    phat = e^{-j pi/4}/sqrt(pi) [ Int_{-inf}^0 W1/(2j W2) e^{-j xi tau} dtau
                                  + Int_0^inf V/W2 e^{-j xi tau} dtau ].

Each integral is moved off the real axis onto a ray where its integrand
decays super-exponentially and no pole (the zeros of W2 lie on arg tau =
-pi/3) is crossed: the first onto tau = r e^{-j 5 pi/6} (from infinity to
0), the second onto tau = r e^{j pi/6}.  These rays are not the oracle's
contours, the quadrature (tanh-sinh) is not its Gauss-Legendre panels, and
the Airy functions are mpmath's at 30 significant digits, so the values pin
the oracle's evaluation rather than repeat it.  For xi < 0 the first
integrand grows like e^{|xi| r / 2} before it decays; at xi = -10 the
cancellation costs about 9 of the 30 digits.

    python tests/golden/make_pekeris_mp.py      (about a minute on 8 cores)
"""
import os
import sys
from multiprocessing import get_context

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "pekeris_mp.txt")
DPS = 30


def xi_points():
    return np.concatenate([np.linspace(-10.0, 1.5, 47), [-9.99, -0.01, 0.01, 1.49]])


def phat_mp(xi, hard, dps=DPS):
    import mpmath as mp
    mp.mp.dps = dps
    xi = mp.mpf(xi)
    w = mp.exp(2j * mp.pi / 3)
    d = 1 if hard else 0
    # W1/(2j W2) and V/W2 through DLMF 9.2.11: W1 = 2 sqrt(pi) e^{j pi/6} Ai(z w),
    # W2 = 2 sqrt(pi) e^{-j pi/6} Ai(z / w); with derivatives the chain rule adds w^{+-1}
    if not hard:
        f = lambda t: mp.exp(1j * mp.pi / 3) * mp.airyai(t * w) / mp.airyai(t / w) / 2j
        g = lambda t: mp.exp(1j * mp.pi / 6) / 2 * mp.airyai(t) / mp.airyai(t / w)
    else:
        f = lambda t: mp.exp(-1j * mp.pi / 3) * mp.airyai(t * w, d) / mp.airyai(t / w, d) / 2j
        g = lambda t: mp.exp(5j * mp.pi / 6) / 2 * mp.airyai(t, d) / mp.airyai(t / w, d)
    en = mp.exp(-5j * mp.pi / 6)
    ep = mp.exp(1j * mp.pi / 6)
    i1 = -mp.quad(lambda r: f(r * en) * mp.exp(-1j * xi * r * en) * en, [0, 2, 6, 15, 30, mp.inf])
    i2 = mp.quad(lambda r: g(r * ep) * mp.exp(-1j * xi * r * ep) * ep, [0, 2, 6, 15, mp.inf])
    v = mp.exp(-1j * mp.pi / 4) / mp.sqrt(mp.pi) * (i1 + i2)
    return complex(v)


def _job(args):
    xi, hard = args
    return xi, hard, phat_mp(xi, hard)


def main():
    jobs = [(float(x), h) for x in xi_points() for h in (False, True)]
    with get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        res = pool.map(_job, jobs)
    val = {(x, h): v for x, h, v in res}
    with open(OUT, "w") as fh:
        fh.write("# regular parts phat = P + c/xi of the soft and hard Fock-Pekeris functions,\n")
        fh.write("# mpmath %d digits on rays off the real axis (tests/golden/make_pekeris_mp.py)\n" % DPS)
        fh.write("# xi  re(phat_s)  im(phat_s)  re(phat_h)  im(phat_h)\n")
        for x in xi_points():
            s, h = val[(float(x), False)], val[(float(x), True)]
            fh.write("%.17g %.17g %.17g %.17g %.17g\n" % (x, s.real, s.imag, h.real, h.imag))
    print("wrote", OUT)


if __name__ == "__main__":
    sys.exit(main())
