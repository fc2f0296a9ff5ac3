"""Reference gradients for the adjoint tests, from the FP64 oracle alone.

The derivative is its definition: central differences of each path's own
field (oracle.evaluate(path_fields=True)) at parameter +- h, with visibility
held fixed by taking exactly the paths of the forward path list (matched by
path code).  A body's parameters move only that body's paths, so its
differences come from a scene with that body alone (the other bodies only
decide visibility, which is fixed); the transmitter and the frequencies move
every path, so theirs come from the whole scene.  The vector-Jacobian product
with dLoss/dE = g is sum over receivers, listed paths, frequencies and
components of Re g * Re dE + Im g * Im dE.
"""
from types import SimpleNamespace

import numpy as np

from oracle import oracle

EN_BODIES = oracle.EN_BODYREFL | oracle.EN_CREEP_SOFT | oracle.EN_CREEP_HARD
BODY_TYPES = (oracle.PT_RB, oracle.PT_CP, oracle.PT_CM, oracle.PT_WCP, oracle.PT_WCM)


def pcode(t, a, b):
    return (int(t) << 56) | (int(a) << 28) | int(b)


def _scene64(sc, bodies=None, tx=None, freqs=None, rx=None):
    return SimpleNamespace(max_enc=getattr(sc, "max_enc", 0), wall_creep=getattr(sc, "wall_creep", False),
                           candidates=getattr(sc, "candidates", None), tri=np.asarray(sc.tri, dtype=np.float64),
                           tri_face=sc.tri_face,
                           bodies=np.asarray(sc.bodies if bodies is None else bodies, dtype=np.float64).reshape(-1, 6),
                           tx=np.asarray(sc.tx if tx is None else tx, dtype=np.float64),
                           pol=np.asarray(sc.pol, dtype=np.float64),
                           freqs=np.asarray(sc.freqs if freqs is None else freqs, dtype=np.float64),
                           rx=sc.rx if rx is None else rx, max_order=sc.max_order,
                           face_eps=getattr(sc, "face_eps", None))


def _path_fields(scene, enable, cap):
    """Per receiver: {code: field [n_f, 3]} of the listed paths."""
    r = oracle.evaluate(scene, enable=enable, cap=cap, path_fields=True)
    out = []
    for i in range(len(r.counts)):
        n = min(int(r.counts[i]), cap)
        out.append({int(r.codes[i, k]): r.path_E[i, k] for k in range(n)})
    return out


def _contract(g, dE):
    return float(np.sum(g.real * dE.real + g.imag * dE.imag))


def vjp(sc, codes, g, bodies=(), h=1e-5, df=1e3, cap=256, tx=True, freqs=True):
    """Reference dLoss/d(params) for scene sc (float32 Scene), forward path
    lists codes (per receiver, iterable of int codes) and g = dLoss/dE as
    complex [n_f, 3, n_rx].  Returns dict(body={b: [4]}, tx=[3], f=[n_f],
    and the sums of |contribution| body_abs / tx_abs / f_abs, skipped = paths
    that vanished at a perturbed point)."""
    codes = [set(int(c) for c in cs) for cs in codes]
    out = dict(body={}, body_abs={}, skipped=0, skipped_paths=[])
    # bodies: a scene with the body alone, the receivers where it has paths
    for b in bodies:
        R = [r for r, cs in enumerate(codes) if any((c >> 56) in BODY_TYPES and ((c >> 28) & 0xFFFFFFF) == b
                                                        for c in cs)]
        grad, absum = np.zeros(4), np.zeros(4)
        if R:
            rx = sc.rx[R]
            for k, col in enumerate((1, 2, 3, 4)):
                fs = []
                for sgn in (+1, -1):
                    row = np.asarray(sc.bodies[b], dtype=np.float64).copy()
                    row[col] += sgn * h
                    fs.append(_path_fields(_scene64(sc, bodies=row[None, :], rx=rx), EN_BODIES, cap))
                for i, r in enumerate(R):
                    for c in codes[r]:
                        if (c >> 56) not in BODY_TYPES or ((c >> 28) & 0xFFFFFFF) != b:
                            continue
                        key = pcode(c >> 56, 0, c & 0xFFFFFFF)     # body 0 of the one-body scene; turns kept
                        if key not in fs[0][i] or key not in fs[1][i]:
                            out["skipped"] += 1
                            out["skipped_paths"].append(("body %d param %d" % (b, k), r, c))
                            continue
                        v = _contract(g[:, :, r], (fs[0][i][key] - fs[1][i][key]) / (2 * h))
                        grad[k] += v
                        absum[k] += abs(v)
        out["body"][b], out["body_abs"][b] = grad, absum
    R = [r for r, cs in enumerate(codes) if cs]
    rx = sc.rx[R]

    def whole(param_fn, step, n_par):
        grad, absum = np.zeros(n_par), np.zeros(n_par)
        for k in range(n_par):
            fs = [_path_fields(param_fn(k, s * step), oracle.EN_ALL, cap) for s in (+1, -1)]
            for i, r in enumerate(R):
                for c in codes[r]:
                    if c not in fs[0][i] or c not in fs[1][i]:
                        out["skipped"] += 1
                        out["skipped_paths"].append(("param %d" % k, r, c))
                        continue
                    v = _contract(g[:, :, r], (fs[0][i][c] - fs[1][i][c]) / (2 * step))
                    grad[k] += v
                    absum[k] += abs(v)
        return grad, absum

    if tx:
        def tx_at(k, d):
            t = np.asarray(sc.tx, dtype=np.float64).copy()
            t[k] += d
            return _scene64(sc, tx=t, rx=rx)
        out["tx"], out["tx_abs"] = whole(tx_at, h, 3)
    if freqs:
        def f_at(k, d):
            f = np.asarray(sc.freqs, dtype=np.float64).copy()
            f[k] += d
            return _scene64(sc, freqs=f, rx=rx)
        out["f"], out["f_abs"] = whole(f_at, df, len(sc.freqs))
    return out
