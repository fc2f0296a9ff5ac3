"""Pins of the oracle's large-scene mode: planar paths of orders 1-3 over a
list of candidate face sequences, and the ray launch that makes the list.

* The ray launch in an empty box finds exactly the realizable sequences:
  order 1 and 2 all faces and ordered pairs; order 3 the triples (f1, f2, f3)
  for which some point X of face f3 is reached from the source by a valid
  two-bounce image path off f1 then f2 (points in their faces, each leg
  crossing its plane), X sampled on a grid -- a test that traces no ray.
* With the list of every sequence of order <= 2, the candidate mode gives the
  enumeration mode's path list and fields (a room with cylinders).
* Order-3 paths in an empty box equal a direct minimisation of the unfolded
  length over three points on the faces (count and field), as the order <= 2
  pin of the enumeration mode does.
"""
import itertools

import numpy as np
import pytest
from scipy.optimize import minimize

from paper_2310_10578_gb300 import scenes
from paper_2310_10578_gb300.scenes import Scene

L_BOX = np.array([10.0, 8.0, 3.0])
FACES = [(2, 0.0), (2, L_BOX[2]), (0, 0.0), (0, L_BOX[0]), (1, 0.0), (1, L_BOX[1])]   # box_triangles ids


def _on_face(f, uv):
    ax, v = FACES[f]
    q = np.empty(3)
    free = [d for d in range(3) if d != ax]
    q[ax] = v; q[free[0]] = uv[0]; q[free[1]] = uv[1]
    return q


def _inside(f, q, tol=1e-9):
    ax, _ = FACES[f]
    return all(-tol <= q[d] <= L_BOX[d] + tol for d in range(3) if d != ax)


def _mirror(X, f):
    ax, v = FACES[f]
    Y = X.copy(); Y[ax] = 2 * v - X[ax]
    return Y


def _two_bounce_to(S, f1, f2, X):
    """Valid image path S -> f1 -> f2 -> X in the empty box?"""
    S1 = _mirror(S, f1); S2 = _mirror(S1, f2)
    ax2, v2 = FACES[f2]
    if not ((S2[ax2] - v2) * (X[ax2] - v2) < 0):
        return False
    Q2 = S2 + (X - S2) * (S2[ax2] - v2) / (S2[ax2] - X[ax2])
    if not _inside(f2, Q2, 0.0):
        return False
    ax1, v1 = FACES[f1]
    if not ((S1[ax1] - v1) * (Q2[ax1] - v1) < 0):
        return False
    Q1 = S1 + (Q2 - S1) * (S1[ax1] - v1) / (S1[ax1] - Q2[ax1])
    return _inside(f1, Q1, 0.0)


def _box_scene(rx, tx=(1.0, 1.0, 2.0)):
    tri, face = scenes.box_triangles(*L_BOX)
    return Scene(tri, face, np.zeros((0, 6)), tx, (0, 0, 1.0), [2.4e9], rx, "box", max_order=3)


def test_ray_launch_finds_the_realizable_sequences(oracle_mod):
    S = np.array([1.0, 1.0, 2.0])
    sc = _box_scene(np.zeros((1, 3), dtype=np.float32))
    c = oracle_mod.candidates(sc, 20000, 3)
    got = {k: set(tuple(int(v) for v in x[:k]) for x in c if (x >= 0).sum() == k) for k in (1, 2, 3)}
    assert got[1] == {(f,) for f in range(6)}
    assert got[2] == {(a, b) for a in range(6) for b in range(6) if a != b}
    real = set()
    for f1, f2, f3 in itertools.product(range(6), repeat=3):
        if f1 == f2 or f2 == f3:
            continue
        ax, _ = FACES[f3]
        free = [d for d in range(3) if d != ax]
        for u in np.linspace(0.01, 0.99, 40):
            for v in np.linspace(0.01, 0.99, 40):
                if _two_bounce_to(S, f1, f2, _on_face(f3, [u * L_BOX[free[0]], v * L_BOX[free[1]]])):
                    real.add((f1, f2, f3))
                    break
            if (f1, f2, f3) in real:
                break
    assert got[3] == real, (sorted(real - got[3]), sorted(got[3] - real))
    # sorted by order, then faces, no repeats
    keys = [((x >= 0).sum(), tuple(x)) for x in c]
    assert keys == sorted(set(keys))


def test_candidate_mode_equals_enumeration(oracle_mod):
    sc = scenes.room(n_cyl=6, nx=14, ny=11, seed=5, freqs=(2.4e9, 28e9))
    sc.max_order = 2
    ref = oracle_mod.evaluate(sc)
    cand = np.array([[a, -1, -1] for a in range(6)] + [[a, b, -1] for a in range(6) for b in range(6) if a != b],
                    dtype=np.int32)
    sc.candidates = cand
    got = oracle_mod.evaluate(sc)
    for r in range(sc.n_rx):
        assert np.array_equal(got.paths[r], ref.paths[r]), r
    assert np.max(np.abs(got.E - ref.E)) <= 1e-12 * np.max(np.abs(ref.E))


def _order3_brute(S, P, seq, k):
    """A genuine three-bounce path through the faces seq, by minimising the
    unfolded length over a point on each face; (valid, length, field)."""
    free = [[d for d in range(3) if d != FACES[f][0]] for f in seq]

    def pts(x):
        return [_on_face(f, x[2 * m:2 * m + 2]) for m, f in enumerate(seq)]

    def fun(x):
        q = [S] + pts(x) + [P]
        return sum(np.linalg.norm(q[m + 1] - q[m]) for m in range(4))

    x0 = []
    for m, f in enumerate(seq):
        x0 += [L_BOX[free[m][0]] / 2, L_BOX[free[m][1]] / 2]
    res = minimize(fun, x0=x0, method="BFGS", options=dict(gtol=1e-12))
    q = [S] + pts(res.x) + [P]
    n = [np.eye(3)[FACES[f][0]] for f in seq]
    ok = all(_inside(f, q[m + 1]) for m, f in enumerate(seq))
    for m in range(3):
        u = (q[m + 1] - q[m]) / np.linalg.norm(q[m + 1] - q[m])
        w = (q[m + 2] - q[m + 1]) / np.linalg.norm(q[m + 2] - q[m + 1])
        # (the law of reflection to the minimiser's accuracy; a minimiser
        # collapsed onto an edge between faces misses it by O(1))
        ok = ok and np.linalg.norm(np.cross(u - w, n[m])) < 1e-4 and np.linalg.norm(q[m + 2] - q[m + 1]) > 1e-3
    if not ok:
        return False, None, None
    d = (q[1] - S) / np.linalg.norm(q[1] - S)
    z = np.array([0, 0, 1.0])
    e = z - (z @ d) * d
    e /= np.linalg.norm(e)
    for m in range(3):
        e = -e + 2 * (n[m] @ e) * n[m]
    return True, res.fun, e * np.exp(-1j * k * res.fun) / res.fun


def test_order3_paths_match_brute_force_in_empty_box(oracle_mod):
    rng = np.random.default_rng(12)
    rx = np.stack([rng.uniform(0.5, 9.5, 2), rng.uniform(0.5, 7.5, 2), rng.uniform(0.3, 2.7, 2)], 1).astype(np.float32)
    sc = _box_scene(rx)
    cand = oracle_mod.candidates(sc, 20000, 3)
    sc.candidates = cand
    r = oracle_mod.evaluate(sc, enable=oracle_mod.EN_PLANAR, path_fields=True)
    k = 2 * np.pi * 2.4e9 / 299792458.0
    S = sc.tx.astype(np.float64)
    n_paths = 0
    for i in range(len(rx)):
        listed = {int(r.codes[i, j]): r.path_E[i, j, 0] for j in range(int(r.counts[i]))}
        o3 = {oracle_mod.decode(c)[1]: E for c, E in listed.items() if oracle_mod.decode(c)[0] == oracle_mod.PT_R3}
        for q, seq in enumerate(cand):
            if (seq >= 0).sum() != 3:
                continue
            ok, _, E = _order3_brute(S, rx[i].astype(np.float64), [int(f) for f in seq], k)
            assert ok == (q in o3), (i, seq, ok)
            if ok:
                assert np.max(np.abs(o3[q] - E)) < 1e-5 * np.max(np.abs(E))
                n_paths += 1
    assert n_paths >= 40, n_paths
