"""Pins of the oracle's wall -> creeping paths (a planar reflection feeding a
creeping ray: S -> Qw on a face -> Q1 -> surface ray -> Q2 -> P).

* Image theory (PEC): above a perfectly conducting plane, the reflected wave
  of a source of polarisation p at S is the wave of an image source at the
  mirror point S' with polarisation p' = -p + 2 (n.p) n (tangential part
  reversed, normal part kept).  So each wall -> creeping path's field equals
  the field of the creeping ray of a scene with no plane, the source moved
  to S' with polarisation p' -- a different code path of the oracle (its
  source polarisation, not the reflection routine), with the same turn count.
  The path exists unless the leg S -> Qw or Qw -> Q1 is blocked (checked by
  dense point sampling).
* Dielectric plane (real eps): the reflected polarisation splits into its
  parts along e_perp = unit(n x s_i) and e_par (Fresnel's angle forms with
  Snell's law, not the oracle's formula); the field is the sum of the two
  image-source creeping fields with those unit polarisations, each weighted
  by its coefficient.
* Geometry: Qw is the point of the plane that minimises |S - Qw| + |Qw - Q1|
  (found here by a direct search), and the path exists only while Qw lies in
  the face (a small face, checked against its rectangle).
"""
from types import SimpleNamespace

import numpy as np
import pytest

from paper_2310_10578_gb300.scenes import BODY_SPHERE, BODY_CYLINDER

EN_CREEP = 8 | 16


def _scene(tri, face, bodies, tx, pol, rx, freqs=(2.4e9, 5.8e9), face_eps=None, max_enc=0, wall=False):
    return SimpleNamespace(tri=np.asarray(tri, dtype=np.float64).reshape(-1, 3, 3),
                           tri_face=np.asarray(face, dtype=np.int32),
                           bodies=np.asarray(bodies, dtype=np.float64).reshape(-1, 6),
                           tx=np.asarray(tx, dtype=np.float64), pol=np.asarray(pol, dtype=np.float64),
                           freqs=np.asarray(freqs, dtype=np.float64), rx=np.asarray(rx, dtype=np.float32),
                           max_order=0, face_eps=face_eps, max_enc=max_enc, wall_creep=wall)


def _quad(c, u, v, half_u, half_v):
    """Two triangles of the rectangle c +- half_u u +- half_v v (one face)."""
    c, u, v = (np.asarray(x, dtype=np.float64) for x in (c, u, v))
    q = [c - half_u * u - half_v * v, c + half_u * u - half_v * v, c + half_u * u + half_v * v,
         c - half_u * u + half_v * v]
    return np.array([[q[0], q[1], q[2]], [q[0], q[2], q[3]]]), np.zeros(2, dtype=np.int32)


def _fields(oracle_mod, sc, enable):
    r = oracle_mod.evaluate(sc, enable=enable, path_fields=True)
    return [{int(r.codes[i, j]): r.path_E[i, j] for j in range(int(r.counts[i]))} for i in range(len(sc.rx))]


def _code(t, b, n):
    return (int(t) << 56) | (int(b) << 28) | int(n)


def _rx_grid(xs, ys, zs):
    X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


CASES = {
    # sphere over a floor (z = 0); receivers behind it, in the shadows of both
    # the source and its image
    "sphere_floor": dict(plane=((0, 0, 0), (1, 0, 0), (0, 1, 0)), normal=(0, 0, 1),
                         body=[BODY_SPHERE, 0.0, 0.0, 1.2, 0.5, 0.0], tx=(3.0, 0.5, 1.5),
                         rx=_rx_grid(np.linspace(-4.0, -1.5, 6), np.linspace(-1.2, 1.2, 5), np.linspace(0.5, 4.5, 9))),
    # cylinder beside a wall (x = 0); the image source is behind the wall
    "cylinder_wall": dict(plane=((0, 0, 1.5), (0, 1, 0), (0, 0, 1)), normal=(1, 0, 0),
                          body=[BODY_CYLINDER, 1.5, 0.0, 0.0, 0.3, 3.0], tx=(3.0, 0.75, 1.0),
                          rx=_rx_grid(np.linspace(0.3, 3.5, 9), np.linspace(-3.0, -0.6, 7), [0.6, 1.2, 2.0])),
}


def _case(name, face_eps=None, max_enc=0, size=50.0):
    cs = CASES[name]
    c, u, v = cs["plane"]
    tri, face = _quad(c, u, v, size, size)
    n = np.asarray(cs["normal"], dtype=np.float64)
    tx = np.asarray(cs["tx"], dtype=np.float64)
    pol = np.array([0.25, 0.5, 0.75])
    S_img = tx - 2 * ((tx - np.asarray(c)) @ n) * n
    return cs, tri, face, n, tx, pol, S_img


@pytest.mark.parametrize("name", sorted(CASES))
def test_pec_wall_creep_is_the_image_sources_creeping_ray(oracle_mod, name):
    cs, tri, face, n, tx, pol, S_img = _case(name)
    pol_img = -pol + 2 * (n @ pol) * n
    A = _scene(tri, face, [cs["body"]], tx, pol, cs["rx"], max_enc=1, wall=True)
    B = _scene(np.zeros((0, 3, 3)), np.zeros(0), [cs["body"]], S_img, pol_img, cs["rx"], max_enc=1)
    fa = _fields(oracle_mod, A, EN_CREEP)
    fb = _fields(oracle_mod, B, EN_CREEP)
    n_cmp = n_blocked = 0
    for i, P in enumerate(cs["rx"].astype(np.float32).astype(np.float64)):
        for turns in (0, 1):
            for t_w, t_c in ((oracle_mod.PT_WCP, oracle_mod.PT_CP), (oracle_mod.PT_WCM, oracle_mod.PT_CM)):
                cw, cc = _code(t_w, 0, turns), _code(t_c, 0, turns)
                if cw in fa[i]:
                    assert cc in fb[i]
                    ref = fb[i][cc]
                    assert np.max(np.abs(fa[i][cw] - ref)) <= 1e-12 * np.max(np.abs(ref)) + 1e-300
                    n_cmp += 1
                elif cc in fb[i]:
                    # the image source's ray exists: a leg from the real source
                    # to the plane, or on to Q1, must be blocked by the body
                    g = oracle_mod.body_creeping(cs["body"], S_img, P, 0 if t_c == oracle_mod.PT_CP else 1, turns)
                    Q1 = g["Q1"]
                    dI, dQ = (S_img - tri[0, 0]) @ n, (Q1 - tri[0, 0]) @ n
                    Qw = S_img + (Q1 - S_img) * dI / (dI - dQ)
                    s = np.linspace(1e-6, 1 - 1e-6, 20001)[:, None]
                    c, a = np.asarray(cs["body"][1:4]), cs["body"][4]
                    pts1 = tx + s * (Qw - tx)
                    pts2 = Qw + s[:-2000] * (Q1 - Qw)         # (short of Q1, where the leg touches the body)
                    if cs["body"][0] == BODY_SPHERE:
                        hit = np.any(np.linalg.norm(pts1 - c, axis=1) < a) or np.any(np.linalg.norm(pts2 - c, axis=1) < a)
                    else:
                        inside = lambda q: (np.hypot(q[:, 0] - c[0], q[:, 1] - c[1]) < a) & (q[:, 2] > c[2]) & \
                            (q[:, 2] < c[2] + cs["body"][5])
                        hit = np.any(inside(pts1)) or np.any(inside(pts2))
                    assert hit or dQ * ((tx - tri[0, 0]) @ n) <= 0, (i, turns)
                    n_blocked += 1
    assert n_cmp >= 20, n_cmp


@pytest.mark.parametrize("eps", [2.5, 7.0])
def test_dielectric_wall_creep_splits_into_fresnel_parts(oracle_mod, eps):
    cs, tri, face, n, tx, pol, S_img = _case("sphere_floor")
    rx = cs["rx"][::7]
    A = _scene(tri, face, [cs["body"]], tx, pol, rx, face_eps=[(1.0, eps, 0.0)], wall=True)
    fa = _fields(oracle_mod, A, EN_CREEP)
    n_cmp = 0
    for i, P in enumerate(rx.astype(np.float32).astype(np.float64)):
        for t_w, t_c, d in ((oracle_mod.PT_WCP, oracle_mod.PT_CP, 0), (oracle_mod.PT_WCM, oracle_mod.PT_CM, 1)):
            cw = _code(t_w, 0, 0)
            if cw not in fa[i]:
                continue
            g = oracle_mod.body_creeping(cs["body"], S_img, P, d, 0)
            Q1 = g["Q1"]
            dI, dQ = (S_img - tri[0, 0]) @ n, (Q1 - tri[0, 0]) @ n
            Qw = S_img + (Q1 - S_img) * dI / (dI - dQ)
            si = (Qw - tx) / np.linalg.norm(Qw - tx)
            sr = (Q1 - Qw) / np.linalg.norm(Q1 - Qw)
            e0 = pol - (pol @ si) * si
            e0 /= np.linalg.norm(e0)
            ep = np.cross(n, si)
            ep /= np.linalg.norm(ep)
            epi, epr = np.cross(ep, si), np.cross(ep, sr)
            inc = np.arccos(abs(si @ n))
            tr = np.arcsin(np.sin(inc) / np.sqrt(eps))
            gs = -np.sin(inc - tr) / np.sin(inc + tr)
            gp = np.tan(inc - tr) / np.tan(inc + tr)
            tot = 0
            for q, w in ((ep, gs * (e0 @ ep)), (epr, gp * (e0 @ epi))):
                B = _scene(np.zeros((0, 3, 3)), np.zeros(0), [cs["body"]], S_img, q, rx[i:i + 1])
                tot = tot + w * _fields(oracle_mod, B, EN_CREEP)[0][_code(t_c, 0, 0)]
            assert np.max(np.abs(fa[i][cw] - tot)) <= 1e-10 * np.max(np.abs(tot)), i
            n_cmp += 1
    assert n_cmp >= 5, n_cmp


def test_reflection_point_minimises_length_and_lies_in_face(oracle_mod):
    """A small floor face (2 x 2 m round the sphere's foot): Qw from a direct
    search over the plane; the path listed exactly when Qw is in the face."""
    from scipy.optimize import minimize
    cs, _, _, n, tx, pol, S_img = _case("sphere_floor")
    tri, face = _quad((0.5, 0, 0), (1, 0, 0), (0, 1, 0), 1.0, 1.0)
    A = _scene(tri, face, [cs["body"]], tx, pol, cs["rx"], wall=True)
    r = oracle_mod.evaluate(A, enable=EN_CREEP)
    listed = [set(int(c) for c in cs_) for cs_ in r.paths]
    n_in = n_out = 0
    for i, P in enumerate(cs["rx"].astype(np.float32).astype(np.float64)):
        for t_w, d in ((oracle_mod.PT_WCP, 0), (oracle_mod.PT_WCM, 1)):
            g = oracle_mod.body_creeping(cs["body"], S_img, P, d, 0)
            if g is None:
                assert _code(t_w, 0, 0) not in listed[i]
                continue
            Q1 = g["Q1"]
            res = minimize(lambda q: np.linalg.norm(tx - [q[0], q[1], 0]) + np.linalg.norm([q[0], q[1], 0] - Q1),
                           x0=[0.0, 0.0], method="Nelder-Mead", options=dict(xatol=1e-10, fatol=1e-13, maxiter=4000))
            Qw = np.array([res.x[0], res.x[1], 0.0])
            dI, dQ = (S_img - tri[0, 0]) @ n, (Q1 - tri[0, 0]) @ n
            Qw_img = S_img + (Q1 - S_img) * dI / (dI - dQ)
            assert np.linalg.norm(Qw - Qw_img) < 1e-6
            inside = -0.5 < Qw_img[0] < 1.5 and -1.0 < Qw_img[1] < 1.0
            margin = min(abs(Qw_img[0] + 0.5), abs(Qw_img[0] - 1.5), abs(Qw_img[1] + 1.0), abs(Qw_img[1] - 1.0))
            if margin < 1e-9:
                continue
            if inside:
                n_in += 1
                # (a leg may still be blocked by the sphere itself)
            else:
                n_out += 1
                assert _code(t_w, 0, 0) not in listed[i]
    assert n_in >= 5 and n_out >= 5, (n_in, n_out)
