"""Pins of the oracle's creeping rays with extra full turns round a body
(the multiply-encircling rays of the smooth-surface UTD, Sec. III.B): a
creeping ray may wind round a convex body any number of times before it
sheds towards the receiver.

* Cylinder: the ray is a helix on the surface, a straight line when the
  surface is unrolled.  With n extra turns the unrolled line is 2 pi a n
  longer in the circumferential direction.  Checked from first principles:
  the attachment and shedding points are tangency points, the path is
  stationary in length (generalised Fermat), the surface length equals that
  of a densely sampled helix of n + dphi/(2 pi) turns, and the ray exists
  exactly when both surface points lie between the cylinder's base and top
  (brute force over heights).
* Sphere: the geodesic is a great circle, so the attachment and shedding
  points do not move with n; the surface length is the base ray's plus
  2 pi a n, and rotating Q1 about the great circle's axis by the arc angle
  lands on Q2 after the extra turns.
* Field: turn n of a ray carries less amplitude than turn n - 1 (the Fock
  attenuation along the longer arc), the scene total with no extra turns is
  unchanged, and every extra-turn path is listed as (CP or CM, body, n).
"""
import numpy as np
import pytest

from paper_2310_10578_gb300 import scenes
from paper_2310_10578_gb300.scenes import BODY_SPHERE, BODY_CYLINDER


def _cyl_case(rng, h=3.0):
    c = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), 0.0])
    a = rng.uniform(0.15, 0.35)
    while True:
        S = np.array([c[0], c[1], 0]) + np.array([*rng.normal(size=2) * 1.5, rng.uniform(0.5, 2.5)])
        P = np.array([c[0], c[1], 0]) + np.array([*rng.normal(size=2) * 1.5, rng.uniform(0.5, 2.5)])
        if np.hypot(*(S - c)[:2]) > 1.3 * a and np.hypot(*(P - c)[:2]) > 1.3 * a:
            return np.array([BODY_CYLINDER, *c, a, h]), S, P


def _helix_length(c, a, Q1, Q2, turns_total, sign, n=20000):
    """Polyline length of the helix from Q1 to Q2 winding `turns_total` turns
    (sign +1 counter-clockwise seen from +z)."""
    ang0 = np.arctan2(Q1[1] - c[1], Q1[0] - c[0])
    u = np.linspace(0.0, 1.0, n + 1)
    ang = ang0 + sign * 2 * np.pi * turns_total * u
    pts = np.stack([c[0] + a * np.cos(ang), c[1] + a * np.sin(ang), Q1[2] + (Q2[2] - Q1[2]) * u], axis=1)
    end_ok = np.linalg.norm(pts[-1] - Q2)
    return np.sum(np.linalg.norm(np.diff(pts, axis=0), axis=1)), end_ok


@pytest.mark.parametrize("trial", range(10))
def test_cylinder_extra_turns_first_principles(oracle_mod, trial):
    rng = np.random.default_rng(300 + trial)
    body, S, P = _cyl_case(rng, h=50.0)          # tall: every turn stays on the body
    c, a = body[1:4], body[4]
    for d in (0, 1):
        g0 = oracle_mod.body_creeping(body, S, P, d, 0)
        if g0 is None:
            continue
        for n in (1, 2, 3):
            g = oracle_mod.body_creeping(body, S, P, d, n)
            assert g is not None
            Q1, Q2 = g["Q1"], g["Q2"]
            # the same azimuths as the base ray (tangency from S and to P)
            for Q, Q0 in ((Q1, g0["Q1"]), (Q2, g0["Q2"])):
                assert abs(np.hypot(*(Q - c)[:2]) - a) < 1e-12
                assert np.allclose(Q[:2], Q0[:2], atol=1e-12)
            assert abs((Q1 - S) @ g["n1"]) < 1e-10 * np.linalg.norm(Q1 - S)
            assert abs((P - Q2) @ g["n2"]) < 1e-10 * np.linalg.norm(P - Q2)
            # the unrolled arc: the base arc plus n full circumferences
            arc0 = np.sqrt(max(g0["t"] ** 2 - (g0["Q2"][2] - g0["Q1"][2]) ** 2, 0.0))
            arc = np.sqrt(max(g["t"] ** 2 - (Q2[2] - Q1[2]) ** 2, 0.0))
            assert abs(arc - (arc0 + 2 * np.pi * a * n)) < 1e-9
            # surface length = a densely sampled helix of that many turns, in
            # the direction the base ray goes round
            n1 = (g0["Q1"] - c)[:2] / a
            f1 = (g0["Q1"] - S)[:2]
            sign = 1.0 if (n1[0] * f1[1] - n1[1] * f1[0]) > 0 else -1.0
            L, end_err = _helix_length(c, a, Q1, Q2, arc / (2 * np.pi * a), sign)
            assert end_err < 1e-9 and abs(L - g["t"]) < 1e-6 * g["t"]
            # Fermat: stationary under moving either surface point along the
            # surface (azimuth and height)
            f2 = (P - Q2)[:2]

            def point(Q, f, dphi, dz):
                nn = np.array([*(Q - c)[:2], 0.0]) / a
                ff = np.array([*f, 0.0]) / np.linalg.norm(f)
                ang = dphi / a
                q = c[:2] + a * (np.cos(ang) * nn[:2] + np.sin(ang) * ff[:2])
                return np.array([q[0], q[1], Q[2] + dz])

            def length(d1, z1, d2, z2):
                q1, q2 = point(Q1, f1, d1, z1), point(Q2, f2, d2, z2)
                travel = arc - d1 + d2
                return np.linalg.norm(q1 - S) + np.hypot(travel, q2[2] - q1[2]) + np.linalg.norm(P - q2)

            assert abs(length(0, 0, 0, 0) - (g["sp"] + g["t"] + g["sq"])) < 1e-10
            hh = 1e-5
            for k in range(4):
                dp = np.zeros(4); dp[k] = hh
                assert abs(length(*dp) - length(*(-dp))) / (2 * hh) < 1e-6


@pytest.mark.parametrize("trial", range(6))
def test_cylinder_extra_turns_exist_by_height(oracle_mod, trial):
    """A short cylinder: turn n exists iff both helix end points lie on the
    side wall (0 <= z - base <= height), computed here from the unrolled line."""
    rng = np.random.default_rng(400 + trial)
    body, S, P = _cyl_case(rng, h=3.0)
    body[3] = rng.uniform(0.2, 1.2)              # base height
    body[5] = rng.uniform(0.4, 1.5)              # height
    c, a = body[1:4], body[4]
    for d in (0, 1):
        tall = body.copy(); tall[3] = -100.0; tall[5] = 1000.0
        for n in range(4):
            gt = oracle_mod.body_creeping(tall, S, P, d, n)
            g = oracle_mod.body_creeping(body, S, P, d, n)
            if gt is None:
                assert g is None
                continue
            ds = np.sqrt(np.hypot(*(S - c)[:2]) ** 2 - a * a)
            dp = np.sqrt(np.hypot(*(P - c)[:2]) ** 2 - a * a)
            arc = np.sqrt(max(gt["t"] ** 2 - (gt["Q2"][2] - gt["Q1"][2]) ** 2, 0.0))
            H = ds + arc + dp
            z1 = S[2] + (P[2] - S[2]) * ds / H
            z2 = S[2] + (P[2] - S[2]) * (ds + arc) / H
            on = all(body[3] <= z <= body[3] + body[5] for z in (z1, z2))
            assert (g is not None) == on, (n, z1, z2)
            if g is not None:
                assert abs(g["Q1"][2] - z1) < 1e-9 and abs(g["Q2"][2] - z2) < 1e-9


@pytest.mark.parametrize("trial", range(6))
def test_sphere_extra_turns_great_circle(oracle_mod, trial):
    rng = np.random.default_rng(500 + trial)
    c = rng.uniform(-1, 1, 3)
    a = rng.uniform(0.2, 0.6)
    S = c + np.array([2.5, 0.3, -0.2]) * rng.uniform(1.0, 1.5)
    P = c + np.array([-2.0, rng.uniform(-1, 1), rng.uniform(-1, 1)])
    body = np.array([BODY_SPHERE, *c, a, 0.0])
    for d in (0, 1):
        g0 = oracle_mod.body_creeping(body, S, P, d, 0)
        if g0 is None:
            continue
        for n in (1, 2):
            g = oracle_mod.body_creeping(body, S, P, d, n)
            assert g is not None
            assert np.allclose(g["Q1"], g0["Q1"], atol=1e-12) and np.allclose(g["Q2"], g0["Q2"], atol=1e-12)
            assert abs(g["t"] - (g0["t"] + 2 * np.pi * a * n)) < 1e-12
            # walk the great circle from Q1, in the plane of S, c and P, by the
            # arc angle: it ends on Q2
            u = (g["Q1"] - c) / a
            w = (g["Q1"] - S) / np.linalg.norm(g["Q1"] - S)      # travel direction, tangent at Q1
            ang = g["t"] / a
            end = c + a * (np.cos(ang) * u + np.sin(ang) * w)
            assert np.linalg.norm(end - g["Q2"]) < 1e-9


def _pcode(t, b, n):
    return (int(t) << 56) | (int(b) << 28) | int(n)


def test_extra_turn_fields_and_codes(oracle_mod):
    sc = scenes.sphere_ring(n_rx=96)
    sc.max_enc = 0
    r0 = oracle_mod.evaluate(sc, path_fields=True)
    sc.max_enc = 2
    r2 = oracle_mod.evaluate(sc, path_fields=True)
    n_extra = 0
    for r in range(sc.n_rx):
        base = set(int(x) for x in r0.paths[r])
        listed = set(int(x) for x in r2.paths[r])
        assert base <= listed
        pf = {int(r2.codes[r, j]): r2.path_E[r, j] for j in range(int(r2.counts[r]))}
        for code in listed - base:
            t, b, n = oracle_mod.decode(code)
            assert t in (oracle_mod.PT_CP, oracle_mod.PT_CM) and n in (1, 2)
            lo = _pcode(t, b, n - 1)
            assert lo in listed                     # the same ray with one turn fewer
            lo_abs = np.linalg.norm(pf[lo])        # (0 on the axis behind a sphere)
            assert np.linalg.norm(pf[code]) < lo_abs or np.linalg.norm(pf[code]) == lo_abs == 0.0
            n_extra += 1
    assert n_extra > 0
    # what the extra turns add is small against the base field
    assert np.all(np.linalg.norm(r2.E - r0.E, axis=1) <= 0.05 * r0.sabs + 1e-300)
