"""Pins of the oracle's ray geometry against first principles.

* Generalised Fermat principle (the paper keeps the ray paths that satisfy it,
  Sec. III.B, Fig. 1): the creeping path S -> Q1 -> geodesic -> Q2 -> P and
  the reflection path S -> Q -> P are stationary in length under every
  perturbation of their surface points; the incident/shed segments are tangent.
* Ray tubes: the GO reflected amplitude^2 (Eq. 3) equals the solid angle per
  unit area of a finite-difference ray tube traced by brute force; the
  transverse spreading of the cylinder's creeping rays equals that of a
  finite-difference family of helices traced in 3-D.
* Visibility: segment-vs-body decisions equal dense point sampling.
"""
import numpy as np
import pytest

from paper_2310_10578_gb300.scenes import BODY_SPHERE, BODY_CYLINDER

RNG = np.random.default_rng(20231016)


def _rand_sphere_case(rng, shadow):
    c = rng.uniform(-1, 1, 3)
    a = rng.uniform(0.2, 0.6)
    while True:
        S = c + rng.normal(size=3) * 2.0
        P = c + rng.normal(size=3) * 2.0
        if np.linalg.norm(S - c) < a * 1.3 or np.linalg.norm(P - c) < a * 1.3:
            continue
        ws, wp = S - c, P - c
        gam = np.arccos(np.clip(ws @ wp / np.linalg.norm(ws) / np.linalg.norm(wp), -1, 1))
        lit = gam < np.arccos(a / np.linalg.norm(ws)) + np.arccos(a / np.linalg.norm(wp))
        if lit != shadow:
            return np.array([BODY_SPHERE, *c, a, 0.0]), S, P


def _rand_cyl_case(rng):
    c = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), 0.0])
    a = rng.uniform(0.15, 0.35)
    h = 3.0
    while True:
        S = np.array([c[0], c[1], 0]) + np.array([*rng.normal(size=2) * 1.5, rng.uniform(0.5, 2.5)])
        P = np.array([c[0], c[1], 0]) + np.array([*rng.normal(size=2) * 1.5, rng.uniform(0.5, 2.5)])
        if np.hypot(*(S - c)[:2]) > 1.3 * a and np.hypot(*(P - c)[:2]) > 1.3 * a:
            return np.array([BODY_CYLINDER, *c, a, h]), S, P


def _tangent_basis(n):
    t = np.array([1.0, 0, 0]) if abs(n[0]) < 0.9 else np.array([0, 1.0, 0])
    e1 = np.cross(n, t); e1 /= np.linalg.norm(e1)
    return e1, np.cross(n, e1)


def _rot_on_sphere(c, a, Q, e, h):
    v = (Q - c) + h * e
    return c + a * v / np.linalg.norm(v)


@pytest.mark.parametrize("trial", range(12))
def test_sphere_creeping_satisfies_fermat(oracle_mod, trial):
    rng = np.random.default_rng(100 + trial)
    body, S, P = _rand_sphere_case(rng, shadow=bool(trial % 2))
    c, a = body[1:4], body[4]
    for d in (0, 1):
        g = oracle_mod.body_creeping(body, S, P, d)
        if g is None:
            continue
        Q1, Q2 = g["Q1"], g["Q2"]
        assert abs(np.linalg.norm(Q1 - c) - a) < 1e-12 and abs(np.linalg.norm(Q2 - c) - a) < 1e-12
        assert abs((Q1 - S) @ g["n1"]) < 1e-10 * np.linalg.norm(Q1 - S)      # tangent incidence
        assert abs((P - Q2) @ g["n2"]) < 1e-10 * np.linalg.norm(P - Q2)      # tangent shedding
        assert abs(g["sp"] - np.linalg.norm(Q1 - S)) < 1e-12
        assert abs(g["sq"] - np.linalg.norm(P - Q2)) < 1e-12
        long_arc = g["t"] / a > np.pi

        def length(q1, q2):
            th = np.arccos(np.clip((q1 - c) @ (q2 - c) / a / a, -1, 1))
            arc = 2 * np.pi - th if long_arc else th
            return np.linalg.norm(q1 - S) + a * arc + np.linalg.norm(P - q2)

        assert abs(length(Q1, Q2) - (g["sp"] + g["t"] + g["sq"])) < 1e-10
        h = 1e-5
        for Q, which in ((Q1, 0), (Q2, 1)):
            for e in _tangent_basis((Q - c) / a):
                qp = _rot_on_sphere(c, a, Q, e, h)
                qm = _rot_on_sphere(c, a, Q, e, -h)
                Lp = length(qp, Q2) if which == 0 else length(Q1, qp)
                Lm = length(qm, Q2) if which == 0 else length(Q1, qm)
                assert abs(Lp - Lm) / (2 * h) < 1e-6


@pytest.mark.parametrize("trial", range(12))
def test_cylinder_creeping_satisfies_fermat(oracle_mod, trial):
    rng = np.random.default_rng(200 + trial)
    body, S, P = _rand_cyl_case(rng)
    c, a = body[1:4], body[4]
    found = 0
    for d in (0, 1):
        g = oracle_mod.body_creeping(body, S, P, d)
        if g is None:
            continue
        found += 1
        Q1, Q2 = g["Q1"], g["Q2"]
        for Q in (Q1, Q2):
            assert abs(np.hypot(*(Q - c)[:2]) - a) < 1e-12
        assert abs((Q1 - S) @ g["n1"]) < 1e-10 * np.linalg.norm(Q1 - S)
        assert abs((P - Q2) @ g["n2"]) < 1e-10 * np.linalg.norm(P - Q2)
        dphi0 = np.sqrt(max(g["t"] ** 2 - (Q2[2] - Q1[2]) ** 2, 0.0)) / a
        f1 = np.array([*(Q1 - S)[:2], 0.0]); f1 /= np.linalg.norm(f1)   # forward tangent at Q1
        f2 = np.array([*(P - Q2)[:2], 0.0]); f2 /= np.linalg.norm(f2)   # forward tangent at Q2

        def point(Q, f, dphi, dz):
            n = np.array([*(Q - c)[:2], 0.0]) / a
            ang = dphi / a
            q = c[:2] + a * (np.cos(ang) * n[:2] + np.sin(ang) * f[:2])
            return np.array([q[0], q[1], Q[2] + dz])

        def length(d1, z1, d2, z2):
            q1, q2 = point(Q1, f1, d1, z1), point(Q2, f2, d2, z2)
            travel = a * dphi0 - d1 + d2
            return np.linalg.norm(q1 - S) + np.hypot(travel, q2[2] - q1[2]) + np.linalg.norm(P - q2)

        assert abs(length(0, 0, 0, 0) - (g["sp"] + g["t"] + g["sq"])) < 1e-10
        h = 1e-5
        for k in range(4):
            dp = np.zeros(4); dp[k] = h
            assert abs(length(*dp) - length(*(-dp))) / (2 * h) < 1e-6
    if trial == 0:
        assert found >= 1


@pytest.mark.parametrize("trial", range(10))
def test_reflection_point_law_of_reflection(oracle_mod, trial):
    rng = np.random.default_rng(300 + trial)
    if trial % 2 == 0:
        body, S, P = _rand_sphere_case(rng, shadow=False)
    else:
        for _ in range(100):
            body, S, P = _rand_cyl_case(rng)
            if oracle_mod.body_reflection(body, S, P) is not None:
                break
    g = oracle_mod.body_reflection(body, S, P)
    assert g is not None
    Q, n = g["Q"], g["n"]
    si, sr = (S - Q) / np.linalg.norm(S - Q), (P - Q) / np.linalg.norm(P - Q)
    assert abs(si @ n - sr @ n) < 1e-9                 # equal angles
    assert abs(np.cross(si, sr) @ n) < 1e-9            # coplanar with the normal
    assert si @ n > 0 and sr @ n > 0


@pytest.mark.parametrize("trial", range(8))
def test_reflection_with_receiver_on_the_source_axis(oracle_mod, trial):
    """Degenerate frames: a receiver straight below the source (the same x, y,
    so on the S-c line of every vertical cylinder in projection) and a receiver
    on a sphere's S-c axis.  The reflection is then a retro-reflection in
    projection: the law of reflection still holds, the reflection point lies on
    the surface, and for the cylinder it sits half way down (equal horizontal
    runs).  Float inputs, as the scenes hold them."""
    rng = np.random.default_rng(700 + trial)
    c = np.array([rng.uniform(-3, 3), rng.uniform(-3, 3), 0.0], dtype=np.float32).astype(np.float64)
    a = float(np.float32(rng.uniform(0.15, 0.3)))
    S = np.array([1.0, 1.0, 2.0])
    if trial % 2 == 0:
        body = np.array([BODY_CYLINDER, *c, a, 1.9])
        P = np.array([S[0], S[1], float(np.float32(rng.uniform(0.3, 1.7)))])
    else:
        body = np.array([BODY_SPHERE, *c, a, 0.0])
        u = (S - c) / np.linalg.norm(S - c)
        P = (c + u * float(rng.uniform(1.5, 3.0)) * a).astype(np.float32).astype(np.float64)
    g = oracle_mod.body_reflection(body, S, P)
    assert g is not None
    Q, n = g["Q"], g["n"]
    si, sr = (S - Q) / np.linalg.norm(S - Q), (P - Q) / np.linalg.norm(P - Q)
    assert abs(si @ n - sr @ n) < 1e-9
    assert abs(np.cross(si, sr) @ n) < 1e-9            # coplanar with the normal
    if body[0] == BODY_CYLINDER:
        assert abs(np.hypot(*(Q - c)[:2]) - a) < 1e-12 and n[2] == 0.0
        assert abs(Q[2] - 0.5 * (S[2] + P[2])) < 1e-9
    else:
        assert abs(np.linalg.norm(Q - c) - a) < 1e-12
    # the creeping rays' frame stays orthonormal: both surface points on the body
    for direction in (0, 1):
        cg = oracle_mod.body_creeping(body, S, P, direction)
        if cg is None:
            continue
        for key in ("Q1", "Q2"):
            rr = np.hypot(*(cg[key] - c)[:2]) if body[0] == BODY_CYLINDER else np.linalg.norm(cg[key] - c)
            assert abs(rr - a) < 1e-12


def _ray_body(S, d, body):
    """First intersection of the ray S + tau d with the body surface (brute force)."""
    c, a = body[1:4], body[4]
    if body[0] == BODY_SPHERE:
        w = S - c
        b = w @ d; cc = w @ w - a * a
        tau = -b - np.sqrt(b * b - cc)
        Q = S + tau * d
        return Q, (Q - c) / a
    w = (S - c)[:2]; dh = d[:2]
    qa = dh @ dh; qb = 2 * w @ dh; qc = w @ w - a * a
    tau = (-qb - np.sqrt(qb * qb - 4 * qa * qc)) / (2 * qa)
    Q = S + tau * d
    n = np.array([*(Q - c)[:2], 0.0]) / a
    return Q, n


@pytest.mark.parametrize("trial", range(10))
def test_reflection_amplitude_equals_ray_tube(oracle_mod, trial):
    rng = np.random.default_rng(400 + trial)
    if trial % 2 == 0:
        body, S, P = _rand_sphere_case(rng, shadow=False)
    else:
        for _ in range(100):
            body, S, P = _rand_cyl_case(rng)
            if oracle_mod.body_reflection(body, S, P) is not None:
                break
    g = oracle_mod.body_reflection(body, S, P)
    Q = g["Q"]
    si, sr = np.linalg.norm(Q - S), np.linalg.norm(P - Q)
    rho1 = 1 / (1 / si + g["inv_f1"]); rho2 = 1 / (1 / si + g["inv_f2"])
    amp2 = (1 / si ** 2) * rho1 * rho2 / ((rho1 + sr) * (rho2 + sr))
    d0 = (Q - S) / si
    e1, e2 = _tangent_basis(d0)
    r0 = (P - Q) / sr

    def land(al, be):
        d = d0 + al * e1 + be * e2
        d /= np.linalg.norm(d)
        q, n = _ray_body(S, d, body)
        r = d - 2 * (d @ n) * n
        lam = ((P - q) @ r0) / (r @ r0)
        return q + lam * r, d

    h = 1e-6
    Xa = (land(h, 0)[0] - land(-h, 0)[0]) / (2 * h)
    Xb = (land(0, h)[0] - land(0, -h)[0]) / (2 * h)
    Da = (land(h, 0)[1] - land(-h, 0)[1]) / (2 * h)
    Db = (land(0, h)[1] - land(0, -h)[1]) / (2 * h)
    area = np.linalg.norm(np.cross(Xa, Xb))
    solid = np.linalg.norm(np.cross(Da, Db))
    assert abs(solid / area / amp2 - 1) < 1e-5


@pytest.mark.parametrize("trial", range(8))
def test_cylinder_creeping_transverse_spreading(oracle_mod, trial):
    """Family of creeping rays grazing the same generator line at varying height
    (the eta direction of the ray tube), traced as explicit 3-D helices."""
    rng = np.random.default_rng(500 + trial)
    for _ in range(200):
        body, S, P = _rand_cyl_case(rng)
        d = trial % 2
        g = oracle_mod.body_creeping(body, S, P, d)
        if g is not None:
            break
    assert g is not None
    c, a = body[1:4], body[4]
    Q1, n1, Q2 = g["Q1"], g["n1"], g["Q2"]
    dphi = np.sqrt(max(g["t"] ** 2 - (Q2[2] - Q1[2]) ** 2, 0.0)) / a
    f1 = np.array([*(Q1 - S)[:2], 0.0]); f1 /= np.linalg.norm(f1)

    def trace(z1):
        q1 = np.array([Q1[0], Q1[1], z1])
        dv = (q1 - S) / np.linalg.norm(q1 - S)          # grazes the same generator line
        dh = np.hypot(dv[0], dv[1])
        tau = a * dphi / dh                              # helix arc length for the same travel
        ang = dphi
        nn = n1[:2] * np.cos(ang) + f1[:2] * np.sin(ang)
        ff = -n1[:2] * np.sin(ang) + f1[:2] * np.cos(ang)
        q2 = np.array([*(c[:2] + a * nn), z1 + dv[2] * tau])
        d2 = np.array([*(ff * dh), dv[2]])
        return q1, q2 + g["sq"] * d2, dv, d2

    h = 1e-6
    q1p, pp, dvp, d2p = trace(Q1[2] + h)
    q1m, pm, dvm, d2m = trace(Q1[2] - h)
    q10, p0, dv0, d20 = trace(Q1[2])
    assert np.linalg.norm(p0 - P) < 1e-9                 # the central ray reaches the receiver
    w1 = (q1p - q1m) / (2 * h); w1 -= (w1 @ dv0) * dv0
    wP = (pp - pm) / (2 * h); wP -= (wP @ d20) * d20
    ratio = np.linalg.norm(wP) / np.linalg.norm(w1)
    # oracle amplitude without the normal-plane 1/sqrt(s) and incident 1/s'
    transverse = (g["amp"] * g["sp"] * np.sqrt(g["sq"])) ** 2
    assert abs(transverse * ratio - 1) < 1e-6


@pytest.mark.parametrize("trial", range(60))
def test_segment_body_visibility_matches_sampling(oracle_mod, trial):
    rng = np.random.default_rng(600 + trial)
    if trial % 2:
        body = np.array([BODY_SPHERE, *rng.uniform(-0.3, 0.3, 3), rng.uniform(0.2, 0.5), 0.0])
    else:
        body = np.array([BODY_CYLINDER, *rng.uniform(-0.3, 0.3, 2), -0.5, rng.uniform(0.2, 0.5), 1.0])
    A = rng.uniform(-1.2, 1.2, 3)
    B = rng.uniform(-1.2, 1.2, 3)
    ts = np.linspace(1e-6, 1 - 1e-6, 200001)
    X = A[None] + ts[:, None] * (B - A)[None]
    c, a = body[1:4], body[4]
    if body[0] == BODY_SPHERE:
        margin = a - np.linalg.norm(X - c, axis=1)
    else:
        margin = np.minimum(np.minimum(a - np.hypot(X[:, 0] - c[0], X[:, 1] - c[1]), X[:, 2] - c[2]),
                            c[2] + body[5] - X[:, 2])
    if np.min(np.abs(margin)) < 1e-3 and np.max(margin) < 1e-3:
        pytest.skip("tangent within sampling resolution")
    inside_any = bool(np.max(margin) > 0)
    if abs(np.max(margin)) < 1e-3:
        pytest.skip("near-tangent")
    assert oracle_mod.seg_hits_body(body, A, B) == inside_any
