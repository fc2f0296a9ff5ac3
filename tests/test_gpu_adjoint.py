"""The adjoint (rt_backward and the autograd.Function over it) against the
FP64 oracle: gradients of a loss through the fields with respect to body
centres and radii, the transmitter position and the frequencies (FP32 dual
numbers by default; FP64 ones where a test says so), with the visibility of
the forward path list held fixed (tests/adjoint_ref.py:
central differences of the oracle's per-path fields, h = 1e-5 m).

Tolerance: 1e-3 relative, where the relative error of a gradient that is a
sum of contributions of both signs is taken against max(|reference|, 1e-3 x
the sum of the contributions' magnitudes).

The receivers are jittered (seeded, by up to 2 cm in x and y) off the regular
grid: on the grid some reflection points fall exactly on an edge between
faces, where a path exists on one side of any perturbation only and has no
central difference.
"""
import numpy as np
import pytest

import adjoint_ref
from paper_2310_10578_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

REL = 1e-3


@pytest.fixture(scope="module")
def creep():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_10578_gb300 import creep as c
    c.load()
    return c


def _jitter(sc, seed, scale=0.02):
    rng = np.random.default_rng(seed)
    sc.rx[:, :2] += rng.uniform(-scale, scale, (sc.n_rx, 2)).astype(np.float32)
    return sc


def _close(got, ref, absum, what):
    tol = REL * max(abs(ref), 1e-3 * absum) + 1e-15
    assert abs(got - ref) <= tol, "%s: gpu %.9e ref %.9e (|contributions| %.3e)" % (what, got, ref, absum)


def _forward(creep, sc, cap=256, precision=None):
    S = creep.Scene.from_scene(sc)
    rx = torch.tensor(sc.rx_soa(), device="cuda")
    opts = creep.options(max_order=sc.max_order, max_encirclements=getattr(sc, "max_enc", 0),
                         enable=creep.RT_EN_ALL | (creep.RT_EN_WALL_CREEP if getattr(sc, "wall_creep", False) else 0),
                         precision=creep.RT_PREC_FP32 if precision is None else precision)
    E = S.evaluate(rx, opts=opts)
    codes, counts, _ = S.paths(rx, cap=cap, opts=opts)
    torch.cuda.synchronize()
    c = codes.cpu().numpy().astype(np.uint64)
    n = counts.cpu().numpy()
    lists = [[int(x) for x in c[r, :min(int(n[r]), cap)]] for r in range(sc.n_rx)]
    return S, rx, opts, E, codes, counts, lists


def _check(creep, sc, bodies, seed, cap=256, tx=True, freqs=True, keep=None, precision=None):
    S, rx, opts, E, codes, counts, lists = _forward(creep, sc, cap, precision)
    if keep is not None:
        # the gradient through the listed paths that pass keep(code) only
        lists = [[c for c in cs if keep(c)] for cs in lists]
        cd = np.zeros((sc.n_rx, cap), dtype=np.uint64)
        for r, cs in enumerate(lists):
            cd[r, :len(cs)] = cs
        codes = torch.tensor(cd.view(np.int64), device="cuda").view(codes.dtype)
        counts = torch.tensor([len(cs) for cs in lists], dtype=counts.dtype, device="cuda")
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((len(sc.freqs), 3, sc.n_rx, 2)).astype(np.float32)
    gb, gt, gf = S.backward(rx, codes, counts, torch.tensor(g, device="cuda"), opts=opts)
    torch.cuda.synchronize()
    gb, gt, gf = gb.cpu().numpy(), gt.cpu().numpy(), gf.cpu().numpy()
    ref = adjoint_ref.vjp(sc, lists, g[..., 0].astype(np.float64) + 1j * g[..., 1], bodies=bodies, cap=cap,
                          tx=tx, freqs=freqs)
    assert ref["skipped"] <= 2, ref["skipped"]
    n_checked = 0
    for b in bodies:
        for k in range(4):
            _close(gb[b, k], ref["body"][b][k], ref["body_abs"][b][k], "body %d param %d" % (b, k))
            n_checked += ref["body_abs"][b][k] > 0
    if tx:
        for k in range(3):
            _close(gt[k], ref["tx"][k], ref["tx_abs"][k], "tx %d" % k)
    if freqs:
        for k in range(len(sc.freqs)):
            _close(gf[k], ref["f"][k], ref["f_abs"][k], "freq %d" % k)
    return n_checked, gb


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_adjoint_room_small(creep, oracle_mod, precision):
    # 12 cylinders, 24 x 20 receivers, two frequencies; every body's gradient,
    # with FP32 dual numbers (the default) and with FP64 ones
    sc = _jitter(scenes.room(n_cyl=12, nx=24, ny=20, freqs=(2.4e9, 28e9), seed=7), 11)
    prec = creep.RT_PREC_FP64 if precision == "fp64" else creep.RT_PREC_FP32
    n_checked, _ = _check(creep, sc, bodies=range(12), seed=1, precision=prec)
    assert n_checked >= 30


def test_adjoint_sphere(creep, oracle_mod):
    # one PEC sphere: direct ray, reflection and both creeping rays (no walls)
    sc = scenes.sphere_ring(n_rx=96, freq=5.8e9)
    sc.rx[:, 2] = 0.3                                       # off the plane of the source: a 3-D frame
    n_checked, gb = _check(creep, sc, bodies=[0], seed=2)
    assert n_checked == 4                                   # x, y, z and radius all move the field


def test_adjoint_extra_turns(creep, oracle_mod):
    """Creeping rays with one or two extra turns round a sphere (off the
    source's plane) and round the room's cylinders: the gradient through
    those paths alone."""
    sc = scenes.sphere_ring(n_rx=96, freq=2.4e9)
    sc.rx[:, 2] = 0.3
    sc.max_enc = 2
    extra = lambda c: (c >> 56) in (4, 5) and (c & 0xFFFFFFF) > 0
    n_checked, _ = _check(creep, sc, bodies=[0], seed=5, keep=extra)
    assert n_checked == 4
    sc = _jitter(scenes.room(n_cyl=12, nx=24, ny=20, freqs=(2.4e9,), seed=7), 11)
    sc.max_enc = 1
    n_checked, _ = _check(creep, sc, bodies=range(12), seed=6, keep=extra)
    assert n_checked >= 8


def _room_with_spheres(n_cyl, nx, ny, freqs, seed):
    """The room with every other cylinder replaced by a sphere of its radius
    centred 0.9 m above its foot."""
    sc = scenes.room(n_cyl=n_cyl, nx=nx, ny=ny, freqs=freqs, seed=seed)
    for k in range(0, n_cyl, 2):
        x, y, a = sc.bodies[k, 1], sc.bodies[k, 2], sc.bodies[k, 4]
        sc.bodies[k] = [scenes.BODY_SPHERE, x, y, 0.9, a, 0.0]
    return sc


def test_adjoint_wall_creep(creep, oracle_mod):
    """Creeping rays fed by a planar reflection (PEC faces, then a dielectric
    floor and walls): the gradient through those paths alone, with respect to
    the spheres' and cylinders' centres and radii, the transmitter and the
    frequencies."""
    walls = (5.31, 0.48)
    for fe in (None, [(4.0, 0.2), None, walls, walls, walls, walls]):
        sc = _jitter(_room_with_spheres(8, 20, 16, (2.4e9, 5.8e9), 17), 18)
        sc.face_eps = None if fe is None else np.asarray(
            [(0.0, 0.0, 0.0) if e is None else (1.0, e[0], e[1]) for e in fe], dtype=np.float32)
        sc.wall_creep = True
        wall = lambda c: (c >> 56) in (6, 7)
        n_checked, _ = _check(creep, sc, bodies=range(8), seed=7, keep=wall)
        assert n_checked >= 20


def test_adjoint_200_cylinders(creep, oracle_mod):
    """The adjoint workload: 200 PEC cylinders (radius U[0.15, 0.25] m) in
    the room, 28 GHz, 64 x 64 receivers; the gradient with respect to every
    body's centre and radius (all 200 bodies, each with its paths), the
    transmitter and the frequency checked."""
    sc = _jitter(scenes.room(n_cyl=200, nx=64, ny=64, freqs=(28e9,)), 12)
    n_checked, gb = _check(creep, sc, bodies=range(200), seed=4)
    # (most of the 200 bodies are hidden from the source by others: about 40
    # have paths on this grid; every body, with or without, is compared)
    assert n_checked >= 120
    assert np.count_nonzero(np.any(gb != 0.0, axis=1)) >= 30


def test_autograd_power_db_over_a_zone(creep, oracle_mod):
    """Loss = sum over a zone of the received power in dB, through
    CreepField.apply and torch autograd; its gradient equals the reference
    vector-Jacobian product with dLoss/dE taken from the same fields."""
    from paper_2310_10578_gb300 import adjoint
    sc = _jitter(scenes.room(n_cyl=30, nx=32, ny=24, freqs=(28e9,), seed=9), 13)
    rx = torch.tensor(sc.rx_soa(), device="cuda")
    st = adjoint.Static.from_scene(sc, rx)
    bp = torch.tensor(sc.bodies[:, 1:5].astype(np.float64), requires_grad=True)
    tx = torch.tensor(sc.tx.astype(np.float64), requires_grad=True)
    fr = torch.tensor(sc.freqs, requires_grad=True)
    E = adjoint.field(bp, tx, fr, st)
    p = (E.detach().double() ** 2).sum(dim=(0, 1, 3))
    zone = torch.nonzero((p > 0) & (torch.tensor(sc.rx[:, 0], device="cuda") > 5.0)).reshape(-1)
    loss = adjoint.power_db(E, zone).sum()
    loss.backward()
    # dLoss/dE from the same fields: (10 / ln 10) 2 E / P on the zone
    En = E.detach().double().cpu().numpy()
    P = p.cpu().numpy()
    g = np.zeros(En.shape[:3], dtype=complex)
    z = zone.cpu().numpy()
    g[:, :, z] = (10.0 / np.log(10.0)) * 2.0 * (En[:, :, z, 0] + 1j * En[:, :, z, 1]) / P[z]
    S2 = creep.Scene.from_scene(sc)
    codes, counts, _ = S2.paths(rx, opts=st.opts)
    c = codes.cpu().numpy().astype(np.uint64)
    n = counts.cpu().numpy()
    lists = [[int(x) for x in c[r, :min(int(n[r]), 256)]] for r in range(sc.n_rx)]
    bodies = sorted({(cc >> 28) & 0xFFFFFFF for r in z for cc in lists[r] if (cc >> 56) >= 3})[:8]
    ref = adjoint_ref.vjp(sc, lists, g, bodies=bodies)
    for b in bodies:
        for k in range(4):
            _close(float(bp.grad[b, k]), ref["body"][b][k], ref["body_abs"][b][k], "body %d param %d" % (b, k))
    for k in range(3):
        _close(float(tx.grad[k]), ref["tx"][k], ref["tx_abs"][k], "tx %d" % k)
    _close(float(fr.grad[0]), ref["f"][0], ref["f_abs"][0], "freq")


def test_adjoint_dielectric_faces(creep, oracle_mod):
    # the planar paths' Fresnel reflections move with the transmitter and the frequency
    walls = (5.31, 0.48)
    sc = _jitter(scenes.room(n_cyl=8, nx=20, ny=16, freqs=(2.4e9, 5.8e9), seed=17,
                             face_eps=[(4.0, 0.2), None, walls, walls, walls, walls]), 19)
    n_checked, _ = _check(creep, sc, bodies=range(3), seed=5)
    assert n_checked >= 6
