"""The large-scene mode on the GPU (a small office: 2 x 2 rooms, wall
panels with doors, furniture boxes, cylinders and spheres; 588 triangles,
so visibility goes through the triangle BVH): the ray launch's candidate
list equals the oracle's; with that list the path lists (orders 1-3) match
the oracle's bit for bit and the fields are within the bound, in FP32 and
FP64; the gradient through the order-3 paths matches the oracle's finite
differences; the limits of the mode are errors."""
import numpy as np
import pytest

import adjoint_ref
from parity import compare_fields, compare_paths
from paper_2310_10578_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def creep():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_10578_gb300 import creep as c
    c.load()
    return c


def _small_office(seed=None):
    kw = {} if seed is None else dict(seed=seed)
    return scenes.office(n_rooms=(2, 2), n_furn=40, n_cyl=6, n_sph=3, n_tx=1, nx=40, ny=32,
                         freqs=(2.4e9, 5.8e9), **kw)


def test_candidates_match_oracle(creep, oracle_mod):
    sc = _small_office()
    S = creep.Scene.from_scene(sc)
    for n_rays, order in ((4096, 3), (1000, 2)):
        got = S.candidates(n_rays, order)
        ref = oracle_mod.candidates(sc, n_rays, order)
        assert np.array_equal(got, ref), (len(got), len(ref))
    assert len(got) > 100


def test_device_candidates_match_oracle(creep, oracle_mod):
    """The ray launch on the device (rt_candidates_device) gives the
    oracle's list, sequence for sequence, in a BVH scene and in the room
    (12 triangles), for several ray counts and orders."""
    sc = _small_office()
    S = creep.Scene.from_scene(sc)
    for n_rays, order in ((4096, 3), (1000, 2), (5461, 3), (333, 1)):
        S.candidates_device(n_rays, order)
        got = S.get_candidates()
        ref = oracle_mod.candidates(sc, n_rays, order)
        assert np.array_equal(got, ref), (n_rays, order, len(got), len(ref))
    room = scenes.room(n_cyl=4, nx=8, ny=8)
    R = creep.Scene.from_scene(room)
    R.candidates_device(2000, 3)
    assert np.array_equal(R.get_candidates(), oracle_mod.candidates(room, 2000, 3))
    with pytest.raises(creep.CreepError):
        S.candidates_device(8000, 3)                 # beyond RT_DEV_CAND_SLOTS prefixes


def test_device_candidates_evaluate_like_a_host_list(creep, oracle_mod):
    """Fields and path lists with the device-built list equal those with the
    same list set from the host (bit for bit); rt_set_tx drops the device
    list and the host list serves again."""
    sc = _small_office()
    S = creep.Scene.from_scene(sc)
    rx = torch.tensor(sc.rx_soa(), device="cuda")
    opts = creep.options(max_order=3)
    S.set_candidates(oracle_mod.candidates(sc, 4096, 3))
    E1 = S.evaluate(rx, opts=opts).clone()
    c1, n1, _ = S.paths(rx, opts=opts)
    S.candidates_device(4096, 3)
    E2 = S.evaluate(rx, opts=opts).clone()
    c2, n2, _ = S.paths(rx, opts=opts)
    torch.cuda.synchronize()
    assert torch.equal(E1, E2) and torch.equal(n1, n2) and torch.equal(c1, c2)
    S.set_tx(sc.tx, sc.pol)
    E3 = S.evaluate(rx, opts=opts)
    torch.cuda.synchronize()
    assert torch.equal(E1, E3)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_office_parity(creep, oracle_mod, precision):
    sc = _small_office()
    S = creep.Scene.from_scene(sc)
    # the oracle's own candidate list (the library's launch is compared with
    # it in test_candidates_match_oracle); the GPU takes the same list
    sc.candidates = oracle_mod.candidates(sc, 4096, 3)
    S.set_candidates(sc.candidates)
    prec = creep.RT_PREC_FP64 if precision == "fp64" else creep.RT_PREC_FP32
    opts = creep.options(max_order=3, precision=prec)
    rx = torch.tensor(sc.rx_soa(), device="cuda")
    fl = torch.zeros(sc.n_rx, dtype=torch.int32, device="cuda")
    E = S.evaluate(rx, flags=fl, opts=opts)
    codes, counts, fl2 = S.paths(rx, opts=opts)
    torch.cuda.synchronize()
    ref = oracle_mod.evaluate(sc)
    compare_paths(codes, counts, ref)
    f = fl.cpu().numpy().astype(np.uint32)
    assert np.array_equal(f & 3, ref.flags & 3)
    Eg = E.cpu().numpy().astype(np.float64)
    compare_fields(Eg[..., 0] + 1j * Eg[..., 1], ref, flags=ref.flags, freqs=sc.freqs)
    types = np.bincount([int(c) >> 56 for cs in ref.paths for c in cs], minlength=9)
    assert types[8] > 500 and types[3:6].sum() > 50, types     # order-3 and body paths present


def test_office_adjoint_order3(creep, oracle_mod):
    """The gradient through the order-3 paths alone (transmitter and
    frequencies) against the oracle's finite differences with the same list."""
    sc = _small_office()
    sc.rx[:, :2] += np.random.default_rng(3).uniform(-0.02, 0.02, (sc.n_rx, 2)).astype(np.float32)
    sc.rx = sc.rx[::4].copy()
    S = creep.Scene.from_scene(sc)
    sc.candidates = oracle_mod.candidates(sc, 4096, 3)
    S.set_candidates(sc.candidates)
    opts = creep.options(max_order=3)
    rx = torch.tensor(sc.rx_soa(), device="cuda")
    codes, counts, _ = S.paths(rx, opts=opts)
    torch.cuda.synchronize()
    c = codes.cpu().numpy().astype(np.uint64)
    n = counts.cpu().numpy()
    lists = [[int(x) for x in c[r, :n[r]] if (int(x) >> 56) == 8] for r in range(sc.n_rx)]
    cd = np.zeros_like(c)
    for r, cs in enumerate(lists):
        cd[r, :len(cs)] = cs
    codes = torch.tensor(cd.view(np.int64), device="cuda")
    counts = torch.tensor([len(cs) for cs in lists], dtype=torch.int32, device="cuda")
    g = np.random.default_rng(4).standard_normal((len(sc.freqs), 3, sc.n_rx, 2)).astype(np.float32)
    gb, gt, gf = S.backward(rx, codes, counts, torch.tensor(g, device="cuda"), opts=opts)
    torch.cuda.synchronize()
    ref = adjoint_ref.vjp(sc, lists, g[..., 0].astype(np.float64) + 1j * g[..., 1], bodies=(), cap=256)
    assert ref["skipped"] <= 2
    assert sum(len(cs) for cs in lists) > 50
    gt, gf = gt.cpu().numpy(), gf.cpu().numpy()
    for k in range(3):
        assert abs(gt[k] - ref["tx"][k]) <= 1e-3 * max(abs(ref["tx"][k]), 1e-3 * ref["tx_abs"][k]), k
    for k in range(len(sc.freqs)):
        assert abs(gf[k] - ref["f"][k]) <= 1e-3 * max(abs(ref["f"][k]), 1e-3 * ref["f_abs"][k]), k


def test_office_limits(creep):
    sc = _small_office()
    S = creep.Scene.from_scene(sc)
    rx = torch.tensor(sc.rx_soa()[:, :64].copy(), device="cuda")
    with pytest.raises(creep.CreepError) as e:              # more than 64 faces and no candidate list
        S.evaluate(rx, opts=creep.options(max_order=1))
    assert e.value.code == creep.RT_ERR_STATE
    S.evaluate(rx, opts=creep.options(max_order=0))        # no planar paths: fine
    for bad in ([[0, 0, -1]], [[-1, 2, -1]], [[1, -1, 3]], [[10 ** 6, -1, -1]]):
        with pytest.raises(creep.CreepError) as e:
            S.set_candidates(np.asarray(bad, dtype=np.int32))
        assert e.value.code == creep.RT_ERR_ARG
    S.set_candidates(S.candidates(256, 2))
    with pytest.raises(creep.CreepError) as e:              # wall -> creeping: small scenes only
        S.evaluate(rx, opts=creep.options(enable=creep.RT_EN_ALL | creep.RT_EN_WALL_CREEP))
    assert e.value.code == creep.RT_ERR_ARG
