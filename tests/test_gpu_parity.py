"""GPU path (libcreep.so through the C ABI) against the FP64 oracle.

Bit-exact: path lists (which direct, reflected and creeping rays exist and are
visible, Eqs. 1-2) and the semantic receiver flags.  Fields: the bound of
tests/parity.py (derived from the FP32 arithmetic) on every receiver, and
|E| within 0.05 dB, phase within 1e-3 rad where the coherent sum is well
conditioned.
"""
import numpy as np
import pytest

from parity import compare_fields, compare_paths, gpu_fields
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


def _run(creep, sc, opts=None, cap=256):
    S = creep.Scene.from_scene(sc)
    rx = torch.tensor(sc.rx_soa(), device="cuda")
    n = sc.n_rx
    fl = torch.zeros(n, dtype=torch.int32, device="cuda")
    if opts is None:
        opts = creep.options(max_order=sc.max_order)
    E = S.evaluate(rx, flags=fl, opts=opts)
    codes, counts, fl2 = S.paths(rx, cap=cap, opts=opts)
    torch.cuda.synchronize()
    return S, gpu_fields(E), codes, counts, fl.cpu().numpy().astype(np.uint32), fl2.cpu().numpy().astype(np.uint32)


def _flags_equal(fl, ref):
    sem = 1 | 2
    assert np.array_equal(fl & sem, ref.flags & sem), np.where((fl & sem) != (ref.flags & sem))[0][:10]


def test_fock_table_matches_oracle(creep):
    from scipy.special import ai_zeros
    from oracle import fock
    xi_lo, step, G, dG, res = creep.fock_table()
    n = G.shape[1]
    xi = xi_lo + step * np.arange(n)
    assert abs(xi[-1] - fock.XI_HI) < 1e-12 and xi_lo == fock.XI_LO
    for k, hard in ((0, False), (1, True)):
        ph = np.array([fock.phat(x, hard) for x in xi])
        ref = ph * np.exp(-1j * xi ** 3 / 12)
        assert np.max(np.abs(G[k] - ref)) < 1e-10
        h = 1e-5
        xs = xi[5:-5:7]
        num = (np.array([fock.phat(x + h, hard) * np.exp(-1j * (x + h) ** 3 / 12) for x in xs]) -
               np.array([fock.phat(x - h, hard) * np.exp(-1j * (x - h) ** 3 / 12) for x in xs])) / (2 * h)
        assert np.max(np.abs(dG[k][5:-5:7] - num)) < 1e-6
    a, ap, ai, aip = ai_zeros(8)
    assert np.allclose(res[0], -a, rtol=1e-13) and np.allclose(res[2], -ap, rtol=1e-13)
    assert np.allclose(res[1], 1 / aip ** 2, rtol=1e-11) and np.allclose(res[3], 1 / (-ap * ai ** 2), rtol=1e-11)


def test_fock_table_p_segment_matches_oracle(creep):
    # the FP32 fields' second table segment, P itself on [1.5, 12], against the
    # oracle's P: its quadrature at 1.5, its 40-term residue series above (taken
    # directly: P = phat - c/xi would cancel to a few digits at xi = 12)
    from oracle import fock
    _, step, _, _, _ = creep.fock_table()
    xi0, Pt, dPt = creep.fock_table_p()
    xi = xi0 + step * np.arange(Pt.shape[1])
    assert abs(xi0 - fock.XI_HI) < 1e-12 and abs(xi[-1] - 12.0) < 1e-12

    def P(x, hard):
        return fock.P_residue(x, hard) if x > fock.XI_HI else fock.P(x, hard)

    h = 1e-5
    for k, hard in ((0, False), (1, True)):
        ref = np.array([P(x, hard) for x in xi])
        assert np.max(np.abs(Pt[k] - ref)) < 1e-10
        assert np.max(np.abs(Pt[k] - ref) / np.abs(ref)) < 1e-6      # FP32 storage needs ~1e-7
        xs = xi[1:-1]
        num = (np.array([P(x + h, hard) for x in xs]) - np.array([P(x - h, hard) for x in xs])) / (2 * h)
        assert np.max(np.abs(dPt[k][1:-1] - num) / np.abs(num)) < 1e-5


@pytest.mark.parametrize("pol", [(0, 0, 1.0), (0, 1.0, 0)])
def test_sphere_ring_parity(creep, oracle_mod, pol):
    sc = scenes.sphere_ring(n_rx=4096, pol=pol)
    S, Eg, codes, counts, fl, fl2 = _run(creep, sc)
    ref = oracle_mod.evaluate(sc)
    compare_paths(codes, counts, ref)
    _flags_equal(fl, ref)
    _flags_equal(fl2, ref)
    st = compare_fields(Eg, ref, flags=ref.flags, freqs=sc.freqs)
    assert st["n_cmp"] > 2500


def test_room_parity_small(creep, oracle_mod):
    # 20 cylinders, 61 x 47 receivers (ragged last block), three frequencies
    sc = scenes.room(n_cyl=20, nx=61, ny=47)
    S, Eg, codes, counts, fl, fl2 = _run(creep, sc)
    ref = oracle_mod.evaluate(sc)
    npaths = compare_paths(codes, counts, ref)
    assert npaths > 20 * sc.n_rx
    _flags_equal(fl, ref)
    compare_fields(Eg, ref, flags=ref.flags, freqs=sc.freqs)


def test_long_paths_phase_at_28ghz(creep, oracle_mod):
    """Phase over long paths: a 30 x 24 x 3 m room at 28 GHz (lambda = 1.07
    cm; direct paths up to 38 m, two-bounce paths beyond 60 m, i.e. several
    thousand wavelengths), 12 cylinders, 48 x 40 receivers.  The FP32 path
    keeps each path's length as double-float and its phase as the FP32
    fraction of L / lambda (the integer wavelength count dropped): every
    compared sample, whatever the conditioning of its sum, within 1e-3 rad
    and 0.05 dB of the FP64 oracle; path lists identical."""
    sc = scenes.room(n_cyl=12, nx=48, ny=40, freqs=(28e9,), size=(30.0, 24.0, 3.0), seed=31)
    S, Eg, codes, counts, fl, fl2 = _run(creep, sc)
    ref = oracle_mod.evaluate(sc)
    compare_paths(codes, counts, ref)
    st = compare_fields(Eg, ref, flags=ref.flags, freqs=sc.freqs)
    assert st["n_all"] > 1500
    assert st["ph_max_all"] <= 1e-3 and st["db_max_all"] <= 0.05, st
    L = np.linalg.norm(sc.rx - sc.tx[None, :], axis=1)
    assert L.max() > 30.0


def test_room_parity_full_size(creep, oracle_mod):
    """The 256 x 256 grid evaluated in one launch on the GPU (the launch the
    benchmark times), compared with the oracle at every receiver."""
    sc = scenes.room()
    S, Eg, codes, counts, fl, _ = _run(creep, sc)
    ref = oracle_mod.evaluate(sc)
    compare_paths(codes, counts, ref)
    assert np.array_equal(fl & 3, ref.flags & 3)
    compare_fields(Eg, ref, flags=ref.flags, freqs=sc.freqs)


def _near_surface_points(bodies, dists, n_ang, z, rng):
    pts = []
    for b in bodies:
        for d in dists:
            for phi in rng.uniform(0, 2 * np.pi, n_ang):
                r = b[4] + d
                if b[0] == 0:                                  # sphere: random direction
                    u = rng.normal(size=3)
                    u /= np.linalg.norm(u)
                    pts.append(b[1:4] + r * u)
                else:
                    pts.append([b[1] + r * np.cos(phi), b[2] + r * np.sin(phi), z])
    return np.asarray(pts, dtype=np.float32)


@pytest.mark.parametrize("kind", ["cylinders", "sphere"])
def test_receivers_near_body_surfaces(creep, oracle_mod, kind):
    """Receivers 10 um to 2 mm outside a body: the reflected leg is far
    shorter than the wavelength and the reflection point far from the FP32
    coordinates' scale, the ill-conditioned end of the curved-surface
    reflection (Eq. 3) and of the shed creeping ray (Eq. 4)."""
    rng = np.random.default_rng(11)
    if kind == "cylinders":
        sc = scenes.room(n_cyl=20, nx=2, ny=2)
        pts = _near_surface_points(sc.bodies[:10], (1e-5, 1e-4, 5e-4, 2e-3), 12, 1.2, rng)
    else:
        sc = scenes.sphere_ring(n_rx=4)
        sc.freqs = np.array([2.4e9, 28e9])
        pts = _near_surface_points(sc.bodies, (1e-5, 1e-4, 5e-4, 2e-3), 60, 0.0, rng)
    sc2 = sc.subset(np.arange(len(pts)) % sc.n_rx)
    sc2.rx = pts
    S, Eg, codes, counts, fl, _ = _run(creep, sc2)
    ref = oracle_mod.evaluate(sc2)
    compare_paths(codes, counts, ref)
    _flags_equal(fl, ref)
    compare_fields(Eg, ref, flags=ref.flags, freqs=sc2.freqs)


def test_grazing_reflection_at_the_shadow_boundary(creep, oracle_mod):
    """Crowd frame 63, receiver 33615: 1.3e-8 rad inside the lit side of a
    cylinder's shadow boundary, so the reflection off it (Eq. 3) has an
    incidence cosine of about 6e-9 and is decided in FP64.  Its divergence
    factor (zero) and Fock-uniform coefficient (pole) must come from the same
    geometry, whose product stays finite; the neighbouring receivers too, in
    FP32 and FP64."""
    cw = scenes.crowd()
    sc = cw.frame(63).subset(np.arange(33600, 33632))
    for prec in (creep.RT_PREC_FP32, creep.RT_PREC_FP64):
        opts = creep.options(max_order=2, precision=prec)
        S, Eg, codes, counts, fl, _ = _run(creep, sc, opts=opts)
        ref = oracle_mod.evaluate(sc)
        compare_paths(codes, counts, ref)
        assert np.all(np.isfinite(Eg))
        compare_fields(Eg, ref, flags=ref.flags, freqs=sc.freqs)


def test_fp64_mode(creep, oracle_mod):
    sc = scenes.room(n_cyl=12, nx=23, ny=19, seed=77)
    opts = creep.options(precision=creep.RT_PREC_FP64)
    S, Eg, codes, counts, fl, _ = _run(creep, sc, opts=opts)
    ref = oracle_mod.evaluate(sc)
    compare_paths(codes, counts, ref)
    err = np.linalg.norm(Eg - ref.E, axis=1)
    assert np.all(err <= 2e-6 * ref.sabs + 1e-13), float(np.max(err / (ref.sabs + 1e-30)))


def test_many_frequencies_and_masks(creep, oracle_mod):
    # five frequencies (two launches of the 4-frequency kernel); contributions
    # switched on one class at a time.  The hard creeping term of a z-polarised
    # source vanishes identically on these cylinders (E^i has no normal
    # component at a tangent point), so the hard-only case uses a y source.
    sc = scenes.room(n_cyl=8, nx=17, ny=13, freqs=(2.0e9, 2.4e9, 5.8e9, 12e9, 28e9), seed=5)
    for enable, order in ((creep.RT_EN_ALL, 1), (creep.RT_EN_CREEP_SOFT, 2), (creep.RT_EN_CREEP_HARD | creep.RT_EN_LOS, 0),
                          (creep.RT_EN_BODYREFL | creep.RT_EN_PLANAR, 2)):
        sc.max_order = order
        sc.pol = np.array([0, 1.0, 0] if enable & creep.RT_EN_CREEP_HARD and not enable & creep.RT_EN_CREEP_SOFT
                          else [0, 0, 1.0], dtype=np.float32)
        opts = creep.options(max_order=order, enable=enable)
        S, Eg, codes, counts, fl, _ = _run(creep, sc, opts=opts)
        ref = oracle_mod.evaluate(sc, enable=enable)
        compare_paths(codes, counts, ref)
        compare_fields(Eg, ref, flags=ref.flags, freqs=sc.freqs)


def test_many_bodies_many_frequencies(creep, oracle_mod):
    # 256 cylinders and 8 frequencies (two chunks): the bodies' data and their
    # occluder masks take so much shared memory that the body kernels keep
    # fewer path records per lane (fewer bodies per geometry pass)
    sc = scenes.room(n_cyl=256, nx=13, ny=11, freqs=tuple(np.linspace(2.4e9, 28e9, 8)), seed=23)
    S, Eg, codes, counts, fl, _ = _run(creep, sc)
    ref = oracle_mod.evaluate(sc)
    compare_paths(codes, counts, ref)
    _flags_equal(fl, ref)
    compare_fields(Eg, ref, flags=ref.flags, freqs=sc.freqs)


def test_receivers_inside_bodies_and_on_axes(creep, oracle_mod):
    sc = scenes.room(n_cyl=10, nx=4, ny=4, seed=9)
    b = sc.bodies
    pts = [[b[0, 1], b[0, 2], 1.0], [b[1, 1] + b[1, 4], b[1, 2], 1.0],      # centre, exactly on the surface
           [b[2, 1], b[2, 2], 1.75], [5.0, 4.0, 1.2], [sc.tx[0], sc.tx[1], 1.2]]
    sc2 = sc.subset(np.arange(len(pts)))
    sc2.rx = np.asarray(pts, dtype=np.float32)
    S, Eg, codes, counts, fl, _ = _run(creep, sc2)
    ref = oracle_mod.evaluate(sc2)
    compare_paths(codes, counts, ref)
    _flags_equal(fl, ref)
    assert fl[0] & 1 and not (fl[2] & 1)              # centre inside; above the top outside
    assert np.all(Eg[:, :, 0] == 0)
    compare_fields(Eg, ref, flags=ref.flags, freqs=sc.freqs)


def test_empty_and_error_paths(creep):
    sc = scenes.room(n_cyl=3, nx=2, ny=2)
    S = creep.Scene.from_scene(sc)
    rx = torch.zeros((3, 0), dtype=torch.float32, device="cuda")
    out = S.evaluate(rx)
    assert out.shape == (3, 3, 0, 2)
    with pytest.raises(creep.CreepError) as e:
        S.set_tx((sc.bodies[0, 1], sc.bodies[0, 2], 1.0), (0, 0, 1))
    assert e.value.code == creep.RT_ERR_GEOM
    with pytest.raises(creep.CreepError) as e:
        S.set_tx((np.nan, 1, 1), (0, 0, 1))
    assert e.value.code == creep.RT_ERR_ARG
    with pytest.raises(creep.CreepError) as e:
        S.set_freqs([])
    assert e.value.code == creep.RT_ERR_ARG
    S2 = creep.Scene(sc.tri, sc.tri_face, sc.bodies)
    with pytest.raises(creep.CreepError) as e:
        S2.evaluate(torch.zeros((3, 4), dtype=torch.float32, device="cuda"))
    assert e.value.code == creep.RT_ERR_STATE
    bad = np.array([[1, 1.0, 1.0, 0.0, 0.3, 1.7], [1, 1.2, 1.0, 0.0, 0.3, 1.7]])
    with pytest.raises(creep.CreepError) as e:
        creep.Scene(sc.tri, sc.tri_face, bad)
    assert e.value.code == creep.RT_ERR_GEOM
    with pytest.raises(creep.CreepError) as e:
        S.evaluate(torch.zeros((3, 4), dtype=torch.float32, device="cuda"), opts=creep.options(max_order=3))
    assert e.value.code == creep.RT_ERR_ARG


def test_host_entry_point_matches_device(creep):
    sc = scenes.room(n_cyl=10, nx=40, ny=33, seed=4)
    S = creep.Scene.from_scene(sc)
    rx = torch.tensor(sc.rx_soa(), device="cuda")
    E = S.evaluate(rx).cpu().numpy()
    Eh, flh = S.evaluate_host(sc.rx_soa(), flags=True)
    assert np.array_equal(E, Eh)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_evaluate_with_paths(creep, precision):
    """Fields and path lists in one call (FP32: from the same kernels): the
    fields of rt_evaluate bit for bit, the path sets of rt_paths (in no
    particular order), the same counts and flags; with a small capacity the
    overflow flag and a subset of the list."""
    sc = scenes.room(n_cyl=20, nx=40, ny=31, freqs=(2.4e9, 28e9), seed=5)
    S = creep.Scene.from_scene(sc)
    rx = torch.tensor(sc.rx_soa(), device="cuda")
    opts = creep.options(max_order=2, precision=creep.RT_PREC_FP64 if precision == "fp64" else creep.RT_PREC_FP32)
    fl0 = torch.zeros(sc.n_rx, dtype=torch.int32, device="cuda")
    E0 = S.evaluate(rx, flags=fl0, opts=opts)
    c0, n0, _ = S.paths(rx, opts=opts)
    E1, c1, n1, fl1 = S.evaluate_with_paths(rx, opts=opts)
    torch.cuda.synchronize()
    assert torch.equal(E0, E1) and torch.equal(n0, n1) and torch.equal(fl0, fl1)
    c0, c1, n = c0.cpu().numpy(), c1.cpu().numpy(), n0.cpu().numpy()
    for r in range(sc.n_rx):
        assert np.array_equal(np.sort(c0[r, :n[r]]), np.sort(c1[r, :n[r]])), r
    E2, c2, n2, fl2 = S.evaluate_with_paths(rx, cap=4, opts=opts)
    torch.cuda.synchronize()
    assert torch.equal(E0, E2) and torch.equal(n0, n2)
    c2, fl2 = c2.cpu().numpy(), fl2.cpu().numpy().astype(np.uint32)
    over = n > 4
    assert over.any() and np.array_equal((fl2 & creep.RT_FLAG_OVERFLOW) != 0, over)
    for r in np.nonzero(over)[0][:200]:
        assert set(c2[r].tolist()) <= set(c0[r, :n[r]].tolist())


def test_scene_tile_shapes_and_tune(creep, oracle_mod):
    """Every tile shape of rt_evaluate gives the oracle's fields within the
    bound; the autotuner keeps a valid shape and evaluates with it."""
    sc = scenes.room(n_cyl=20, nx=61, ny=47, seed=3)
    S = creep.Scene.from_scene(sc)
    rx = torch.tensor(sc.rx_soa(), device="cuda")
    opts = creep.options(max_order=2)
    ref = oracle_mod.evaluate(sc)
    base = S.evaluate(rx, opts=opts).clone()
    for shape in [(1, 3, 1), (2, 6, 4), (4, 12, 2), (1, 1, 1)]:
        S.set_shape(*shape)
        E = S.evaluate(rx, opts=opts)
        torch.cuda.synchronize()
        assert torch.max(torch.abs(E - base)).item() <= 1e-5 * torch.max(torch.abs(base)).item(), shape
        compare_fields(gpu_fields(E), ref, flags=ref.flags, freqs=sc.freqs)
    shape = S.tune(rx, opts=opts)
    assert S.shape() == shape and shape[0] in (1, 2, 4) and 12 % shape[1] == 0
    compare_fields(gpu_fields(S.evaluate(rx, opts=opts)), ref, flags=ref.flags, freqs=sc.freqs)
    with pytest.raises(creep.CreepError) as e:
        S.set_shape(4, 4, 5)
    assert e.value.code == creep.RT_ERR_ARG


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_dielectric_faces(creep, oracle_mod, precision):
    """Dielectric (Fresnel) walls and floor, PEC ceiling: the oracle's fields
    within the bound, its path lists bit for bit (materials change no
    visibility)."""
    walls = (5.31, 0.48)
    sc = scenes.room(n_cyl=20, nx=61, ny=47, seed=8, face_eps=[(4.0, 0.2), None, walls, walls, walls, walls])
    opts = creep.options(max_order=2, precision=creep.RT_PREC_FP64 if precision == "fp64" else creep.RT_PREC_FP32)
    S, Eg, codes, counts, fl, _ = _run(creep, sc, opts=opts)
    ref = oracle_mod.evaluate(sc)
    compare_paths(codes, counts, ref)
    _flags_equal(fl, ref)
    compare_fields(Eg, ref, flags=ref.flags, freqs=sc.freqs)
    pec = oracle_mod.evaluate(scenes.room(n_cyl=20, nx=61, ny=47, seed=8))
    assert np.max(np.abs(ref.E - pec.E)) > 0.1 * np.max(np.abs(pec.E))     # the materials matter
    with pytest.raises(creep.CreepError) as e:
        S.set_face_materials([(1, -2.0, 0.0)] * 6)
    assert e.value.code == creep.RT_ERR_ARG


def test_alu_peaks(creep):
    """The measured FFMA and SFU rates are near the device's unit counts x
    clock: FFMA within [0.5, 1.2] of SMs x 128 lanes x 2 x the maximum clock,
    SFU at least 8 per SM per clock."""
    ffma, mufu = creep.alu_peaks()
    p = torch.cuda.get_device_properties(0)
    clock_ghz = 2.1           # GB300 maximum SM clock, about
    derived = p.multi_processor_count * 128 * 2 * clock_ghz / 1e3          # TFLOP/s
    assert 0.5 * derived <= ffma <= 1.2 * derived, (ffma, derived)
    assert mufu >= p.multi_processor_count * 8 * clock_ghz * 0.5, mufu      # Gop/s


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_extra_turns(creep, oracle_mod, precision):
    """Creeping rays with up to two extra turns round each body: the path
    lists bit for bit (CP / CM, body, turns), the fields within the bound;
    a sphere (both polarisations' shadow fields) and the room's cylinders,
    where the heights decide which turns stay on the body."""
    prec = creep.RT_PREC_FP64 if precision == "fp64" else creep.RT_PREC_FP32
    for sc in (scenes.sphere_ring(n_rx=1024, pol=(0, 1.0, 0)), scenes.room(n_cyl=20, nx=61, ny=47, seed=8)):
        sc.max_enc = 2
        opts = creep.options(max_order=sc.max_order, precision=prec, max_encirclements=2)
        S, Eg, codes, counts, fl, _ = _run(creep, sc, opts=opts)
        ref = oracle_mod.evaluate(sc)
        compare_paths(codes, counts, ref)
        _flags_equal(fl, ref)
        compare_fields(Eg, ref, flags=ref.flags, freqs=sc.freqs)
        turns = {int(c) & 0xFFFFFFF for cs in ref.paths for c in cs if (int(c) >> 56) in (4, 5)}
        assert turns == {0, 1, 2}
    with pytest.raises(creep.CreepError) as e:
        S.evaluate(torch.zeros((3, 4), dtype=torch.float32, device="cuda"),
                   opts=creep.options(max_encirclements=5))
    assert e.value.code == creep.RT_ERR_ARG


def _room_with_spheres(n_cyl, nx, ny, seed):
    """The room with every other cylinder replaced by a sphere of its radius
    centred 0.9 m above its foot."""
    sc = scenes.room(n_cyl=n_cyl, nx=nx, ny=ny, seed=seed)
    for k in range(0, n_cyl, 2):
        x, y, a = sc.bodies[k, 1], sc.bodies[k, 2], sc.bodies[k, 4]
        sc.bodies[k] = [scenes.BODY_SPHERE, x, y, 0.9, a, 0.0]
    return sc


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_wall_creep(creep, oracle_mod, precision):
    """Creeping rays fed by a planar reflection (RT_EN_WALL_CREEP): the
    20-cylinder room with PEC faces, the same with a dielectric floor and
    walls and one extra turn, and a room of spheres and cylinders; path lists
    bit for bit (WCP / WCM, body, 16 face + turns), flags, fields within the
    bound."""
    prec = creep.RT_PREC_FP64 if precision == "fp64" else creep.RT_PREC_FP32
    walls = (5.31, 0.48)
    cases = [(scenes.room(n_cyl=20, nx=61, ny=47, seed=8), 0),
             (scenes.room(n_cyl=20, nx=61, ny=47, seed=8, face_eps=[(4.0, 0.2), None, walls, walls, walls, walls]), 1),
             (_room_with_spheres(12, 40, 32, 9), 0)]
    for sc, enc in cases:
        sc.wall_creep = True
        sc.max_enc = enc
        opts = creep.options(max_order=2, precision=prec, enable=creep.RT_EN_ALL | creep.RT_EN_WALL_CREEP,
                             max_encirclements=enc)
        S, Eg, codes, counts, fl, fl2 = _run(creep, sc, opts=opts)
        ref = oracle_mod.evaluate(sc)
        compare_paths(codes, counts, ref)
        _flags_equal(fl, ref)
        _flags_equal(fl2, ref)
        compare_fields(Eg, ref, flags=ref.flags, freqs=sc.freqs)
        n_wall = sum(1 for cs in ref.paths for c in cs if (int(c) >> 56) in (6, 7))
        assert n_wall > 20000, n_wall


def test_received_power_dbm(creep):
    """rt_power_dbm: the Friis form from the field.  The direct ray alone
    (free space) gives P_t + 20 log10(lambda / (4 pi R)) exactly; on the
    sphere ring the map equals 10 log10 of the field's |E|^2 (or |E.p|^2)
    plus P_t + 20 log10(lambda / 4 pi); no field gives -inf."""
    C0 = 299792458.0
    f = 2.4e9
    S = creep.Scene(np.zeros((0, 3, 3)), None, np.array([[scenes.BODY_SPHERE, 50.0, 50.0, 50.0, 0.1, 0.0]]))
    S.set_tx(np.array([0.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0]))
    S.set_freqs([f])
    S.set_tx_power(40.0)
    R = np.array([0.5, 1.0, 2.0, 5.0, 10.0, 37.0])
    rx = torch.tensor(np.stack([R, np.zeros_like(R), np.zeros_like(R)]).astype(np.float32), device="cuda")
    E = S.evaluate(rx, opts=creep.options(max_order=0, enable=creep.RT_EN_LOS))
    P = S.power_dbm(E).cpu().numpy()[0]
    Pz = S.power_dbm(E, rx_pol=(0.0, 0.0, 2.0)).cpu().numpy()[0]
    want = 40.0 + 20 * np.log10(C0 / f / (4 * np.pi * R))
    assert np.max(np.abs(P - want)) < 1e-4 and np.max(np.abs(Pz - want)) < 1e-4
    sc = scenes.sphere_ring(n_rx=256)
    S = creep.Scene.from_scene(sc)
    S.set_tx_power(40.0)
    rx = torch.tensor(sc.rx_soa(), device="cuda")
    fl = torch.zeros(sc.n_rx, dtype=torch.int32, device="cuda")
    E = S.evaluate(rx, flags=fl)
    P = S.power_dbm(E).cpu().numpy()[0]
    Py = S.power_dbm(E, rx_pol=(0.0, 0.6, 0.8)).cpu().numpy()[0]
    e = E.cpu().numpy().astype(np.float64)[0]
    c0 = 40.0 + 20 * np.log10(C0 / sc.freqs[0] / (4 * np.pi))
    m2 = np.sum(e[..., 0] ** 2 + e[..., 1] ** 2, axis=0)
    my2 = (0.6 * e[1, :, 0] + 0.8 * e[2, :, 0]) ** 2 + (0.6 * e[1, :, 1] + 0.8 * e[2, :, 1]) ** 2
    ok, oky = m2 > 0, my2 > 1e-30
    assert np.max(np.abs(P[ok] - (c0 + 10 * np.log10(m2[ok])))) < 1e-3
    assert np.max(np.abs(Py[oky] - (c0 + 10 * np.log10(my2[oky])))) < 1e-3
    assert np.all(np.isneginf(P[~ok]))
