"""Batched frames (rt_batch_*): every frame of one launch per path class
against the FP64 oracle, and bit for bit against the single-frame entry point
(rt_evaluate) on the same receivers; the captured graph against the direct
launch; the error paths.

The frames are those of scenes.crowd: walking PEC cylinders in the 10 x 8 x 3
m room (Sec. III's dynamic scenes), each frame with its own frequencies and
receiver count.
"""
import numpy as np
import pytest

from parity import compare_fields, gpu_fields
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


def _batch(creep, cw, max_body=None):
    S = creep.Scene(cw.tri, cw.tri_face, np.zeros((0, 6)))
    S.set_tx(cw.tx, cw.pol)
    mb = max(len(b) for b in cw.bodies) if max_body is None else max_body
    B = creep.Batch(S, cw.n_rx, len(cw.freqs[0]), mb)
    for i in range(cw.n_frames):
        B.set_frame(i, cw.bodies[i], cw.freqs[i])
    rx = torch.tensor(B.rx_pack([r.T for r in cw.rx]), device="cuda")
    return S, B, rx


def _single(creep, cw, i, opts):
    sc = cw.frame(i)
    S = creep.Scene.from_scene(sc)
    n = sc.n_rx
    fl = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
    E = S.evaluate(torch.tensor(sc.rx_soa(), device="cuda"), flags=fl, opts=opts)
    return E.cpu().numpy(), fl[:n].cpu().numpy().astype(np.uint32)


def _small_crowd():
    """Six frames: ragged receiver counts (0, 1, 97, ...), one frame with a
    third of the bodies, one with none, six frequencies (a full and a partial
    chunk of four)."""
    cw = scenes.crowd(n_frames=6, n_cyl=12, n_freq=6, rx_range=(150, 700), seed=11)
    cw.rx[1] = cw.rx[1][:0]
    cw.rx[2] = cw.rx[2][:1]
    cw.rx[3] = cw.rx[3][:97]
    cw.bodies[4] = cw.bodies[4][:4]
    cw.bodies[5] = cw.bodies[5][:0]
    return cw


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_small_parity_and_single_equality(creep, oracle_mod, precision):
    cw = _small_crowd()
    opts = creep.options(max_order=2, precision=creep.RT_PREC_FP64 if precision == "fp64" else creep.RT_PREC_FP32)
    S, B, rx = _batch(creep, cw)
    fl = torch.zeros(max(B.total_rx, 1), dtype=torch.int32, device="cuda")
    out = B.evaluate(rx, flags=fl, opts=opts)
    torch.cuda.synchronize()
    flags = fl.cpu().numpy().astype(np.uint32)
    for i in range(cw.n_frames):
        Eb = B.frame_fields(out, i).cpu().numpy()
        fb = flags[B.rx_off[i]:B.rx_off[i + 1]]
        Es, fs = _single(creep, cw, i, opts)
        assert np.array_equal(Eb, Es), "frame %d differs from the single-frame evaluation" % i
        assert np.array_equal(fb, fs)
        if cw.n_rx[i] == 0:
            continue
        ref = oracle_mod.evaluate(cw.frame(i))
        assert np.array_equal(fb & 3, ref.flags & 3)
        compare_fields(gpu_fields(B.frame_fields(out, i)), ref, flags=ref.flags, freqs=cw.freqs[i])
    st = B.stats()
    # three for the receivers' spatial order; FP32: one planar launch for both
    # chunks, one per body class; FP64: three per chunk
    assert st["kernel_launches"] == 3 + (3 if precision == "fp32" else 6)


def test_batch_full_size_crowd(creep, oracle_mod):
    """The 64-frame crowd (50 walking cylinders, 16 frequencies in 24-30 GHz,
    1k-64k receivers a frame) in the launches the benchmark times: every
    frame bit for bit equal to its single-frame evaluation, and sampled
    receivers of eight frames against the oracle."""
    cw = scenes.crowd()
    opts = creep.options(max_order=2)
    S, B, rx = _batch(creep, cw)
    fl = torch.zeros(B.total_rx, dtype=torch.int32, device="cuda")
    out = B.evaluate(rx, flags=fl, opts=opts)
    torch.cuda.synchronize()
    assert B.stats()["kernel_launches"] == 6
    flags = fl.cpu().numpy().astype(np.uint32)
    for i in range(cw.n_frames):
        Es, fs = _single(creep, cw, i, opts)
        assert np.array_equal(B.frame_fields(out, i).cpu().numpy(), Es), "frame %d" % i
        assert np.array_equal(flags[B.rx_off[i]:B.rx_off[i + 1]], fs)
    rng = np.random.default_rng(5)
    for i in rng.choice(cw.n_frames, 8, replace=False):
        n = cw.n_rx[i]
        idx = np.sort(rng.choice(n, min(n, 400), replace=False))
        ref = oracle_mod.evaluate(cw.frame(i, idx))
        Eg = gpu_fields(B.frame_fields(out, i))[:, :, idx]
        assert np.array_equal(flags[B.rx_off[i] + idx] & 3, ref.flags & 3)
        compare_fields(Eg, ref, flags=ref.flags, freqs=cw.freqs[i])


def test_batch_graph_replay(creep):
    """A captured graph gives the direct launch's fields bit for bit, and
    reads the frames when it runs: frames set between replays take effect."""
    cw = scenes.crowd(n_frames=5, n_cyl=20, n_freq=7, rx_range=(300, 3000), seed=21)
    S, B, rx = _batch(creep, cw)
    opts = creep.options(max_order=2)
    ref = B.evaluate(rx, opts=opts).clone()
    side = torch.cuda.Stream()
    out = torch.full_like(ref, float("nan"))
    side.wait_stream(torch.cuda.current_stream())
    B.capture(rx, out, opts=opts, stream=side)
    torch.cuda.synchronize()
    assert torch.isnan(out).all()          # capture runs nothing
    for _ in range(2):
        B.replay(stream=side)
        side.synchronize()
        assert torch.equal(out, ref)
    # move the crowd: frame i takes frame i+1's bodies
    cw2 = scenes.crowd(n_frames=5, n_cyl=20, n_freq=7, rx_range=(300, 3000), seed=21)
    for i in range(cw.n_frames):
        B.set_frame(i, cw2.bodies[(i + 1) % cw.n_frames], cw2.freqs[i])
    B.replay(stream=side)
    side.synchronize()
    ref2 = B.evaluate(rx, opts=opts)
    torch.cuda.synchronize()
    assert torch.equal(out, ref2) and not torch.equal(ref2, ref)


def test_batch_errors(creep):
    cw = scenes.crowd(n_frames=3, n_cyl=5, n_freq=2, rx_range=(10, 40), seed=31)
    S = creep.Scene(cw.tri, cw.tri_face, np.zeros((0, 6)))
    with pytest.raises(creep.CreepError) as e:       # transmitter not set
        B = creep.Batch(S, cw.n_rx, 2, 5)
        B.set_frame(0, cw.bodies[0], cw.freqs[0])
    assert e.value.code == creep.RT_ERR_STATE
    S.set_tx(cw.tx, cw.pol)
    B = creep.Batch(S, cw.n_rx, 2, 5)
    rx = torch.tensor(B.rx_pack([r.T for r in cw.rx]), device="cuda")
    B.set_frame(0, cw.bodies[0], cw.freqs[0])
    B.set_frame(1, cw.bodies[1], cw.freqs[1])
    with pytest.raises(creep.CreepError) as e:       # frame 2 not set
        B.evaluate(rx)
    assert e.value.code == creep.RT_ERR_STATE
    with pytest.raises(creep.CreepError) as e:       # more bodies than max_body
        B.set_frame(2, np.concatenate([cw.bodies[2], cw.bodies[2][:1] + [0, 0, 0, 2.0, 0, 0]]), cw.freqs[2])
    assert e.value.code == creep.RT_ERR_OVERFLOW
    on_tx = cw.bodies[2].copy()
    on_tx[0] = [0, cw.tx[0], cw.tx[1], cw.tx[2], 0.2, 0.0]     # a sphere round the transmitter
    with pytest.raises(creep.CreepError) as e:       # transmitter inside a body
        B.set_frame(2, on_tx, cw.freqs[2])
    assert e.value.code == creep.RT_ERR_GEOM
    with pytest.raises(creep.CreepError) as e:
        B.set_frame(2, cw.bodies[2], [0.0, 1e9])
    assert e.value.code == creep.RT_ERR_ARG
    with pytest.raises(creep.CreepError) as e:
        B.set_frame(3, cw.bodies[2], cw.freqs[2])
    assert e.value.code == creep.RT_ERR_ARG
    B.set_frame(2, cw.bodies[2], cw.freqs[2])
    B.evaluate(rx)
    with pytest.raises(creep.CreepError) as e:       # wall -> creeping paths: single scenes only
        B.evaluate(rx, opts=creep.options(enable=creep.RT_EN_ALL | creep.RT_EN_WALL_CREEP))
    assert e.value.code == creep.RT_ERR_ARG
    S.set_tx(cw.tx + np.float32(0.01), cw.pol)       # every frame must be set again
    with pytest.raises(creep.CreepError) as e:
        B.evaluate(rx)
    assert e.value.code == creep.RT_ERR_STATE
    with pytest.raises(creep.CreepError) as e:
        B.replay()
    assert e.value.code == creep.RT_ERR_STATE
    with pytest.raises(creep.CreepError) as e:       # no capture on the legacy default stream
        B.capture(rx, torch.empty(6 * 2 * B.total_rx, device="cuda"), stream=torch.cuda.default_stream())
    assert e.value.code == creep.RT_ERR_ARG
    with pytest.raises(creep.CreepError) as e:
        creep.Batch(S, [3, -1], 2, 5)
    assert e.value.code == creep.RT_ERR_ARG
    with pytest.raises(creep.CreepError) as e:
        creep.Batch(S, [3, 4], 2, 5000)
    assert e.value.code == creep.RT_ERR_OVERFLOW
    # all frames empty: a no-op
    E = creep.Batch(S, [0, 0], 2, 5)
    for i in range(2):
        E.set_frame(i, cw.bodies[i], cw.freqs[i])
    out = E.evaluate(torch.zeros(0, dtype=torch.float32, device="cuda"))
    assert out.numel() == 0


def test_batch_tile_shapes(creep, oracle_mod):
    """Every tile shape gives the oracle's fields within the bound, the same
    flags, and the default shape's fields up to the rounding of the sums
    over a tile's warps."""
    cw = _small_crowd()
    S, B, rx = _batch(creep, cw)
    opts = creep.options(max_order=2)
    fl0 = torch.zeros(max(B.total_rx, 1), dtype=torch.int32, device="cuda")
    ref = B.evaluate(rx, flags=fl0, opts=opts).clone()
    assert B.shape() == (4, 4, 4)
    for shape in [(1, 1, 1), (2, 2, 2), (1, 3, 1), (4, 6, 2), (2, 12, 1), (4, 12, 4)]:
        B.set_shape(*shape)
        fl = torch.zeros_like(fl0)
        out = B.evaluate(rx, flags=fl, opts=opts)
        torch.cuda.synchronize()
        assert torch.equal(fl, fl0), shape
        scale = torch.max(torch.abs(ref)).item()
        assert torch.max(torch.abs(out - ref)).item() <= 1e-5 * scale, shape
        if shape == (1, 3, 1):
            for i in (0, 3, 4):
                oref = oracle_mod.evaluate(cw.frame(i))
                compare_fields(gpu_fields(B.frame_fields(out, i)), oref, flags=oref.flags, freqs=cw.freqs[i])
    with pytest.raises(creep.CreepError) as e:
        B.set_shape(3, 4, 4)
    assert e.value.code == creep.RT_ERR_ARG
    with pytest.raises(creep.CreepError) as e:
        B.set_shape(4, 5, 4)
    assert e.value.code == creep.RT_ERR_ARG


def test_batch_tune(creep):
    """The autotuner keeps a valid shape whose evaluation is that of the
    shape set by hand, and a batch of the same size takes it from its cache."""
    cw = scenes.crowd(n_frames=6, n_cyl=30, n_freq=8, rx_range=(2000, 8000), seed=41)
    S, B, rx = _batch(creep, cw)
    opts = creep.options(max_order=2)
    out = torch.empty(6 * 8 * B.total_rx, device="cuda")
    shape = B.tune(rx, out, opts=opts)
    assert shape[0] in (1, 2, 4) and 12 % shape[1] == 0 and 1 <= shape[2] <= 2
    assert B.shape() == shape
    a = B.evaluate(rx, opts=opts).clone()
    B2 = creep.Batch(S, cw.n_rx, 8, max(len(b) for b in cw.bodies))
    for i in range(cw.n_frames):
        B2.set_frame(i, cw.bodies[i], cw.freqs[i])
    B2.set_shape(*shape)
    b = B2.evaluate(rx, opts=opts)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    import time
    B3 = creep.Batch(S, cw.n_rx, 8, max(len(b) for b in cw.bodies))
    for i in range(cw.n_frames):
        B3.set_frame(i, cw.bodies[i], cw.freqs[i])
    t0 = time.perf_counter()
    assert B3.tune(rx, out, opts=opts) == shape
    assert time.perf_counter() - t0 < 0.05          # cached: no timing runs
