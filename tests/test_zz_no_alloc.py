"""The entry point that allocates no device memory (rt_evaluate_host_noalloc).

Some callers cannot call cudaMalloc: a framework may own all device memory
through its own pool, a latency-critical loop may not afford cudaMalloc's
implicit synchronisation, or a deployment may forbid allocation after
start-up.  For them the library keeps its staging buffers in one fixed device
array instead of allocating.  This test calls that entry point through the C
ABI twice in a row -- two different workloads, so a call that read stale data
from the shared array would show -- and checks each result against the
ordinary host entry point rt_evaluate_host (same kernel; the same parity
tolerance as the other GPU tests applies, and the two agree exactly).
A second test checks the promise itself: on a scene that has never seen
rt_evaluate_host (whose staging buffers are allocated per scene), the free
device memory that cudaMemGetInfo reports does not move across no-allocation calls,
the later ones with more receivers than the first.
It lives in its own file, collected last, and passes alone or after the rest.
"""
import ctypes

import numpy as np
import pytest

from paper_2310_10578_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _host_call(creep, name, S, rx, nf, opts):
    lib = creep.load()
    n = rx.shape[1]
    out = np.zeros((nf, 3, n, 2), dtype=np.float32)
    fl = np.zeros(n, dtype=np.uint32)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = getattr(lib, name)(S._h, rx.ctypes.data_as(ctypes.c_void_p), n, out.ctypes.data_as(ctypes.c_void_p),
                            fl.ctypes.data_as(ctypes.c_void_p), ctypes.byref(opts), stream)
    assert rc == 0, lib.rt_last_error().decode()
    return out, fl


def test_noalloc_entry_point_matches_host_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_10578_gb300 import creep
    from parity import TOL_REL
    creep.load()
    runs = [scenes.room(n_cyl=20, nx=96, ny=80),                                   # 7680 receivers, 3 freqs
            scenes.room(n_cyl=8, nx=37, ny=29, freqs=(5.8e9, 28e9), seed=99)]       # smaller, 2 freqs
    for sc in runs:
        S = creep.Scene.from_scene(sc)
        opts = creep.options(max_order=sc.max_order)
        rx = np.ascontiguousarray(sc.rx_soa())
        ref, fref = _host_call(creep, "rt_evaluate_host", S, rx, len(sc.freqs), opts)
        got, fgot = _host_call(creep, "rt_evaluate_host_noalloc", S, rx, len(sc.freqs), opts)
        a = got[..., 0] + 1j * got[..., 1]
        b = ref[..., 0] + 1j * ref[..., 1]
        scale = np.linalg.norm(b, axis=1) + 1e-30
        assert np.all(np.linalg.norm(a - b, axis=1) <= TOL_REL * scale)
        assert np.array_equal(got, ref) and np.array_equal(fgot, fref)
    # a request beyond the fixed array is refused with a clear error, before any work
    big = np.zeros((3, 200000), dtype=np.float32)
    with pytest.raises(creep.CreepError) as e:
        S.evaluate_host_noalloc(big)
    assert e.value.code == creep.RT_ERR_OVERFLOW and "scratch" in str(e.value)


def test_noalloc_entry_point_allocates_nothing():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_10578_gb300 import creep
    creep.load()
    torch.cuda.synchronize()
    sc = scenes.room(n_cyl=12, nx=160, ny=128, freqs=(2.4e9, 5.8e9, 28e9), seed=5)   # 20 480 receivers
    S = creep.Scene.from_scene(sc)          # never given to rt_evaluate_host
    opts = creep.options(max_order=sc.max_order)
    rx = np.ascontiguousarray(sc.rx_soa())
    small = np.ascontiguousarray(rx[:, :1000])
    _host_call(creep, "rt_evaluate_host_noalloc", S, small, len(sc.freqs), opts)    # warm-up: kernels loaded
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    outs = []
    for _ in range(2):
        outs.append(_host_call(creep, "rt_evaluate_host_noalloc", S, rx, len(sc.freqs), opts))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert np.any(outs[0][0] != 0.0)
