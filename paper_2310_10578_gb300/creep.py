"""Python binding of the C ABI in include/creep.h (argument marshalling only).

Every step of the field evaluation runs in the CUDA library libcreep.so; this
module loads it with ctypes and passes pointers.  PyTorch provides device
memory and streams.  There is no CPU fallback: if the library is missing or
no CUDA device is present, the calls raise.
"""
import ctypes
import os

import numpy as np

from . import build as _build

RT_OK, RT_ERR_ARG, RT_ERR_GEOM, RT_ERR_CUDA, RT_ERR_TIMEOUT, RT_ERR_OVERFLOW, RT_ERR_STATE = range(7)
RT_BODY_SPHERE, RT_BODY_CYLINDER = 0, 1
RT_EN_LOS, RT_EN_PLANAR, RT_EN_BODYREFL, RT_EN_CREEP_SOFT, RT_EN_CREEP_HARD = 1, 2, 4, 8, 16
RT_EN_ALL = 31
RT_EN_WALL_CREEP = 32        # creeping rays fed by one planar reflection (not in RT_EN_ALL)
RT_PREC_FP32, RT_PREC_FP64 = 0, 1
RT_FLAG_INSIDE, RT_FLAG_CAUSTIC, RT_FLAG_ESCALATED, RT_FLAG_OVERFLOW = 1, 2, 4, 8
RT_PATH_LOS, RT_PATH_R1, RT_PATH_R2, RT_PATH_RB, RT_PATH_CP, RT_PATH_CM, RT_PATH_WCP, RT_PATH_WCM = range(8)
FOCK_NRES = 8

EXPORTS = ("rt_scene_create", "rt_scene_destroy", "rt_set_tx", "rt_set_freqs", "rt_evaluate",
           "rt_evaluate_host", "rt_evaluate_host_noalloc", "rt_paths", "rt_get_stats", "rt_fock_table",
           "rt_fock_table_p",
           "rt_last_error", "rt_batch_create", "rt_batch_destroy", "rt_batch_set_frame", "rt_batch_evaluate",
           "rt_batch_capture", "rt_batch_replay", "rt_batch_get_stats", "rt_backward", "rt_alu_peaks",
           "rt_evaluate_with_paths", "rt_batch_set_shape", "rt_batch_get_shape", "rt_batch_tune",
           "rt_set_shape", "rt_get_shape", "rt_tune", "rt_set_face_materials", "rt_candidates",
           "rt_set_candidates", "rt_candidates_mesh", "rt_candidates_device", "rt_get_candidates",
           "rt_set_tx_power", "rt_power_dbm", "rt_l2_peak")
RT_DEV_CAND_SLOTS = 16384
RT_NOALLOC_SCRATCH_BYTES = 8 << 20


class CreepError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("creep error %d: %s" % (code, msg))
        self.code = code


class rt_body(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("c", ctypes.c_float * 3), ("a", ctypes.c_float), ("h", ctypes.c_float)]


class rt_options(ctypes.Structure):
    _fields_ = [("max_order", ctypes.c_int), ("enable", ctypes.c_uint), ("precision", ctypes.c_int),
                ("max_encirclements", ctypes.c_int)]


class rt_stats(ctypes.Structure):
    _fields_ = [("escalated_candidates", ctypes.c_ulonglong), ("kernel_launches", ctypes.c_ulonglong)]


_lib = None


def load(build_if_missing=True):
    """Load libcreep.so (building it in-tree first if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise OSError("libcreep.so not built: run paper_2310_10578_gb300.build.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    P, I, U = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint
    lib.rt_scene_create.argtypes = [P, P, I, P, I, ctypes.POINTER(P)]
    lib.rt_scene_destroy.argtypes = [P]
    lib.rt_scene_destroy.restype = None
    lib.rt_set_tx.argtypes = [P, P, P]
    lib.rt_set_freqs.argtypes = [P, P, I]
    lib.rt_evaluate.argtypes = [P, P, I, P, P, P, P]
    lib.rt_evaluate_host.argtypes = [P, P, I, P, P, P, P]
    lib.rt_evaluate_host_noalloc.argtypes = [P, P, I, P, P, P, P]
    lib.rt_paths.argtypes = [P, P, I, P, P, I, P, P, P]
    lib.rt_get_stats.argtypes = [P, P]
    lib.rt_fock_table.argtypes = [P, P, P, P, P, P]
    lib.rt_fock_table_p.argtypes = [P, P, P, P]
    lib.rt_last_error.restype = ctypes.c_char_p
    lib.rt_batch_create.argtypes = [P, I, P, I, I, ctypes.POINTER(P)]
    lib.rt_batch_destroy.argtypes = [P]
    lib.rt_batch_destroy.restype = None
    lib.rt_batch_set_frame.argtypes = [P, I, P, I, P]
    lib.rt_batch_evaluate.argtypes = [P, P, P, P, P, P]
    lib.rt_batch_capture.argtypes = [P, P, P, P, P, P]
    lib.rt_batch_replay.argtypes = [P, P]
    lib.rt_batch_get_stats.argtypes = [P, P]
    lib.rt_backward.argtypes = [P, P, I, P, P, I, P, P, P, P, P, P]
    lib.rt_alu_peaks.argtypes = [P, P, P]
    lib.rt_evaluate_with_paths.argtypes = [P, P, I, P, P, P, I, P, P, P]
    lib.rt_batch_set_shape.argtypes = [P, P]
    lib.rt_batch_get_shape.argtypes = [P, P]
    lib.rt_batch_tune.argtypes = [P, P, P, P, P, P, P]
    lib.rt_set_shape.argtypes = [P, P]
    lib.rt_get_shape.argtypes = [P, P]
    lib.rt_tune.argtypes = [P, P, I, P, P, P, P, P]
    lib.rt_set_face_materials.argtypes = [P, P, I]
    lib.rt_candidates.argtypes = [P, I, I, P, I, ctypes.POINTER(I)]
    lib.rt_set_candidates.argtypes = [P, P, I]
    lib.rt_candidates_mesh.argtypes = [P, P, I, P, I, I, P, I, ctypes.POINTER(I)]
    lib.rt_candidates_device.argtypes = [P, I, I, P]
    lib.rt_get_candidates.argtypes = [P, P, I, ctypes.POINTER(I)]
    lib.rt_set_tx_power.argtypes = [P, ctypes.c_float]
    lib.rt_l2_peak.argtypes = [P, P]
    lib.rt_power_dbm.argtypes = [P, P, I, P, P, P]
    _lib = lib
    return lib


def _check(code):
    if code != RT_OK:
        raise CreepError(code, _lib.rt_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(a.data_ptr())


def options(max_order=2, enable=RT_EN_ALL, precision=RT_PREC_FP32, max_encirclements=0):
    return rt_options(max_order, enable, precision, max_encirclements)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _bodies_arr(bodies):
    bodies = np.asarray(bodies, dtype=np.float64).reshape(-1, 6)
    arr = (rt_body * max(1, len(bodies)))()
    for i, b in enumerate(bodies):
        arr[i].type = int(b[0])
        arr[i].c[0], arr[i].c[1], arr[i].c[2] = float(b[1]), float(b[2]), float(b[3])
        arr[i].a, arr[i].h = float(b[4]), float(b[5])
    return arr, len(bodies)


class Scene:
    """A scene on the current CUDA device: planar faces (triangles grouped into
    coplanar reflecting faces) and convex PEC bodies (spheres, vertical
    cylinders), one transmitter and a frequency list."""

    def __init__(self, tri, tri_face, bodies):
        lib = load()
        tri = np.ascontiguousarray(np.asarray(tri, dtype=np.float32).reshape(-1, 9))
        n_tri = tri.shape[0]
        tf = None if tri_face is None else np.ascontiguousarray(np.asarray(tri_face, dtype=np.int32))
        arr, nb = _bodies_arr(bodies)
        self._h = ctypes.c_void_p()
        _check(lib.rt_scene_create(_ptr(tri) if n_tri else None, _ptr(tf), n_tri, ctypes.cast(arr, ctypes.c_void_p),
                                   nb, ctypes.byref(self._h)))
        self.n_body = nb
        self.n_f = 0

    @classmethod
    def from_scene(cls, sc):
        """Build from a paper_2310_10578_gb300.scenes.Scene (also sets Tx and frequencies)."""
        s = cls(sc.tri, sc.tri_face, sc.bodies)
        s.set_tx(sc.tx, sc.pol)
        s.set_freqs(sc.freqs)
        if getattr(sc, "face_eps", None) is not None:
            s.set_face_materials(sc.face_eps)
        if getattr(sc, "candidates", None) is not None:
            s.set_candidates(sc.candidates)
        return s

    def candidates(self, n_rays, max_order=3):
        """Candidate face sequences [n, 3] int32 (-1 padded) of the ray launch
        from the transmitter (rt_candidates; host computation)."""
        n = ctypes.c_int(0)
        _check(_lib.rt_candidates(self._h, int(n_rays), int(max_order), None, 0, ctypes.byref(n)))
        out = np.zeros((max(n.value, 1), 3), dtype=np.int32)
        _check(_lib.rt_candidates(self._h, int(n_rays), int(max_order), _ptr(out), n.value, ctypes.byref(n)))
        return out[:n.value]

    def candidates_device(self, n_rays, max_order=3, stream=None):
        """The same ray launch on the device, installed as the candidate list
        (rt_candidates_device; asynchronous on the stream)."""
        _check(_lib.rt_candidates_device(self._h, int(n_rays), int(max_order), _stream_handle(stream)))

    def get_candidates(self):
        """The current candidate list [n, 3] int32 (rt_get_candidates)."""
        n = ctypes.c_int(0)
        _check(_lib.rt_get_candidates(self._h, None, 0, ctypes.byref(n)))
        out = np.zeros((max(n.value, 1), 3), dtype=np.int32)
        _check(_lib.rt_get_candidates(self._h, _ptr(out), n.value, ctypes.byref(n)))
        return out[:n.value]

    def set_candidates(self, seq):
        """The planar paths' candidate list (rt_set_candidates); None clears it."""
        if seq is None:
            _check(_lib.rt_set_candidates(self._h, None, 0))
            return
        a = np.ascontiguousarray(np.asarray(seq, dtype=np.int32).reshape(-1, 3))
        _check(_lib.rt_set_candidates(self._h, _ptr(a), a.shape[0]))

    def set_face_materials(self, mat):
        """Per face (kind, eps', eps''): kind 0 PEC, 1 dielectric (eps' - j eps''); None: all PEC."""
        if mat is None:
            _check(_lib.rt_set_face_materials(self._h, None, 0))
            return
        m = np.ascontiguousarray(np.asarray(mat, dtype=np.float32).reshape(-1, 3))
        _check(_lib.rt_set_face_materials(self._h, _ptr(m), m.shape[0]))

    def close(self):
        if self._h:
            _lib.rt_scene_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tx(self, tx, pol):
        tx = np.ascontiguousarray(np.asarray(tx, dtype=np.float32).reshape(3))
        pol = np.ascontiguousarray(np.asarray(pol, dtype=np.float32).reshape(3))
        _check(_lib.rt_set_tx(self._h, _ptr(tx), _ptr(pol)))

    def set_tx_power(self, power_dbm):
        """The transmitter's power in dBm (rt_set_tx_power)."""
        _check(_lib.rt_set_tx_power(self._h, float(power_dbm)))

    def power_dbm(self, E, rx_pol=None, out=None, stream=None):
        """Received power in dBm [n_f, n] from fields E [n_f, 3, n, 2]
        (rt_power_dbm); rx_pol: the receiving antenna's polarisation, or
        None for the power over all polarisations."""
        import torch
        n = E.shape[2]
        if out is None:
            out = torch.empty((E.shape[0], n), dtype=torch.float32, device=E.device)
        pol = None if rx_pol is None else np.ascontiguousarray(np.asarray(rx_pol, dtype=np.float32).reshape(3))
        _check(_lib.rt_power_dbm(self._h, _ptr(E.contiguous()), n, _ptr(pol), _ptr(out), _stream_handle(stream)))
        return out

    def set_freqs(self, freqs):
        f = np.ascontiguousarray(np.asarray(freqs, dtype=np.float64).reshape(-1))
        _check(_lib.rt_set_freqs(self._h, _ptr(f), len(f)))
        self.n_f = len(f)

    def evaluate(self, rx_soa, out=None, flags=None, opts=None, stream=None):
        """Field at receivers. rx_soa: CUDA float32 tensor [3, n]; returns (and
        fills) out: CUDA float32 tensor [n_f, 3, n, 2]."""
        import torch
        n = rx_soa.shape[1]
        assert rx_soa.is_cuda and rx_soa.dtype == torch.float32 and rx_soa.is_contiguous()
        if out is None:
            out = torch.empty((self.n_f, 3, n, 2), dtype=torch.float32, device=rx_soa.device)
        _check(_lib.rt_evaluate(self._h, _ptr(rx_soa), n, _ptr(out), _ptr(flags),
                                ctypes.byref(opts) if opts is not None else None, _stream_handle(stream)))
        return out

    def evaluate_host(self, rx_soa, flags=False, opts=None, stream=None):
        """Same from/to host memory (numpy): copies inside the call."""
        rx_soa = np.ascontiguousarray(np.asarray(rx_soa, dtype=np.float32))
        n = rx_soa.shape[1]
        out = np.empty((self.n_f, 3, n, 2), dtype=np.float32)
        fl = np.empty(n, dtype=np.uint32) if flags else None
        _check(_lib.rt_evaluate_host(self._h, _ptr(rx_soa), n, _ptr(out), _ptr(fl),
                                     ctypes.byref(opts) if opts is not None else None, _stream_handle(stream)))
        return (out, fl) if flags else out

    def evaluate_host_noalloc(self, rx_soa, flags=False, opts=None, stream=None):
        """evaluate_host through the entry point that allocates no device
        memory (fixed 8 MiB device array shared by all calls on a device)."""
        rx_soa = np.ascontiguousarray(np.asarray(rx_soa, dtype=np.float32))
        n = rx_soa.shape[1]
        out = np.empty((self.n_f, 3, n, 2), dtype=np.float32)
        fl = np.empty(n, dtype=np.uint32) if flags else None
        _check(_lib.rt_evaluate_host_noalloc(self._h, _ptr(rx_soa), n, _ptr(out), _ptr(fl),
                                             ctypes.byref(opts) if opts is not None else None,
                                             _stream_handle(stream)))
        return (out, fl) if flags else out

    def paths(self, rx_soa, cap=256, opts=None, stream=None):
        """Path lists: (codes [n, cap] int64 tensor, counts [n] int32, flags [n] int32)."""
        import torch
        n = rx_soa.shape[1]
        codes = torch.zeros((n, cap), dtype=torch.int64, device=rx_soa.device)
        counts = torch.zeros(n, dtype=torch.int32, device=rx_soa.device)
        fl = torch.zeros(n, dtype=torch.int32, device=rx_soa.device)
        _check(_lib.rt_paths(self._h, _ptr(rx_soa), n, _ptr(codes), _ptr(counts), cap, _ptr(fl),
                             ctypes.byref(opts) if opts is not None else None, _stream_handle(stream)))
        return codes, counts, fl

    def set_shape(self, planar_warps, body_warps, planar_chunks):
        sh = (ctypes.c_int * 3)(planar_warps, body_warps, planar_chunks)
        _check(_lib.rt_set_shape(self._h, sh))

    def shape(self):
        sh = (ctypes.c_int * 3)()
        _check(_lib.rt_get_shape(self._h, sh))
        return tuple(sh)

    def tune(self, rx_soa, out=None, opts=None, stream=None):
        """Autotune the tile shape of evaluate on these receivers (rt_tune)."""
        import torch
        n = rx_soa.shape[1]
        if out is None:
            out = torch.empty((self.n_f, 3, n, 2), dtype=torch.float32, device=rx_soa.device)
        sh = (ctypes.c_int * 3)()
        _check(_lib.rt_tune(self._h, _ptr(rx_soa), n, _ptr(out), None,
                            ctypes.byref(opts) if opts is not None else None, _stream_handle(stream), sh))
        return tuple(sh)

    def evaluate_with_paths(self, rx_soa, cap=256, out=None, opts=None, stream=None):
        """Fields and, from the same kernels, the path lists (codes unordered
        per receiver): (E [n_f, 3, n, 2], codes [n, cap] int64, counts [n]
        int32, flags [n] int32)."""
        import torch
        n = rx_soa.shape[1]
        dev = rx_soa.device
        if out is None:
            out = torch.empty((self.n_f, 3, n, 2), dtype=torch.float32, device=dev)
        codes = torch.zeros((n, cap), dtype=torch.int64, device=dev)
        counts = torch.zeros(n, dtype=torch.int32, device=dev)
        fl = torch.zeros(n, dtype=torch.int32, device=dev)
        _check(_lib.rt_evaluate_with_paths(self._h, _ptr(rx_soa), n, _ptr(out), _ptr(codes), _ptr(counts), cap,
                                           _ptr(fl), ctypes.byref(opts) if opts is not None else None,
                                           _stream_handle(stream)))
        return out, codes, counts, fl

    def backward(self, rx_soa, codes, counts, grad_e, opts=None, stream=None):
        """Adjoint of evaluate (rt_backward): dLoss/d(body centres and radii
        [n_body, 4], transmitter [3], frequencies [n_f]) as float64 CUDA
        tensors, from grad_e = dLoss/dE [n_f, 3, n, 2] and the path list
        (codes [n, cap], counts [n]) of the same receivers."""
        import torch
        n = rx_soa.shape[1]
        dev = rx_soa.device
        gb = torch.zeros((max(self.n_body, 1), 4), dtype=torch.float64, device=dev)
        gt = torch.zeros(3, dtype=torch.float64, device=dev)
        gf = torch.zeros(self.n_f, dtype=torch.float64, device=dev)
        ge = grad_e.contiguous().to(torch.float32)
        _check(_lib.rt_backward(self._h, _ptr(rx_soa), n, _ptr(codes), _ptr(counts), codes.shape[1], _ptr(ge),
                                _ptr(gb), _ptr(gt), _ptr(gf), ctypes.byref(opts) if opts is not None else None,
                                _stream_handle(stream)))
        return gb[:self.n_body], gt, gf

    def stats(self):
        st = rt_stats()
        _check(_lib.rt_get_stats(self._h, ctypes.byref(st)))
        return {"escalated_candidates": int(st.escalated_candidates), "kernel_launches": int(st.kernel_launches)}


def candidates_mesh(tri, tri_face, tx, n_rays, max_order=3):
    """The ray launch of rt_candidates for a mesh and a transmitter, host
    only (rt_candidates_mesh): [n, 3] int32 face sequences, -1 padded."""
    lib = load()
    tri = np.ascontiguousarray(np.asarray(tri, dtype=np.float32).reshape(-1, 9))
    tf = None if tri_face is None else np.ascontiguousarray(np.asarray(tri_face, dtype=np.int32))
    t = np.ascontiguousarray(np.asarray(tx, dtype=np.float32).reshape(3))
    n = ctypes.c_int(0)
    _check(lib.rt_candidates_mesh(_ptr(tri), _ptr(tf), tri.shape[0], _ptr(t), int(n_rays), int(max_order), None, 0,
                                  ctypes.byref(n)))
    out = np.zeros((max(n.value, 1), 3), dtype=np.int32)
    _check(lib.rt_candidates_mesh(_ptr(tri), _ptr(tf), tri.shape[0], _ptr(t), int(n_rays), int(max_order),
                                  _ptr(out), n.value, ctypes.byref(n)))
    return out[:n.value]


class Batch:
    """Frames of one scene evaluated together (rt_batch_*): each frame has its
    own bodies, n_f frequencies and receivers; the triangles and transmitter
    are the scene's.  Receivers of all frames are one [3, sum n_rx] tensor of
    per-frame [3, n_rx[f]] blocks (see rx_pack); fields one flat tensor of
    per-frame [n_f, 3, n_rx[f], 2] blocks (see frame_fields)."""

    def __init__(self, scene, n_rx, n_f, max_body):
        self.scene = scene                  # keeps the scene alive
        self.n_rx = [int(n) for n in n_rx]
        self.n_f = int(n_f)
        self.rx_off = np.concatenate([[0], np.cumsum(self.n_rx)]).astype(np.int64)
        n = np.ascontiguousarray(np.asarray(self.n_rx, dtype=np.int32))
        self._h = ctypes.c_void_p()
        _check(_lib.rt_batch_create(scene._h, len(self.n_rx), _ptr(n), self.n_f, int(max_body),
                                    ctypes.byref(self._h)))

    @property
    def n_frames(self):
        return len(self.n_rx)

    @property
    def total_rx(self):
        return int(self.rx_off[-1])

    def close(self):
        if self._h:
            _lib.rt_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_frame(self, frame, bodies, freqs):
        arr, nb = _bodies_arr(bodies)
        f = np.ascontiguousarray(np.asarray(freqs, dtype=np.float64).reshape(-1))
        if len(f) != self.n_f:
            raise ValueError("frame %d: %d frequencies, the batch has %d" % (frame, len(f), self.n_f))
        _check(_lib.rt_batch_set_frame(self._h, int(frame), ctypes.cast(arr, ctypes.c_void_p), nb, _ptr(f)))

    def rx_pack(self, rx_per_frame):
        """Per-frame [3, n_rx[f]] float32 arrays -> one flat float32 array."""
        return np.concatenate([np.ascontiguousarray(r, dtype=np.float32).reshape(3, n).ravel()
                               for r, n in zip(rx_per_frame, self.n_rx)] or [np.zeros(0, np.float32)])

    def frame_fields(self, out, frame):
        """View of frame's [n_f, 3, n_rx, 2] block in the flat output."""
        a, n = int(self.rx_off[frame]), self.n_rx[frame]
        return out[6 * self.n_f * a: 6 * self.n_f * (a + n)].reshape(self.n_f, 3, n, 2)

    def evaluate(self, rx_flat, out=None, flags=None, opts=None, stream=None):
        import torch
        assert rx_flat.is_cuda and rx_flat.dtype == torch.float32 and rx_flat.is_contiguous()
        assert rx_flat.numel() == 3 * self.total_rx
        if out is None:
            out = torch.empty(6 * self.n_f * self.total_rx, dtype=torch.float32, device=rx_flat.device)
        _check(_lib.rt_batch_evaluate(self._h, _ptr(rx_flat), _ptr(out), _ptr(flags),
                                      ctypes.byref(opts) if opts is not None else None, _stream_handle(stream)))
        return out

    def capture(self, rx_flat, out, flags=None, opts=None, stream=None):
        _check(_lib.rt_batch_capture(self._h, _ptr(rx_flat), _ptr(out), _ptr(flags),
                                     ctypes.byref(opts) if opts is not None else None, _stream_handle(stream)))

    def set_shape(self, planar_warps, body_warps, planar_chunks):
        sh = (ctypes.c_int * 3)(planar_warps, body_warps, planar_chunks)
        _check(_lib.rt_batch_set_shape(self._h, sh))

    def shape(self):
        sh = (ctypes.c_int * 3)()
        _check(_lib.rt_batch_get_shape(self._h, sh))
        return tuple(sh)

    def tune(self, rx_flat, out, flags=None, opts=None, stream=None):
        """Autotune the tile shape on this batch (rt_batch_tune); returns it."""
        sh = (ctypes.c_int * 3)()
        _check(_lib.rt_batch_tune(self._h, _ptr(rx_flat), _ptr(out), _ptr(flags),
                                  ctypes.byref(opts) if opts is not None else None, _stream_handle(stream), sh))
        return tuple(sh)

    def replay(self, stream=None):
        _check(_lib.rt_batch_replay(self._h, _stream_handle(stream)))

    def stats(self):
        st = rt_stats()
        _check(_lib.rt_batch_get_stats(self._h, ctypes.byref(st)))
        return {"escalated_candidates": int(st.escalated_candidates), "kernel_launches": int(st.kernel_launches)}


def alu_peaks(stream=None):
    """Measured FP32 FFMA (TFLOP/s) and SFU (Gop/s) rates of the current device."""
    lib = load()
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib.rt_alu_peaks(ctypes.byref(a), ctypes.byref(b), _stream_handle(stream)))
    return a.value, b.value


def l2_peak(stream=None):
    """Measured L2 read bandwidth (GB/s) of the current device."""
    lib = load()
    a = ctypes.c_double()
    _check(lib.rt_l2_peak(ctypes.byref(a), _stream_handle(stream)))
    return a.value


def fock_table():
    """The device's Fock--Pekeris table: (xi_lo, step, G [2, n] complex, dG [2, n], res [4, 8])."""
    lib = load()
    xi_lo, step, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(lib.rt_fock_table(ctypes.byref(xi_lo), ctypes.byref(step), ctypes.byref(n), None, None, None))
    g = np.zeros((2, n.value, 2))
    dg = np.zeros((2, n.value, 2))
    res = np.zeros((4, FOCK_NRES))
    _check(lib.rt_fock_table(None, None, None, _ptr(g), _ptr(dg), _ptr(res)))
    return xi_lo.value, step.value, g[..., 0] + 1j * g[..., 1], dg[..., 0] + 1j * dg[..., 1], res


def fock_table_p():
    """The table's P segment (FP32 fields above xi0): (xi0, P [2, n] complex, dP [2, n])."""
    lib = load()
    xi0, n = ctypes.c_double(), ctypes.c_int()
    _check(lib.rt_fock_table_p(ctypes.byref(xi0), ctypes.byref(n), None, None))
    p = np.zeros((2, n.value, 2))
    dp = np.zeros((2, n.value, 2))
    _check(lib.rt_fock_table_p(None, None, _ptr(p), _ptr(dp)))
    return xi0.value, p[..., 0] + 1j * p[..., 1], dp[..., 0] + 1j * dp[..., 1]


def decode(code):
    code = int(code) & 0xFFFFFFFFFFFFFFFF
    return (code >> 56) & 0xFF, (code >> 28) & 0xFFFFFFF, code & 0xFFFFFFF
