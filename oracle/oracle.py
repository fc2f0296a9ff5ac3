"""ctypes front end of the FP64 C oracle (oracle/creep_oracle.c).

TEST INFRASTRUCTURE: imported only by tests, the smoke check and the CPU legs
of bench.py.  ``build()`` compiles the C file with gcc (-O2, OpenMP); the
Fock--Pekeris quadrature rule comes from ``oracle.fock`` (scipy Airy).
"""
import ctypes
import os
import subprocess
import time

import numpy as np

from . import fock

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "creep_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")

# enable mask (same meaning as the C enum)
EN_LOS, EN_PLANAR, EN_BODYREFL, EN_CREEP_SOFT, EN_CREEP_HARD = 1, 2, 4, 8, 16
EN_ALL = 31
EN_WALL_CREEP = 32          # wall -> creeping paths (also switched on by scene.wall_creep)
# receiver flags
FL_INSIDE, FL_CAUSTIC, FL_OVERFLOW = 1, 2, 8
# path types
PT_LOS, PT_R1, PT_R2, PT_RB, PT_CP, PT_CM, PT_WCP, PT_WCM, PT_R3 = range(9)
COUNTER_NAMES = ("seg_tri", "seg_body", "inside_tri", "image_cand", "body_refl", "creep_geom",
                 "paths", "fock_evals")

_lib = None
_tables = None


def build(force=False):
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".%d.tmp" % os.getpid()
        # -ffp-contract=off: every operation rounds as written (no fused
        # multiply-add), so results do not depend on the host ISA.
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(LIB)
        P = ctypes.c_void_p
        i = ctypes.c_int
        d = ctypes.c_double
        _lib.oracle_eval.argtypes = [P, P, i, P, i, P, P, P, i, P, i,
                                     P, P, P, P, P, P, P, i, P, P, P, P, i, d, d,
                                     i, i, P, P, P, i, P, P, i, P, P, P, i, P, i]
        _lib.oracle_eval.restype = i
        _lib.oracle_transition_F.argtypes = [P, i, P]
        _lib.oracle_fock_bracket.argtypes = [P, P, P, P, P, P, P, i, P, P, P, P, i, d, d, P, P, i, P]
        _lib.oracle_body_reflection.argtypes = [P, P, P, P]
        _lib.oracle_body_creeping.argtypes = [P, P, P, i, i, P]
        _lib.oracle_seg_hits_body.argtypes = [P, P, P]
        _lib.oracle_reflect.argtypes = [P, P, P, P, i, d, d, P]
        _lib.oracle_reflect.restype = None
        _lib.oracle_candidates.argtypes = [P, P, i, P, i, i, P, i]
        _lib.oracle_candidates.restype = i
    return _lib


def _fock_arrays():
    global _tables
    if _tables is None:
        t = fock.c_tables()
        _tables = dict(
            tau_re=np.ascontiguousarray(t["tau"].real), tau_im=np.ascontiguousarray(t["tau"].imag),
            ws_re=np.ascontiguousarray(t["Ws"].real), ws_im=np.ascontiguousarray(t["Ws"].imag),
            wh_re=np.ascontiguousarray(t["Wh"].real), wh_im=np.ascontiguousarray(t["Wh"].imag),
            offsets=np.ascontiguousarray(t["offsets"], dtype=np.int32),
            res_alpha=t["res_alpha"], res_cs=t["res_cs"], res_beta=t["res_beta"], res_ch=t["res_ch"])
    return _tables


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _fock_args():
    T = _fock_arrays()
    return [_p(T["tau_re"]), _p(T["tau_im"]), _p(T["ws_re"]), _p(T["ws_im"]), _p(T["wh_re"]), _p(T["wh_im"]),
            _p(T["offsets"]), len(T["offsets"]) - 1,
            _p(T["res_alpha"]), _p(T["res_cs"]), _p(T["res_beta"]), _p(T["res_ch"]), len(T["res_alpha"]),
            fock.XI_LO, fock.XI_HI]


class Result:
    pass


def evaluate(scene, rx=None, enable=EN_ALL, cap=256, threads=0, want_paths=True, path_fields=False):
    """FP64 field of ``scene`` at its receivers (or at ``rx`` [n,3]).

    Returns an object with E [n_f][3][n_rx] complex128, sabs [n_f][n_rx] (sum of
    |E_path|), paths (list of sorted uint64 arrays), flags [n_rx] uint32,
    counters dict and seconds; with path_fields, also codes [n_rx][cap]
    (enumeration order), counts [n_rx] and path_E [n_rx][cap][n_f][3]
    complex128, each listed path's own field.  The scene's arrays are read as
    float64 (pass float64 arrays for coordinates finer than float32)."""
    lib = _load()
    rx = scene.rx if rx is None else rx
    rx64 = np.ascontiguousarray(np.asarray(rx, dtype=np.float32).astype(np.float64))
    n_rx = rx64.shape[0]
    tri = np.ascontiguousarray(scene.tri.astype(np.float64).reshape(-1))
    tf = np.ascontiguousarray(scene.tri_face.astype(np.int32))
    bodies = np.ascontiguousarray(scene.bodies.astype(np.float64).reshape(-1))
    tx = np.ascontiguousarray(scene.tx.astype(np.float64))
    pol = np.ascontiguousarray(scene.pol.astype(np.float64))
    fr = np.ascontiguousarray(scene.freqs.astype(np.float64))
    n_f = len(fr)
    E = np.zeros((n_f, 3, n_rx, 2), dtype=np.float64)
    codes = np.zeros((n_rx, cap), dtype=np.uint64) if want_paths else None
    counts = np.zeros(n_rx, dtype=np.int32)
    flags = np.zeros(n_rx, dtype=np.uint32)
    ctr = np.zeros(8, dtype=np.int64)
    sabs = np.zeros((n_f, n_rx), dtype=np.float64)
    pE = np.zeros((n_rx, cap, n_f, 3, 2), dtype=np.float64) if (path_fields and want_paths) else None
    # face materials: [n_face][3] (dielectric flag, eps', eps''), eps_r = eps' - j eps''; None: PEC
    fe = getattr(scene, "face_eps", None)
    fe = None if fe is None else np.ascontiguousarray(np.asarray(fe, dtype=np.float64).reshape(-1, 3))
    # candidate face sequences [n][3] (-1 padded): planar paths of orders 1-3 from them only
    cand = getattr(scene, "candidates", None)
    cand = None if cand is None else np.ascontiguousarray(np.asarray(cand, dtype=np.int32).reshape(-1, 3))
    t0 = time.perf_counter()
    lib.oracle_eval(_p(tri), _p(tf), scene.tri.shape[0], _p(bodies), scene.bodies.shape[0],
                    _p(tx), _p(pol), _p(fr), n_f, _p(rx64), n_rx, *_fock_args(),
                    scene.max_order, enable | (EN_WALL_CREEP if getattr(scene, "wall_creep", False) else 0), _p(E),
                    _p(codes) if want_paths else None, _p(counts), cap if want_paths else 0,
                    _p(flags), _p(ctr), threads, _p(sabs), _p(pE) if pE is not None else None,
                    _p(fe) if fe is not None else None, int(getattr(scene, "max_enc", 0)),
                    _p(cand) if cand is not None else None, 0 if cand is None else cand.shape[0])
    res = Result()
    res.seconds = time.perf_counter() - t0
    res.E = E[..., 0] + 1j * E[..., 1]
    res.flags = flags
    res.sabs = sabs
    res.counts = counts
    if want_paths:
        res.paths = [np.sort(codes[r, :min(counts[r], cap)]) for r in range(n_rx)]
    if pE is not None:
        res.codes = codes
        res.path_E = pE[..., 0] + 1j * pE[..., 1]
    res.counters = dict(zip(COUNTER_NAMES, (int(c) for c in ctr)))
    return res


def candidates(scene, n_rays, max_order=3, cap=1 << 20):
    """Candidate face sequences [n][3] int32 (-1 padded) of the ray launch from
    the scene's transmitter (see oracle_candidates in creep_oracle.c)."""
    lib = _load()
    tri = np.ascontiguousarray(scene.tri.astype(np.float64).reshape(-1))
    tf = np.ascontiguousarray(scene.tri_face.astype(np.int32))
    tx = np.ascontiguousarray(np.asarray(scene.tx, dtype=np.float64))
    out = np.zeros((cap, 3), dtype=np.int32)
    n = lib.oracle_candidates(_p(tri), _p(tf), scene.tri.shape[0], _p(tx), int(n_rays), int(max_order), _p(out), cap)
    return out[:n].copy()


def transition_F(X):
    lib = _load()
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64).reshape(-1))
    out = np.zeros(2 * len(X))
    lib.oracle_transition_F(_p(X), len(X), _p(out))
    return out[0::2] + 1j * out[1::2]


def fock_bracket(xi, K):
    """(B_s, B_h) = phat - c F((K xi)^2)/xi from the C oracle."""
    lib = _load()
    xi = np.ascontiguousarray(np.asarray(xi, dtype=np.float64).reshape(-1))
    K = np.ascontiguousarray(np.broadcast_to(np.asarray(K, dtype=np.float64), xi.shape).copy())
    out = np.zeros(4 * len(xi))
    lib.oracle_fock_bracket(*_fock_args(), _p(xi), _p(K), len(xi), _p(out))
    return out[0::4] + 1j * out[1::4], out[2::4] + 1j * out[3::4]


def decode(code):
    code = int(code)
    return (code >> 56) & 0xFF, (code >> 28) & 0xFFFFFFF, code & 0xFFFFFFF


def _d3(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1))


def body_reflection(body6, S, P):
    """Reflection geometry on one body: dict(Q, n, inv_f1, inv_f2, rho_g) or None."""
    lib = _load()
    out = np.zeros(9)
    b, s, p = _d3(body6), _d3(S), _d3(P)
    if not lib.oracle_body_reflection(_p(b), _p(s), _p(p), _p(out)):
        return None
    return dict(Q=out[0:3], n=out[3:6], inv_f1=out[6], inv_f2=out[7], rho_g=out[8])


def body_creeping(body6, S, P, direction, turns=0):
    """Creeping-ray geometry (direction 0 short way, 1 long way; `turns` extra
    full turns round the body) or None."""
    lib = _load()
    out = np.zeros(19)
    b, s, p = _d3(body6), _d3(S), _d3(P)
    if not lib.oracle_body_creeping(_p(b), _p(s), _p(p), int(direction), int(turns), _p(out)):
        return None
    return dict(Q1=out[0:3], Q2=out[3:6], n1=out[6:9], n2=out[9:12], sp=out[12], t=out[13], sq=out[14],
                amp=out[15], rho_g=out[16], caustic_j=bool(out[17]), dperp_P=out[18])


def seg_hits_body(body6, A, B):
    lib = _load()
    b, a_, bb = _d3(body6), _d3(A), _d3(B)
    return bool(lib.oracle_seg_hits_body(_p(b), _p(a_), _p(bb)))


def reflect(n, si, sr, E, eps=None):
    """One reflection of the complex field vector E at a face of unit normal
    n (ray along si in, sr out): PEC (eps None) or a dielectric half-space
    eps = (eps', eps''), eps_r = eps' - j eps''."""
    lib = _load()
    e = np.ascontiguousarray(np.stack([np.real(E), np.imag(E)], axis=1).reshape(-1).astype(np.float64))
    out = np.zeros(6)
    lib.oracle_reflect(_p(_d3(n)), _p(_d3(si)), _p(_d3(sr)), _p(e), 0 if eps is None else 1,
                       0.0 if eps is None else float(eps[0]), 0.0 if eps is None else float(eps[1]), _p(out))
    return out[0::2] + 1j * out[1::2]
