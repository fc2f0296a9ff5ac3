"""Differentiable field evaluation: a torch.autograd.Function over the C ABI.

forward  -- rt_evaluate_with_paths: the FP32 fields and, from the same
            kernels, the path list at fixed receivers for the given body
            centres/radii, transmitter position and frequencies;
backward -- rt_backward: the adjoint of the evaluation with the path list of
            the forward pass held fixed (visibility frozen), each path's
            geometry and field recomputed in dual numbers: FP64 ones by
            default (Static.grad_precision), FP32 ones on request.

Argument marshalling only: every step runs in libcreep.so.  The loss is the
caller's (PyTorch) function of the fields, e.g. received power in dB over a
zone (see ``power_db``).
"""
import numpy as np
import torch

from . import creep


class Static:
    """What stays fixed across evaluations: the triangles (and their faces),
    every body's type and height, the polarisation, the receivers (CUDA
    float32 tensor [3, n]), the options, the path-list capacity, the face
    materials and (large scenes) the candidate face sequences."""

    def __init__(self, tri, tri_face, body_type, body_h, pol, rx_soa, opts=None, cap=256, face_mat=None,
                 candidates=None, grad_precision=None):
        self.tri = np.asarray(tri, dtype=np.float32)
        self.tri_face = None if tri_face is None else np.asarray(tri_face, dtype=np.int32)
        self.body_type = np.asarray(body_type, dtype=np.float64).reshape(-1)
        self.body_h = np.asarray(body_h, dtype=np.float64).reshape(-1)
        self.pol = np.asarray(pol, dtype=np.float32).reshape(3)
        self.rx = rx_soa
        self.opts = opts if opts is not None else creep.options(max_order=2)
        self.cap = int(cap)
        self.face_mat = face_mat              # per face (kind, eps', eps'') or None (PEC)
        self.candidates = candidates          # candidate face sequences [n, 3] (large scenes) or None
        # the adjoint's dual numbers: FP64 by default -- a loss like received
        # power in dB seeds dLoss/dE = E/|E|^2, which multiplies the field
        # derivatives' FP32 error by the sum's conditioning near interference
        # nulls; creep.RT_PREC_FP32 for the faster FP32 form
        o = self.opts
        self.grad_opts = creep.options(o.max_order, o.enable,
                                       creep.RT_PREC_FP64 if grad_precision is None else grad_precision,
                                       o.max_encirclements)

    @classmethod
    def from_scene(cls, sc, rx_soa, opts=None, cap=256):
        return cls(sc.tri, sc.tri_face, sc.bodies[:, 0], sc.bodies[:, 5], sc.pol, rx_soa,
                   opts if opts is not None else creep.options(
                       max_order=sc.max_order, max_encirclements=getattr(sc, "max_enc", 0),
                       enable=creep.RT_EN_ALL | (creep.RT_EN_WALL_CREEP if getattr(sc, "wall_creep", False) else 0)),
                   cap,
                   getattr(sc, "face_eps", None), getattr(sc, "candidates", None))

    def scene(self, body_params, tx, freqs):
        """An rt_scene for parameters body_params [n, 4] (cx, cy, cz, a), tx [3], freqs [n_f]."""
        p = body_params.detach().cpu().numpy().astype(np.float64).reshape(-1, 4)
        bodies = np.stack([self.body_type, p[:, 0], p[:, 1], p[:, 2], p[:, 3], self.body_h], axis=1)
        S = creep.Scene(self.tri, self.tri_face, bodies)
        S.set_tx(tx.detach().cpu().numpy(), self.pol)
        S.set_freqs(freqs.detach().cpu().numpy().astype(np.float64))
        if self.face_mat is not None:
            S.set_face_materials(self.face_mat)
        if self.candidates is not None:
            S.set_candidates(self.candidates)
        return S


class CreepField(torch.autograd.Function):
    """E [n_f, 3, n, 2] (float32) as a function of body_params [n_body, 4],
    tx [3] and freqs [n_f] (any float dtype; gradients come back in it)."""

    @staticmethod
    def forward(ctx, body_params, tx, freqs, static):
        S = static.scene(body_params, tx, freqs)
        E, codes, counts, _ = S.evaluate_with_paths(static.rx, cap=static.cap, opts=static.opts)
        ctx.S, ctx.static = S, static
        ctx.save_for_backward(codes, counts)
        ctx.dtypes = (body_params.dtype, tx.dtype, freqs.dtype)
        ctx.devs = (body_params.device, tx.device, freqs.device)
        return E

    @staticmethod
    def backward(ctx, grad_E):
        codes, counts = ctx.saved_tensors
        gb, gt, gf = ctx.S.backward(ctx.static.rx, codes, counts, grad_E, opts=ctx.static.grad_opts)
        (db, dt, df), (vb, vt, vf) = ctx.dtypes, ctx.devs
        return gb.to(device=vb, dtype=db), gt.to(device=vt, dtype=dt), gf.to(device=vf, dtype=df), None


def field(body_params, tx, freqs, static):
    return CreepField.apply(body_params, tx, freqs, static)


def power_db(E, zone=None):
    """Received power per receiver in dB, 10 log10(sum over frequencies and
    components of |E|^2), over the receivers of `zone` (index tensor or mask)."""
    p = (E.to(torch.float64) ** 2).sum(dim=(0, 1, 3))
    if zone is not None:
        p = p[zone]
    return 10.0 * torch.log10(p)


# ---- several GPUs: receivers are independent, so each rank evaluates a
# contiguous share of them and the parameter gradients (body centres and
# radii, transmitter, frequencies) are summed over the ranks: the one
# collective of the adjoint (shard.py holds both).
from .shard import allreduce_gradients, shard  # noqa: E402,F401
