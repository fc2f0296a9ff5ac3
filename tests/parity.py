"""Shared comparison helpers for the GPU-vs-oracle parity tests.

Tolerance (derived from the arithmetic).  Each path's contribution is
computed in FP32 with double-float path lengths:
  * amplitude and Fock-function error: a few 1e-6 relative (table
    interpolation, residue truncation, FP32 transcendental functions);
  * phase: the straight legs are exact double-float lengths, but the surface
    arc t = a * dpsi of a creeping ray and the reflection-point angles come
    from FP32 angles (about 1 ulp each at ~pi), i.e. a length error of at most
    DL_FP32 = 3e-7 m, a phase error k * DL_FP32 (2e-4 rad at 28 GHz).
So every receiver satisfies
    |E_gpu - E_oracle| <= (TOL_REL + k DL_FP32) * sum_paths |E_path|
whatever the cancellation between paths.  Where the coherent sum is well
conditioned (kappa = sum|E_path| / |E| <= KAPPA_MAX) this bounds the |E|
error by 0.05 dB and the phase error by 1e-3 rad, the targets, which are
asserted there too; max and p99 over all compared receivers are reported.
"""
import numpy as np

TOL_REL = 2e-5
DL_FP32 = 3e-7
KAPPA_MAX = 5.0
C0 = 299792458.0
FLAG_SEMANTIC = 1 | 2        # inside, caustic


def gpu_fields(t):
    a = t.detach().cpu().numpy().astype(np.float64)
    return a[..., 0] + 1j * a[..., 1]


def compare_fields(Eg, ref, flags=None, freqs=None, tol_rel=TOL_REL, dl=DL_FP32, kappa_max=KAPPA_MAX,
                   db_tol=0.05, ph_tol=1e-3, check=True):
    """Compare GPU fields Eg [n_f, 3, n] with the oracle's; assert the bounds
    (check=True) or only report them (check=False).  The statistics count
    the receivers beyond the field bound (n_over_bound) and the compared
    (frequency, receiver) samples beyond the dB / phase targets (n_over_db_ph)."""
    Eo, sabs = ref.E, ref.sabs
    err = np.linalg.norm(Eg - Eo, axis=1)                  # [n_f, n]
    if freqs is None:
        freqs = np.zeros(Eo.shape[0])
    k = 2 * np.pi * np.asarray(freqs, dtype=np.float64) / C0
    tol = (tol_rel + k * dl)[:, None]
    bound = tol * sabs + 1e-12
    worst = float(np.max(err / (sabs + 1e-30)))
    rel = err / (tol * sabs + 1e-30)
    fi, ri = np.unravel_index(np.argmax(rel), rel.shape)
    n_over = int(np.sum(np.any(err > bound, axis=0)))
    assert not check or n_over == 0, "max |dE|/sum|E_path| = %.3e (worst vs bound at f=%d rx=%d: %.3e of %.3e; E_gpu=%s E_ref=%s)" % (
        worst, fi, ri, err[fi, ri] / (sabs[fi, ri] + 1e-30), tol[fi, 0], Eg[fi, :, ri], Eo[fi, :, ri])
    amp_o = np.linalg.norm(Eo, axis=1)
    amp_g = np.linalg.norm(Eg, axis=1)
    ok = (amp_o > 0) & (sabs <= kappa_max * amp_o)
    if flags is not None:
        ok &= (np.asarray(flags)[None, :] & FLAG_SEMANTIC) == 0
    stats = dict(rel=worst, worst_over_bound=float(rel[fi, ri]), n_over_bound=n_over, n_cmp=int(ok.sum()))
    if ok.any():
        db = np.abs(20 * np.log10(amp_g[ok] / amp_o[ok]))
        # phase of the dominant component
        idx = np.argmax(np.abs(Eo), axis=1)                 # [n_f, n]
        Eo_d = np.take_along_axis(Eo, idx[:, None, :], 1)[:, 0, :]
        Eg_d = np.take_along_axis(Eg, idx[:, None, :], 1)[:, 0, :]
        ph = np.abs(np.angle(Eg_d[ok] / Eo_d[ok]))
        stats.update(db_max=float(db.max()), db_p99=float(np.percentile(db, 99)),
                     ph_max=float(ph.max()), ph_p99=float(np.percentile(ph, 99)),
                     n_over_db_ph=int(np.sum((db > db_tol) | (ph > ph_tol))))
        if check:
            assert db.max() <= db_tol, stats
            assert ph.max() <= ph_tol, stats
    stats.update(all_samples(Eg, Eo, sabs, flags, db_tol, ph_tol))
    return stats


KAPPA_BINS = (1.0, 2.0, 5.0, 10.0, 100.0, 1e3, np.inf)


def all_samples(Eg, Eo, sabs, flags=None, db_tol=0.05, ph_tol=1e-3):
    """|dB| and phase errors over EVERY compared sample (each frequency and
    receiver with a field and no semantic flag), whatever its conditioning,
    with the histogram of kappa = sum|E_path| / |E| and the worst errors per
    kappa bin.  Reported beside the kappa <= KAPPA_MAX statistics; nothing is
    asserted here (the per-sample bound of compare_fields is the assertion)."""
    amp_o = np.linalg.norm(Eo, axis=1)
    amp_g = np.linalg.norm(Eg, axis=1)
    ok = amp_o > 0
    if flags is not None:
        ok &= (np.asarray(flags)[None, :] & FLAG_SEMANTIC) == 0
    out = {"n_all": int(ok.sum())}
    if not ok.any():
        return out
    kap = sabs[ok] / amp_o[ok]
    with np.errstate(divide="ignore"):
        db = np.abs(20 * np.log10(np.maximum(amp_g[ok], 1e-300) / amp_o[ok]))
    idx = np.argmax(np.abs(Eo), axis=1)
    Eo_d = np.take_along_axis(Eo, idx[:, None, :], 1)[:, 0, :]
    Eg_d = np.take_along_axis(Eg, idx[:, None, :], 1)[:, 0, :]
    ph = np.abs(np.angle(Eg_d[ok] / Eo_d[ok]))
    # the same error measured against the scale of the paths: |dE| / sum|E_path|
    rel = np.linalg.norm(Eg - Eo, axis=1)[ok] / sabs[ok]
    out.update(db_max_all=float(db.max()), db_p99_all=float(np.percentile(db, 99)),
               ph_max_all=float(ph.max()), ph_p99_all=float(np.percentile(ph, 99)),
               n_all_over_db_ph=int(np.sum((db > db_tol) | (ph > ph_tol))),
               rel_to_path_sum_max_all=float(rel.max()))
    hist = []
    lo = 0.0
    for hi in KAPPA_BINS:
        m = (kap > lo) & (kap <= hi) if lo > 0 else (kap <= hi)
        if m.any():
            hist.append({"kappa": [lo, None if np.isinf(hi) else hi], "n": int(m.sum()),
                         "db_max": float(db[m].max()), "ph_max": float(ph[m].max())})
        lo = hi
    out["kappa_hist"] = hist
    return out


def path_mismatches(codes, counts, ref):
    """Receivers whose GPU path list differs from the oracle's (indices)."""
    codes = np.asarray(codes).astype(np.uint64)
    counts = np.asarray(counts)
    return [r for r in range(len(counts))
            if counts[r] != ref.counts[r] or not np.array_equal(np.sort(codes[r, :counts[r]]), ref.paths[r])]


def compare_paths(codes, counts, ref, idx=None):
    codes = codes.detach().cpu().numpy().astype(np.uint64)
    counts = counts.detach().cpu().numpy()
    n = len(counts)
    bad = []
    for r in range(n):
        ro = r if idx is None else idx[r]
        if counts[r] != ref.counts[ro] or not np.array_equal(np.sort(codes[r, :counts[r]]), ref.paths[ro]):
            bad.append(r)
    assert not bad, "path lists differ at %d receivers, first %s" % (len(bad), bad[:5])
    return int(counts.sum())
