"""Throughput of the creeping-wave field evaluator (one JSON line on stdout).

Workload (one step): the 10 x 8 x 3 m room with 6 PEC faces (12 triangles)
and 20 PEC cylinders standing in for people, source at (1, 1, 2) m, the
256 x 256 receiver grid at z = 1.2 m, 2.4 / 5.8 / 28 GHz, planar reflections
up to order 2, the first creeping ray each way round every cylinder, FP32
bulk arithmetic: 65 536 receivers x 3 frequencies = 196 608 field samples.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

At N = 1 the line also carries "batched": the batched form on 64 crowd frames
(50 walking PEC cylinders, 16 frequencies in 24-30 GHz per frame, 1k-64k
receivers per frame, 1.12 M receivers in all) replayed from a captured CUDA
graph, with its own roofline and oracle comparison (--no-batched skips it),
"adjoint": one gradient step (fields, path list, rt_backward) on the room
with 200 PEC cylinders at 28 GHz, 64 x 64 receivers (--no-adjoint skips it),
and "extended_paths": the room workload with dielectric floor and walls,
creeping rays with up to two extra turns and wall-reflection -> creeping
paths, against the oracle on 512 sampled receivers (--no-extended skips it),
and "office": the large office (about 194k triangles, 110 bodies, 1M
receivers, reflections up to order 3 from a ray-launch candidate list, four
transmitters) (--no-office skips it).

N > 1 runs under torch.distributed (one process per GPU): one job of
256 x 256 N receivers, each rank evaluating its contiguous range of 65 536
with no data-path collective, the slices gathered on rank 0 after the timed
region; value = all ranks' samples / max-over-ranks time ("weak").
--impl reference times the FP64 oracle (oracle/) on the host cores instead.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "receiver field samples/s (GO+UTD creeping), error vs FP64 oracle (dB/rad)"
UNIT = "samples/s"
WORKLOAD = "room 10x8x3 m, 12 PEC triangles + 20 PEC cylinders, 256x256 rx at z=1.2 m, 2.4/5.8/28 GHz, refl<=2"

# Algorithmic FP32 work per unit (FFMA = 2 flops), the work model of the
# scope table: visibility tests, surface-ray geometry, image construction,
# Fock evaluation and per-path phase/accumulation.
UNIT_FLOPS = dict(seg_tri=30, seg_body=25, inside_tri=60, image_cand=60, body_refl=150, creep_geom=150,
                  fock_evals=60, path_freq=30)
# special-function (SFU) operations per unit: creeping geometry (tangent
# angles, sincos of the attachment angles, sqrt), Fock evaluation per
# polarisation pair (exp, sincos), the phase of a path at one frequency
# (sincos), reflection geometry (acos, atan2, sqrt), image normalisation.
UNIT_MUFU = dict(creep_geom=6, fock_evals=3, path_freq=2, body_refl=4, image_cand=1)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched crowd-frames measurement")
    ap.add_argument("--batched-steps", type=int, default=10)
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint (gradient) measurement")
    ap.add_argument("--no-office", action="store_true", help="skip the large-office measurement")
    ap.add_argument("--no-extended", action="store_true",
                    help="skip the extended path set (dielectric faces, extra turns, wall->creeping)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 form of the room workload")
    ap.add_argument("--office-rooms", type=int, nargs=2, default=(20, 15), metavar=("NX", "NY"),
                    help="rooms of the office building (a smaller building keeps an ncu capture small)")
    ap.add_argument("--only-office", action="store_true",
                    help="time the office alone (no room line extras); for profiling captures")
    ap.add_argument("--no-ring", action="store_true", help="skip the sphere-ring workload")
    ap.add_argument("--cpu-seconds", type=float, default=20.0, help="target CPU time of the oracle sample")
    return ap.parse_args()


def make_scene(rank=0, world=1):
    """The workload of one rank.  One job: the room with a 256 x (256 world)
    receiver grid at z = 1.2 m (cell centres; at one GPU the 256 x 256 grid).
    Rank r evaluates the contiguous receiver range shard(n, r, world) of it,
    65 536 receivers each (weak scaling), with no data-path exchange; the
    ranks' output slices gather into the single-rank layout."""
    from paper_2310_10578_gb300 import scenes, shard
    sc = scenes.room(nx=256, ny=256 * world)
    if world > 1:
        lo, hi = shard.shard(sc.n_rx, rank, world)
        sc.rx = np.ascontiguousarray(sc.rx[lo:hi])
    return sc


def max_over_ranks(values, device="cpu"):
    """Element-wise maximum of a list of floats over all ranks (the slowest
    rank's time decides the job's time); the identity on one process."""
    import torch
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def job_throughput(samples_per_rank, world, seconds):
    """Whole-job samples/s: every rank's samples over the max-over-ranks time."""
    return world * samples_per_rank / seconds


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return self.clocks_now()

    def clocks_now(self):
        """Summary of the samples taken so far (None if none)."""
        if not self.samples:
            return None
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for nm, v in zip(names, s[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# the class kernels' translation unit: its source and the headers it includes
KERNEL_SOURCES = ("paper_2310_10578_gb300/csrc/eval_fields.cu", "paper_2310_10578_gb300/csrc/devmath.cuh",
                  "paper_2310_10578_gb300/csrc/dual.cuh", "paper_2310_10578_gb300/csrc/internal.h",
                  "include/creep.h")


def _kernel_source_hash():
    """sha256[:16] of the concatenated kernel sources (the key of the ncu summaries)."""
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, rel), "rb").read())
    return h.hexdigest()[:16]


def _profiled(name="k_eval_room20_traffic.txt", key="dram_bytes_per_evaluation_full_workload"):
    """A per-evaluation counter from a committed ncu summary under profiles/,
    if it was taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    kv = {}
    for line in open(p):
        # "key: value" -- split at the first ": " (keys may hold a colon, e.g. sha256[:16])
        if ": " in line:
            k, v = line.split(": ", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel sources sha256[:16]") != _kernel_source_hash():
        return None
    try:
        return float(kv[key])
    except (KeyError, ValueError):
        return None


def _profiled_traffic():
    """DRAM bytes of one evaluation of the room (the three class kernels)."""
    return _profiled()


def _profiled_timed_step_read():
    """DRAM bytes read by the three class kernels of a timed room step (L2 as
    the bench leaves it after its flush), from the committed summary."""
    return _profiled(key="dram_read_bytes_per_evaluation_timed_step")


def hbm_peak():
    """The measured copy bandwidth of this machine's GPUs (MEASURED_PEAKS.json),
    else the stated fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(p))["hbm_gbs"]), "measured: MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback: 6.8 TB/s (no MEASURED_PEAKS.json)"


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle
    sc = make_scene()
    rng = np.random.default_rng(12345)
    oracle.build()
    cores = os.cpu_count() or 1
    # size one step: a few seconds of oracle work, and the whole run (warm-up
    # included) within about two minutes
    rate = _oracle_rate(oracle, sc, rng)
    step_s = min(4.0, 120.0 / max(1, args.steps + args.warmup))
    per_step = int(np.clip(rate * step_s, 64, sc.n_rx))
    times = []
    for it in range(args.warmup + args.steps):
        sub = sc.subset(rng.choice(sc.n_rx, per_step, replace=False))
        t0 = time.perf_counter()
        oracle.evaluate(sub, want_paths=False)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    samples = per_step * len(sc.freqs)
    value = samples * len(times) / sum(times)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "step": "%d random receivers x %d frequencies" % (per_step, len(sc.freqs))},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d random receivers of the 256x256 grid per step" % per_step},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _oracle_rate(oracle, sc, rng, probe_n=1024, threads=0):
    """Receivers per second of the oracle on this host (a warm-up call, then a
    timed random probe)."""
    oracle.evaluate(sc.subset(rng.choice(sc.n_rx, 64, replace=False)), want_paths=False, threads=threads)
    idx = rng.choice(sc.n_rx, probe_n, replace=False)
    t0 = time.perf_counter()
    oracle.evaluate(sc.subset(idx), want_paths=False, threads=threads)
    return probe_n / max(time.perf_counter() - t0, 1e-3)


# ---------------------------------------------------------------- CPU baseline + accuracy
def cpu_baseline_and_accuracy(sc, E_gpu, paths_fn, target_s):
    """The oracle (as it stands, all host cores) on a bounded random sample of
    the workload (the whole grid when it fits in target_s): its throughput, the
    GPU fields and path lists against it, the work counters of the sample, and
    a one-core throughput on a smaller sample."""
    from oracle import oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from parity import compare_fields, path_mismatches
    oracle.build()
    rng = np.random.default_rng(2024)
    rate = _oracle_rate(oracle, sc, rng)
    n = int(np.clip(rate * target_s, 512, sc.n_rx))
    idx = np.arange(sc.n_rx) if n >= sc.n_rx else np.sort(rng.choice(sc.n_rx, n, replace=False))
    sub = sc.subset(idx)
    t0 = time.perf_counter()
    ref = oracle.evaluate(sub)
    dt = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    st = compare_fields(E_gpu[:, :, idx], ref, flags=ref.flags, freqs=sc.freqs, check=False)
    codes, counts = paths_fn(idx)
    st["path_list_mismatches"] = len(path_mismatches(codes, counts, ref))
    rate1 = _oracle_rate(oracle, sc, rng, probe_n=256, threads=1)
    what = "all %d receivers" % n if n == sc.n_rx else "%d random receivers" % n
    base = {"value": n * len(sc.freqs) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%s of the 256x256 grid x %d freqs (%.1f s)" % (what, len(sc.freqs), dt),
            "value_1core": rate1 * len(sc.freqs)}
    return base, st, ref.counters, n


def algorithmic_flops(counters, n_sample, n_rx, n_f, units=UNIT_FLOPS):
    w = 0.0
    for k, c in units.items():
        if k == "path_freq":
            w += c * counters["paths"] * n_f
        else:
            w += c * counters[k]
    return w * n_rx / n_sample


# ---------------------------------------------------------------- batched crowd frames
def batched_crowd(args, creep, dev, flush, peak_fn):
    """The batched form: 64 crowd frames in one launch per path class,
    replayed from a captured graph; throughput, roofline and accuracy on
    sampled receivers of eight frames against the oracle."""
    import torch
    from paper_2310_10578_gb300 import scenes
    cw = scenes.crowd()
    n_f = len(cw.freqs[0])
    S = creep.Scene(cw.tri, cw.tri_face, np.zeros((0, 6)))
    S.set_tx(cw.tx, cw.pol)
    B = creep.Batch(S, cw.n_rx, n_f, max(len(b) for b in cw.bodies))
    for i in range(cw.n_frames):
        B.set_frame(i, cw.bodies[i], cw.freqs[i])
    rx = torch.tensor(B.rx_pack([r.T for r in cw.rx]), device=dev)
    out = torch.empty(6 * n_f * B.total_rx, dtype=torch.float32, device=dev)
    opts = creep.options(max_order=2)
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream())
    shape = B.tune(rx, out, opts=opts, stream=side)          # the batch's autotuner (tile shape)
    B.capture(rx, out, opts=opts, stream=side)
    for _ in range(3):
        B.replay(stream=side)
    side.synchronize()
    st, en = [], []
    for i in range(args.batched_steps):
        with torch.cuda.stream(side):
            flush.fill_(float(i))
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(side)
            B.replay(stream=side)
            b.record(side)
        st.append(a)
        en.append(b)
    side.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in zip(st, en)]))
    samples = B.total_rx * n_f
    stats = B.stats()
    res = {"workload": cw.name, "value": samples / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
           "steps": args.batched_steps, "frames": cw.n_frames, "n_rx_total": B.total_rx, "n_freq": n_f,
           "launch": "captured CUDA graph: counter resets + %d kernels (receiver spatial order: 3; planar, body "
                     "reflection, creeping)" % stats["kernel_launches"],
           "gpu_launches_per_step": stats["kernel_launches"],
           "tile_shape": {"planar_warps_per_tile": shape[0], "body_warps_per_tile": shape[1],
                          "planar_chunks_per_launch": shape[2], "chosen_by": "rt_batch_tune"},
           "fp64_escalated_candidates": stats["escalated_candidates"],
           "l2": "flushed between timed steps (256 MiB write)"}
    if not args.no_cpu_baseline:
        from oracle import oracle
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        from parity import compare_fields
        oracle.build()
        rng = np.random.default_rng(77)
        flat = out.detach().cpu().numpy().astype(np.float64)
        flops_frames = 0.0          # algorithmic work of the sampled frames (scaled to their receivers)
        mufu_frames = 0.0
        rx_frames = 0
        n_s = 0
        worst = {}
        t_cpu = 0.0
        for fr in rng.choice(cw.n_frames, 8, replace=False):
            idx = np.sort(rng.choice(cw.n_rx[fr], 256, replace=False))
            t0 = time.perf_counter()
            ref = oracle.evaluate(cw.frame(fr, idx))
            t_cpu += time.perf_counter() - t0
            a = int(B.rx_off[fr])
            n = cw.n_rx[fr]
            Eg = flat[6 * n_f * a: 6 * n_f * (a + n)].reshape(n_f, 3, n, 2)
            Eg = (Eg[..., 0] + 1j * Eg[..., 1])[:, :, idx]
            acc = compare_fields(Eg, ref, flags=ref.flags, freqs=cw.freqs[fr], check=False)
            for k, v in acc.items():
                if k.startswith("n_"):
                    worst[k] = worst.get(k, 0) + v
                elif isinstance(v, (int, float)):
                    worst[k] = max(worst.get(k, v), v)
            flops_frames += algorithmic_flops(ref.counters, len(idx), n, n_f)
            mufu_frames += algorithmic_flops(ref.counters, len(idx), n, n_f, UNIT_MUFU)
            rx_frames += n
            n_s += len(idx)
        # the sampled frames stand for all 64, in proportion to receivers
        flops = flops_frames * B.total_rx / rx_frames
        mufu = mufu_frames * B.total_rx / rx_frames
        res["roofline"] = peak_fn(flops, mufu, ms, None)
        res["roofline"]["kernel"] = "evaluation: k_eval<float, false, 1|2|4> over all frames"
        res["accuracy_vs_fp64_oracle"] = dict(worst, sample_receivers=n_s,
                                              sample="256 random receivers of each of 8 random frames")
        res["cpu_baseline"] = {"value": n_s * n_f / t_cpu, "unit": UNIT, "cores": os.cpu_count() or 1,
                               "kind": "oracle", "sample": "the accuracy sample (%.1f s)" % t_cpu}
    return res


# ---------------------------------------------------------------- adjoint
ZONE = ((6.0, 8.0), (4.0, 6.0))     # the adjoint workload's target zone: x in [6, 8] m, y in [4, 6] m


def zone_of(sc):
    (x0, x1), (y0, y1) = ZONE
    return np.nonzero((sc.rx[:, 0] >= x0) & (sc.rx[:, 0] <= x1) & (sc.rx[:, 1] >= y0) & (sc.rx[:, 1] <= y1))[0]


def _seed_zone_db(E, zone_mask):
    """dLoss/dE of the loss = sum over the zone's receivers of the received
    power in dB, 10 log10 sum|E|^2: 20/ln10 E/|E|^2 on the zone (zero where
    a zone receiver has no field), zero elsewhere."""
    import torch
    p = (E.double() ** 2).sum(dim=(0, 1, 3))
    g = torch.where((p > 0) & zone_mask, 20.0 / np.log(10.0) / torch.clamp(p, min=1e-300), torch.zeros_like(p))
    return (E.double() * g[None, None, :, None]).float()


def adjoint_room200(args, creep, dev, flush):
    """The adjoint form: the room with 200 PEC cylinders, 28 GHz, 64 x 64
    receivers; loss = sum over the target zone (x in [6, 8] m, y in [4, 6] m)
    of the received power in dB.  One gradient step = the fields with their
    path list (rt_evaluate_with_paths), the loss seed, and the adjoint
    (rt_backward), timed with FP64 dual numbers (the line's value) and with
    FP32 ones (beside it); the fields alone (rt_evaluate) beside both."""
    import torch
    from paper_2310_10578_gb300 import scenes
    sc = scenes.room(n_cyl=200, nx=64, ny=64, freqs=(28e9,))
    S = creep.Scene.from_scene(sc)
    rx = torch.tensor(sc.rx_soa(), device=dev)
    opts = creep.options(max_order=2)
    bopts = {"fp64": creep.options(max_order=2, precision=creep.RT_PREC_FP64),
             "fp32": creep.options(max_order=2, precision=creep.RT_PREC_FP32)}
    n = sc.n_rx
    zone = zone_of(sc)
    zmask = torch.zeros(n, dtype=torch.bool, device=dev)
    zmask[torch.tensor(zone, device=dev)] = True
    E = torch.empty((1, 3, n, 2), dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()
    out = {}
    for name, bo in bopts.items():
        for _ in range(3):
            _, codes, counts, _ = S.evaluate_with_paths(rx, cap=64, out=E, opts=opts)
            S.backward(rx, codes, counts, _seed_zone_db(E, zmask), opts=bo)
        torch.cuda.synchronize()
        marks = []
        for i in range(args.batched_steps):
            flush.fill_(float(i))
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(st)
            S.evaluate(rx, out=E, opts=opts)
            ev[1].record(st)
            _, codes, counts, _ = S.evaluate_with_paths(rx, cap=64, out=E, opts=opts)
            ev[2].record(st)
            gb, gt, gf = S.backward(rx, codes, counts, _seed_zone_db(E, zmask), opts=bo)
            ev[3].record(st)
            marks.append(ev)
        torch.cuda.synchronize()
        t = np.array([[m[k].elapsed_time(m[k + 1]) for k in range(3)] for m in marks])
        fwd, paths, bwd = (float(np.mean(t[:, k])) for k in range(3))
        out[name] = dict(fwd=fwd, paths=paths, bwd=bwd, gb=gb, gt=gt, n_paths=int(counts.sum()))
    o = out["fp64"]
    res = {"workload": "room 10x8x3 m, 12 PEC triangles + 200 PEC cylinders, 64x64 rx at z=1.2 m, 28 GHz, refl<=2",
           "loss": "sum over the target zone x in [6, 8] m, y in [4, 6] m (%d receivers) of received power in dB "
                   "(seed dLoss/dE = 20/ln10 E/|E|^2 on the zone)" % len(zone),
           "ms_fields_only": o["fwd"], "ms_fields_with_path_list": o["paths"], "ms_backward_incl_seed": o["bwd"],
           "ms_step": o["paths"] + o["bwd"],
           "value": n / ((o["paths"] + o["bwd"]) / 1e3), "unit": "receiver gradients/s (fields with path list + adjoint)",
           "duals": "FP64 (RT_PREC_FP64)",
           "paths": o["n_paths"], "steps": args.batched_steps,
           "gradients": "d/d(200 x (cx, cy, cz, a)), d/d(Tx), d/d(f)",
           "fp32_duals": {"ms_backward_incl_seed": out["fp32"]["bwd"],
                          "ms_step": out["fp32"]["paths"] + out["fp32"]["bwd"],
                          "value": n / ((out["fp32"]["paths"] + out["fp32"]["bwd"]) / 1e3),
                          "note": "RT_PREC_FP32: FP32 dual numbers on direct, planar and creeping paths, FP64 on "
                                  "reflections off bodies"},
           "l2": "flushed between timed steps (256 MiB write)"}
    if not args.no_cpu_baseline:
        try:
            acc = adjoint_oracle_sample(creep, S, sc, dev, opts, zone, {k: (v["gb"], v["gt"]) for k, v in out.items()})
            res.update(acc)
        except Exception as e:                      # the measurement above stands without it
            res["cpu_baseline"] = {"error": "%s: %s" % (type(e).__name__, e)}
    return res


def adjoint_oracle_sample(creep, S, sc, dev, opts, zone, grads):
    """The oracle beside the adjoint: the zone loss's gradient with respect
    to every body's centre and radius and the transmitter, by rt_backward
    (the timed steps' results, grads = {duals: (g_body, g_tx)}) and by the
    oracle's central differences of its per-path fields with the same path
    lists (visibility held fixed); the worst relative difference of each
    and the oracle's rate."""
    import torch
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import adjoint_ref
    from oracle import oracle
    oracle.build()
    rx = torch.tensor(sc.rx_soa(), device=dev)
    E, codes, counts, _ = S.evaluate_with_paths(rx, cap=64, opts=opts)
    zmask = torch.zeros(sc.n_rx, dtype=torch.bool, device=dev)
    zmask[torch.tensor(zone, device=dev)] = True
    gE = _seed_zone_db(E, zmask)
    torch.cuda.synchronize()
    c = codes.cpu().numpy().astype(np.uint64)
    k = counts.cpu().numpy()
    zset = set(int(r) for r in zone)
    # paths of the zone's receivers only (the seed is zero elsewhere)
    lists = [[int(x) for x in c[r, :min(int(k[r]), 64)]] if r in zset else [] for r in range(sc.n_rx)]
    g = gE.cpu().numpy().astype(np.float64)
    bodies = sorted({(cc >> 28) & 0xFFFFFFF for cs in lists for cc in cs if (cc >> 56) >= 3})
    t0 = time.perf_counter()
    ref = adjoint_ref.vjp(sc, lists, g[..., 0] + 1j * g[..., 1], bodies=bodies, freqs=False, cap=64)
    t_cpu = time.perf_counter() - t0

    def rel(got, want, absum):
        return abs(got - want) / max(abs(want), 1e-3 * absum, 1e-300)

    acc = {"bodies_checked": len(bodies), "zone_receivers": len(zone),
           "paths_skipped_by_reference": int(ref["skipped"]),
           "tolerance": "1e-3 relative (against max(|ref|, 1e-3 sum|contributions|))"}
    idle = [b for b in range(sc.bodies.shape[0]) if b not in set(bodies)]
    for name, (gb, gt) in grads.items():
        gb, gt = gb.cpu().numpy(), gt.cpu().numpy()
        acc[name] = {"tx_gradient_rel_err_max": float(max(rel(gt[i], ref["tx"][i], ref["tx_abs"][i]) for i in range(3))),
                     "body_gradient_rel_err_max": float(max([rel(gb[b, j], ref["body"][b][j], ref["body_abs"][b][j])
                                                             for b in bodies for j in range(4)] or [0.0])),
                     # bodies without a path to the zone must get exactly zero
                     "bodies_without_zone_paths_nonzero_gradient":
                         int(np.count_nonzero(np.any(gb[idle] != 0.0, axis=1))) if idle else 0}
    return {"accuracy_vs_fp64_oracle": acc,
            "cpu_baseline": {"value": len(zone) / t_cpu,
                             "unit": "receiver gradients/s (every body with zone paths + transmitter)",
                             "cores": os.cpu_count() or 1, "kind": "oracle central differences (h = 1e-5 m)",
                             "sample": "the zone's %d receivers (%.1f s)" % (len(zone), t_cpu)}}


def _time_eval(S, rx, out, opts, flush, steps, flags=None):
    """Mean CUDA-event time (ms) of S.evaluate over `steps` evaluations, the
    L2 flushed before each, after three untimed ones."""
    import torch
    st = torch.cuda.current_stream()
    for _ in range(3):
        S.evaluate(rx, out=out, flags=flags, opts=opts)
    torch.cuda.synchronize()
    ev = []
    for i in range(steps):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        S.evaluate(rx, out=out, flags=flags, opts=opts)
        e1.record(st)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in ev]))


def room_fp64(args, creep, dev, flush, base_ms):
    """The bench workload computed entirely in FP64 (RT_PREC_FP64: geometry,
    decisions, Fock evaluation, fields): its time beside the FP32 form's, and
    its fields and path lists against the oracle on sampled receivers."""
    import torch
    sc = make_scene()
    S = creep.Scene.from_scene(sc)
    rx = torch.tensor(sc.rx_soa(), device=dev)
    n, n_f = sc.n_rx, len(sc.freqs)
    opts = creep.options(max_order=2, precision=creep.RT_PREC_FP64)
    out = torch.empty((n_f, 3, n, 2), dtype=torch.float32, device=dev)
    ms = _time_eval(S, rx, out, opts, flush, max(3, args.batched_steps // 2))
    res = {"workload": WORKLOAD + ", FP64", "value": n * n_f / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
           "dtype": "f64", "fp64_over_fp32_time": ms / base_ms,
           "gpu_launches_per_step": S.stats()["kernel_launches"],
           "l2": "flushed between timed steps (256 MiB write)"}
    if not args.no_cpu_baseline:
        from oracle import oracle
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        from parity import compare_fields, path_mismatches
        oracle.build()
        idx = np.sort(np.random.default_rng(97).choice(n, 2048, replace=False))
        ref = oracle.evaluate(sc.subset(idx))
        Eg = out.detach().cpu().numpy().astype(np.float64)
        Eg = (Eg[..., 0] + 1j * Eg[..., 1])[:, :, idx]
        acc = compare_fields(Eg, ref, flags=ref.flags, freqs=sc.freqs, tol_rel=2e-6, dl=0.0, check=False)
        codes, counts, _ = S.paths(torch.tensor(sc.subset(idx).rx_soa(), device=dev), opts=opts)
        torch.cuda.synchronize()
        acc["path_list_mismatches"] = len(path_mismatches(codes.cpu().numpy(), counts.cpu().numpy(), ref))
        res["accuracy_vs_fp64_oracle"] = dict(acc, sample_receivers=len(idx),
                                              tolerance="|dE| <= 2e-6 sum|E_path| per receiver (FP64 mode)")
    return res


def sphere_ring_bench(args, creep, dev, flush):
    """The analytical-sphere workload (Sec. IV.A's validation case): PEC
    sphere a = 0.5 m, source at (3, 0, 0) m, 4096 receivers on the r = 2 m
    ring, 2.4 GHz, direct ray + GO reflection + first creeping ray each way;
    z-polarised (soft) and y-polarised (hard) source; FP64 (the
    configuration's precision) and FP32.  Every receiver against the oracle."""
    import torch
    from paper_2310_10578_gb300 import scenes
    res = {"workload": "PEC sphere a=0.5 m, Tx (3,0,0) m, 4096 rx on the r=2 m ring, 2.4 GHz, z- and y-polarised",
           "unit": UNIT, "l2": "flushed between timed steps (256 MiB write)", "cases": {}}
    for pol in ((0.0, 0.0, 1.0), (0.0, 1.0, 0.0)):
        sc = scenes.sphere_ring(pol=pol)
        S = creep.Scene.from_scene(sc)
        rx = torch.tensor(sc.rx_soa(), device=dev)
        n = sc.n_rx
        for prec, name in ((creep.RT_PREC_FP64, "fp64"), (creep.RT_PREC_FP32, "fp32")):
            opts = creep.options(max_order=0, precision=prec)
            out = torch.empty((1, 3, n, 2), dtype=torch.float32, device=dev)
            fl = torch.zeros(n, dtype=torch.int32, device=dev)
            ms = _time_eval(S, rx, out, opts, flush, args.batched_steps, flags=fl)
            case = {"value": n / (ms / 1e3), "ms_per_step": ms}
            if not args.no_cpu_baseline:
                from oracle import oracle
                sys.path.insert(0, os.path.join(ROOT, "tests"))
                from parity import compare_fields, path_mismatches
                oracle.build()
                t0 = time.perf_counter()
                ref = oracle.evaluate(sc)
                t_cpu = time.perf_counter() - t0
                Eg = out.detach().cpu().numpy().astype(np.float64)
                kw = dict(tol_rel=2e-6, dl=0.0) if name == "fp64" else {}
                acc = compare_fields(Eg[..., 0] + 1j * Eg[..., 1], ref, flags=ref.flags, freqs=sc.freqs,
                                     check=False, **kw)
                codes, counts, _ = S.paths(rx, opts=opts)
                torch.cuda.synchronize()
                acc["path_list_mismatches"] = len(path_mismatches(codes.cpu().numpy(), counts.cpu().numpy(), ref))
                acc["flags_equal"] = bool(np.array_equal(fl.cpu().numpy().astype(np.uint32) & 3, ref.flags & 3))
                case["accuracy_vs_fp64_oracle"] = acc
                case["cpu_baseline"] = {"value": n / t_cpu, "unit": UNIT, "cores": os.cpu_count() or 1,
                                        "kind": "oracle", "sample": "all 4096 receivers (%.2f s)" % t_cpu}
            res["cases"]["%s_%s" % ("zpol" if pol[2] else "ypol", name)] = case
    return res


def extended_room(args, creep, dev, flush, peak_fn, base_ms):
    """The room workload (20 cylinders, 256 x 256 receivers, 3 frequencies)
    with the extended path set: a dielectric floor and walls (PEC ceiling),
    creeping rays with up to two extra turns, and wall-reflection -> creeping
    paths.  Its time per evaluation beside the first-order set's, and the
    fields and path lists of 512 sampled receivers against the oracle."""
    import torch
    from paper_2310_10578_gb300 import scenes
    walls = (5.31, 0.48)
    sc = scenes.room(face_eps=[(4.0, 0.2), None, walls, walls, walls, walls])
    sc.max_enc = 2
    sc.wall_creep = True
    S = creep.Scene.from_scene(sc)
    rx = torch.tensor(sc.rx_soa(), device=dev)
    n, n_f = sc.n_rx, len(sc.freqs)
    opts = creep.options(max_order=2, enable=creep.RT_EN_ALL | creep.RT_EN_WALL_CREEP, max_encirclements=2)
    out = torch.empty((n_f, 3, n, 2), dtype=torch.float32, device=dev)
    shape = S.tune(rx, out=out, opts=opts)
    for _ in range(3):
        S.evaluate(rx, out=out, opts=opts)
    st = torch.cuda.current_stream()
    torch.cuda.synchronize()
    ms = []
    for i in range(args.batched_steps):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        S.evaluate(rx, out=out, opts=opts)
        e1.record(st)
        ms.append((e0, e1))
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ms]))
    stats = S.stats()
    res = {"workload": "room 10x8x3 m, dielectric floor (eps 4.0-0.2j) and walls (5.31-0.48j), PEC ceiling, "
                       "20 PEC cylinders, 256x256 rx, 2.4/5.8/28 GHz, refl<=2, creeping with <=2 extra turns, "
                       "wall->creeping paths",
           "value": n * n_f / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": args.batched_steps,
           "vs_first_order_set": ms / base_ms, "gpu_launches_per_step": stats["kernel_launches"],
           "tile_shape": {"planar_warps_per_tile": shape[0], "body_warps_per_tile": shape[1],
                          "planar_chunks_per_launch": shape[2], "chosen_by": "rt_tune"},
           "fp64_escalated_candidates": stats["escalated_candidates"],
           "l2": "flushed between timed steps (256 MiB write)"}
    if not args.no_cpu_baseline:
        from oracle import oracle
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        from parity import compare_fields, path_mismatches
        oracle.build()
        idx = np.sort(np.random.default_rng(91).choice(n, 512, replace=False))
        t0 = time.perf_counter()
        ref = oracle.evaluate(sc.subset(idx))
        t_cpu = time.perf_counter() - t0
        Eg = out.detach().cpu().numpy().astype(np.float64)
        Eg = (Eg[..., 0] + 1j * Eg[..., 1])[:, :, idx]
        acc = compare_fields(Eg, ref, flags=ref.flags, freqs=sc.freqs, check=False)
        codes, counts, _ = S.paths(torch.tensor(sc.subset(idx).rx_soa(), device=dev), opts=opts)
        torch.cuda.synchronize()
        acc["path_list_mismatches"] = len(path_mismatches(codes.cpu().numpy(), counts.cpu().numpy(), ref))
        res["accuracy_vs_fp64_oracle"] = dict(acc, sample_receivers=len(idx))
        flops = algorithmic_flops(ref.counters, len(idx), n, n_f)
        mufu = algorithmic_flops(ref.counters, len(idx), n, n_f, UNIT_MUFU)
        res["roofline"] = peak_fn(flops, mufu, ms, None)
        res["roofline"]["kernel"] = "evaluation: k_eval<float, false, 1|2|4|8> (planar, body reflection, creeping x3, " \
                                    "wall->creeping x3)"
        res["cpu_baseline"] = {"value": len(idx) * n_f / t_cpu, "unit": UNIT, "cores": os.cpu_count() or 1,
                               "kind": "oracle", "sample": "the accuracy sample (%.1f s)" % t_cpu}
    return res


def office_large(args, creep, dev, flush):
    """The large office: about 194k triangles (rooms, wall panels with doors,
    furniture boxes), 100 PEC cylinders and 10 PEC spheres, 1M receivers at
    1.2 m, 5.8 GHz, reflections up to order 3 from the candidate list of a
    4096-ray launch per transmitter, first-order creeping; four transmitters
    in turn.  A transmitter's step = its ray launch (candidate list), the
    list's upload, and the evaluation of every receiver, timed end to end
    on the host clock around a synchronised step (the evaluation alone with
    CUDA events beside it).  Against the oracle: the first transmitter's
    candidate list (the oracle's own launch, whole office), then 256 sampled
    receivers within 10 m of it (half among those with a path) evaluated by
    the oracle with ITS list."""
    import torch
    from paper_2310_10578_gb300 import scenes
    nrx, nry = args.office_rooms
    if (nrx, nry) == (20, 15):
        sc = scenes.office()
    else:
        # the same building recipe at a smaller size: furniture, bodies and
        # receivers in proportion to the floor area
        frac = nrx * nry / 300.0
        sc = scenes.office(n_rooms=(nrx, nry), n_furn=int(15000 * frac), n_cyl=max(4, int(100 * frac)),
                           n_sph=max(2, int(10 * frac)), nx=int(62.5 * nrx), ny=int(53.34 * nry))
    S = creep.Scene.from_scene(sc)
    n, n_f = sc.n_rx, len(sc.freqs)
    rx = torch.tensor(sc.rx_soa(), device=dev)
    out = torch.empty((n_f, 3, n, 2), dtype=torch.float32, device=dev)
    opts = creep.options(max_order=3)
    st = torch.cuda.current_stream()
    step_ms, cand_ms, host_ms, n_cand, cands, esc = [], [], [], [], [], []
    for i, t in enumerate(sc.txs):
        S.set_tx(t, sc.pol)
        # the host launch of the same rule, for reference (not in the step)
        t0 = time.perf_counter()
        host_list = S.candidates(4096, 3)
        host_ms.append(1e3 * (time.perf_counter() - t0))
        S.candidates_device(4096, 3)                     # warm-up of this transmitter
        S.evaluate(rx, out=out, opts=opts)
        torch.cuda.synchronize()
        stp, cdm = [], []
        for k in range(2):
            flush.fill_(float(k))
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(st)
            S.candidates_device(4096, 3)                 # the ray launch, on the device
            e1.record(st)
            S.evaluate(rx, out=out, opts=opts)
            e2.record(st)
            torch.cuda.synchronize()
            stp.append(e0.elapsed_time(e2))
            cdm.append(e0.elapsed_time(e1))
        step_ms.append(float(np.mean(stp)))
        cand_ms.append(float(np.mean(cdm)))
        esc.append(int(S.stats()["escalated_candidates"]))
        cand = S.get_candidates()
        n_cand.append(int(len(cand)))
        cands.append(cand)
        res_equal = bool(np.array_equal(cand, host_list))
        if i == 0:
            E0 = out.detach().cpu().numpy().astype(np.float64)
            dev_equals_host = [res_equal]
        else:
            dev_equals_host.append(res_equal)
    total_ms = float(np.sum(step_ms))
    res = {"workload": sc.name, "value": len(sc.txs) * n * n_f / (total_ms / 1e3), "unit": UNIT,
           "ms_per_step": total_ms,
           "step": "per transmitter: the device ray launch (4096 rays, candidate list) + the evaluation, one stream",
           "ms_per_tx": step_ms, "ms_candidates_per_tx": cand_ms, "ms_host_launch_per_tx_reference": host_ms,
           "device_list_equals_host_launch": dev_equals_host,
           "candidates_per_tx": n_cand, "n_triangles": int(sc.tri.shape[0]),
           "fp64_escalated_candidates_per_tx": esc,
           "gpu_launches_per_step": (S.stats()["kernel_launches"] + 2) * len(sc.txs), "roofline": None,
           "l2": "flushed between timed steps (256 MiB write)"}
    # roofline of the traversal-bound evaluation (transmitter 0): DRAM and L2
    # bytes of one evaluation from the committed ncu summary of the same
    # kernel source, over the evaluation's time in this run
    dram = _profiled("k_eval_office_traffic.txt")
    l2b = _profiled("k_eval_office_traffic.txt", "l2_bytes_per_evaluation_full_workload")
    if dram is not None and (nrx, nry) == (20, 15):
        t_eval = (step_ms[0] - cand_ms[0]) / 1e3
        peak, basis = hbm_peak()
        l2peak = creep.l2_peak()
        res["roofline"] = {
            "bound": "hbm", "achieved": dram / t_eval / 1e9, "peak": peak, "unit": "GB/s",
            "frac": dram / t_eval / 1e9 / peak, "traffic": dram, "peak_basis": basis,
            "kernel": "evaluation of transmitter 0: k_eval<float, false, 16|2|4> (candidate list, body "
                      "reflection, creeping), BVH visibility",
            "l2": {"achieved": l2b / t_eval / 1e9, "peak": l2peak, "unit": "GB/s", "frac": l2b / t_eval / 1e9 / l2peak,
                   "bytes": l2b, "peak_basis": "measured: L2 read microbenchmark rt_l2_peak in this run"},
            "note": "the BVH (194k triangles) and the scene stay in the 129 MB L2: DRAM carries the receivers and "
                    "fields only, the traversal reads the L2"}
    if not args.no_cpu_baseline:
        from oracle import oracle
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        from parity import compare_fields, path_mismatches
        oracle.build()
        sc.tx = np.asarray(sc.txs[0], dtype=np.float32)
        t0 = time.perf_counter()
        ocand = oracle.candidates(sc, 4096, 3)
        t_cand = time.perf_counter() - t0
        res["candidate_list_equals_oracle"] = bool(np.array_equal(ocand, cands[0]))
        res["oracle_candidates_s"] = t_cand
        sc.candidates = ocand
        # (receivers within 10 m of the transmitter: most of the building is
        # walled off from it and has no path at all)
        near = np.nonzero(np.hypot(sc.rx[:, 0] - sc.txs[0][0], sc.rx[:, 1] - sc.txs[0][1]) < 10.0)[0]
        # and, as the furniture hides most of them, half of the sample among
        # those with at least one path
        S.set_tx(sc.txs[0], sc.pol)
        S.set_candidates(ocand)
        _, cnt_near, _ = S.paths(torch.tensor(sc.subset(near).rx_soa(), device=dev), opts=opts)
        torch.cuda.synchronize()
        lit = near[cnt_near.cpu().numpy() > 0]
        rng = np.random.default_rng(93)
        idx = np.unique(np.concatenate([rng.choice(near, 128, replace=False),
                                        rng.choice(lit, min(128, len(lit)), replace=False)]))
        sub = sc.subset(idx)
        t0 = time.perf_counter()
        ref = oracle.evaluate(sub)
        t_cpu = time.perf_counter() - t0
        Eg = S.evaluate(torch.tensor(sub.rx_soa(), device=dev), opts=opts).cpu().numpy().astype(np.float64)
        acc = compare_fields(Eg[..., 0] + 1j * Eg[..., 1], ref, flags=ref.flags, freqs=sc.freqs, check=False)
        if res["candidate_list_equals_oracle"]:
            # the timed evaluation's own output at those receivers
            Et = (E0[..., 0] + 1j * E0[..., 1])[:, :, idx]
            acc["timed_output_equals_sample_evaluation"] = bool(np.array_equal(Et, Eg[..., 0] + 1j * Eg[..., 1]))
        codes, counts, _ = S.paths(torch.tensor(sub.rx_soa(), device=dev), opts=opts)
        torch.cuda.synchronize()
        acc["path_list_mismatches"] = len(path_mismatches(codes.cpu().numpy(), counts.cpu().numpy(), ref))
        res["accuracy_vs_fp64_oracle"] = dict(acc, sample_receivers=len(idx), transmitter=0,
                                              candidate_list="the oracle's own ray launch")
        res["cpu_baseline"] = {"value": len(idx) * n_f / t_cpu, "unit": UNIT, "cores": os.cpu_count() or 1,
                               "kind": "oracle (brute-force visibility)",
                               "sample": "the accuracy sample (%.1f s)" % t_cpu}
    return res


# ---------------------------------------------------------------- GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2310_10578_gb300 import build, creep
    build.build()
    if args.only_office:
        dev = torch.device("cuda", torch.cuda.current_device())
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        print(json.dumps({"office": office_large(args, creep, dev, flush)}), flush=True)
        return 0
    sc = make_scene(rank, world)
    S = creep.Scene.from_scene(sc)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    rx = torch.tensor(sc.rx_soa(), device=dev)
    n_rx, n_f = sc.n_rx, len(sc.freqs)
    out = torch.empty((n_f, 3, n_rx, 2), dtype=torch.float32, device=dev)
    opts = creep.options(max_order=2)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2
    shape = S.tune(rx, out=out, opts=opts)          # the scene's autotuner (tile shape), before any timing

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 3)):
        S.evaluate(rx, out=out, opts=opts)
    barrier()
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    nvtx = torch.cuda.nvtx      # names the timed evaluations for a profiler's range filter
    for i in range(args.steps):
        flush.fill_(float(i))                        # evict L2 between timed steps
        starts[i].record(stream)
        nvtx.range_push("room_step")
        S.evaluate(rx, out=out, opts=opts)
        nvtx.range_pop()
        ends[i].record(stream)
    barrier()
    dev_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    # ---- e2e: host buffers through rt_evaluate_host, copies inside the timed region
    rx_host = torch.tensor(sc.rx_soa()).pin_memory()
    out_host = torch.empty((n_f, 3, n_rx, 2), dtype=torch.float32).pin_memory()
    lib = creep.load()
    import ctypes
    h = S._h

    def e2e_once():
        rc = lib.rt_evaluate_host(h, ctypes.c_void_p(rx_host.data_ptr()), n_rx, ctypes.c_void_p(out_host.data_ptr()),
                                  None, ctypes.byref(opts), ctypes.c_void_p(stream.cuda_stream))
        if rc != 0:
            raise RuntimeError(lib.rt_last_error().decode())

    for _ in range(3):
        e2e_once()
    barrier()
    e2e_t = []
    for i in range(args.steps):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_once()
        e2e_t.append(time.perf_counter() - t0)
    barrier()
    gathered = None
    if world > 1:
        # the optional gather of the ranks' slices into the job's layout
        # (after the timed regions; the evaluation itself exchanges nothing)
        from paper_2310_10578_gb300 import shard
        full = shard.gather_fields(out, 256 * 256 * world)
        if rank == 0:
            gathered = {"shape": list(full.shape), "finite": bool(torch.isfinite(full).all())}
    props = torch.cuda.get_device_properties(dev)
    # measured FP32 FFMA and SFU rates (microbenchmarks of the library), the
    # roofline's denominators; the peak derived from unit counts and clock
    # is kept beside them
    ffma_meas, mufu_meas = creep.alu_peaks()

    def peak_fn(flops, mufu, ms_eval, traffic):
        c = (sampler.clocks_now() if sampler else None) or {}
        sm_max = c.get("sm_max_mhz") or 2070.0
        derived = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
        achieved = flops / (ms_eval / 1e3) / 1e12
        mufu_rate = mufu / (ms_eval / 1e3) / 1e9
        return {"bound": "alu", "achieved": achieved, "peak": ffma_meas, "unit": "TFLOP/s",
                "frac": achieved / ffma_meas, "traffic": traffic,
                "peak_basis": "measured: FFMA microbenchmark rt_alu_peaks in this run",
                "peak_derived": derived,
                "peak_derived_basis": "%d SMs x 128 FP32 lanes x 2 x %.0f MHz" % (props.multi_processor_count, sm_max),
                "work_per_evaluation_flops": flops,
                "sfu": {"achieved": mufu_rate, "peak": mufu_meas, "unit": "Gop/s", "frac": mufu_rate / mufu_meas,
                        "peak_basis": "measured: ex2.approx microbenchmark rt_alu_peaks in this run",
                        "work_per_evaluation_ops": mufu}}

    batched = None
    if world == 1 and not args.no_batched:
        batched = batched_crowd(args, creep, dev, flush, peak_fn)
    adj = None
    if world == 1 and not args.no_adjoint:
        adj = adjoint_room200(args, creep, dev, flush)
    office = None
    if world == 1 and not args.no_office:
        office = office_large(args, creep, dev, flush)
    ext = None
    if world == 1 and not args.no_extended:
        ext = extended_room(args, creep, dev, flush, peak_fn, float(np.mean(dev_ms)))
    fp64 = ring = None
    if world == 1 and not args.no_fp64:
        fp64 = room_fp64(args, creep, dev, flush, float(np.mean(dev_ms)))
    if world == 1 and not args.no_ring:
        ring = sphere_ring_bench(args, creep, dev, flush)
    clocks = sampler.stop() if sampler else None

    ms, e2e_s = max_over_ranks([np.mean(dev_ms), np.mean(e2e_t)], device=dev)
    samples = n_rx * n_f
    value = job_throughput(samples, world, ms / 1e3)
    e2e_value = job_throughput(samples, world, e2e_s)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    launches_per_step = S.stats()["kernel_launches"]      # our kernels per evaluation (one step)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_rx": n_rx, "n_freq": n_f, "n_cylinders": int(sc.bodies.shape[0]),
                       "n_triangles": int(sc.tri.shape[0]), "max_refl_order": 2, "precision": "fp32",
                       "l2": "flushed between timed steps (256 MiB write)",
                       "tile_shape": {"planar_warps_per_tile": shape[0], "body_warps_per_tile": shape[1],
                                      "planar_chunks_per_launch": shape[2], "chosen_by": "rt_tune"}},
            "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 3 * 4 * n_rx,
                    "d2h_bytes_per_step": n_f * 3 * n_rx * 8},
            "gpu_launches": launches_per_step * args.steps,
            "roofline": None, "cpu_baseline": None}
    stats = S.stats()
    line["config"]["fp64_escalated_candidates"] = stats["escalated_candidates"]
    if world > 1:
        line["config"]["sharding"] = {"job_receivers": 256 * 256 * world, "per_rank": n_rx,
                                      "partition": "contiguous receiver ranges, no data-path collective",
                                      "gathered_on_rank0": gathered}
    if world == 1 and not args.no_cpu_baseline:
        E_gpu = out.detach().cpu().numpy().astype(np.float64)
        E_gpu = E_gpu[..., 0] + 1j * E_gpu[..., 1]

        def paths_fn(idx):
            rx_sub = torch.tensor(sc.subset(idx).rx_soa(), device=dev)
            codes, counts, _ = S.paths(rx_sub, opts=opts)
            torch.cuda.synchronize()
            return codes.cpu().numpy(), counts.cpu().numpy()

        base, acc, counters, n_s = cpu_baseline_and_accuracy(sc, E_gpu, paths_fn, args.cpu_seconds)
        line["cpu_baseline"] = base
        line["accuracy_vs_fp64_oracle"] = dict(acc, sample_receivers=n_s)
        flops = algorithmic_flops(counters, n_s, n_rx, n_f)
        mufu = algorithmic_flops(counters, n_s, n_rx, n_f, UNIT_MUFU)
        # the unit timed is one evaluation: the three class kernels, which
        # overlap through programmatic dependent launch (their durations are
        # not separable with events); per-kernel shares are in the ncu launch
        # list under profiles/
        line["roofline"] = peak_fn(flops, mufu, ms, _profiled_traffic())
        line["roofline"]["traffic_basis"] = ("ncu, caches flushed before each of the three class kernels: the "
                                             "body kernels' read-modify-writes of the outputs read DRAM")
        line["roofline"]["timed_step_dram_read"] = _profiled_timed_step_read()
        line["roofline"]["algorithmic_bytes"] = n_rx * (12 + 24 * n_f)
        line["roofline"]["kernel"] = "evaluation: k_eval<float, false, 1|2|4> (planar, body reflection, creeping)"
    if batched is not None:
        line["batched"] = batched
    if adj is not None:
        line["adjoint"] = adj
    if ext is not None:
        line["extended_paths"] = ext
    if office is not None:
        line["office"] = office
    if fp64 is not None:
        line["fp64"] = fp64
    if ring is not None:
        line["sphere_ring"] = ring
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
