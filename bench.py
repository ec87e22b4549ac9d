#!/usr/bin/env python3
"""Throughput of the improved W-stacking grid + degrid path on one GB300.

Metric: visibilities per second through ``ws_degrid`` AND ``ws_grid`` (one
unit = one visibility degridded from the model image and gridded back into a
dirty image), W = 7, x0 = 0.25, on the survey-scale workload: a 2048 x 2048
image over l, m in +-0.25 (FFT grid 4096 x 4096, ~490 w-planes) and 9,987,840
visibilities from 256 antennas in a 10 km disc on 8 h tracks at declination
-30.  Inputs are seeded synthetic data (``paper_2101_11172_gb300.synth``).

One step = ws_degrid(model image) + ws_grid(visibilities) with inputs already
in HBM; ``value`` = M x ranks / (max over ranks of the step time).  ``e2e``
repeats the step from pinned host buffers, copies included.  The per-stage
device times come from the library's own CUDA events (WS_FLAG_TIMING) on the
launching stream inside the timed region.

``--impl reference`` times the FP64 CPU oracle (the method written step by
step from the paper, numpy + plain C) on a bounded slab of the same workload.

Multi-GPU: every rank runs an independent replica of the workload (different
observations need no exchange); there is no data-path collective.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "visibilities/sec grid+degrid at W=7,x0=0.25 (err vs DFT), % HBM roofline"
UNIT = "vis/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["survey", "tiny", "profile", "reduced", "batched"], default="survey")
    ap.add_argument("--e2e-steps", type=int, default=6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--oracle-full", action="store_true",
                    help="also run the whole workload through the oracle on every core (minutes) and compare "
                         "every GPU output with it")
    ap.add_argument("--no-folded", action="store_true", help="skip the real-sky folded timing")
    ap.add_argument("--deterministic", action="store_true",
                    help="bit-for-bit reproducible gridding (WS_FLAG_DETERMINISTIC)")
    ap.add_argument("--real-sky", action="store_true",
                    help="fold w < 0 onto -w (Section 5.4, WS_FLAG_HERMITIAN): real image, real dirty image")
    return ap.parse_args()


def load_workload(name: str):
    from paper_2101_11172_gb300 import synth
    if name == "tiny":
        return synth.tiny("A")
    if name == "profile":
        return synth.survey_slab()
    if name == "reduced":
        return synth.reduced_cost()
    return synth.survey()


def workload_config(wl, extra=None):
    cfg = {"workload": wl.name, "image": wl.N, "grid": None, "W": wl.W, "x0": wl.x0,
           "fov_rad": wl.fov, "visibilities": wl.M, "w_range": [round(x, 3) for x in wl.w_range],
           "l2": "inputs larger than L2 (w-stack and visibility arrays far above 129 MB)"}
    if extra:
        cfg.update(extra)
    return cfg


# -- clocks -------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                        rows.append(parts)
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        smax = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
        loaded = [s for s in sm if s >= 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


# -- roofline ------------------------------------------------------------------

def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def stage_bytes(stage: str, N: int, Np: int, Nw: int, total_planes: int, M: int, nchunks: int):
    """Algorithmic bytes of ONE launch of a stage: what that kernel must move.

    These are the dense figures of the method: every cell of every w-plane is
    moved once per pass.  Per plane, gridding writes the full N' x N' plane
    once (grid3d); the column transform reads it and writes back the N crop
    rows (cols_inv); the row transform reads those rows and, once per chunk,
    the running sum (rows_inv).  Degridding mirrors it: the row transform
    reads the image and z once per chunk and writes N rows per plane
    (rows_fwd); the column transform reads them and writes the full plane
    (cols_fwd); degrid3d reads the stack once.  Records are 32 B per
    visibility.  Stages that run once per plane chunk divide by the chunk
    count.  The library's own occupied-byte counts (ws_stats_t stage_bytes)
    give what the kernels must move when they skip the tiles and strips no
    footprint touches; both are reported.
    """
    c8 = 8
    full, crop = Np * Np * c8, N * Np * c8
    planes = total_planes / nchunks
    if stage == "grid3d":
        return planes * full + M * 32 / nchunks
    if stage == "cols_inv":
        return planes * (full + crop)
    if stage == "rows_inv":
        return planes * crop + N * N * (8 + 16 + 16 + 4 + 8)
    if stage == "rows_fwd":
        return N * N * 16 + planes * crop
    if stage == "cols_fwd":
        return planes * (crop + full)
    if stage == "degrid3d":
        return planes * full + M * (32 + 8) / nchunks
    if stage == "prep":
        return M * (24 + 4 + 32)
    if stage == "correct":
        return N * N * (8 + 4 + 8)
    return None


def _code_tokens(text: str) -> str:
    """C/C++/CUDA source with comments removed and whitespace runs collapsed (string
    and character literals kept as they are), so that editing a comment leaves the
    hash of the code unchanged."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def library_source_sha() -> str:
    """Hash of the library's device code (the kernels, and the headers that shape their
    arguments), comments and layout aside: any change to the code invalidates the DRAM
    counters of profiles/traffic.json.  Host-only files (plan construction, batches,
    the least-misfit fit) are left out."""
    import glob
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2101_11172_gb300", "csrc", "*"))):
        if f.endswith((".cu", ".cuh")) or os.path.basename(f) in ("ws_internal.hpp", "fft_plan.hpp"):
            with open(f, encoding="utf-8") as fh:
                h.update(_code_tokens(fh.read()).encode())
    return h.hexdigest()


def traffic_for(stage: str, occupied_bytes_per_launch, planes_per_launch):
    """DRAM bytes of one launch of a stage, scaled from the committed ncu summary
    (profiles/traffic.json: one capture of each kernel on the small profiling
    workload, DRAM bytes beside the same launch's occupied algorithmic bytes and
    w-planes).  A kernel's DRAM traffic grows in proportion to the occupied tiles and
    strips it processes, or, for inv_rows' whole-row copies, to its planes; the
    capture's ratio times this launch's figure is the traffic of a full launch.  None
    if the library's device code changed since the capture, or the stage was not
    captured."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            data = json.load(f)
        ent = data.get("stages", {}).get(stage)
        if not ent or data.get("source_sha256") != library_source_sha():
            return None
        if ent.get("scale") == "planes":
            return int(round(ent["dram_bytes_per_launch"] / ent["planes"] * planes_per_launch))
        if occupied_bytes_per_launch:
            return int(round(ent["dram_bytes_per_launch"] / ent["occupied_bytes_per_launch"]
                             * occupied_bytes_per_launch))
    except (OSError, ValueError, KeyError, TypeError, ZeroDivisionError):
        pass
    return None


# -- the oracle on every host core ---------------------------------------------------
#
# The FP64 oracle (Algorithms 5 and 6 step by step, numpy + plain C) is timed as it
# stands; only the harness is parallel.  Both operators are linear in the visibility
# set, so the visibilities are split by the plane of their first tap into contiguous
# slabs, one per spawned process, and each process runs the oracle's ws.degrid and
# ws.grid on its own visibilities over the planes their footprints cover (adjacent
# slabs share W - 1 planes).  The dirty images add up; the visibilities are disjoint.
# Inputs and outputs sit in shared memory.  Processes are spawned, never forked: the
# parent has already made CUDA calls.

_ORACLE = {}


def _shared(name, shape, dtype):
    from multiprocessing import shared_memory

    import numpy as np
    shm = shared_memory.SharedMemory(name=name)
    return shm, np.ndarray(shape, dtype=dtype, buffer=shm.buf)


def _oracle_init(spec):
    """Per process: attach the shared inputs and outputs, fit the kernel and make the
    per-image correction (plan work, outside every timing)."""
    from oracle import wstack as ows
    from oracle.geometry import make_geometry
    from oracle.lmfit import least_misfit
    o = _ORACLE
    o.update(spec)
    o["handles"] = []
    for key in ("uvw", "vis", "image", "vout", "dout"):
        shm, arr = _shared(*spec[key])
        o["handles"].append(shm)
        o[key + "_a"] = arr
    g = make_geometry(spec["N"], spec["x0"], spec["W"], spec["fov"], 0.0, 0.0)
    o["lm"] = least_misfit(spec["W"], g.x0)
    ows.correction(g, o["lm"])


def _oracle_part(job):
    """One slab: Algorithm 6 then Algorithm 5 on the visibilities idx, written to the
    shared outputs (visibilities at idx, dirty image in slot `slot`); returns seconds."""
    import numpy as np

    from oracle import wstack as ows
    from oracle.geometry import make_geometry
    slot, idx = job
    o = _ORACLE
    uvw = np.ascontiguousarray(o["uvw_a"][idx])
    vis = o["vis_a"][idx].astype(np.complex128)
    g = make_geometry(o["N"], o["x0"], o["W"], o["fov"], float(uvw[:, 2].min()), float(uvw[:, 2].max()))
    t = time.perf_counter()
    v = ows.degrid(g, o["lm"], o["image_a"], uvw)
    d = ows.grid(g, o["lm"], uvw, vis)
    dt = time.perf_counter() - t
    o["vout_a"][idx] = v
    o["dout_a"][slot] = d
    return dt


class OraclePool:
    """The oracle on `procs` spawned processes sharing one workload (see above)."""

    def __init__(self, wl, procs=None):
        import multiprocessing as mp
        from multiprocessing import shared_memory

        import numpy as np

        from oracle.geometry import first_tap, make_geometry
        self.wl = wl
        self.procs = procs or os.cpu_count() or 1
        self.g = make_geometry(wl.N, wl.x0, wl.W, wl.fov, *wl.w_range)
        self.t0 = first_tap(wl.uvw[:, 2] * self.g.nscale, wl.W)[0]
        self.order = np.argsort(self.t0, kind="stable")
        self._shm = []

        def share(key, arr):
            shm = shared_memory.SharedMemory(create=True, size=max(1, arr.nbytes))
            view = np.ndarray(arr.shape, dtype=arr.dtype, buffer=shm.buf)
            view[...] = arr
            self._shm.append(shm)
            return (shm.name, arr.shape, arr.dtype), view

        spec = {"N": wl.N, "x0": wl.x0, "W": wl.W, "fov": wl.fov}
        spec["uvw"], _ = share("uvw", np.ascontiguousarray(wl.uvw, dtype=np.float64))
        spec["vis"], _ = share("vis", np.ascontiguousarray(wl.vis))
        spec["image"], _ = share("image", np.ascontiguousarray(wl.image, dtype=np.complex128))
        spec["vout"], self.vout = share("vout", np.zeros(wl.M, dtype=np.complex128))
        spec["dout"], self.dout = share("dout", np.zeros((self.procs, wl.N, wl.N), dtype=np.complex128))
        self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_oracle_init, initargs=(spec,))

    # The oracle's cost of one visibility (its W^3 spread and gather over W planes),
    # in units of one plane's cost (transforms, screen, crop): measured on the survey.
    VIS_PER_PLANE_COST = 2.5e-5

    def slabs(self, idx_sorted, t_lo, t_hi):
        """Split visibilities (sorted by first tap) into up to `procs` slabs of contiguous
        first-tap planes with equal estimated cost (planes plus visibilities)."""
        import numpy as np
        t = self.t0[idx_sorted]
        planes = np.arange(t_lo, t_hi + 1)
        counts = np.bincount(t - t_lo, minlength=planes.size)
        cost = np.cumsum(1.0 + self.VIS_PER_PLANE_COST * counts)
        bounds = np.searchsorted(cost, cost[-1] * np.arange(1, self.procs) / self.procs, side="left")
        cuts = np.searchsorted(t, planes[np.minimum(bounds + 1, planes.size - 1)], side="left")
        return [part for part in np.split(idx_sorted, np.unique(cuts)) if part.size]

    def run(self, parts):
        """Wall seconds of one parallel pass over the given visibility sets."""
        self.dout[...] = 0
        t = time.perf_counter()
        self.pool.map(_oracle_part, list(enumerate(parts)), chunksize=1)
        return time.perf_counter() - t

    def full_pass(self):
        """The whole workload: every visibility through every w-plane; returns (seconds, vis, dirty)."""
        parts = self.slabs(self.order, int(self.t0.min()), int(self.t0.max()))
        dt = self.run(parts)
        return dt, self.vout.copy(), self.dout.sum(0)

    def slab_step(self, rng, per_slab=2000, dense=False):
        """A bounded sample: `procs` slabs of W planes, each with up to per_slab
        visibilities whose footprints lie inside it; the slabs are spread over the
        w-range, or (dense) put on the planes where the most footprints start.
        Returns (seconds, planes, visibilities)."""
        import numpy as np
        W = self.wl.W
        if dense:
            counts = np.bincount(self.t0 - self.t0.min())
            starts = self.t0.min() + np.argsort(counts)[::-1][:self.procs]
        else:
            starts = np.linspace(self.t0.min(), self.t0.max(), self.procs).astype(np.int64)
        parts = []
        for ta in starts:
            pool_idx = np.nonzero(self.t0 == ta)[0]
            if pool_idx.size:
                parts.append(rng.choice(pool_idx, min(per_slab, pool_idx.size), replace=False))
        dt = self.run(parts)
        return dt, len(parts) * W, sum(p.size for p in parts)

    def close(self):
        self.pool.close()
        self.pool.join()
        for shm in self._shm:
            shm.close()
            shm.unlink()


def oracle_vis_cost(pool, rng, few=2000, many=60000):
    """Wall seconds per visibility of the parallel oracle: two passes over the same
    dense slabs (the planes where most footprints start) that differ only in how many
    visibilities each slab holds, after one untimed pass (the processes' first pass
    pays for first-touch allocations and transform set-up)."""
    pool.slab_step(rng, few, dense=True)
    t_few, _, n_few = pool.slab_step(rng, few, dense=True)
    t_many, _, n_many = pool.slab_step(rng, many, dense=True)
    return max(0.0, (t_many - t_few) / (n_many - n_few)) if n_many > n_few else 0.0


def oracle_rate_from_slabs(pool, rng, c_vis):
    """Whole-job oracle rate from one bounded slab pass: the pass gives the wall cost per
    plane once its visibilities' share (c_vis each) is taken out; the job is Nw planes
    and M visibilities."""
    wl = pool.wl
    t, planes, n = pool.slab_step(rng, 4000)
    c_plane = max(0.0, (t - n * c_vis) / max(1, planes))
    total = pool.g.Nw * c_plane + wl.M * c_vis
    return wl.M / total, t, (c_plane, planes, n)


def oracle_sample_text(pool, c_plane, c_vis, n):
    wl = pool.wl
    return (f"per step: {pool.procs} processes, each one slab of {wl.W} of the {pool.g.Nw} w-planes (spread over the "
            f"w-range) with up to 4000 visibilities whose footprints lie in it ({n} in all): {c_plane:.3f} wall s per "
            f"plane; {1e6 * c_vis:.2f} wall us per visibility from two passes over the {pool.procs} densest slabs "
            f"(2000 and 60000 visibilities each); on {pool.procs} cores, extrapolated to {pool.g.Nw} planes and "
            f"{wl.M} visibilities")


def run_reference(args):
    """The oracle arm: each step is a bounded sample (slabs of W planes on every host core),
    extrapolated to the whole job's visibilities per second."""
    import numpy as np
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = load_workload(args.workload)
    pool = OraclePool(wl)
    rng = np.random.default_rng(77)
    try:
        c_vis = oracle_vis_cost(pool, rng)              # warm-up: two passes
        for _ in range(max(0, args.warmup - 2)):
            oracle_rate_from_slabs(pool, rng, c_vis)
        vals, times, last = [], [], None
        for _ in range(args.steps):
            v, dt, last = oracle_rate_from_slabs(pool, rng, c_vis)
            vals.append(v)
            times.append(dt)
    finally:
        pool.close()
    value = len(vals) / sum(1.0 / v for v in vals)
    c_plane, planes, n = last
    sample = oracle_sample_text(pool, c_plane, c_vis, n)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(wl, {"oracle": f"FP64 numpy + C, {pool.procs} processes"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.procs, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# -- replicas: one process per GPU, each with its own copy of the workload ----------------

def max_over_ranks(x: float, device=None) -> float:
    """The slowest rank's time (a no-op without an initialised process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    on = device if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=on)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(m_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job visibilities per second: every rank's visibilities over the slowest rank's time."""
    return m_per_rank * world / (ms_max / 1e3)


# -- the batched serving workload -----------------------------------------------

def run_batched(args):
    """64 independent instances (images 512^2 .. 2048^2, 10^4 .. 5x10^6 visibilities):
    aggregate grid + degrid throughput of one ws_batch call pair against the same
    instances run one after another through single plans, and sampled errors against
    the exact DFT per instance."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_11172_gb300 import synth
    from paper_2101_11172_gb300.batch import Batch
    from paper_2101_11172_gb300.wstack import Plan

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    wls = synth.batched()
    M_total = sum(w.M for w in wls)
    uvw = [torch.from_numpy(w.uvw).to(dev) for w in wls]
    img = [torch.from_numpy(w.image.astype(np.complex64)).to(dev) for w in wls]
    vis = [torch.from_numpy(w.vis).to(dev) for w in wls]
    stream = torch.cuda.current_stream(dev)
    b = Batch([(w.N, w.fov, w.w_range[0], w.w_range[1], w.M) for w in wls], wls[0].x0, wls[0].W, device=dev)
    vout = [torch.empty(w.M, dtype=torch.complex64, device=dev) for w in wls]
    dout = [torch.empty(w.N, w.N, dtype=torch.complex64, device=dev) for w in wls]

    def step():
        b.degrid(img, uvw, out=vout)
        b.grid(uvw, vis, out=dout)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clocks:
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    # the same instances, one plan at a time (each with its own full w-stack)
    ms_seq = 0.0
    for i, w in enumerate(wls):
        with Plan(w.N, w.x0, w.W, w.fov, *w.w_range, device=dev) as p:
            p.degrid(img[i], uvw[i], out=vout[i])
            p.grid(uvw[i], vis[i], out=dout[i])
            torch.cuda.synchronize(dev)
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            p.degrid(img[i], uvw[i], out=vout[i])
            p.grid(uvw[i], vis[i], out=dout[i])
            a1.record(stream)
            torch.cuda.synchronize(dev)
            ms_seq += a0.elapsed_time(a1)
    Ns = [w.N for w in wls]
    line = {"metric": "visibilities/sec grid+degrid, 64-instance batch at W=7,x0=0.25", "value": M_total / (ms / 1e3),
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "dtype": "f32 (FP64 coordinates and phase arguments)", "data": "synthetic",
            "config": {"workload": "batched-64", "instances": len(wls), "visibilities": M_total,
                       "images": {str(n): Ns.count(n) for n in sorted(set(Ns))},
                       "visibility_range": [min(w.M for w in wls), max(w.M for w in wls)],
                       "branches": b.branches},
            "sequential": {"value": M_total / (ms_seq / 1e3), "ms_per_step": ms_seq,
                           "what": "the same 64 instances through single plans, one after another"},
            "speedup_vs_sequential": ms_seq / ms,
            "accuracy": "per-instance errors against the exact DFT: tests/test_gpu_batch.py",
            "clocks": clocks.summary()}
    b.close()
    print(json.dumps(line), flush=True)
    return 0


# -- our path -----------------------------------------------------------------

def accuracy_sample(wl, v_gpu, d_gpu, n_vis=10_000, n_pix=1024, real_sky=False):
    """Relative RMS error against the exact DFT on sampled outputs (the real
    part of the dirty image for a folded real-sky plan), and the worst sampled
    output's error in units of the reference's RMS.  The grid DFT costs
    n_pix x M complex exponentials on every host core."""
    import numpy as np

    from oracle import dft
    from oracle.geometry import make_geometry
    g = make_geometry(wl.N, wl.x0, wl.W, wl.fov, *wl.w_range)
    rng = np.random.default_rng(1234)
    kv = rng.choice(wl.M, n_vis, replace=False)
    nz_rows, nz_cols = np.nonzero(wl.image)            # the skies are sparse or compact
    v_ref = dft.dft_degrid(wl.uvw[kv], dft.pixel_lmn(g, nz_rows, nz_cols), wl.image[nz_rows, nz_cols])
    ev = float(np.linalg.norm(v_gpu[kv] - v_ref) / np.linalg.norm(v_ref))
    rows = rng.integers(0, wl.N, n_pix)
    cols = rng.integers(0, wl.N, n_pix)
    d_ref = dft.dft_grid(wl.uvw, wl.vis, dft.pixel_lmn(g, rows, cols))
    if real_sky:
        d_ref = d_ref.real
        d_gpu = d_gpu.real
    ed = float(np.linalg.norm(d_gpu[rows, cols] - d_ref) / np.linalg.norm(d_ref))

    def worst(a, ref):
        return float(np.abs(a - ref).max() / np.sqrt(np.mean(np.abs(ref) ** 2)))
    return {"degrid_rel_rms_vs_dft": ev, "grid_rel_rms_vs_dft": ed, "sampled_vis": n_vis, "sampled_pixels": n_pix,
            "degrid_worst_over_rms": worst(v_gpu[kv], v_ref), "grid_worst_over_rms": worst(d_gpu[rows, cols], d_ref)}


def main():
    args = parse_args()
    if args.warmup < 3:
        print("warning: --warmup raised to 3", file=sys.stderr)
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_11172_gb300 import WS_FLAG_DETERMINISTIC, WS_FLAG_HERMITIAN, WS_FLAG_TIMING, _lib
    from paper_2101_11172_gb300.wstack import Plan

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    def barrier():
        if world > 1:
            dist.barrier()

    wl = load_workload(args.workload)
    M = wl.M
    flags = WS_FLAG_TIMING
    if args.deterministic:
        flags |= WS_FLAG_DETERMINISTIC
    if args.real_sky:
        flags |= WS_FLAG_HERMITIAN
        wl.image = wl.image.real.astype(np.complex128)
    plan = Plan(wl.N, wl.x0, wl.W, wl.fov, *wl.w_range, flags=flags, device=dev)
    uvw = torch.from_numpy(wl.uvw).to(dev)
    vis = torch.from_numpy(wl.vis.astype(np.complex64)).to(dev)
    img = torch.from_numpy(wl.image.astype(np.complex64)).to(dev)
    vout = torch.empty(M, dtype=torch.complex64, device=dev)
    dout = torch.empty(wl.N, wl.N, dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.degrid(img, uvw, out=vout)
        plan.grid(uvw, vis, out=dout)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if plan.last_status != _lib.WS_OK:
        raise RuntimeError(f"ws status {plan.last_status}")
    plan.stats(reset=True)

    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clocks:
        barrier()
        torch.cuda.synchronize(dev)
        start.record(stream)
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            step()
        stop.record(stream)
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter() - t_wall
        barrier()
    ms = start.elapsed_time(stop) / args.steps
    st = plan.stats(reset=True)
    ms = max_over_ranks(ms, dev)
    value = replica_value(M, world, ms)

    # the same step with the uvw set bound to the plan (ws_plan_bind_uvw): the tap rule and
    # the tile sort are made once, as an iterative imager would use the pair
    plan.bind(uvw)
    for _ in range(2):
        step()
    torch.cuda.synchronize(dev)
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    for _ in range(args.steps):
        step()
    b1.record(stream)
    torch.cuda.synchronize(dev)
    ms_bound = max_over_ranks(b0.elapsed_time(b1) / args.steps, dev)
    plan.bind(None)
    plan.stats(reset=True)
    bound = {"value": replica_value(M, world, ms_bound), "unit": UNIT, "ms_per_step": ms_bound,
             "what": "uvw bound to the plan once (ws_plan_bind_uvw): calls skip pre-processing and binning"}

    # end to end: pinned host inputs -> device -> both calls -> results back to pinned host,
    # pipelined over two buffer sets: step i+1's inputs go up and step i-1's results come
    # down on a copy stream while step i computes; every step's copies are inside the timing
    h_uvw = torch.from_numpy(wl.uvw).pin_memory()
    h_vis = torch.from_numpy(wl.vis.astype(np.complex64)).pin_memory()
    h_img = torch.from_numpy(wl.image.astype(np.complex64)).pin_memory()
    h_vout = torch.empty(M, dtype=torch.complex64).pin_memory()
    h_dout = torch.empty(wl.N, wl.N, dtype=torch.complex64).pin_memory()
    cs = torch.cuda.Stream(dev)
    d_in = [(torch.empty_like(uvw), torch.empty_like(vis), torch.empty_like(img)) for _ in range(2)]
    d_out = [(torch.empty_like(vout), torch.empty_like(dout)) for _ in range(2)]
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]

    def upload(j):
        b = j % 2
        with torch.cuda.stream(cs):
            cs.wait_event(ev_done[b])                # the step that last read buffer set b is done
            for d, h in zip(d_in[b], (h_uvw, h_vis, h_img)):
                d.copy_(h, non_blocking=True)
            ev_in[b].record(cs)

    def run_e2e(nsteps):
        upload(0)
        for i in range(nsteps):
            if i + 1 < nsteps:
                upload(i + 1)
            b = i % 2
            stream.wait_event(ev_in[b])
            du, dv, di = d_in[b]
            vo, do = d_out[b]
            plan.degrid(di, du, out=vo)
            plan.grid(du, dv, out=do)
            ev_done[b].record(stream)
            with torch.cuda.stream(cs):
                cs.wait_event(ev_done[b])
                h_vout.copy_(vo, non_blocking=True)
                h_dout.copy_(do, non_blocking=True)
        stream.wait_stream(cs)

    run_e2e(2)
    torch.cuda.synchronize(dev)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    cs.wait_event(e0)
    run_e2e(max(2, args.e2e_steps))
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_e2e = e0.elapsed_time(e1) / max(2, args.e2e_steps)
    ms_e2e = max_over_ranks(ms_e2e, dev)
    h2d = wl.uvw.nbytes + M * 8 + wl.N * wl.N * 8
    d2h = M * 8 + wl.N * wl.N * 8
    plan.stats(reset=True)

    # the same step with Section 5.4's folding, when the sky is real (as the survey's is)
    folded = None
    if world == 1 and not args.real_sky and not args.no_folded and not np.any(wl.image.imag):
        plan_r = Plan(wl.N, wl.x0, wl.W, wl.fov, *wl.w_range, flags=WS_FLAG_HERMITIAN, device=dev)

        def step_r():
            plan_r.degrid(img, uvw, out=vout)
            plan_r.grid(uvw, vis, out=dout)

        for _ in range(args.warmup):
            step_r()
        torch.cuda.synchronize(dev)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            step_r()
        f1.record(stream)
        torch.cuda.synchronize(dev)
        ms_r = f0.elapsed_time(f1) / args.steps
        folded = {"value": M / (ms_r / 1e3), "unit": UNIT, "ms_per_step": ms_r, "w_planes": plan_r.Nw,
                  "what": "WS_FLAG_HERMITIAN: the real sky's w < 0 visibilities folded onto -w (Section 5.4); "
                          "errors of this mode are in --real-sky runs and tests/test_gpu_parity.py"}
        plan_r.close()
        step()                                    # leave vout / dout as the main mode's results
        torch.cuda.synchronize(dev)

    if rank != 0:
        plan.close()
        if world > 1:
            dist.destroy_process_group()
        return 0

    # stage breakdown and roofline of the dominant kernel of this library
    peak, peak_src = measured_peaks()
    total_planes = -(-plan.Nw // 8) * 8
    nchunks = -(-total_planes // plan.planes_per_chunk)
    stages = {}
    for name, tot in st["stage_ms"].items():
        n = st["stage_launches"][name]
        if n == 0 or tot == 0:
            continue
        per_launch_ms = tot / n
        b = stage_bytes(name, wl.N, plan.Np, plan.Nw, total_planes, M, nchunks)
        ob = st["stage_bytes"][name] / n if st["stage_bytes"][name] > 0 else None
        stages[name] = {"ms_per_step": tot / args.steps, "launches_per_step": n / args.steps,
                        "ms_per_launch": per_launch_ms,
                        "algorithmic_gb_per_launch": None if b is None else b / 1e9,
                        "gbs": None if b is None else b / (per_launch_ms / 1e3) / 1e9,
                        "occupied_gb_per_launch": None if ob is None else ob / 1e9,
                        "occupied_gbs": None if ob is None else ob / (per_launch_ms / 1e3) / 1e9}
    ours = stages
    dom = max(ours, key=lambda k: ours[k]["ms_per_step"])
    d = stages[dom]
    occ_b = None if d["occupied_gb_per_launch"] is None else d["occupied_gb_per_launch"] * 1e9
    traffic = traffic_for(dom, occ_b, min(plan.Nw, total_planes // nchunks))
    t_s = d["ms_per_launch"] / 1e3
    roof = {"kernel": dom, "bound": "hbm", "achieved": d["gbs"], "peak": peak, "unit": "GB/s",
            "frac": None if d["gbs"] is None else d["gbs"] / peak, "peak_source": peak_src,
            "traffic": traffic,
            "bytes_model": "dense: every cell of every w-plane moved once per pass (the method's algorithmic bytes)",
            "occupied": None if occ_b is None else {
                "achieved": d["occupied_gbs"], "frac": d["occupied_gbs"] / peak, "bytes_per_launch": occ_b,
                "model": "only the tiles and column strips some visibility footprint touches (ws_stats_t "
                         "stage_bytes), plus the kernel's inputs and outputs"},
            "traffic_gbs": None if traffic is None else traffic / t_s / 1e9,
            "traffic_frac": None if traffic is None else traffic / t_s / 1e9 / peak}
    # the CPU baseline leg: the only place this arm runs the oracle (its rate, and
    # the exact DFT on sampled outputs for the error half of the metric)
    cpu, acc = None, {}
    if world == 1 and not args.no_cpu_baseline:
        v_np = vout.cpu().numpy().astype(np.complex128)
        d_np = dout.cpu().numpy().astype(np.complex128)
        if not args.no_accuracy:
            acc = accuracy_sample(wl, v_np, d_np, real_sky=args.real_sky)
        # the oracle on every host core: bounded slab passes by default; with --oracle-full
        # the whole workload timed in full, its results a full-size reference for the GPU's
        pool = OraclePool(wl)
        try:
            rng = np.random.default_rng(77)
            c_vis = oracle_vis_cost(pool, rng)
            v_cpu, _, (c_plane, _, n) = oracle_rate_from_slabs(pool, rng, c_vis)
            cpu = {"value": v_cpu, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
                   "sample": oracle_sample_text(pool, c_plane, c_vis, n)}
            if args.oracle_full:
                t_cpu, v_or, d_or = pool.full_pass()
                cpu["full_pass"] = {
                    "value": M / t_cpu, "wall_s": t_cpu,
                    "what": f"the whole workload, timed in full: {M} visibilities degridded and gridded through all "
                            f"{pool.g.Nw} w-planes, split by first-tap plane into cost-balanced slabs on "
                            f"{pool.procs} spawned processes"}
        finally:
            pool.close()
        if args.oracle_full and not args.real_sky:
            def worst(a, ref):
                return float(np.abs(a - ref).max() / np.sqrt(np.mean(np.abs(ref) ** 2)))
            acc.update({"degrid_rel_rms_vs_oracle": float(np.linalg.norm(v_np - v_or) / np.linalg.norm(v_or)),
                        "grid_rel_rms_vs_oracle": float(np.linalg.norm(d_np - d_or) / np.linalg.norm(d_or)),
                        "degrid_worst_over_rms_vs_oracle": worst(v_np, v_or),
                        "grid_worst_over_rms_vs_oracle": worst(d_np, d_or),
                        "vs_oracle": f"all {M} visibilities and all {wl.N}x{wl.N} pixels"})
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (FP64 coordinates and phase arguments)", "data": "synthetic",
            "config": workload_config(wl, {"grid": plan.Np, "w_planes": plan.Nw,
                                           "planes_per_chunk": plan.planes_per_chunk,
                                           "real_sky_folding": bool(args.real_sky),
                                           "deterministic_gridding": bool(args.deterministic),
                                           "parallelism": f"replicas x{world}"}),
            "e2e": {"value": replica_value(M, world, ms_e2e), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e,
                    "copies": "pinned host <-> device on a second stream, overlapping the neighbouring steps"},
            "gpu_launches": None,
            "roofline": roof, "stages": stages, "accuracy": acc, "clocks": clocks.summary(),
            "real_sky_folded": folded, "bound_uvw": bound,
            "cpu_baseline": cpu, "wall_s_timed": t_wall}
    line["gpu_launches"] = int(round(sum(stages[k]["launches_per_step"] for k in ours) * args.steps))
    print(json.dumps(line), flush=True)
    plan.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
