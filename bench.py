"""Benchmark: Gpixels/s of bit-exact morphological reconstruction on GB300.

Default workload (one step): the 512-image uneven batch (sides log-uniform in
256..4096, u8 / u16 with p = 1/2, the first half h-dome dilations, the second half
fill-holes, 8-connectivity; 970 Mpx), reconstructed as "batched + learned": the
learned work estimator orders the batch's tiles (features, MLP, counting sort) and
one persistent launch reconstructs every image, both replayed from CUDA graphs.
Inputs are seeded synthetic data resident in HBM; markers are restored by a device
copy and L2 is flushed (256 MiB write) before every timed step, both outside the
timed events. The same line reports, on the same images, the plain per-image loop
(one iwpp_reconstruct call per image) and the batched static form, the dominant
kernel's roofline, an end-to-end number through the C ABI from pinned host buffers,
and the CPU oracle on the host's cores; `forms` repeats the three forms on the other
four workloads (512^2 noise blur, 4096^2 tissue with conn 8 and 4, the 16384^2
sparse-seed image, the 256-image batch).

Prints ONE JSON line (rank 0). `--impl reference` times the CPU oracle (Vincent's
hybrid in C, one image per host thread) on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Gpixels/s morph. reconstruction (bit-exact); batched+learned vs plain; %HBM peak"
UNIT = "Gpixels/s"
L2_FLUSH_BYTES = 256 << 20


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def host_cores() -> int:
    return len(os.sched_getaffinity(0))


# ---- the five workloads -------------------------------------------------------------------
WORKLOADS = {
    "noiseblur512": "C1: noise-blur 512x512 u8 (5x5 box mean of uniform noise), marker = mask-40, dilation conn 8",
    "tissue4096": ("C2: tissue 4096x4096 u8 (2000 blobs r 5-40, peak 80-255, over U{0..30} noise), h-dome "
                   "marker h=30, dilation with conn 8 and with conn 4 (2 images)"),
    "seeds16384": ("C3: blob field 16384x16384 u8 (2000 blobs), marker 0 except 1000 seed pixels equal to "
                   "the mask, dilation conn 8"),
    "batch256": ("C4: 256 images, sides log-uniform 256-4096, u8/u16, first half h-dome dilation "
                 "(h 10-60), second half fill-holes (erosion), conn 8"),
    "batch512": ("C5: 512 images generated like C4 (another seed stream), the learned schedule's test "
                 "batch; estimator trained on 50k 64x64 blocks from runs of C1-C3"),
}


def load_workload(name: str):
    from paper_1605_00930_gb300 import synth
    if name == "noiseblur512":
        return [synth.noise_blur_case()]
    if name == "tissue4096":
        c = synth.tissue_case()
        return [c, synth.Case(c.marker, c.mask, 4, "dilate")]
    if name == "seeds16384":
        return [synth.sparse_seed_case()]
    if name == "batch256":
        return synth.mixed_batch(256, workload_id=4, workers=min(16, host_cores()))
    if name == "batch512":
        return synth.mixed_batch(512, workload_id=5, workers=min(16, host_cores()))
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """Samples nvidia-smi clocks / throttle reasons in the background."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.rows, self.proc, self.gpu = [], None, gpu_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [x.strip() for x in line.split(",")]))

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self, t0: float, t1: float):
        if not self.rows:
            return None
        inside = [r for t, r in self.rows if t0 <= t <= t1] or [self.rows[-1][1]]
        sm = [float(r[1]) for r in inside if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in inside if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in inside:
            for k, n in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(inside)}


# The sources the reconstruction kernels are built and launched from (their digest keys the
# ncu traffic record: a change to any of them makes the record stale).
KERNEL_SOURCES = ["paper_1605_00930_gb300/csrc/iwpp_api.cu",
                  "paper_1605_00930_gb300/csrc/iwpp_engine.cuh", "paper_1605_00930_gb300/csrc/iwpp_host.h",
                  "paper_1605_00930_gb300/csrc/iwpp_kern_reg.cu", "paper_1605_00930_gb300/csrc/iwpp_regtile.cuh",
                  "paper_1605_00930_gb300/csrc/iwpp_kern_coop.cu", "paper_1605_00930_gb300/csrc/iwpp_coop.cuh",
                  "paper_1605_00930_gb300/csrc/iwpp_scan.cuh", "paper_1605_00930_gb300/csrc/iwpp_feat.cuh",
                  "paper_1605_00930_gb300/csrc/iwpp_spread.h", "paper_1605_00930_gb300/csrc/iwpp_sched.cu"]


def kernel_digest() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def _traffic_from_profiles(kernel: str, workload: str):
    """ncu DRAM bytes per launch recorded under profiles/ for this kernel, workload and the
    current kernel sources (None when there is no such record)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    digest = kernel_digest()
    name = kernel.replace(" ", "")   # records name the kernel without spaces
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and parts[0] == name and parts[1] == workload and parts[2] == digest:
            return float(parts[3])
    return None


def max_over_ranks(x: float, world: int, device) -> float:
    """The slowest rank's time: every rank of the replicas contributes, all get the max."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_gpx_s(world: int, pix_per_step: int, ms_per_step: float) -> float:
    """Whole-job throughput of `world` replicas, each doing `pix_per_step` pixels per step,
    timed by the slowest rank."""
    return world * pix_per_step / (ms_per_step * 1e-3) / 1e9


def _align(x: int, a: int = 256) -> int:
    return (x + a - 1) // a * a


class DeviceBatch:
    """A workload's images in two device arenas (markers, masks; each image at a 256-byte
    aligned offset) plus a copy of the initial markers, so that restoring every marker is
    one device copy and host <-> device transfers are one copy per arena."""

    def __init__(self, cases, dev):
        import torch
        self.cases = cases
        self.offs, total = [], 0
        for c in cases:
            self.offs.append(total)
            total += _align(c.mask.nbytes)
        self.nbytes = total
        host = np.zeros(total, np.uint8)
        hmask = np.zeros(total, np.uint8)
        for c, o in zip(cases, self.offs):
            host[o:o + c.mask.nbytes] = c.marker.reshape(-1).view(np.uint8)
            hmask[o:o + c.mask.nbytes] = c.mask.reshape(-1).view(np.uint8)
        self.host_marker, self.host_mask = host, hmask
        self.init = torch.from_numpy(host).to(dev)
        self.marker = self.init.clone()
        self.mask = torch.from_numpy(hmask).to(dev)
        self.items = [(self.view(self.marker, i), self.view(self.mask, i), c.conn, c.op)
                      for i, c in enumerate(cases)]
        self.pixels = sum(int(c.mask.size) for c in cases)
        self.alg_bytes = 3 * sum(int(c.mask.nbytes) for c in cases)   # read J, read I, write J

    def view(self, arena, i):
        import torch
        c, o = self.cases[i], self.offs[i]
        t = arena[o:o + c.mask.nbytes]
        return (t.view(torch.uint16) if c.mask.dtype == np.uint16 else t).view(c.mask.shape)

    def restore(self):
        self.marker.copy_(self.init)

    def outputs(self):
        """Host copies of every image's current marker (the results after a run)."""
        h = self.marker.cpu().numpy()
        return [h[o:o + c.mask.nbytes].view(c.mask.dtype).reshape(c.mask.shape)
                for c, o in zip(self.cases, self.offs)]


def _capture(fn):
    """A CUDA graph of fn(stream), captured on a side stream."""
    import torch
    cur = torch.cuda.current_stream()
    s = torch.cuda.Stream()
    s.wait_stream(cur)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            fn(s)
    cur.wait_stream(s)
    return g


class Forms:
    """The three forms of one workload on one DeviceBatch: plain per-image loop, batched
    static (the spread order of the initial frontier), batched + learned schedule. Each batched form is two graphs
    (prepare + scan, then the persistent drain) so that the drain can be timed alone."""

    def __init__(self, db, sch, plan, dev):
        from paper_1605_00930_gb300 import iwpp
        self.db, self.sch, self.plan, self.dev = db, sch, plan, dev
        self.Rs = [iwpp.Reconstructor(m.shape[0], m.shape[1], m.dtype, None, dev) for m, _, _, _ in db.items]
        self.Bs = iwpp.Batch(db.items, plan)
        self.Bl = iwpp.Batch(db.items, plan)
        import torch
        stream = torch.cuda.current_stream()
        # one uncaptured call of each form first (kernel attributes, schedule buffers)
        self.Bs(stream=stream)
        if sch is not None:
            if sch.reconstruct(self.Bl, stream) != 0:
                raise RuntimeError("learned batch call failed")
        else:
            self.Bl(stream=stream)
        torch.cuda.synchronize()
        db.restore()
        self.g = {
            "batched_static": (_capture(lambda s: self._scan(self.Bs, None, s)),
                               _capture(lambda s: self._drain(self.Bs, None, s))),
            "batched_learned": (_capture(lambda s: self._scan(self.Bl, sch, s)),
                                _capture(lambda s: self._drain(self.Bl, sch, s))),
        }

    def _scan(self, B, sch, s):
        # the learned form: schedule made inside the batch call (features from the scan kernel)
        rc = sch.reconstruct(B, s, phases=1) if sch is not None else B.phase("scan", stream=s)
        if rc != 0:
            raise RuntimeError(f"batch scan phase failed: {rc}")

    def _drain(self, B, sch, s):
        rc = sch.reconstruct(B, s, phases=2) if sch is not None else B.phase("drain", stream=s)
        if rc != 0:
            raise RuntimeError(f"batch drain phase failed: {rc}")

    def plain(self, stream):
        for R, (m, I, conn, op) in zip(self.Rs, self.db.items):
            if R(m, I, conn, op, stream) != 0:
                raise RuntimeError("plain call failed")

    def launches(self, form: str) -> int:
        """Kernel launches of the library in one step of `form`."""
        from paper_1605_00930_gb300 import iwpp
        n = len(self.db.items)
        if form == "plain":   # per image: scan, queue compaction, queue finalisation, drain
            return 4 * n
        if form == "batched_static":
            return iwpp.iwpp_batch_launch_count(n, 3)
        fused = (self.plan.local_solver == iwpp.IWPP_SOLVER_COOP and self.plan.tile_h == 64 and
                 self.plan.tile_w == 64 and len({c.conn for c in self.db.cases}) == 1)
        if fused:   # features in the scan
            return iwpp.iwpp_batch_launch_count(n, 7)
        return (n + 31) // 32 + 5 + iwpp.iwpp_batch_launch_count(n, 3)

    def run(self, form: str, flush, ev=None):
        """One step of `form` on the current stream (events: start, after scan, end)."""
        import torch
        stream = torch.cuda.current_stream()
        if ev is not None:
            ev[0].record(stream)
        if form == "plain":
            self.plain(stream)
            if ev is not None:
                ev[1].record(stream)
        else:
            gs, gd = self.g[form]
            gs.replay()
            if ev is not None:
                ev[1].record(stream)
            gd.replay()
        if ev is not None:
            ev[2].record(stream)

    def status(self, form: str) -> int:
        import torch
        stream = torch.cuda.current_stream()
        if form == "plain":
            return max(R.status(stream) for R in self.Rs)
        return (self.Bs if form == "batched_static" else self.Bl).status(stream)

    def timed(self, form: str, flush, reps: int):
        """Per-rep (total ms, drain ms), markers restored and L2 flushed before each rep."""
        import torch
        out = []
        for _ in range(reps):
            self.db.restore()
            flush.fill_(1)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            self.run(form, flush, ev)
            torch.cuda.synchronize()
            out.append((ev[0].elapsed_time(ev[2]), ev[1].elapsed_time(ev[2])))
        st = self.status(form)
        if st != 0:
            from paper_1605_00930_gb300 import iwpp
            raise RuntimeError(f"{form}: device status {iwpp.STATUS.get(st, st)}")
        return out


def _stats(ts):
    a = np.asarray(ts, dtype=np.float64)
    med = float(np.median(a))
    return med, (float(a.std() / a.mean()) if a.size > 1 and a.mean() > 0 else 0.0)


def drain_kernel_name(db, plan) -> str:
    """Name of the persistent kernel a batch call of this workload launches."""
    from paper_1605_00930_gb300 import iwpp
    kinds = {(c.mask.dtype.itemsize, c.conn) for c in db.cases}
    solver = {iwpp.IWPP_SOLVER_QUEUE: "drain_kernel", iwpp.IWPP_SOLVER_REGISTER: "drain_reg_kernel",
              iwpp.IWPP_SOLVER_COOP: "drain_coop_kernel"}[plan.local_solver]
    if len(kinds) == 1:
        (size, conn), = kinds
        return f"{solver}<{'u16' if size == 2 else 'u8'}, {conn}>"
    conns = {k[1] for k in kinds}
    if plan.local_solver == iwpp.IWPP_SOLVER_COOP and len(conns) == 1:
        return f"{solver}<u8|u16, {conns.pop()}>"
    return f"{solver}<mixed>"


def measure_forms(name, db, sch, plan, dev, flush, reps, peak):
    """Plain, batched static and batched + learned on one workload: median time and CV over
    `reps`, Gpx/s, the drain kernel's HBM fraction of the compulsory 3 s bytes per pixel,
    and every form's output compared with the plain form's."""
    import torch
    F = Forms(db, sch, plan, dev)
    res = {"workload": WORKLOADS[name], "images": len(db.items), "pixels": db.pixels,
           "plan": plan.as_dict(), "drain_kernel": drain_kernel_name(db, plan)}
    ref = None
    for form in ("plain", "batched_static", "batched_learned"):
        ts = F.timed(form, flush, reps)
        med, cv = _stats([t[0] for t in ts])
        dmed, _ = _stats([t[1] for t in ts])
        out = db.marker.clone()
        if ref is None:
            ref = out
            same = True
        else:
            same = bool(torch.equal(out, ref))
        r = {"ms": round(med, 4), "cv": round(cv, 4), "gpx_s": round(db.pixels / med / 1e6, 3),
             "same_output_as_plain": same, "launches_per_step": F.launches(form)}
        if form != "plain":
            ach = db.alg_bytes / (dmed * 1e-3) / 1e9
            r.update({"drain_ms": round(dmed, 4), "drain_hbm_gbs": round(ach, 1),
                      "drain_frac": round(ach / peak, 5)})
        res[form] = r
    for form in ("batched_static", "batched_learned"):
        res[form]["speedup_vs_plain"] = round(res["plain"]["ms"] / res[form]["ms"], 3)
    return res, F


def oracle_check(cases, gpu_outputs, threads):
    """Every image reconstructed by the CPU oracle on `threads` host threads and compared
    pixel for pixel with the GPU's result. Returns (all equal, seconds)."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    outs = oracle.reconstruct_many([(c.marker, c.mask, c.conn, c.op) for c in cases], threads=threads)
    dt = time.perf_counter() - t0
    return all(np.array_equal(o, g) for o, g in zip(outs, gpu_outputs)), dt


def cpu_baseline(cases, gpu_outputs, threads):
    """The oracle on the host's cores: the whole workload on `threads` threads (one image per
    thread at a time; its outputs are also compared with the GPU's), and a one-core figure
    on a strided sample of the images (about 5 s of work)."""
    import oracle
    oracle.build()
    exact, dt = oracle_check(cases, gpu_outputs, threads)
    px = sum(int(c.mask.size) for c in cases)
    # one core: every k-th image, about 5 s at the N-core rate divided by N
    budget_px = px / dt / threads * 5.0
    k = max(1, int(round(px / max(budget_px, 1.0))))
    sample = cases[::k]
    t0 = time.perf_counter()
    for c in sample:
        oracle.reconstruct(c.marker, c.mask, c.conn, c.op)
    dt1 = time.perf_counter() - t0
    spx = sum(int(c.mask.size) for c in sample)
    return {"value": round(px / dt / 1e9, 5), "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": (f"the whole workload ({len(cases)} images, {px} px) on {threads} host threads, one "
                       f"image per thread at a time, single-threaded C oracle per image"),
            "seconds": round(dt, 2),
            "one_core": {"value": round(spx / dt1 / 1e9, 5), "unit": UNIT, "cores": 1,
                         "sample": f"every {k}-th image ({len(sample)} images, {spx} px) on one thread",
                         "seconds": round(dt1, 2)},
            "gpu_output_bit_exact": bool(exact)}


def train_estimator(sets_cases, dev):
    """The learned work estimator, trained on labels from runs of the given workloads."""
    from paper_1605_00930_gb300 import learned
    import torch
    sets = []
    for cases in sets_cases:
        items = []
        for c in cases:
            items.append((torch.from_numpy(c.marker).to(dev), torch.from_numpy(c.mask).to(dev), c.conn, c.op))
        sets.append(items)
    t0 = time.time()
    sch, report = learned.train_from_workloads(sets, n_samples=50000, epochs=60)
    report["seconds"] = round(time.time() - t0, 2)
    del sets
    torch.cuda.empty_cache()
    return sch, report


def choose_plan(db, dev):
    """The batch plan the library's autotuner picks on this workload (markers restored)."""
    from paper_1605_00930_gb300 import iwpp
    B = iwpp.Batch(db.items, iwpp.iwpp_default_batch_plan())
    plan, _ = B.autotune(reps=2)
    db.restore()
    del B
    return plan


def run_profile(args):
    """A lean run for profilers: one form of the workload only (default plan, no autotuning,
    no training, no other forms), W warm-up steps then K timed steps. A batched form's
    persistent drain of timed step k is the library's drain launch number 2 + W + k of the
    process (0-based: two uncaptured batch set-up calls come first); the plain form launches
    one drain per image and step after those two. That is what an ncu -k / -s / -c selection
    needs. The learned form uses an untrained estimator whose sweep output is fixed at 0 (as
    the trained one predicts on these workloads): the kernels it launches and their cost do
    not depend on the weights otherwise."""
    import torch
    from paper_1605_00930_gb300 import build as B
    B.build()
    from paper_1605_00930_gb300 import iwpp, learned
    cases = load_workload(args.workload)
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    db = DeviceBatch(cases, dev)
    sch = None
    if args.profile_form == "batched_learned":
        p = learned.init_params(11)
        n1 = 16 * 64 + 64 + 64 * 64 + 64          # the last layer's weights [64][2], then 2 biases
        p[n1 + 1:n1 + 128:2] = 0.0
        p[-1] = 0.0
        sch = learned.LearnedScheduler(p, dev)
    F = Forms(db, sch, iwpp.iwpp_default_batch_plan(), dev)
    form = args.profile_form
    for _ in range(args.warmup):
        db.restore()
        flush.fill_(1)
        F.run(form, flush)
    ts = F.timed(form, flush, args.steps)
    return {"profile_run": args.workload, "form": form, "steps": args.steps, "warmup": args.warmup,
            "ms": [round(t[0], 4) for t in ts], "drain_ms": [round(t[1], 4) for t in ts],
            "drain_kernel": drain_kernel_name(db, F.plan), "launches_per_step": F.launches(form)}


def run_profile_ops():
    """A lean run for profilers: one call each of the distance transform, the watershed and
    SKIZ, in that order, on the 4096^2 inputs the full run times (run_edt's tissue mask above
    60, run_watershed's inverted blob field with 2000 labelled markers, run_skiz's porous
    domain with 2000 markers), so that an ncu selection of the three drains
    (-k regex:"edt_drain|ws_drain|sk_drain" -c 3) takes one launch of each."""
    import torch
    from paper_1605_00930_gb300 import iwpp, synth
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    f = synth.tissue_case().mask
    H, W = f.shape
    fg = torch.from_numpy((f > 60).astype(np.uint8)).to(dev)
    site = torch.empty((H, W), dtype=torch.int32, device=dev)
    T = iwpp.DistanceTransform(H, W, dev)
    if T(fg, site, None, 8) != 0 or T.status() != 0:
        raise RuntimeError("edt call failed")
    rng = synth.rng_for(9)
    markers = np.zeros((H, W), np.int32)
    markers[rng.integers(0, H, 2000), rng.integers(0, W, 2000)] = np.arange(1, 2001)
    iwpp.watershed(torch.from_numpy(markers).to(dev), torch.from_numpy((255 - f).astype(np.uint8)).to(dev), 8)
    sk_markers, sk_mask = synth.porous_skiz_case()
    iwpp.skiz(torch.from_numpy(sk_markers.astype(np.int32)).to(dev), torch.from_numpy(sk_mask).to(dev), 8)
    torch.cuda.synchronize()
    return {"profile_run": "operators", "calls": ["iwpp_edt", "iwpp_watershed", "iwpp_skiz"], "H": H, "W": W}


def run_ours(args, rank: int, world: int):
    import torch
    from paper_1605_00930_gb300 import build as B
    B.build()
    from paper_1605_00930_gb300 import iwpp
    if args.profile_ops:
        return run_profile_ops()
    if args.profile:
        return run_profile(args)

    full = rank == 0 and world == 1 and not args.quick
    head_cases = load_workload(args.workload)   # generator processes start before any CUDA work
    other = {}
    if full:
        for name in WORKLOADS:
            if name != args.workload:
                other[name] = load_workload(name)
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    peak, peak_kind = _peaks()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    # the learned estimator: labels from runs of the 512^2, 4096^2 (conn 8, 4) and 16384^2 workloads
    def train_cases():
        got = {n: (other.get(n) or (head_cases if n == args.workload else None))
               for n in ("noiseblur512", "tissue4096", "seeds16384")}
        return [got[n] if got[n] is not None else load_workload(n) for n in ("noiseblur512", "tissue4096", "seeds16384")]
    sch, estimator = (None, None) if args.static else train_estimator(
        [[c] for cs in train_cases() for c in cs], dev)

    db = DeviceBatch(head_cases, dev)
    plan = choose_plan(db, dev)
    forms, F = measure_forms(args.workload, db, sch, plan, dev, flush, max(3, args.form_reps), peak)
    form = "batched_static" if sch is None else "batched_learned"
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        db.restore()
        flush.fill_(1)
        F.run(form, flush)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    gpu_index = dev.index
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0]
    with ClockSampler(int(vis) if vis.isdigit() else gpu_index) as cs:
        time.sleep(0.25)
        t0 = time.time()
        for i in range(args.steps):
            db.restore()
            flush.fill_(1)
            F.run(form, flush, evs[i])
        torch.cuda.synchronize()
        t1 = time.time()
        if t1 - t0 < 0.3:
            time.sleep(0.3 - (t1 - t0))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    st = F.status(form)
    if st != 0:
        raise RuntimeError(f"device status {iwpp.STATUS.get(st, st)}")
    step_ms = [e[0].elapsed_time(e[2]) for e in evs]
    drain_ms = [e[1].elapsed_time(e[2]) for e in evs]
    ms_per_step = max_over_ranks(sum(step_ms) / args.steps, world, dev)
    value = job_gpx_s(world, db.pixels, ms_per_step)
    gpu_out = db.outputs()
    head_arena = db.marker.cpu().numpy()

    # end to end through the C ABI from pinned host buffers, as a user streaming batches runs
    # it: per step the H2D copy of every marker and mask (the two arenas), the learned batch
    # call and the D2H copy of every result. Three device buffer sets and three streams: input
    # copies on one, the batch calls on another (consecutive steps' kernels run in order), the
    # result copies on a third; a step's input copy waits only for the result copy out of the
    # same buffer set three steps earlier, so the two copy directions and the kernels overlap.
    hm = torch.from_numpy(db.host_marker).pin_memory()
    hI = torch.from_numpy(db.host_mask).pin_memory()
    dbs = [db] + [DeviceBatch(head_cases, dev) for _ in range(2)]
    Bks = [F.Bl if sch is not None else F.Bs] + [iwpp.Batch(d.items, plan) for d in dbs[1:]]
    K = len(dbs)
    s_in, s_run, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    hos = [torch.empty_like(hm).pin_memory() for _ in range(K)]

    def e2e_run(nsteps):
        freed = [None] * K   # per buffer set: its last result copy has been read out
        for i in range(nsteps):
            k = i % K
            d, Bk = dbs[k], Bks[k]
            with torch.cuda.stream(s_in):
                if freed[k] is not None:
                    s_in.wait_event(freed[k])
                d.marker.copy_(hm, non_blocking=True)
                d.mask.copy_(hI, non_blocking=True)
                loaded = torch.cuda.Event()
                loaded.record(s_in)
            s_run.wait_event(loaded)
            rc = sch.reconstruct(Bk, s_run) if sch is not None else Bk(stream=s_run)
            if rc != 0:
                raise RuntimeError(f"batch call failed: {rc}")
            done = torch.cuda.Event()
            done.record(s_run)
            with torch.cuda.stream(s_out):
                s_out.wait_event(done)
                hos[k].copy_(d.marker, non_blocking=True)
                freed[k] = torch.cuda.Event()
                freed[k].record(s_out)

    e2e_run(K)
    torch.cuda.synchronize()
    n_e2e = max(4, args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s_in)
    s_run.wait_event(e0)
    s_out.wait_event(e0)
    e2e_run(n_e2e)
    s_in.wait_stream(s_run)
    s_in.wait_stream(s_out)
    e1.record(s_in)
    torch.cuda.synchronize()
    e2e_ts = [e0.elapsed_time(e1) / n_e2e]
    ok = all(Bks[k].status(s_run) == 0 for k in range(K))
    if not ok or not all(np.array_equal(h.numpy(), head_arena) for h in hos):
        raise RuntimeError("end-to-end run failed or differs from the device-resident run")
    del dbs, Bks
    e2e_ms = max_over_ranks(float(np.mean(e2e_ts)), world, dev)
    if rank != 0:
        return None

    kname = drain_kernel_name(db, plan)
    dmean = float(np.mean(drain_ms))
    achieved = db.alg_bytes / (dmean * 1e-3) / 1e9
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8/u16 (16-bit integer lanes)", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "name": args.workload, "images": len(head_cases),
                   "pixels_per_step": db.pixels,
                   "form": ("batched + learned schedule: one iwpp_reconstruct_batch_learned call (features "
                            "out of the scan kernel, MLP, tile order, one persistent launch over every image), "
                            "replayed from CUDA graphs" if sch is not None else
                            "batched, static tile order, CUDA graphs"),
                   "plan": plan.as_dict(),
                   "l2": "flushed before every timed step (256 MiB write); the inputs also exceed L2",
                   "timing": "CUDA events on the launching stream around each step (schedule + batch call)",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "plain": forms["plain"], "batched_static": forms["batched_static"],
        "batched_learned": forms["batched_learned"],
        "speedup_vs_plain": round(forms["plain"]["ms"] / ms_per_step, 3),
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1), "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 5),
                     "traffic": _traffic_from_profiles(kname, args.workload),
                     "alg_bytes_per_launch": db.alg_bytes,
                     "drain_ms_per_launch": round(dmean, 4),
                     "path_frac": round(db.alg_bytes / (ms_per_step * 1e-3) / 1e9 / peak, 5)},
        "e2e": {"value": round(world * db.pixels / e2e_ms / 1e6, 3), "unit": UNIT,
                "h2d_bytes_per_step": 2 * db.nbytes, "d2h_bytes_per_step": db.nbytes,
                "ms_per_step": round(e2e_ms, 3),
                "steps": n_e2e,
                "form": ("per step: pinned H2D of every marker and mask (two arena copies), the learned "
                         "batch call through the C ABI (iwpp_reconstruct_batch_learned), D2H of every result; "
                         "three device buffer sets, input copies, batch calls and result copies on three "
                         "streams: a step's input copy overlaps the previous step's kernels and the result "
                         "copy before it, the kernels of consecutive steps run in order; CUDA events around "
                         "all steps (pipeline fill and drain included), mean per step; inputs exceed L2 (no "
                         "flush between steps)")},
        "gpu_launches": F.launches(form) * args.steps,
        "clocks": cs.summary(t0, t1),
        "estimator": estimator,
    }
    if full:
        other_out = {}
        res_forms = {}
        for name, cases in other.items():
            d2 = DeviceBatch(cases, dev)
            p2 = choose_plan(d2, dev)
            r, F2 = measure_forms(name, d2, sch, p2, dev, flush, max(3, args.form_reps), peak)
            other_out[name] = (cases, d2.outputs())
            res_forms[name] = r
            del F2, d2
            torch.cuda.empty_cache()
        out["forms"] = res_forms
        out["edt"] = run_edt(args, dev, peak)
        out["watershed"] = run_watershed(args, dev)
        out["skiz"] = run_skiz(args, dev)
        out["host_bands"] = run_host_bands(args, dev)
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(head_cases, gpu_out, host_cores())
        if full:
            for name, (cases, outs) in other_out.items():
                ok, dt = oracle_check(cases, outs, host_cores())
                out["forms"][name]["oracle_bit_exact"] = ok
                out["forms"][name]["oracle_seconds"] = round(dt, 2)
    return out


def run_edt(args, dev, peak):
    """The distance transform (Algorithm 8 on the tile engine) on tissue-like masks: the
    blob fields of the 4096^2 and 16384^2 workloads thresholded above 60 (objects = blobs).
    Reports time, Gpixels/s, the HBM fraction of the compulsory 5 bytes per pixel (read the
    mask, write the site map) and, against scipy's exact transform, the share of pixels
    whose distance is exact and the largest error in pixels."""
    import torch
    from paper_1605_00930_gb300 import iwpp, synth
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    out = {}
    for name, c in (("tissue4096", synth.tissue_case()), ("seeds16384_mask", None)):
        mask = synth.sparse_seed_case().mask if c is None else c.mask
        fg = (mask > 60).astype(np.uint8)
        H, W = fg.shape
        if H > 32767 or W > 32767:
            continue
        m = torch.from_numpy(fg).to(dev)
        site = torch.empty((H, W), dtype=torch.int32, device=dev)
        T = iwpp.DistanceTransform(H, W, dev)
        ts = []
        for r in range(max(3, args.form_reps) + 1):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if T(m, site, None, 8, stream) != 0:
                raise RuntimeError("edt call failed")
            e1.record(stream)
            torch.cuda.synchronize()
            if r > 0:
                ts.append(e0.elapsed_time(e1))
        if T.status(stream) != 0:
            raise RuntimeError("edt device error")
        ms = float(np.median(ts))
        res = {"pixels": H * W, "foreground": round(float(fg.mean()), 4), "conn": 8, "ms": round(ms, 3),
               "gpx_s": round(H * W / ms / 1e6, 3),
               "hbm_frac": round(5 * H * W / (ms * 1e-3) / 1e9 / peak, 5)}
        cnt = T.counters(stream)
        res["visits"] = int(cnt["visits"])
        if H * W <= 4096 * 4096:
            try:
                from scipy import ndimage
                s = site.cpu().numpy().view(np.uint32).astype(np.int64)
                yy, xx = np.mgrid[0:H, 0:W]
                d2 = (yy - (s >> 16)) ** 2 + (xx - (s & 0xFFFF)) ** 2
                ex = ndimage.distance_transform_edt(fg)
                res["exact_fraction"] = round(float(np.mean(d2 == np.rint(ex ** 2))), 5)
                res["max_error_px"] = round(float(np.max(np.sqrt(d2) - ex)), 4)
            except ImportError:
                pass
        out[name] = res
        del m, site, T
    return out


def run_watershed(args, dev):
    """Marker-controlled watershed by flooding on the 4096^2 tissue image: the gradient is
    the inverted blob field (blobs become basins), 2000 seeded markers with distinct labels.
    Reports time and Gpixels/s of the whole call (initialisation, flooding, labels)."""
    import torch
    from paper_1605_00930_gb300 import iwpp, synth
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    f = synth.tissue_case().mask
    grad = torch.from_numpy((255 - f).astype(np.uint8)).to(dev)
    H, W = f.shape
    rng = synth.rng_for(9)
    markers = np.zeros((H, W), np.int32)
    markers[rng.integers(0, H, 2000), rng.integers(0, W, 2000)] = np.arange(1, 2001)
    mk = torch.from_numpy(markers).to(dev)
    labels = torch.empty((H, W), dtype=torch.int32, device=dev)
    ws = iwpp.alloc_workspace(iwpp.iwpp_watershed_workspace_bytes(H, W), dev)
    ts = []
    for r in range(max(3, args.form_reps) + 1):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = iwpp.iwpp_watershed(ctypes_ptr(mk), ctypes_ptr(grad), iwpp.IWPP_U8, ctypes_ptr(labels), None, H, W, 8,
                                 ctypes_ptr(ws), ws.numel(), stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if rc != 0:
            raise RuntimeError("watershed call failed")
        if r > 0:
            ts.append(e0.elapsed_time(e1))
    if iwpp.iwpp_sync_status(ctypes_ptr(ws), stream.cuda_stream) != 0:
        raise RuntimeError("watershed device error")
    ms = float(np.median(ts))
    cnt = iwpp.iwpp_work_counters(ctypes_ptr(ws), stream.cuda_stream)
    return {"tissue4096": {"pixels": H * W, "markers": 2000, "conn": 8, "ms": round(ms, 3),
                           "gpx_s": round(H * W / ms / 1e6, 3), "visits": int(cnt["visits"])}}


def run_skiz(args, dev):
    """Geodesic influence zones on the 4096^2 porous domain (blob field above 8: blobs plus
    ~70 % of the noisy background), 2000 markers with distinct labels, 8-connectivity.
    Reports time and Gpixels/s of the whole call (initialisation, propagation, zones)."""
    import torch
    from paper_1605_00930_gb300 import iwpp, synth
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    markers, mask = synth.porous_skiz_case()
    H, W = mask.shape
    mk = torch.from_numpy(markers.astype(np.int32)).to(dev)
    m = torch.from_numpy(mask).to(dev)
    zone = torch.empty((H, W), dtype=torch.int32, device=dev)
    ws = iwpp.alloc_workspace(iwpp.iwpp_skiz_workspace_bytes(H, W), dev)
    ts = []
    for r in range(max(3, args.form_reps) + 1):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = iwpp.iwpp_skiz(ctypes_ptr(mk), ctypes_ptr(m), ctypes_ptr(zone), None, None, H, W, 8,
                            ctypes_ptr(ws), ws.numel(), stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if rc != 0:
            raise RuntimeError("skiz call failed")
        if r > 0:
            ts.append(e0.elapsed_time(e1))
    if iwpp.iwpp_sync_status(ctypes_ptr(ws), stream.cuda_stream) != 0:
        raise RuntimeError("skiz device error")
    ms = float(np.median(ts))
    cnt = iwpp.iwpp_work_counters(ctypes_ptr(ws), stream.cuda_stream)
    return {"porous4096": {"pixels": H * W, "markers": 2000, "conn": 8, "ms": round(ms, 3),
                           "gpx_s": round(H * W / ms / 1e6, 3), "visits": int(cnt["visits"])}}


def run_host_bands(args, dev):
    """Out-of-core form: a 32768^2 sparse-seed image (1 GiB per plane, 8000 blobs, 4000
    seeds; the 16384^2 workload's density) in pinned host memory, reconstructed in bands of
    4096 rows (iwpp_reconstruct_host; the whole blocking call is timed, copies included),
    against the same image reconstructed in HBM (CUDA events, inputs resident). The two
    results are compared pixel for pixel."""
    import time
    import torch
    from paper_1605_00930_gb300 import iwpp, synth
    c = synth.sparse_seed_case(32768, 32768, nblobs=8000, nseeds=4000)
    H, W = c.mask.shape
    band = 4096
    m0 = torch.from_numpy(c.marker)
    m = m0.clone().pin_memory()
    I = torch.from_numpy(c.mask).pin_memory()
    R = iwpp.HostReconstructor(H, W, torch.uint8, band, dev)
    ts = []
    for r in range(3):
        m.copy_(m0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc = R(m, I, 8, "dilate")
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        if rc != 0:
            raise RuntimeError(f"host-band reconstruction failed with status {rc}")
        if r > 0:
            ts.append((t1 - t0) * 1e3)
    ms = float(np.median(ts))
    host_ws = R.ws.numel()
    visits = R.band_visits
    del R
    md = m0.to(dev)
    Id = I.to(dev)
    md0 = md.clone()
    Rd = iwpp.Reconstructor(H, W, torch.uint8, None, dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    dts = []
    for r in range(3):
        md.copy_(md0)
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Rd(md, Id, 8, "dilate")
        e1.record(stream)
        torch.cuda.synchronize()
        if r > 0:
            dts.append(e0.elapsed_time(e1))
    if Rd.status() != 0:
        raise RuntimeError("in-HBM reconstruction failed")
    same = bool(torch.equal(md.cpu(), m))
    dms = float(np.median(dts))
    in_hbm_bytes = Rd.ws.numel() + 2 * H * W
    del md, Id, md0, Rd, flush
    return {"seeds32768": {"pixels": H * W, "band_rows": band, "bands": (H + band - 1) // band,
                           "band_visits": int(visits), "ms": round(ms, 2),
                           "gpx_s": round(H * W / ms / 1e6, 3), "device_bytes": host_ws,
                           "in_hbm_ms": round(dms, 2), "in_hbm_gpx_s": round(H * W / dms / 1e6, 3),
                           "in_hbm_device_bytes": in_hbm_bytes, "same_as_in_hbm": same}}


def ctypes_ptr(t):
    import ctypes
    return ctypes.c_void_p(t.data_ptr())


REFERENCE_BUDGET_S = 120.0   # wall-clock target of the whole --impl reference run


def run_reference(args, rank: int, world: int):
    """The oracle arm: the C oracle (one image per host thread, on every core of the host)
    timed on the same workload, metric and unit. When the requested steps of the whole
    workload would not fit the time budget, every step is a bounded sample of it, sized from
    a timed pass of the whole workload: every k-th image of a batch (the same mix of sizes,
    pixel types, dilations and fill-holes), or the first rows of each image of a
    single-image workload."""
    if rank != 0:
        return None
    import oracle
    oracle.build()
    cases = load_workload(args.workload)
    threads = host_cores()
    items = [(c.marker, c.mask, c.conn, c.op) for c in cases]
    full_px = sum(int(c.mask.size) for c in cases)
    t0 = time.perf_counter()
    oracle.reconstruct_many(items, threads=threads)
    full_s = time.perf_counter() - t0
    nsteps = args.steps + max(0, args.warmup - 1)
    sample_desc = f"every step is the whole workload ({len(items)} images, {full_px} px)"
    if nsteps * full_s > REFERENCE_BUDGET_S:
        frac = REFERENCE_BUDGET_S / (nsteps * full_s)
        if len(items) >= 8:
            k = int(np.ceil(1.0 / frac))
            items = items[::k]
            sample_desc = f"every step: every {k}-th image"
        else:
            rows = max(16, int(cases[0].mask.shape[0] * frac))
            items = [(np.ascontiguousarray(m[:rows]), np.ascontiguousarray(i[:rows]), conn, op)
                     for (m, i, conn, op) in items]
            sample_desc = f"every step: the first {rows} rows of each image"
        spx = sum(int(it[1].size) for it in items)
        sample_desc += (f" ({len(items)} images, {spx} of {full_px} px; the whole workload takes the oracle "
                        f"{full_s:.2f} s on {threads} threads)")
    pix = sum(int(it[1].size) for it in items)
    for _ in range(max(0, args.warmup - 1)):
        oracle.reconstruct_many(items, threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.reconstruct_many(items, threads=threads)
    dt = (time.perf_counter() - t0) / args.steps
    value = pix / dt / 1e9
    return {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8/u16",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "name": args.workload, "pixels_per_step": pix},
            "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample_desc + "; single-threaded C oracle per image, one image per "
                                                     "thread at a time"},
            "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch512", choices=list(WORKLOADS))
    ap.add_argument("--static", action="store_true", help="time the static schedule instead of the learned one")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--quick", action="store_true", help="headline workload only (no other forms or operators)")
    ap.add_argument("--form-reps", type=int, default=10)
    ap.add_argument("--profile", action="store_true",
                    help="profiler run: one batched form of the workload only (see run_profile)")
    ap.add_argument("--profile-form", default="batched_static", choices=["batched_static", "batched_learned", "plain"])
    ap.add_argument("--profile-ops", action="store_true",
                    help="profiler run: one call each of the distance transform, watershed and SKIZ (see run_profile_ops)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    out = run_reference(args, rank, world) if args.impl == "reference" else run_ours(args, rank, world)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if world > 1 and args.impl == "ours":
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
