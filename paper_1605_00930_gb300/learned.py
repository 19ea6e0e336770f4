"""Learned work estimator for batch schedules: training-data generation and training.

The estimator itself (features, MLP inference, the counting sort that turns
predictions into a tile order and per-tile sweep counts) runs in the CUDA library;
this module only drives it through the C ABI:

  * labels come from runs of the reconstruction itself: for every sweep count s of
    SWEEP_OPTIONS the batch is reconstructed with every tile forced to s sweeps and
    per-tile work counters on; per 64 x 64 block the work label is log(1 + SM cycles spent
    on the block's tiles) in the run with the plan's own sweep count, and the sweep label
    is the smallest s that no larger option beats by more than SWEEP_MARGIN (cycle counts
    of single runs are noisy; extra sweeps must pay for themselves clearly); the estimator's
    sweep output learns whether that label is above 0;
  * training runs the library's hand-written FP32 backpropagation and Adam kernels;
  * weights are saved as raw float32 plus a JSON header; a missing or corrupt file
    means the static schedule is used.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from . import iwpp

SWEEP_OPTIONS = (0, 1, 2, 4, 8)
SWEEP_MARGIN = 0.25
WEIGHTS_VERSION = 2


def init_params(seed: int = 0) -> np.ndarray:
    """He-uniform weights, zero biases (seeded), in the library's flat layout."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, shape in [(16, (16, 64)), (0, (64,)), (64, (64, 64)), (0, (64,)), (64, (64, 2)), (0, (2,))]:
        if fan_in:
            lim = math.sqrt(6.0 / fan_in)
            parts.append(rng.uniform(-lim, lim, size=shape).ravel())
        else:
            parts.append(np.zeros(shape).ravel())
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == iwpp.MLP_PARAMS
    return p


def _descs(items):
    descs = (iwpp.Image * len(items))()
    for i, (m, I, conn, op) in enumerate(items):
        descs[i] = iwpp.Image(m.data_ptr(), I.data_ptr(), m.shape[0], m.shape[1], int(conn), iwpp.OPS[op],
                              iwpp._dtype_code(m), 0)
    return descs


def features(items, device="cuda"):
    """Per-block features of a batch (torch float32 [nblocks, 16] on the device)."""
    import torch
    descs = _descs(items)
    nb = iwpp.iwpp_batch_block_count(descs)
    sws = iwpp.alloc_workspace(iwpp.iwpp_sched_workspace_bytes(descs), device)
    feats = torch.empty((nb, iwpp.NFEAT), dtype=torch.float32, device=device)
    iwpp.iwpp_batch_features(descs, feats, sws)
    return feats


def sweep_label(cycles, options=SWEEP_OPTIONS, margin: float = SWEEP_MARGIN):
    """Per block (columns of `cycles`, one row per option in increasing order): the smallest
    option that no larger option beats by more than `margin` of its cycles."""
    best = np.full(cycles.shape[1], float(options[0]))
    cur = cycles[0].copy()
    for oi in range(1, len(options)):
        better = cycles[oi] < (1.0 - margin) * cur
        best = np.where(better, float(options[oi]), best)
        cur = np.where(better, cycles[oi], cur)
    return best


def block_labels(items, plan=None, options=SWEEP_OPTIONS, reps: int = 1):
    """Run the batch once per sweep option with work counters; returns (log-work label:
    log(1 + cycles) of the run with the plan's sweep count, sweep label per block, cycles
    per option) as numpy arrays. The markers are restored after every run."""
    import torch
    init = [m.clone() for m, _, _, _ in items]
    B = iwpp.Batch(items, plan)
    nt = B.ntiles
    nb = iwpp.iwpp_batch_block_count(B.descs)
    sws = iwpp.alloc_workspace(iwpp.iwpp_sched_workspace_bytes(B.descs, plan), init[0].device)
    cycles = np.zeros((len(options), nb))
    own = (plan if plan is not None else iwpp.iwpp_default_batch_plan()).sweeps
    for oi, s in enumerate(options):
        for _ in range(reps):
            for (m, _, _, _), m0 in zip(items, init):
                m.copy_(m0)
            work = torch.zeros(2 * nt, dtype=torch.int32, device=init[0].device)
            sweeps = torch.full((nt,), s, dtype=torch.uint8, device=init[0].device)
            rc = B(sweeps=sweeps, work=work)
            if rc != 0 or B.status() != 0:
                raise iwpp.IwppError(rc or B.status(), "label run")
            bw = torch.zeros(2 * nb, dtype=torch.int64, device=init[0].device)
            iwpp.iwpp_tile_work_to_blocks(B.descs, plan, work, bw, sws)
            bw = bw.cpu().numpy().astype(np.float64)
            cycles[oi] += bw[nb:] / reps
    for (m, _, _, _), m0 in zip(items, init):
        m.copy_(m0)
    oi = options.index(own) if own in options else 0
    return np.log1p(cycles[oi]), sweep_label(cycles, options), cycles


class LearnedScheduler:
    """MLP weights on the device plus the calls that turn a batch into a schedule."""

    def __init__(self, params=None, device="cuda", meta=None):
        import torch
        p = init_params(0) if params is None else np.asarray(params, dtype=np.float32)
        self.params = torch.from_numpy(p.copy()).to(device)
        self.meta = dict(meta or {})
        self.device = device

    # -- training -------------------------------------------------------------------------
    def train(self, X, T, epochs: int = 60, batch: int = 512, lr: float = 1e-3, w=(1.0, 1.0), seed: int = 1):
        import torch
        X = torch.as_tensor(X, dtype=torch.float32, device=self.device).contiguous()
        T = torch.as_tensor(T, dtype=torch.float32, device=self.device).contiguous()
        m = torch.zeros(iwpp.MLP_PARAMS, dtype=torch.float32, device=self.device)
        v = torch.zeros_like(m)
        g = torch.zeros_like(m)
        iwpp.iwpp_mlp_train(self.params, m, v, g, X, T, epochs, batch, lr, w[0], w[1], seed, 0)
        torch.cuda.synchronize()
        return self

    def predict(self, X):
        import torch
        X = torch.as_tensor(X, dtype=torch.float32, device=self.device).contiguous()
        Y = torch.empty((X.shape[0], 2), dtype=torch.float32, device=self.device)
        iwpp.iwpp_mlp_forward(self.params, X, Y)
        return Y

    # -- scheduling -----------------------------------------------------------------------
    def _buffers(self, batch):
        import torch
        dev = batch.ws.device
        if not hasattr(batch, "_sched_ws"):
            batch._sched_ws = iwpp.alloc_workspace(iwpp.iwpp_sched_workspace_bytes(batch.descs, batch.plan), dev)
            batch._order = torch.empty(batch.ntiles, dtype=torch.int32, device=dev)
            batch._sweeps = torch.empty(batch.ntiles, dtype=torch.uint8, device=dev)

    def schedule(self, batch: "iwpp.Batch", stream=None):
        """Device tile order and sweep counts for `batch` (no host synchronisation)."""
        self._buffers(batch)
        iwpp.iwpp_schedule_learned(batch.descs, batch.plan, self.params, batch._order, batch._sweeps,
                                   batch._sched_ws, stream)
        return batch._order, batch._sweeps

    def reconstruct(self, batch: "iwpp.Batch", stream=None, phases: int = 3) -> int:
        """Reconstruct `batch` with the schedule made inside the call (iwpp_reconstruct_batch_learned:
        features from the scan kernel under the default plan). Returns the host status; the
        schedule lands in batch._order / batch._sweeps."""
        import ctypes
        self._buffers(batch)
        P = ctypes.c_void_p
        return iwpp.iwpp_reconstruct_batch_learned(
            batch.descs, batch.plan, P(self.params.data_ptr()), P(batch._order.data_ptr()),
            P(batch._sweeps.data_ptr()), P(batch._sched_ws.data_ptr()), batch._sched_ws.numel(), phases,
            P(batch.ws.data_ptr()), batch.ws.numel(), iwpp._stream_handle(stream))

    def features_of(self, batch: "iwpp.Batch"):
        """The features the last reconstruct() call wrote (float32 [nblocks, 16], a view)."""
        import torch
        off = iwpp.iwpp_sched_features_offset(batch.descs, batch.plan)
        nb = iwpp.iwpp_batch_block_count(batch.descs)
        return batch._sched_ws[off:off + nb * iwpp.NFEAT * 4].view(torch.float32).view(nb, iwpp.NFEAT)

    # -- persistence ----------------------------------------------------------------------
    def save(self, path: str):
        hdr = {"version": WEIGHTS_VERSION, "nparams": iwpp.MLP_PARAMS, **self.meta}
        with open(path + ".json", "w") as f:
            json.dump(hdr, f)
        self.params.cpu().numpy().astype("<f4").tofile(path)

    @classmethod
    def load(cls, path: str, device="cuda"):
        """Returns None when the file is missing or does not match (static fallback)."""
        try:
            with open(path + ".json") as f:
                hdr = json.load(f)
            if hdr.get("version") != WEIGHTS_VERSION or hdr.get("nparams") != iwpp.MLP_PARAMS:
                return None
            p = np.fromfile(path, dtype="<f4")
            if p.size != iwpp.MLP_PARAMS or not np.all(np.isfinite(p)):
                return None
            return cls(p, device, hdr)
        except (OSError, ValueError):
            return None


def train_from_workloads(item_sets, n_samples: int = 50000, epochs: int = 60, seed: int = 7, plan=None,
                         device="cuda", reps: int = 2):
    """Generate labels from runs of each batch in `item_sets` (cycles averaged over `reps`
    runs per sweep option), sample n_samples blocks and train a scheduler. The sweep output is
    trained on "do sweeps pay here" (1 if the block's sweep label is > 0, else 0), so that the
    schedule runs one sweep pair where the estimator expects it to pay and none elsewhere.
    Returns (scheduler, report)."""
    Xs, T0s, T1s, Ls = [], [], [], []
    for items in item_sets:
        Xs.append(features(items, device).cpu().numpy())
        lw, best, _ = block_labels(items, plan, reps=reps)
        T0s.append(lw)
        T1s.append((best > 0).astype(np.float64))
        Ls.append(best)
    X = np.concatenate(Xs)
    T = np.stack([np.concatenate(T0s), np.concatenate(T1s)], axis=1)
    labels = np.concatenate(Ls)
    rng = np.random.default_rng(seed)
    idx = rng.permutation(X.shape[0])[:min(n_samples, X.shape[0])]
    ntr = int(len(idx) * 0.9)
    tr, te = idx[:ntr], idx[ntr:]
    sch = LearnedScheduler(init_params(seed), device)
    sch.train(X[tr], T[tr], epochs=epochs)
    pred = sch.predict(X[te]).cpu().numpy()
    base = T[tr].mean(0)
    report = {
        "samples": int(len(idx)), "train": int(ntr), "test": int(len(te)),
        "mae_logwork": float(np.mean(np.abs(pred[:, 0] - T[te, 0]))),
        "mae_logwork_const": float(np.mean(np.abs(base[0] - T[te, 0]))),
        "mae_sweeps": float(np.mean(np.abs(np.clip(np.rint(pred[:, 1]), 0, 8) - T[te, 1]))),
        "mae_sweeps_const": float(np.mean(np.abs(np.rint(base[1]) - T[te, 1]))),
        "sweeps_predicted_share": round(float(np.mean(np.rint(pred[:, 1]) >= 1)), 4),
        "sweep_label_share": {str(o): round(float(np.mean(labels == o)), 4) for o in SWEEP_OPTIONS},
    }
    sch.meta.update({"report": report})
    return sch, report
