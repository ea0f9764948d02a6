"""Autotuner for the launch configuration of the GPU forms.

It picks, per scene, the thread-block size, the wavefront depth (tracking steps a thread takes
between connection regroupings, `regroup`) and the empty-space cell size (`skip_cell`), or local
majorants (`macro_cell`), by timing short renders of a slice of the workload with CUDA events. All
candidates evaluate the same estimator on the same paths, so the objective is events per second.
The batched form is tuned over its block size and resident blocks per SM.

The search itself (`select`) is plain host logic and takes any timing function, so it is testable
without a GPU.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field


@dataclass(frozen=True)
class Candidate:
    form: str = "wavefront"
    block_size: int = 256
    regroup: int = 4
    skip_cell: int = 0
    macro_cell: int = 0

    def kwargs(self):
        return {"form": self.form, "block_size": self.block_size, "regroup": self.regroup,
                "skip_cell": self.skip_cell, "macro_cell": self.macro_cell}


@dataclass
class Result:
    best: Candidate
    trials: list = field(default_factory=list)   # (candidate, events_per_s)


def default_candidates(has_grid=True, max_cell=8):
    """Block- or warp-level regrouping, wavefront depth 1..8, blocks of 128 or 256 (the warp form:
    128), empty-space cells 0 (off) .. max_cell, a few local-majorant cell sizes, and the path-pool
    form (regrouping by event type; blocks of 128, one free flight per round) with each cell size."""
    cells = [0] + ([c for c in (1, 2, 4, 8) if c <= max_cell] if has_grid else [])
    out = []
    for form, block, regroup, skip in itertools.product(("wavefront", "wavefront_warp"), (256, 128),
                                                        (1, 2, 4, 8), cells):
        if form == "wavefront_warp" and block > 128:
            continue   # the warp-regrouped form runs blocks of at most 128 threads
        out.append(Candidate(form, block, regroup, skip, 0))
    for skip in cells:
        out.append(Candidate("wavefront_pool", 128, 1, skip, 0))
    if has_grid:
        for block, regroup, mc in itertools.product((256,), (2, 4), (4, 8)):
            out.append(Candidate("wavefront", block, regroup, 0, mc))
    return out


def select(candidates, measure, prune=1.6):
    """Coordinate search: time every candidate once (measure(candidate) -> events/s), then re-time
    the ones within a factor `prune` of the best and keep the best of the re-timed set."""
    if not candidates:
        raise ValueError("no candidates")
    trials = [(c, float(measure(c))) for c in candidates]
    top = max(v for _, v in trials)
    finalists = [c for c, v in trials if v * prune >= top]
    retimed = [(c, float(measure(c))) for c in finalists]
    trials += retimed
    best = max(retimed, key=lambda cv: cv[1])[0]
    return Result(best=best, trials=trials)


def tune_render(scene, n_paths, candidates=None, repeats=2, path_offset=0):
    """Tune the single-scene render of `scene` (a Scene) on n_paths paths."""
    import torch

    if candidates is None:
        candidates = default_candidates(has_grid=scene.conc_t is not None or
                                        scene.solv_t is not None)
    stream = torch.cuda.current_stream(scene.device)

    def measure(c):
        kw = c.kwargs()
        scene.render(n_paths=n_paths, path_offset=path_offset, film=True, **kw)   # warm-up
        best = float("inf")
        for _ in range(repeats):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            scene.render(n_paths=n_paths, path_offset=path_offset, film=True, **kw)
            b.record(stream)
            b.synchronize()
            best = min(best, a.elapsed_time(b))
        events = scene.read()["counters"]["events"]
        return events / (best / 1000.0)

    return select(candidates, measure)


def tune_batch(make_batch, candidates=((256, 0), (128, 0), (256, 2), (128, 4)), repeats=2):
    """Tune the batched launch: make_batch(block_size, blocks_per_sm) -> Batch."""
    import torch

    cands = [Candidate("batch", b, bps, 0, 0) for b, bps in candidates]

    def measure(c):
        bt = make_batch(c.block_size, c.regroup)
        bt.launch()
        best = float("inf")
        for _ in range(repeats):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            bt.launch()
            b.record()
            b.synchronize()
            best = min(best, a.elapsed_time(b))
        events = bt.read()["counters"]["events"]
        bt.close()
        return events / (best / 1000.0)

    return select(cands, measure)
