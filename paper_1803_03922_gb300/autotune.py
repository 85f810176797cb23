"""Autotuner for the level loop: picks the degree threshold TH (Sec. VI-B: the
threshold balances delegates against normal-vertex edges; the paper sweeps it
and picks from the measured rates), Beamer's alpha/beta, the CTAs per SM, the
direction rule (alpha/beta or the paper's FV/BV rule, Sec. IV-B, with its
factor0), and a per-level direction schedule, by timing BFS runs from sample
sources on the device.  The search only changes which work is done, never the
result (Sec. IV-B), so any tuned schedule gives the same depth and parent.

The search logic (coordinate descent, greedy per-level mask) is independent of
the GPU: it takes an `evaluate(options) -> seconds` callable, so it can be
tested with a synthetic cost model.
"""
from __future__ import annotations

import dataclasses
import itertools
from typing import Callable, Dict, Iterable, List, Optional, Sequence, Tuple

# tunables of bfs_options searched at run time (the graph stays built)
RUN_SPACE: Dict[str, Sequence] = {
    "alpha": (5, 10, 15, 30, 60),
    "beta": (9, 18, 36, 72),
    "blocks_per_sm": (1, 2, 3),
}
PAPER_FACTOR0 = (0.05, 0.1, 0.5, 1.0, 2.0)
TH_SPACE = (32, 64, 128, 256)


def th_for_scale(scale: int) -> int:
    """Degree threshold suggested for an RMAT graph of 2^scale vertices (Sec. VI-B):
    the best TH grows by about sqrt(2) per scale, and 64 is the value taken at
    scale 30 (128 at scale 32), so TH = 64 * 2^((scale - 30) / 2), rounded, >= 1."""
    return max(1, int(round(64 * 2.0 ** ((scale - 30) / 2.0))))


def th_goals(row: dict, n: int, p: int = 1) -> dict:
    """The paper's two goals for TH (Sec. VI-B) on one row of Graph.degree_classes:
    delegates under 4 n / p, and nn entries under 10 % of all entries."""
    return {"delegates_under_4n_over_p": row["delegates"] <= 4 * n // p, "nn_under_10pct": row["nn_pct"] < 10.0}


def th_space_for_scale(scale: int):
    """TH candidates: the fixed sweep plus the per-scale rule's value and its
    neighbours a factor 2 away."""
    t = th_for_scale(scale)
    return tuple(sorted(set(TH_SPACE) | {max(1, t // 2), t, 2 * t}))
BEAMER, PAPER, MASK, BEAMER_STAY = 0, 5, 4, 7


@dataclasses.dataclass
class TuneResult:
    th: int
    options: Dict[str, object]
    seconds: float
    baseline_seconds: float
    trials: List[Tuple[Dict[str, object], float]]

    @property
    def speedup(self) -> float:
        return self.baseline_seconds / self.seconds if self.seconds > 0 else 0.0


def coordinate_descent(evaluate: Callable[[Dict[str, object]], float], start: Dict[str, object],
                       space: Dict[str, Sequence], rounds: int = 2,
                       trials: Optional[list] = None) -> Tuple[Dict[str, object], float]:
    """Minimise evaluate over the product of `space`, one coordinate at a time."""
    best = dict(start)
    best_t = evaluate(best)
    if trials is not None:
        trials.append((dict(best), best_t))
    for _ in range(rounds):
        improved = False
        for key, values in space.items():
            for v in values:
                if best.get(key) == v:
                    continue
                cand = dict(best, **{key: v})
                t = evaluate(cand)
                if trials is not None:
                    trials.append((dict(cand), t))
                if t < best_t:
                    best, best_t, improved = cand, t, True
        if not improved:
            break
    return best, best_t


def greedy_mask(evaluate: Callable[[Dict[str, object]], float], base: Dict[str, object],
                directions: Sequence[int], trials: Optional[list] = None,
                tolerance: float = 0.0) -> Tuple[Dict[str, object], float]:
    """Per-level schedule: start from the directions a heuristic took (bit L of
    the mask = level L backward) and flip one level at a time, keeping a flip
    when it lowers the time by more than `tolerance` (relative)."""
    mask = 0
    for L, d in enumerate(directions[:63]):
        if d:
            mask |= 1 << L
    if len(directions) > 63 and directions[-1]:
        mask |= 1 << 63
    best = dict(base, schedule=MASK, schedule_mask=mask)
    best_t = evaluate(best)
    if trials is not None:
        trials.append((dict(best), best_t))
    for L in range(min(len(directions), 64)):
        cand = dict(best, schedule_mask=best["schedule_mask"] ^ (1 << L))
        t = evaluate(cand)
        if trials is not None:
            trials.append((dict(cand), t))
        if t < best_t * (1.0 - tolerance):
            best, best_t = cand, t
    return best, best_t


def tune(evaluate_for_th: Callable[[int], Callable[[Dict[str, object]], float]],
         directions_for_th: Callable[[int, Dict[str, object]], Sequence[int]],
         ths: Iterable[int] = TH_SPACE, defaults: Optional[Dict[str, object]] = None,
         mask_search: bool = True, baseline_th: int = 64) -> TuneResult:
    """Full search.  evaluate_for_th(th) returns an evaluate(options) for a graph
    built with that threshold; directions_for_th(th, options) returns the
    per-level directions the options produce on a representative source."""
    defaults = dict(defaults or {"schedule": BEAMER_STAY, "alpha": 10, "beta": 18, "blocks_per_sm": 2})
    trials: list = []
    baseline_t = None
    per_th = {}
    for th in ths:
        ev = evaluate_for_th(th)
        t = ev(defaults)
        trials.append((dict(defaults, th=th), t))
        per_th[th] = t
        if th == baseline_th:
            baseline_t = t
    th_best = min(per_th, key=per_th.get)
    if baseline_t is None:
        baseline_t = per_th[th_best]
    ev = evaluate_for_th(th_best)
    best, best_t = coordinate_descent(ev, defaults, RUN_SPACE, trials=trials)
    paper, paper_t = coordinate_descent(ev, dict(best, schedule=PAPER, factor0=0.5),
                                        {"factor0": PAPER_FACTOR0}, rounds=1, trials=trials)
    if paper_t < best_t:
        best, best_t = paper, paper_t
    if mask_search:
        dirs = directions_for_th(th_best, best)
        masked, masked_t = greedy_mask(ev, best, dirs, trials=trials, tolerance=0.02)
        if masked_t < best_t:
            best, best_t = masked, masked_t
    return TuneResult(th=th_best, options=best, seconds=best_t, baseline_seconds=baseline_t, trials=trials)


# ---- the device runner ------------------------------------------------------------------------

def device_tuner(src, dst, n: int, sources: Sequence[int], runs: int = 2, ths: Iterable[int] = TH_SPACE,
                 mask_search: bool = True) -> Tuple[TuneResult, "object"]:
    """Tunes on the GPU for the edge list (device tensors) and sample sources.
    Returns the result and a Graph built with the chosen TH and options."""
    import torch

    from . import Graph

    graphs = {}

    def graph_for(th):
        if th not in graphs:
            graphs[th] = Graph(src, dst, n, th=th)
        return graphs[th]

    depth = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")

    def evaluate_for_th(th):
        g = graph_for(th)

        def ev(opts):
            g.set_options(**{k: v for k, v in opts.items() if k != "th"})
            for s in sources[:2]:  # warm-up
                g.run(int(s), depth, parent)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(runs):
                for s in sources:
                    g.run(int(s), depth, parent)
            b.record()
            torch.cuda.synchronize()
            g.wait()
            return a.elapsed_time(b) / 1e3
        return ev

    def directions_for_th(th, opts):
        g = graph_for(th)
        g.set_options(**{k: v for k, v in opts.items() if k != "th"})
        _, _, st = g.run(int(sources[0]), depth, parent, stats=True)
        return [st.level[i].direction for i in range(st.logged_levels)]

    res = tune(evaluate_for_th, directions_for_th, ths=ths, mask_search=mask_search)
    best = graph_for(res.th)
    best.set_options(**{k: v for k, v in res.options.items() if k != "th"})
    for th, g in graphs.items():
        if th != res.th:
            g.close()
    return res, best


BATCH_ALPHA = (2, 5, 15, 30, 60, 120)


def tune_batch_alpha(graph, sources, alphas: Iterable[int] = BATCH_ALPHA, batches: int = 2,
                     with_parents: bool = True) -> Tuple[int, Dict[int, float]]:
    """Schedule of the 64-lane batched form: its direction rule is Beamer's alpha on
    the union frontier (once backward, it stays backward), so the search is over
    alpha.  Times `batches` batches of 64 of `sources` per candidate on the device;
    returns the best alpha and the seconds per batch of every candidate.  The
    graph's alpha is left at the best value."""
    import torch

    from . import Batch

    b = Batch(graph, with_parents=with_parents)
    n = graph.n
    depth = torch.empty((64, n), dtype=torch.uint8, device="cuda")
    parent = torch.empty((64, n), dtype=torch.int32, device="cuda") if with_parents else None
    times = {}
    for a in alphas:
        graph.set_options(alpha=int(a))
        b.run(sources[:64], depth, parent)  # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(batches):
            b.run(sources[64 * i:64 * (i + 1)], depth, parent)
        e1.record()
        torch.cuda.synchronize()
        b.wait()
        times[int(a)] = e0.elapsed_time(e1) / 1e3 / batches
    best = min(times, key=times.get)
    graph.set_options(alpha=best)
    b.close()
    return best, times
