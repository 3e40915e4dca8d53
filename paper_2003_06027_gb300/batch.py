"""Batched FWI over many independent inversion instances of uneven grid size.

Two ways to run the same gradient sweep (J_i and dJ_i/dc_i of every instance i):

* ``plain``: the per-shot scheme of the paper's multi-GPU experiment
  (Performance Benchmarking: shots split across devices, gradients summed): one
  instance after the other, one shot per fwi_misfit_grad call, on one stream,
  the per-shot gradients summed.
* ``batched``: every instance's shots in one fwi_misfit_grad call (shots are a
  batch axis of every step kernel), and W instances in flight at once, each on
  its own CUDA stream and library context (a pool of W persistent host threads,
  one per stream; the library call releases the GIL). Instances are handed out
  largest first.
* ``graph``: every instance's gradient call is recorded once as a CUDA graph
  (fwi.GradGraph, one library context per instance); a sweep is then one graph
  launch per instance, spread over W streams from a single host thread, so the
  host issues one launch per instance instead of tens of thousands of step
  kernels.
* ``persistent``: the instances split into W groups (round robin over the
  instances sorted by size), each group one fwi.Batch on its own stream: each
  time step of a group is ONE persistent launch whose CTAs walk the (instance,
  shot, tile) work items of every instance of the group, and a group's whole
  sweep is one recorded CUDA graph. W = 1 puts every instance into each
  step's launch; larger W trades launch count for L2 locality (a step of one
  launch touches all its instances' fields). Results equal the per-instance
  calls bit for bit.

``autotune`` measures a sweep on the instances themselves for each candidate
(mode, W, checkpoint interval K) and keeps the fastest. Both modes compute the same
gradients (up to the order of the shot sum), so an FWI loop reaches the same
misfit in the same number of iterations; what differs is GPU time per iteration.
All wave propagation and all gradients run in the library's kernels; the model
update and the plain mode's shot sum are torch element-wise operations.
"""

from __future__ import annotations

import threading
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import fwi, optim


@dataclass
class Instance:
    name: str
    c: torch.Tensor          # [nz][nx] current model (updated in place by fwi_iterations)
    stf: torch.Tensor        # [S][nt]
    x0: torch.Tensor         # [S][2]
    rec_iz: torch.Tensor
    rec_ix: torch.Tensor
    observed: torch.Tensor   # [S][nrec][nt]
    kw: dict
    cell_steps: int          # S * padded cells * nt: one forward sweep

    @property
    def shots(self) -> int:
        return int(self.stf.shape[0])


def prepare(problems, device=0) -> list:
    """Device copies of synth problem dicts, with observed data from each true model."""
    dev = torch.device("cuda", device)
    out = []
    for d in problems:
        cu = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev)
        kw = fwi.problem_kwargs(d)
        c, stf, x0, iz, ix = cu(d["c"]), cu(d["stf"]), cu(d["x0"]), cu(d["rec_iz"]), cu(d["rec_ix"])
        obs = fwi.forward(cu(d["c_true"]), stf, x0, iz, ix, **kw)
        S, nt = d["stf"].shape
        cells = S * (d["nz"] + 2 * d["npml"]) * (d["nx"] + 2 * d["npml"]) * nt
        out.append(Instance(d["name"], c, stf, x0, iz, ix, obs, kw, cells))
    torch.cuda.synchronize(dev)
    return out


def _grad_batched(inst: Instance, K: int, groups=(0, 0), tile_rows: int = 0):
    fwi.set_shot_groups(*groups, device=inst.c.device.index)
    fwi.set_tile_shape(tile_rows, device=inst.c.device.index)
    J, g, _, _, _ = fwi.misfit_grad(inst.c, inst.stf, inst.x0, inst.rec_iz, inst.rec_ix, inst.observed,
                                    ckpt_every=K, want_src=False, **inst.kw)
    return J, g


def _grad_per_shot(inst: Instance, K: int):
    J = None
    g = None
    for s in range(inst.shots):
        Js, gs, _, _, _ = fwi.misfit_grad(inst.c, inst.stf[s:s + 1], inst.x0[s:s + 1], inst.rec_iz, inst.rec_ix,
                                          inst.observed[s:s + 1], ckpt_every=K, want_src=False, **inst.kw)
        J = Js if J is None else J + Js
        g = gs if g is None else g + gs
    return J, g


_graphs = {}
_graph_streams = {}


def _graph_of(inst: Instance, K: int, groups=(0, 0), tile_rows: int = 0) -> fwi.GradGraph:
    key = (id(inst), K, tuple(groups), tile_rows)
    g = _graphs.get(key)
    if g is None or g._a.c.data_ptr() != inst.c.data_ptr():
        g = fwi.GradGraph(inst.c, inst.stf, inst.x0, inst.rec_iz, inst.rec_ix, inst.observed, ckpt_every=K,
                          groups=groups, tile_rows=tile_rows, **inst.kw)
        _graphs[key] = g
    return g


_batches = {}


def _batch_of(instances, K: int) -> fwi.Batch:
    key = (tuple(id(i) for i in instances), K)
    b = _batches.get(key)
    if b is None or any(b._calls[k].c.data_ptr() != inst.c.data_ptr() for k, inst in enumerate(instances)):
        if b is not None:
            b.close()
        b = fwi.Batch([(i.c, i.stf, i.x0, i.rec_iz, i.rec_ix, i.observed, i.kw) for i in instances], ckpt_every=K)
        _batches[key] = b
    return b


def close_graphs():
    """Free the recorded graphs, batches and their contexts."""
    for k in list(_graphs):
        _graphs.pop(k).close()
    for k in list(_batches):
        _batches.pop(k).close()


def _streams(W: int, device: int):
    key = (W, device)
    if key not in _graph_streams:
        _graph_streams[key] = [torch.cuda.Stream(device) for _ in range(W)]
    return _graph_streams[key]


class _Pool:
    """W persistent host threads, each with its own CUDA stream and library
    context (so its device arena is reused from sweep to sweep)."""

    def __init__(self, workers: int, device: int):
        import queue

        self.q = queue.Queue()
        self.device = device
        self.threads = [threading.Thread(target=self._loop, daemon=True) for _ in range(workers)]
        for t in self.threads:
            t.start()

    def _loop(self):
        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream()
        while True:
            job = self.q.get()
            if job is None:
                fwi.release_context()
                self.q.task_done()
                return
            fn, done = job
            try:
                with torch.cuda.stream(stream):
                    fn()
                stream.synchronize()
            except Exception as e:  # surfaced by run()
                done.append(e)
            self.q.task_done()

    def run(self, fns):
        errors = []
        for fn in fns:
            self.q.put((fn, errors))
        self.q.join()
        if errors:
            raise errors[0]

    def close(self):
        for _ in self.threads:
            self.q.put(None)
        self.q.join()


_pools = {}


def pool(workers: int, device: int = 0) -> _Pool:
    key = (workers, device)
    if key not in _pools:
        _pools[key] = _Pool(workers, device)
    return _pools[key]


def close_pools():
    """Stop the worker threads and free their library contexts."""
    for k in list(_pools):
        _pools.pop(k).close()


def sweep(instances, mode: str = "batched", workers: int = 4, ckpt_every: int = 100, groups=(0, 0),
          tile_rows: int = 0):
    """One gradient sweep over all instances; returns ([J_i], [g_i], seconds).
    The time is host wall time with the device idle on both sides (every
    library call ends with a stream synchronisation). ``tile_rows``: tile
    height of the forward steps (fwi_set_tile_shape; the persistent mode runs
    32-row tiles)."""
    n = len(instances)
    Js, gs = [None] * n, [None] * n
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if mode == "plain":
        for i, inst in enumerate(instances):
            Js[i], gs[i] = _grad_per_shot(inst, min(ckpt_every, int(inst.stf.shape[1])))
    elif mode == "batched":
        def job(i):
            def fn():
                inst = instances[i]
                Js[i], gs[i] = _grad_batched(inst, min(ckpt_every, int(inst.stf.shape[1])), groups, tile_rows)
            return fn

        order = sorted(range(n), key=lambda i: -instances[i].cell_steps)  # largest first
        pool(max(1, min(workers, n)), torch.cuda.current_device()).run([job(i) for i in order])
    elif mode == "graph":
        order = sorted(range(n), key=lambda i: -instances[i].cell_steps)  # largest first
        graphs = {i: _graph_of(instances[i], min(ckpt_every, int(instances[i].stf.shape[1])), groups, tile_rows)
                  for i in order}
        streams = _streams(max(1, min(workers, n)), torch.cuda.current_device())
        main = torch.cuda.current_stream()
        for s in streams:
            s.wait_stream(main)
        for k, i in enumerate(order):
            graphs[i].launch(streams[k % len(streams)])
        for k, i in enumerate(order):
            graphs[i].check(streams[k % len(streams)])
            Js[i], gs[i] = graphs[i].misfit.clone(), graphs[i].grad.clone()
    elif mode == "persistent":
        W = max(1, min(workers, n))
        order = sorted(range(n), key=lambda i: -instances[i].cell_steps)  # largest first, dealt round robin
        groups = [order[k::W] for k in range(W)]
        batches = [_batch_of([instances[i] for i in grp], ckpt_every) for grp in groups]
        streams = _streams(W, torch.cuda.current_device())
        torch.cuda.synchronize()
        t0 = time.perf_counter()  # creation (the first sweep and its recording) is not part of a sweep
        for b, st in zip(batches, streams):
            b.launch(st)
        for b, st, grp in zip(batches, streams, groups):
            b.check(st)
            for j, i in enumerate(grp):
                Js[i], gs[i] = b.misfit[j:j + 1].clone(), b.grads[j].clone()
    else:
        raise ValueError(f"unknown mode {mode!r}")
    torch.cuda.synchronize()
    return Js, gs, time.perf_counter() - t0


def _close_batches_but(instances, best):
    """Free the persistent-mode batches except those of the candidate `best`."""
    keep = set()
    if best is not None and best[0] == "persistent":
        W = max(1, min(best[1], len(instances)))
        order = sorted(range(len(instances)), key=lambda i: -instances[i].cell_steps)
        keep = {(tuple(id(instances[i]) for i in order[k::W]), best[2]) for k in range(W)}
    for key in [k for k in _batches if k not in keep]:
        _batches.pop(key).close()
    torch.cuda.synchronize()


def autotune(instances, workers=(1, 2, 4, 8), ckpt=(50, 100, 200), modes=("batched",), groups=((0, 0),),
             tiles=(0,)):
    """Pick (mode, workers, ckpt_every, shot groups, tile height) by timing one
    sweep per candidate on the given instances (the first sweep of each
    candidate also sizes the arenas or records the graphs, so each candidate is
    run twice and the second run counts). ``groups`` lists (forward, adjoint)
    shot-group counts, the step kernels' launch shape (fwi_set_shot_groups);
    ``tiles`` lists forward tile heights (fwi_set_tile_shape: 0 or 32, 64; the
    persistent mode runs 32-row tiles only). A candidate's key is (mode, W, K),
    followed by the shot groups if more than one is listed and by the tile
    height if more than one is listed (`candidate` unpacks it). The pools of
    the losing worker counts are closed, and the graphs and batches the winner
    does not use are freed."""
    best = None
    table = {}
    dev = torch.cuda.current_device()
    for mode in modes:
        for W in workers:
            prev = best
            for K in ckpt:
                for grp in groups:
                    grp = tuple(grp)
                    for tile in (tiles if mode != "persistent" else tiles[:1]):
                        sweep(instances, mode, W, K, grp, tile)
                        _, _, t = sweep(instances, mode, W, K, grp, tile)
                        key = (mode, W, K) + ((grp,) if len(groups) > 1 else ()) + ((tile,) if len(tiles) > 1 else ())
                        table[key] = t
                        if best is None or t < table[best]:
                            best = key
                        _close_batches_but(instances, best)  # each grouping holds every instance's workspace
            if mode == "batched":  # keep at most the best pool alive between candidates
                bw = best[1] if best[0] == "batched" else None
                loser = W if bw != W else (prev[1] if prev is not None and prev[0] == "batched" and prev[1] != W
                                           else None)
                if loser is not None and (loser, dev) in _pools:
                    _pools.pop((loser, dev)).close()
    _, _, bK, bgrp, btile = candidate(best, groups, tiles)
    for key in [k for k in _graphs if not (best[0] == "graph" and k[1:] == (bK, bgrp, btile))]:
        _graphs.pop(key).close()  # graphs the winner does not use
    _close_batches_but(instances, best)
    return best, table


def candidate(key, groups=((0, 0),), tiles=(0,)):
    """(mode, workers, ckpt_every, shot groups, tile height) of an autotune key."""
    mode, W, K = key[:3]
    rest = list(key[3:])
    grp = tuple(rest.pop(0)) if len(groups) > 1 else tuple(groups[0])
    tile = rest.pop(0) if len(tiles) > 1 else tiles[0]
    return mode, W, K, grp, tile


def fwi_iterations(instances, iters: int, mode: str = "batched", workers: int = 4, ckpt_every: int = 100,
                   step: float = 20.0, vmin: float = 1500.0, vmax: float = 4500.0):
    """Steepest descent with a normalised step (at most ``step`` m/s per cell per
    iteration) on every instance; returns per-iteration total misfit and time."""
    hist = []
    for _ in range(iters):
        Js, gs, t = sweep(instances, mode, workers, ckpt_every)
        hist.append((float(sum(float(J[0]) for J in Js)), t))
        with torch.no_grad():
            for inst, g in zip(instances, gs):
                inst.c.sub_(step * g / g.abs().max().clamp_min(1e-30)).clamp_(vmin, vmax)
    return hist


def fwi_lbfgs(inst: Instance, iters: int, ckpt_every: int = 100, step0: float = 40.0, m: int = 5,
              vmin: float = 1500.0, vmax: float = 4500.0):
    """FWI of one instance with the paper's outer loop, L-BFGS (optim.lbfgs,
    velocity bounds [vmin, vmax], first step at most ``step0`` m/s per cell),
    each misfit/gradient evaluation one launch of the instance's recorded
    graph. Updates ``inst.c``; returns the optimiser's log."""
    K = min(ckpt_every, int(inst.stf.shape[1]))
    g = _graph_of(inst, K)

    def fun_grad(c):
        with torch.no_grad():
            inst.c.copy_(c)
        g.launch()
        g.check()
        return float(g.misfit[0]), g.grad.clone()

    c, log = optim.lbfgs(fun_grad, inst.c, iters, m=m, step0=step0, lower=vmin, upper=vmax)
    with torch.no_grad():
        inst.c.copy_(c)
    return log
