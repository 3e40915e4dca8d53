#!/usr/bin/env python
"""Benchmark of the acoustic FWI gradient (forward + adjoint) on GB300.

Workload: 201 x 601 physical grid (+32 CPML cells per side = 265 x 665), 8th
order in space, dt = 0.8 ms, 3000 steps, 16 Ricker shots (8 Hz), 301
receivers, checkpoint every 100 steps; seeded dipping-layer model with faults
(observed data) and its Gaussian-smoothed start model (the gradient is taken
there). One bench step = one full misfit + gradient evaluation
(fwi_misfit_grad). Metric: Gcell-steps/s = shots x padded cells x nt / time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs the same per-GPU workload (shots are
independent; no collective on the data path: weak scaling); rank 0 prints one
JSON line with the max-over-ranks time.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FWI Gcell-steps/s (fwd+adjoint), % HBM roofline, batched/learned vs plain"
UNIT = "Gcell-steps/s"

# Algorithmic HBM bytes per cell-step of each step kernel (FP32): every field
# streamed once per step, halos assumed cached.
#   forward (recording):  read u^n, u^{n-1}, m; write u^{n+1}                         16 B
#   forward (storing):    + write the fluxes p_x, p_z to the segment slot             24 B
#   adjoint:              read lam_{n+1}, lam_{n+2}, m, p_x, p_z, g; write lam_n, g   32 B
# plus, per cell inside an x- or z-CPML strip and per active axis, 16 B:
#   forward psi and zeta read+write; adjoint Z and P read+write.
BYTES = {"fwd": (16, 16), "store": (24, 16), "adj": (32, 16)}
# Whole-path algorithmic bytes per cell-step (one sweep of every field per step,
# halos cached, CPML memory not counted): acoustic forward 16 B; acoustic
# gradient 48 B (forward 16, stored wavefield 4 + reload 4, adjoint 16, FP32
# gradient partial r/w 8); elastic forward 52 B (5 fields r/w, 3 parameters);
# elastic gradient 168 B (forward 52, stored 20 + reload 20, adjoint 52, 3
# partials r/w 24). The kernels move more (two kernels per elastic step, stored
# fluxes instead of wavefields, recomputation), so these fractions are lower
# than the per-kernel ones.
PATH_BYTES = {"acoustic_forward": 16, "acoustic_gradient": 48, "elastic_forward": 52, "elastic_gradient": 168}
# Elastic step kernels, per cell-step of one step (velocity and stress kernels together):
#   forward:   vel 36 B (read sxx, szz, sxz, vx, vz, bx, bz; write vx, vz) + str 44 B (read vx, vz, sxx, szz,
#              sxz, lambda, lambda+2mu, mu_xz; write sxx, szz, sxz)                                        80 B
#   recompute: + the stored forces fx, fz and strains ex, ez, exz                                          100 B
#   adjoint:   str 76 B (adjoint stresses read through TMA, adjoint velocities r/w, lambda, lambda+2mu,
#              mu_xz, stored strains, 3 partials r/w) + vel 64 B (adjoint velocities read, adjoint
#              stresses r/w, bx, bz, stored forces, 2 partials r/w)                                        140 B
# plus 32 B per cell and CPML axis (two memory variables r/w in each of the two kernels).
ELA_BYTES = {"fwd": (80, 32), "store": (100, 32), "adj": (140, 32)}


def padded(d):
    return d["nz"] + 2 * d["npml"], d["nx"] + 2 * d["npml"]


def launch_bytes(d, kind):
    Nz, Nx = padded(d)
    S = d["stf"].shape[0]
    cells = Nz * Nx
    pml_cells = Nz * 2 * d["npml"] + Nx * 2 * d["npml"]  # (cell, axis) pairs in CPML strips
    base, per_pml = BYTES[kind]
    return S * (base * cells + per_pml * pml_cells)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def adj_source_hash():
    """sha256 of the source the acoustic adjoint kernel is compiled from: the
    part of csrc/acoustic_kernels.cu before the forward-step section (shared
    definitions), its adjoint-step section (up to the bounded-wait self-test),
    and the two headers it includes. Edits elsewhere in the file (the forward
    kernels, the launch code) leave it unchanged."""
    csrc = os.path.join(ROOT, "paper_2003_06027_gb300", "csrc")
    src = open(os.path.join(csrc, "acoustic_kernels.cu")).read()
    a = src.index("// Forward step n:")
    b = src.index("// Adjoint step n (")
    c = src.index("// Self-test of the bounded wait")
    h = hashlib.sha256()
    for part in (src[:a], src[b:c], open(os.path.join(csrc, "tma.cuh")).read(),
                 open(os.path.join(csrc, "fwi_internal.cuh")).read()):
        h.update(part.encode())
    return h.hexdigest()


def load_traffic():
    """DRAM bytes per adjoint step from the committed ncu summary, if the
    adjoint kernel's source is unchanged since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    kv = {}
    for line in open(p):
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    try:
        if kv.get("adj_source_sha256") != adj_source_hash():
            return None
        return float(kv["adj_dram_bytes_per_launch_full"])
    except (KeyError, ValueError, OSError):
        return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = str(gpu_index)
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", self.gpu, "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def elastic_measure(steps):
    """fwd+adjoint and forward throughput of the 300 x 800 elastic workload
    (32 moment-tensor shots, 4000 steps, 4th order, checkpoint every 100)."""
    import torch

    from paper_2003_06027_gb300 import fwi, synth

    d = synth.elastic_layered()
    kw = fwi.problem_kwargs(d)
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    args = [cu(d[k]) for k in ("vp", "vs", "rho", "stf", "x0", "mt", "rec_iz", "rec_ix")]
    obs = fwi.forward_elastic(*args, **kw)
    Nz, Nx = padded(d)
    S, nt = d["stf"].shape
    cs = S * Nz * Nx * nt
    fwi.misfit_grad_elastic(*args, obs, ckpt_every=d["ckpt_every"], **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fwi.misfit_grad_elastic(*args, obs, ckpt_every=d["ckpt_every"], **kw)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    t = fwi.last_timing()
    e0.record()
    for _ in range(steps):
        fwi.forward_elastic(*args, out=obs, **kw)
    e1.record()
    torch.cuda.synchronize()
    fms = e0.elapsed_time(e1) / steps
    peak, kind = load_peaks()
    path = {k: {"bytes_per_cell_step": b, "GBps": b * cs / (tm / 1e3) / 1e9, "frac": b * cs / (tm / 1e3) / 1e9 / peak,
                "peak_source": kind} for k, b, tm in (("forward", PATH_BYTES["elastic_forward"], fms),
                                                     ("gradient", PATH_BYTES["elastic_gradient"], ms))}
    cells = S * Nz * Nx
    pml_pairs = S * (Nz * 2 * d["npml"] + Nx * 2 * d["npml"])
    kern = {}
    for k, tms in (("fwd", t.fwd_step_ms), ("store", t.store_step_ms), ("adj", t.adj_step_ms)):
        base, per_pml = ELA_BYTES[k]
        gbs = (base * cells + per_pml * pml_pairs) / (tms / 1e3) / 1e9
        kern[k] = {"step_ms": tms, "algorithmic_GBps": gbs, "frac": gbs / peak, "peak_source": kind}
    return {"workload": d["name"] + "-ckpt100", "value": cs / (ms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": ms,
            "path_roofline": path, "kernels": kern,
            "forward": {"value": cs / (fms / 1e3) / 1e9, "ms_per_step": fms},
            "cell_steps_per_step": cs, "step_launch_ms": {"fwd_vel+str": t.fwd_step_ms,
                                                          "recompute_vel+str": t.store_step_ms,
                                                          "adjoint_str+vel": t.adj_step_ms}}


def acoustic_xl_measure(peak):
    """Per-launch HBM bandwidth of the acoustic step kernels when one step's
    working set (256 shots x 265 x 665 cells, ~1 GB per step) is far larger
    than L2: the same discretisation as the headline workload, 300 steps."""
    import torch

    from paper_2003_06027_gb300 import fwi, synth

    d = synth.acoustic_xl(nshots=256, nt=300)
    kw = fwi.problem_kwargs(d)
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    c, stf, x0, iz, ix = cu(d["c"]), cu(d["stf"]), cu(d["x0"]), cu(d["rec_iz"]), cu(d["rec_ix"])
    obs = fwi.forward(c, stf, x0, iz, ix, **kw)
    for _ in range(2):
        fwi.misfit_grad(c, stf, x0, iz, ix, obs, ckpt_every=100, **kw)
    torch.cuda.synchronize()
    t = fwi.last_timing()
    out = {"workload": d["name"] + "-ckpt100", "shots": 256, "nt": 300,
           "working_set_per_step_MB": round(5 * 256 * (265 * 665) * 4 / 1e6)}
    for k, ms in (("fwd", t.fwd_step_ms), ("store", t.store_step_ms), ("adj", t.adj_step_ms)):
        gbs = launch_bytes(d, k) / (ms / 1e3) / 1e9
        out[k] = {"avg_launch_ms": ms, "algorithmic_GBps": gbs, "frac": gbs / peak}
    return out


def graph_ms(args_dev, obs, K, kw, steps):
    """Mean device time of one replay of the gradient call recorded as a CUDA
    graph (recorded and replayed once before timing)."""
    import torch

    from paper_2003_06027_gb300 import fwi

    g = fwi.GradGraph(*args_dev, obs, ckpt_every=K, want_src=True, **kw)
    try:
        st = torch.cuda.current_stream()
        g.launch(st)
        g.check(st)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            g.launch(st)
        e1.record()
        g.check(st)
        return e0.elapsed_time(e1) / steps
    finally:
        g.close()


def store_all_measure(d, args_dev, obs, kw, value_k, steps=3):
    """The headline gradient with ckpt_every = nt: the forward sweep stores the
    fluxes of every step (2 nt fields in HBM) and no step is recomputed, the
    memory-for-time trade the GPU's HBM allows on this workload (timed as a
    recorded-graph replay, like the headline)."""
    Nz, Nx = padded(d)
    S, nt = d["stf"].shape
    cs = S * Nz * Nx * nt
    ms = graph_ms(args_dev, obs, nt, kw, steps)
    pitch = -(-Nx // 64) * 64 + 16
    rows = -(-Nz // 64) * 64 + 16
    return {"workload": d["name"] + f"-ckpt{nt}", "value": cs / (ms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": ms,
            "stored_flux_GB": 2 * nt * S * pitch * rows * 4 / 1e9, "vs_ckpt": value_k and cs / (ms / 1e3) / 1e9 / value_k,
            "path_frac": PATH_BYTES["acoustic_gradient"] * cs / (ms / 1e3) / 1e9 / load_peaks()[0]}


def laplacian_op_measure(peak, steps=2):
    """The c^2 Laplacian operator variant (FWI_OP_LAPLACIAN, the persistent
    TMA step kernels' Laplacian instantiation) on the headline workload: gradient and forward throughput, with
    whole-path fractions by the same per-cell-step byte model as the
    divergence form (48 and 16 B)."""
    import torch

    from paper_2003_06027_gb300 import fwi, synth

    d = dict(synth.acoustic_fwi(), op=1)
    kw = fwi.problem_kwargs(d)
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    c, stf, x0, iz, ix = cu(d["c"]), cu(d["stf"]), cu(d["x0"]), cu(d["rec_iz"]), cu(d["rec_ix"])
    obs = fwi.forward(cu(d["c_true"]), stf, x0, iz, ix, **kw)
    Nz, Nx = padded(d)
    S, nt = d["stf"].shape
    cs = S * Nz * Nx * nt
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    for name, call, b in (("gradient", lambda: fwi.misfit_grad(c, stf, x0, iz, ix, obs, ckpt_every=d["ckpt_every"],
                                                                **kw), PATH_BYTES["acoustic_gradient"]),
                          ("forward", lambda: fwi.forward(c, stf, x0, iz, ix, out=obs, **kw),
                           PATH_BYTES["acoustic_forward"])):
        call()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            call()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        v = cs / (ms / 1e3) / 1e9
        res[name] = {"value": v, "unit": UNIT, "ms_per_step": ms, "bytes_per_cell_step": b,
                     "path_frac": b * v / peak}
    # the gradient as a recorded-graph replay, like the headline (the direct call's number above)
    ms = graph_ms((c, stf, x0, iz, ix), obs, d["ckpt_every"], kw, steps)
    v = cs / (ms / 1e3) / 1e9
    res["gradient"] = {"value": v, "unit": UNIT, "ms_per_step": ms, "bytes_per_cell_step": PATH_BYTES["acoustic_gradient"],
                       "path_frac": PATH_BYTES["acoustic_gradient"] * v / peak, "execution": "recorded graph",
                       "direct_call": res["gradient"]}
    return {"workload": d["name"] + "-c2laplacian-ckpt100", "kernels": "acu_fwd_step / acu_adj_step, Laplacian variant", **res}


def batched_measure(n_inst=16):
    """Batched vs plain per-shot gradient sweeps over the first ``n_inst``
    instances of the seeded uneven workload (seed 4; grids 128..512 x
    128..1024, nt 1000..4000, 4..16 shots). The batched sweep's mode (one
    persistent launch per step over all instances in one recorded graph, one
    recorded graph per instance on W streams, or host threads on W streams),
    streams and checkpoint interval come from the autotuner run on the same
    instances."""
    from paper_2003_06027_gb300 import batch, synth

    inst = batch.prepare([synth.uneven_instance(4, i) for i in range(n_inst)])
    cells = sum(i.cell_steps for i in inst)
    modes, tiles = ("persistent", "graph", "batched"), (32, 64)
    best, table = batch.autotune(inst, workers=(1, 2, 4, 8), ckpt=(100,), modes=modes, tiles=tiles)
    mode, W, K, _, tile = batch.candidate(best, tiles=tiles)
    _, _, tb = batch.sweep(inst, mode, W, K, tile_rows=tile)
    batch.close_graphs()
    batch.close_pools()
    batch.sweep(inst, "plain", ckpt_every=100)
    _, _, tp = batch.sweep(inst, "plain", ckpt_every=100)
    best_of = {m: min(t for key, t in table.items() if key[0] == m) for m in modes}
    best_tile = {tt: min(t for key, t in table.items() if key[0] != "persistent" and key[-1] == tt) for tt in tiles}
    batch.close_graphs()
    return {"workload": f"uneven-seed4-{n_inst}-instances", "cell_steps_per_sweep": cells,
            "batched": {"value": cells / tb / 1e9, "unit": UNIT, "s_per_sweep": tb, "mode": mode,
                        "streams": W, "ckpt_every": K, "forward_tile_rows": tile},
            "tile_rows_best": {str(tt): {"value": cells / v / 1e9, "s_per_sweep": v} for tt, v in best_tile.items()},
            "persistent": {"value": cells / best_of["persistent"] / 1e9, "s_per_sweep": best_of["persistent"],
                           "launches": "W groups of instances, each one graph whose time steps are one persistent "
                                       "launch over the group's instances (W = 1: all instances in every launch)"},
            "graphs_best": {"value": cells / best_of["graph"] / 1e9, "s_per_sweep": best_of["graph"]},
            "threads_best": {"value": cells / best_of["batched"] / 1e9, "s_per_sweep": best_of["batched"]},
            "plain_per_shot": {"value": cells / tp / 1e9, "unit": UNIT, "s_per_sweep": tp},
            "speedup": tp / tb,
            "autotune_s": {"-".join(str(x) for x in key): t for key, t in table.items()},
            "timing": "host wall time per sweep, device idle before and after (each sweep ends synchronised)"}


def uneven_all_measure(mode="graph", workers=2, waves=2, tile_rows=0):
    """The whole 64-instance uneven workload (seed 4, 479 G cell-steps per
    gradient sweep) in a batched mode. Its workspace at K = 100 (300 GB)
    exceeds the GPU's memory, so it runs as `waves` sets of consecutive
    instances, one after the other; the time is the sum of their sweeps."""
    from paper_2003_06027_gb300 import batch, synth

    per = (64 + waves - 1) // waves
    cells, secs = 0, 0.0
    for w in range(waves):
        inst = batch.prepare([synth.uneven_instance(4, i) for i in range(w * per, min(64, (w + 1) * per))])
        cells += sum(i.cell_steps for i in inst)
        batch.sweep(inst, mode, workers, ckpt_every=100, tile_rows=tile_rows)  # creation: the first sweep
        _, _, t = batch.sweep(inst, mode, workers, ckpt_every=100, tile_rows=tile_rows)
        secs += t
        batch.close_graphs()
        batch.close_pools()
        del inst
    return {"workload": "uneven-seed4-64-instances", "cell_steps_per_sweep": cells, "mode": mode,
            "streams": workers, "forward_tile_rows": tile_rows, "waves": waves, "value": cells / secs / 1e9, "unit": UNIT, "s_per_sweep": secs,
            "timing": "host wall time per sweep, each wave's sweep timed after its creation sweep"}


def learned_measure():
    """Training throughput of the start-model network (its 3x3 convolutions are
    the project's one dense contraction: BF16 tensor-core GEMMs with FP32
    accumulation): one Adam step on a batch of 32 surveys (16 x 1000 x 64
    inputs, 128 x 256 targets), synthetic inputs of those shapes, against the
    measured sustained BF16 GEMM rate."""
    import torch

    from paper_2003_06027_gb300 import learned as L

    peak = None
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        peak = float(json.load(open(p)).get("bf16_tflops_sustained", 0.0)) or None
    B = 32
    g = torch.Generator(device="cuda").manual_seed(0)
    X = torch.randn((L.NSHOT, B, L.NT, L.NREC), device="cuda", generator=g) * 0.1
    Y = torch.randn((1, B, L.NZ, L.NX), device="cuda", generator=g) * 0.1
    net = L.Net(0, seed=0)

    def step():
        out = net.forward(X)
        _, dout = L.mse(net.h, out, Y)
        net.backward(dout)
        net.step(1e-4)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = 10
    e0.record()
    for _ in range(n):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    tfl = 3.0 * L.network_flops_per_sample() * B / (ms / 1e3) / 1e12
    return {"workload": f"start-model CNN training step, batch {B}, {net.nparams} parameters",
            "ms_per_step": ms, "samples_per_s": B / (ms / 1e3),
            "roofline": {"bound": "tensor", "achieved": tfl, "peak": peak, "unit": "TFLOP/s",
                         "frac": tfl / peak if peak else None, "peak_source": "measured sustained bf16"}}


def learned_fwi_measure(n_train=3072, epochs=12, n_models=4, iters=20):
    """The learned start against plain FWI, live and small: the start-model
    network trained on `n_train` solver-generated surveys, then FWI (L-BFGS,
    `iters` iterations, every evaluation one replay of the recorded gradient) on
    `n_models` held-out models from the smoothed true model (plain start), the
    network's prediction and the mean training model (no survey information).
    Reports the GPU time each start needs to reach the plain start's final
    misfit."""
    import torch

    from paper_2003_06027_gb300 import learned as L

    t0 = time.perf_counter()
    X, Y, _ = L.make_dataset(n_train, seed=5)
    net = L.Net(0, seed=0)
    log = L.train(net, X, Y, epochs=epochs, batch=32, lr=1e-3)
    mean_model = (L.V_MID + L.V_HALF * Y[0].mean(dim=0)).contiguous()
    del X, Y
    torch.cuda.empty_cache()
    _, s = L.compare_fwi(net, n_models=n_models, seed=1005, iters=iters, mean_model=mean_model)
    s = {k: v for k, v in s.items()}
    s.update(train_samples=n_train, epochs=epochs, params=net.nparams, train_seconds=log.seconds,
             total_seconds=time.perf_counter() - t0,
             timing="GPU seconds of the misfit/gradient evaluations of each FWI run (recorded graphs)")
    return s


def dist_setup(backend: str = "nccl"):
    """(world size, rank, local rank) from the torchrun environment; joins the
    process group when there is more than one rank (NCCL on GPUs; the host-side
    logic below also runs under gloo, which the CPU tests use)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist

        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(ws, x, local):
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = f"cuda:{local}" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ws, units_per_rank, ms):
    """Whole-job throughput (weak scaling: every rank processes its own
    units_per_rank, no data-path collective): all ranks' units / the max-over-
    ranks time, in G units per second."""
    return ws * units_per_rank / (ms / 1e3) / 1e9


def host_cores():
    """Cores this process may run on (its CPU affinity), and the machine's count."""
    try:
        usable = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        usable = os.cpu_count() or 1
    return usable, os.cpu_count() or usable


def cpu_oracle_sample(d, shots, nt, repeats=1):
    """Time the FP64 oracle (as it stands) on a bounded sample of the
    workload: `shots` shots, `nt` steps, same grid, run `repeats` times.
    The oracle runs its shots in parallel (OpenMP over shots), so `shots` =
    the thread count keeps every core busy. Returns (Gcell-steps/s, seconds,
    threads)."""
    import oracle

    g = dict(nz=d["nz"], nx=d["nx"], npml=d["npml"], order=d["order"], nt=nt, dz=d["dz"], dx=d["dx"],
             dt=d["dt"], src_kind=d["src_kind"], pml_R=d["pml_R"], pml_vmax=d["pml_vmax"],
             pml_f0=d["pml_f0"], rec_iz=d["rec_iz"], rec_ix=d["rec_ix"])
    stf = np.float64(d["stf"][:shots, :nt])
    x0 = np.float64(d["x0"][:shots])
    c = np.float64(d["c"])
    obs = np.zeros((shots, len(d["rec_iz"]), nt))
    oracle.lib()
    t0 = time.perf_counter()
    for _ in range(repeats):
        oracle.acoustic_misfit_grad(g, c, stf, x0, obs)
    sec = time.perf_counter() - t0
    Nz, Nx = padded(d)
    return repeats * shots * Nz * Nx * nt / sec / 1e9, sec, min(oracle.num_threads(), shots)


def cpu_uneven_sample(n_inst=4, shots=2, nt=100):
    """The FP64 oracle on a bounded subset of the uneven batched workload: the
    first ``n_inst`` instances (seed 4), ``shots`` shots and ``nt`` steps of
    each. Returns (Gcell-steps/s over the subset, seconds, threads)."""
    from paper_2003_06027_gb300 import synth

    cells, sec, cores = 0, 0.0, 1
    for i in range(n_inst):
        d = synth.uneven_instance(4, i)
        v, t, c = cpu_oracle_sample(d, shots, nt)
        cells += v * 1e9 * t
        sec += t
        cores = max(cores, c)
    return cells / sec / 1e9, sec, cores


def run_reference(args, ws, rank):
    """The oracle, timed on the host cores, on bounded samples of the workload."""
    if rank != 0:
        return
    from paper_2003_06027_gb300 import synth

    d = synth.acoustic_fwi()
    import oracle

    # one shot per oracle thread (all of the host cores this process may use)
    shots = max(1, oracle.num_threads())
    nt = 100
    for _ in range(args.warmup):
        cpu_oracle_sample(d, shots, nt)
    vals, secs = [], []
    for _ in range(args.steps):
        v, s, cores = cpu_oracle_sample(d, shots, nt)
        vals.append(v)
        secs.append(s)
    value = statistics.mean(vals)
    sample = f"{shots} shots x {nt} steps of the 265x665 (padded) 8th-order grid per step, FP64 oracle fwd+adjoint"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * statistics.mean(secs),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(d),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                            "host_cores": dict(zip(("usable", "machine"), host_cores()))},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def workload_config(d):
    Nz, Nx = padded(d)
    S, nt = d["stf"].shape
    return {"workload": d["name"] + f"-ckpt{d['ckpt_every']}", "grid_physical": [d["nz"], d["nx"]],
            "grid_padded": [Nz, Nx], "order": d["order"], "npml": d["npml"], "shots": S, "nt": nt,
            "receivers": int(len(d["rec_iz"])), "ckpt_every": d["ckpt_every"],
            "cell_steps_per_step": S * Nz * Nx * nt,
            "l2": "no explicit flush: each step writes and reads back ~80 GB of stored fluxes (28 MB per time "
                  "step) and 2.5 GB of checkpoints through HBM, far more than the 129 MB L2",
            "parallelism": "shots batched on one GPU; N GPUs = N independent replicas"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the elastic and 256-shot measurements")
    ap.add_argument("--uneven-all", action="store_true",
                    help="also time the whole 64-instance uneven workload (persistent mode, two waves)")
    args = ap.parse_args()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import torch

    from paper_2003_06027_gb300 import fwi, synth

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    d = synth.acoustic_fwi()
    kw = fwi.problem_kwargs(d)
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev)
    c, stf, x0, iz, ix = cu(d["c"]), cu(d["stf"]), cu(d["x0"]), cu(d["rec_iz"]), cu(d["rec_ix"])
    obs = fwi.forward(cu(d["c_true"]), stf, x0, iz, ix, **kw)
    K = d["ckpt_every"]
    out = {"misfit": torch.empty(1, dtype=torch.float64, device=dev), "grad": torch.empty_like(c),
           "grad_stf": torch.empty_like(stf), "grad_x0": torch.empty_like(x0)}
    Nz, Nx = padded(d)
    S, nt = d["stf"].shape
    cell_steps = S * Nz * Nx * nt

    # the whole gradient call recorded once as a CUDA graph (outside the timed
    # region) and replayed per step: the same kernels in the same order as a
    # direct call, without the host issuing each of its ~30k launches
    gg = fwi.GradGraph(c, stf, x0, iz, ix, obs, ckpt_every=K, want_src=True, **kw)

    def step():
        gg.launch()
        gg.check()  # one synchronisation and status read per call, as a direct call does
        return gg.timing()

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    kms = {"fwd": [], "store": [], "adj": []}
    launches = 0
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        t = step()
        kms["fwd"].append(t.fwd_step_ms)
        kms["store"].append(t.store_step_ms)
        kms["adj"].append(t.adj_step_ms)
        launches += t.launches
    e1.record()
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop() if sampler else None
    ms = max_over_ranks(ws, e0.elapsed_time(e1) / args.steps, local)
    value = job_value(ws, cell_steps, ms)
    gg.close()

    # the same call issued directly (the host launches every kernel), for comparison
    def direct():
        fwi.misfit_grad(c, stf, x0, iz, ix, obs, ckpt_every=K, out=out, **kw)

    direct()
    torch.cuda.synchronize()
    nd = max(3, args.steps // 2)
    e0.record()
    for _ in range(nd):
        direct()
    e1.record()
    torch.cuda.synchronize()
    direct_ms = max_over_ranks(ws, e0.elapsed_time(e1) / nd, local)

    # forward only (same workload), for reference beside the gradient
    for _ in range(2):
        fwi.forward(c, stf, x0, iz, ix, out=obs, **kw)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    nf = max(3, args.steps // 2)
    for _ in range(nf):
        fwi.forward(c, stf, x0, iz, ix, out=obs, **kw)
    f1.record()
    torch.cuda.synchronize()
    fwd_ms = f0.elapsed_time(f1) / nf

    # end to end with host (pinned) buffers: the recorded call copies the inputs in
    # and the results out at every replay (its own copy nodes), and each step
    # waits for the status word on the host
    pin = lambda a, dt_: torch.as_tensor(np.ascontiguousarray(a, dtype=dt_)).pin_memory()
    h = [pin(d["c"], np.float32), pin(d["stf"], np.float32), pin(d["x0"], np.float32), pin(d["rec_iz"], np.int32),
         pin(d["rec_ix"], np.int32), obs.cpu().pin_memory()]
    gh = fwi.GradGraph(*h, ckpt_every=K, want_src=True, device=local, **kw)
    hout = [gh.misfit, gh.grad, gh.grad_stf, gh.grad_x0]
    h2d = sum(t.numel() * t.element_size() for t in h)
    d2h = sum(t.numel() * t.element_size() for t in hout)
    st_e2e = torch.cuda.current_stream()
    gh.launch(st_e2e)
    gh.check(st_e2e)
    barrier(ws)
    t0 = time.perf_counter()
    ne = max(3, args.steps // 2)
    for _ in range(ne):
        gh.launch(st_e2e)
        gh.check(st_e2e)
    e2e_ms = max_over_ranks(ws, (time.perf_counter() - t0) * 1e3 / ne, local)
    gh.close()
    # the same with the direct call (the host issues every launch), for comparison
    hd = {"misfit": torch.empty(1, dtype=torch.float64).pin_memory(), "grad": torch.empty_like(h[0]).pin_memory(),
          "grad_stf": torch.empty_like(h[1]).pin_memory(), "grad_x0": torch.empty_like(h[2]).pin_memory()}
    fwi.misfit_grad(*h, ckpt_every=K, out=hd, **kw)
    t0 = time.perf_counter()
    for _ in range(ne):
        fwi.misfit_grad(*h, ckpt_every=K, out=hd, **kw)
    e2e_direct_ms = max_over_ranks(ws, (time.perf_counter() - t0) * 1e3 / ne, local)

    if rank != 0:
        return
    # roofline of the dominant kernel (largest device time per step)
    # steps of each kernel per call: the last checkpoint segment is stored by the forward sweep, not recomputed
    nrec_steps = ((nt + K - 1) // K - 1) * K
    tot = {k: statistics.mean(v) * (nrec_steps if k == "store" else nt) for k, v in kms.items()}
    dom = max(tot, key=tot.get)
    peak, peak_kind = load_peaks()
    avg_ms = statistics.mean(kms[dom])
    achieved = launch_bytes(d, dom) / (avg_ms / 1e3) / 1e9
    kernel_names = {"fwd": "acu_fwd_step<4,record>", "store": "acu_fwd_step<4,store>", "adj": "acu_adj_step<4>"}
    groups = min(2 if dom == "adj" else 4, S)  # shot groups per step of the kernel (the library's choice)
    roof = {"bound": "hbm", "kernel": kernel_names[dom], "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_kind, "launches_per_step": groups,
            "note": f"one step of the kernel is {groups} concurrent launches (one per shot group, own stream); "
                    "achieved = the step's algorithmic bytes / the step's duration, traffic likewise per step",
            "traffic": load_traffic() if dom == "adj" else None,
            "algorithmic_bytes_per_launch": launch_bytes(d, dom), "avg_launch_ms": avg_ms}
    kernels = {k: {"avg_launch_ms": statistics.mean(v), "algorithmic_GBps": launch_bytes(d, k) / (statistics.mean(v) / 1e3) / 1e9,
                   "share_of_step": tot[k] / ms} for k, v in kms.items()}
    res = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(d),
           "roofline": roof, "kernels": kernels, "gpu_launches": launches,
           "path_roofline": {k: {"bytes_per_cell_step": PATH_BYTES[b], "GBps": PATH_BYTES[b] * v,
                                 "frac": PATH_BYTES[b] * v / peak, "peak_source": peak_kind}
                             for k, b, v in (("gradient", "acoustic_gradient", value / ws),
                                             ("forward", "acoustic_forward", cell_steps / (fwd_ms / 1e3) / 1e9))},
           "forward": {"value": ws * cell_steps / (fwd_ms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": fwd_ms},
           "execution": "each step replays the whole gradient call recorded once as a CUDA graph "
                        "(fwi_misfit_grad_graph, outside the timed region); kernel times from its phase marks",
           "direct_call": {"value": job_value(ws, cell_steps, direct_ms), "unit": UNIT, "ms_per_step": direct_ms,
                           "note": "fwi_misfit_grad issued directly (host launches every kernel)"},
           "e2e": {"value": ws * cell_steps / (e2e_ms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": e2e_ms,
                   "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                   "path": "fwi_misfit_grad_graph on pinned host buffers, replayed per step (host wall time)",
                   "direct_call": {"value": ws * cell_steps / (e2e_direct_ms / 1e3) / 1e9,
                                   "ms_per_step": e2e_direct_ms, "path": "fwi_misfit_grad with the same host buffers"}},
           "clocks": clocks}
    if not args.no_extra:
        res["elastic"] = elastic_measure(2)
        res["acoustic_xl"] = acoustic_xl_measure(peak)
        res["laplacian_op"] = laplacian_op_measure(peak)
        res["store_all"] = store_all_measure(d, (c, stf, x0, iz, ix), obs, kw, value)
        res["batched_uneven"] = batched_measure()
        if args.uneven_all:
            b = res["batched_uneven"]["batched"]
            res["uneven_all"] = uneven_all_measure(b["mode"], b["streams"], tile_rows=b["forward_tile_rows"])
        res["learned"] = learned_measure()
        res["learned"]["fwi"] = learned_fwi_measure()
    # a compact summary of the extra measurements, placed right after the contract keys so that it
    # survives a capture that keeps only the head of this long line
    summ = {}
    if "elastic" in res:
        e = res["elastic"]
        summ["elastic"] = {"gradient": round(e["value"], 2), "forward": round(e["forward"]["value"], 2),
                           "adj_pair_frac": round(e["kernels"]["adj"]["frac"], 3),
                           "fwd_pair_frac": round(e["kernels"]["fwd"]["frac"], 3)}
    if "acoustic_xl" in res:
        summ["acoustic_xl_frac"] = {k: round(res["acoustic_xl"][k]["frac"], 3) for k in ("fwd", "store", "adj")}
    if "batched_uneven" in res:
        b = res["batched_uneven"]
        summ["batched_uneven"] = {"best": round(b["batched"]["value"], 2), "mode": b["batched"]["mode"],
                                  "persistent": round(b["persistent"]["value"], 2),
                                  "plain_per_shot": round(b["plain_per_shot"]["value"], 2)}
    if "learned" in res:
        lf = res["learned"].get("fwi", {})
        summ["learned"] = {"train_step_ms": round(res["learned"]["ms_per_step"], 2),
                           "bf16_frac": res["learned"]["roofline"]["frac"],
                           "learned_over_mean_final_misfit": lf.get("learned_over_mean_final_misfit"),
                           "learned_reaches_plain_final": lf.get("learned_reaches_plain_final")}
    if "store_all" in res:
        summ["store_all"] = round(res["store_all"]["value"], 2)
    if "laplacian_op" in res:
        summ["laplacian_op"] = {k: round(res["laplacian_op"][k]["value"], 2) for k in ("gradient", "forward")}
    if summ:
        head = list(res.items())
        k = [i for i, (key, _) in enumerate(head) if key == "config"][0] + 1
        res = dict(head[:k] + [("summary", summ)] + head[k:])
    if ws == 1 and not args.no_cpu_baseline:
        import oracle

        # one shot per oracle thread, so that every usable host core runs a shot
        shots = max(1, oracle.num_threads())
        v, sec, cores = cpu_oracle_sample(d, shots, 100, repeats=4)
        res["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "host_cores": dict(zip(("usable", "machine"), host_cores())),
                               "sample": f"4 x ({shots} shots x 100 steps) of the same 265x665 8th-order grid, "
                                         f"FP64 oracle fwd+adjoint, one shot per thread, {sec:.1f} s"}
        # the oracle parallelises over shots only: a one-shot sample runs on one thread
        v1, sec1, _ = cpu_oracle_sample(d, 1, 150)
        res["cpu_baseline"]["single_thread"] = {"value": v1, "unit": UNIT, "cores": 1,
                                                "sample": f"1 shot x 150 steps of the same grid, {sec1:.1f} s"}
        if not args.no_extra:
            vu, secu, cu_ = cpu_uneven_sample()
            res["cpu_baseline"]["uneven_subset"] = {
                "value": vu, "unit": UNIT, "cores": cu_,
                "sample": f"instances 0-3 of the uneven workload (seed 4), 2 shots x 100 steps each, {secu:.1f} s",
                "gpu_batched_value": res["batched_uneven"]["batched"]["value"]}
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
