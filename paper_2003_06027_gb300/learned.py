"""Learned starting model for FWI (the project's learned part; not from the paper).

The paper's Limitations section names the starting model as FWI's weak point:
from a poor start the misfit has local minima (cycle skipping). Here a small
encoder-decoder CNN maps the 16 shot gathers of a survey (64 receivers x 1000
samples) to a 128 x 256 velocity model. It is trained on gathers that the
library's own forward modelling computes from random layered models, and its
prediction is then used as the start of ordinary FWI. Plain smooth-start FWI
stays the fallback and the yardstick: `compare_fwi` runs both from the same data.

Network (activations channel-major [C][B][H][W]; H = time or depth, W = receivers
or x; every conv 3x3, pad 1, ReLU except the last):
  encoder  16 -> 32 (stride 4,1) -> 32 -> 64 (2,2) -> 64 -> 128 (2,1) -> 192 (2,1) -> 256 (2,1) -> 256
           i.e. 1000 x 64 -> 250 x 64 -> 125 x 32 -> 63 x 32 -> 32 x 32 -> 16 x 32
  decoder  3 x (2x nearest upsampling, conv): 256 -> 192 -> 64 -> 32 at 32x64, 64x128, 128x256,
           then conv 32 -> 1 (no ReLU); velocity = 3000 + 1500 * output (m/s).
About 2.0 M parameters (1 969 217). Weights are FP32 with a BF16 copy for the tensor-core
GEMMs (BF16 operands, FP32 accumulation); every layer runs in libfwi's kernels
(include/fwi_cnn.h); torch only holds the device memory.
"""

from __future__ import annotations

import ctypes
import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import fwi

NZ, NX = 128, 256              # model grid (cells), dx = 10 m
NT, DT, F0 = 1000, 1e-3, 8.0
NSHOT, NREC = 16, 64
V_MID, V_HALF = 3000.0, 1500.0  # output scaling: v = V_MID + V_HALF * out

# encoder layers (C_in, C_out, stride_h, stride_w); decoder layers (C_in, C_out), each after a 2x upsampling
ENCODER = [(16, 32, 4, 1), (32, 32, 1, 1), (32, 64, 2, 2), (64, 64, 1, 1), (64, 128, 2, 1), (128, 192, 2, 1),
           (192, 256, 2, 1), (256, 256, 1, 1)]
DECODER = [(256, 192), (192, 64), (64, 32)]


def _lib():
    L = fwi.library()
    if not getattr(L, "_cnn_declared", False):
        P, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
        L.fwi_cnn_create.argtypes = [ctypes.POINTER(P), ctypes.c_int]
        L.fwi_cnn_destroy.argtypes = [P]
        L.fwi_cnn_check.argtypes = [P, P]
        L.fwi_cnn_set_conv_gather.argtypes = [P, i32]
        L.fwi_cnn_gemm_bt.argtypes = [P, P, i64, P, i64, i64, i32, i64, P, i64, P, i32, i32, P]
        L.fwi_cnn_conv_forward.argtypes = [P, P, i32, i32, i32, i32, P, P, i32, i32, i32, i32, P, P]
        L.fwi_cnn_conv_backward.argtypes = [P, P, i32, i32, i32, i32, P, i32, i32, i32, i32, P, P, P, P, P, P]
        L.fwi_cnn_upsample2.argtypes = [P, i32, i32, i32, i32, P, P]
        L.fwi_cnn_upsample2_backward.argtypes = [P, i32, i32, i32, i32, P, P]
        L.fwi_cnn_mse.argtypes = [P, P, P, i64, P, P, P]
        L.fwi_cnn_adam.argtypes = [P, P, P, P, i64, i32, f32, f32, f32, f32, P, P]
        L.fwi_cnn_to_bf16.argtypes = [P, P, i64, P]
        for f in ("fwi_cnn_create", "fwi_cnn_destroy", "fwi_cnn_check", "fwi_cnn_gemm_bt", "fwi_cnn_conv_forward",
                  "fwi_cnn_conv_backward",
                  "fwi_cnn_upsample2", "fwi_cnn_upsample2_backward", "fwi_cnn_mse", "fwi_cnn_adam",
                  "fwi_cnn_to_bf16"):
            getattr(L, f).restype = ctypes.c_int
        L._cnn_declared = True
    return L


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _st():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _chk(st):
    fwi._check(st)


class Handle:
    """The CNN layers' handle on one device (workspace and GEMM status word).
    Its calls must be issued in order on one stream."""

    def __init__(self, device=0):
        self.h = ctypes.c_void_p()
        _chk(_lib().fwi_cnn_create(ctypes.byref(self.h), int(device)))

    def check(self):
        """Wait for the current stream; raise if a GEMM wait timed out."""
        _chk(_lib().fwi_cnn_check(self.h, _st()))

    def set_conv_gather(self, on: bool):
        """Gather the convolution GEMMs' tap operand in the GEMM (default) or
        build the im2col matrix first (fwi_cnn_set_conv_gather)."""
        _chk(_lib().fwi_cnn_set_conv_gather(self.h, int(bool(on))))

    def __del__(self):
        try:
            _lib().fwi_cnn_destroy(self.h)
        except Exception:
            pass


def conv_out(n, s):
    return (n - 1) // s + 1


def to_bf16(x: torch.Tensor) -> torch.Tensor:
    y = torch.empty(x.shape, dtype=torch.int16, device=x.device)
    _chk(_lib().fwi_cnn_to_bf16(_p(x), _p(y), x.numel(), _st()))
    return y


def gemm_bt(h: Handle, A, B, out=None, bias=None, relu=False, splits=1):
    """out[n][m] = act(sum_k A[m][k] B[n][k] + bias[n]) for BF16 (int16-viewed)
    A [M][lda], B [N][ldb] with the contraction over their first K columns,
    K = A.shape[1] = B.shape[1] (fwi_cnn_gemm_bt)."""
    M, K = A.shape
    N = B.shape[0]
    if out is None:
        out = torch.empty((N, M), dtype=torch.float32, device=A.device)
    _chk(_lib().fwi_cnn_gemm_bt(h.h, _p(A), A.stride(0), _p(B), B.stride(0), M, N, K, _p(out), out.stride(0),
                                _p(bias), int(relu), int(splits), _st()))
    return out


def conv_forward(h: Handle, x, w_bf16, bias, sh, sw, relu):
    """x [C][B][H][W] -> y [O][B][Ho][Wo] (fwi_cnn_conv_forward)."""
    C, B, H, W = x.shape
    O = bias.shape[0]
    Ho, Wo = conv_out(H, sh), conv_out(W, sw)
    y = torch.empty((O, B, Ho, Wo), dtype=torch.float32, device=x.device)
    _chk(_lib().fwi_cnn_conv_forward(h.h, _p(x), C, B, H, W, _p(w_bf16), _p(bias), O, sh, sw, int(relu), _p(y),
                                     _st()))
    return y


def conv_backward(h: Handle, x, w_bf16, y, dy, sh, sw, relu, need_dx=True):
    """(dx or None, dw, db); dy is overwritten with the pre-activation gradient."""
    C, B, H, W = x.shape
    O = dy.shape[0]
    dev = x.device
    dx = torch.empty_like(x) if need_dx else None
    dw = torch.empty((O, C, 3, 3), dtype=torch.float32, device=dev)
    db = torch.empty(O, dtype=torch.float32, device=dev)
    _chk(_lib().fwi_cnn_conv_backward(h.h, _p(x), C, B, H, W, _p(w_bf16), O, sh, sw, int(relu), _p(y), _p(dy),
                                      _p(dx), _p(dw), _p(db), _st()))
    return dx, dw, db


def upsample2(x):
    C, B, H, W = x.shape
    y = torch.empty((C, B, 2 * H, 2 * W), dtype=torch.float32, device=x.device)
    _chk(_lib().fwi_cnn_upsample2(_p(x), C, B, H, W, _p(y), _st()))
    return y


def upsample2_backward(dy):
    C, B, H2, W2 = dy.shape
    dx = torch.empty((C, B, H2 // 2, W2 // 2), dtype=torch.float32, device=dy.device)
    _chk(_lib().fwi_cnn_upsample2_backward(_p(dy), C, B, H2 // 2, W2 // 2, _p(dx), _st()))
    return dx


def mse(h: Handle, p, t):
    """(loss as a 1-element FP64 tensor, dL/dp)."""
    loss = torch.empty(1, dtype=torch.float64, device=p.device)
    dp = torch.empty_like(p)
    _chk(_lib().fwi_cnn_mse(h.h, _p(p), _p(t), p.numel(), _p(loss), _p(dp), _st()))
    return loss, dp


class Net:
    """The encoder-decoder, its flat FP32 parameters (with BF16 copy, gradient
    and Adam moments) and the activations of the last forward pass."""

    def __init__(self, device=0, seed=0):
        self.dev = torch.device("cuda", device)
        self.h = Handle(device)
        specs = [dict(C=c, O=o, sh=sh, sw=sw, relu=True, up=False) for c, o, sh, sw in ENCODER]
        specs += [dict(C=c, O=o, sh=1, sw=1, relu=True, up=True) for c, o in DECODER]
        specs.append(dict(C=DECODER[-1][1], O=1, sh=1, sw=1, relu=False, up=False))
        self.layers = specs
        n = sum(L["O"] * L["C"] * 9 + L["O"] for L in specs)
        self.nparams = n
        g = torch.Generator().manual_seed(seed)
        theta = torch.empty(n, dtype=torch.float32)
        off = 0
        for L in specs:
            nw = L["O"] * L["C"] * 9
            theta[off:off + nw] = torch.randn(nw, generator=g) * math.sqrt(2.0 / (9 * L["C"]))  # He
            theta[off + nw:off + nw + L["O"]] = 0.0
            L["off"] = off
            off += nw + L["O"]
        self.theta = theta.to(self.dev)
        self.grad = torch.zeros_like(self.theta)
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.theta_bf16 = to_bf16(self.theta)
        self.t = 0
        self.acts = None

    def _w(self, L, buf):
        nw = L["O"] * L["C"] * 9
        return buf[L["off"]:L["off"] + nw]

    def _b(self, L, buf):
        nw = L["O"] * L["C"] * 9
        return buf[L["off"] + nw:L["off"] + nw + L["O"]]

    def forward(self, x):
        """x [16][B][1000][64] -> normalised model [1][B][128][256]."""
        acts = []
        for L in self.layers:
            xin = upsample2(x) if L["up"] else x
            y = conv_forward(self.h, xin, self._w(L, self.theta_bf16), self._b(L, self.theta), L["sh"], L["sw"],
                             L["relu"])
            acts.append((x, xin, y))
            x = y
        self.acts = acts
        return x

    def backward(self, dout):
        """Parameter gradients into self.grad from dL/d(output)."""
        d = dout
        for k in range(len(self.layers) - 1, -1, -1):
            L = self.layers[k]
            x, xin, y = self.acts[k]
            need_dx = k > 0
            dxin, dw, db = conv_backward(self.h, xin, self._w(L, self.theta_bf16), y, d.contiguous(), L["sh"],
                                         L["sw"], L["relu"], need_dx=need_dx)
            self._w(L, self.grad).copy_(dw.reshape(-1))
            self._b(L, self.grad).copy_(db)
            if need_dx:
                d = upsample2_backward(dxin) if L["up"] else dxin

    def step(self, lr, b1=0.9, b2=0.999, eps=1e-8):
        self.t += 1
        _chk(_lib().fwi_cnn_adam(_p(self.theta), _p(self.grad), _p(self.m), _p(self.v), self.nparams, self.t,
                                 float(lr), float(b1), float(b2), float(eps), _p(self.theta_bf16), _st()))

    def predict(self, x):
        """Velocity models [B][128][256] (m/s) for inputs [16][B][1000][64]."""
        out = self.forward(x)
        return (V_MID + V_HALF * out[0]).clamp(1400.0, 4600.0)


# ---------------------------------------------------------------- data from the solver
def survey_problem(c: np.ndarray) -> dict:
    """The learned part's survey on a 128 x 256 model: dx = 10 m, dt = 1 ms, 1000
    samples, 8th order, 32 CPML cells, 16 Ricker (8 Hz) point sources and 64
    receivers (every 4th cell) at iz = 2."""
    x0 = np.stack([np.linspace(0, NX - 1, NSHOT) * 10.0, np.full(NSHOT, 20.0)], 1).astype(np.float32)
    return dict(nz=NZ, nx=NX, dz=10.0, dx=10.0, dt=DT, nt=NT, order=8, npml=32, pml_R=1e-5, pml_vmax=4500.0,
                pml_f0=F0, src_kind=0, c=np.ascontiguousarray(c, np.float32),
                stf=np.tile(fwi_ricker(), (NSHOT, 1)), x0=x0, rec_iz=np.full(NREC, 2, np.int32),
                rec_ix=(np.arange(NREC) * 4).astype(np.int32), ckpt_every=100)


def fwi_ricker():
    from . import synth

    return synth.ricker(F0, DT, NT)


def random_model(seed: int) -> np.ndarray:
    """3-10 dipping layers, 1500-4500 m/s, no faults (seeded)."""
    from . import synth

    return synth.layered_model(seed, NZ, NX, 10.0, n_layers=(3, 10), n_faults=0)


def gathers_to_input(seis: torch.Tensor) -> torch.Tensor:
    """[S][nrec][nt] seismograms -> one network input [16][1000][64]: time-gained
    (t / T) and scaled by the peak of the gained data."""
    t = torch.arange(1, NT + 1, device=seis.device, dtype=torch.float32) / NT
    g = seis * t
    g = g / g.abs().amax().clamp_min(1e-30)
    return g.permute(0, 2, 1).contiguous()


def make_dataset(n: int, seed: int, device=0, workers: int = 4):
    """(inputs [16][n][1000][64], targets [1][n][128][256] normalised, models [n][128][256]).
    The surveys are modelled by `workers` host threads, each with its own CUDA
    stream and library context (one forward call per sample is launch-bound, so
    concurrent calls keep the GPU busy); sample i depends only on its seed."""
    import threading

    dev = torch.device("cuda", device)
    X = torch.empty((NSHOT, n, NT, NREC), dtype=torch.float32, device=dev)
    Y = torch.empty((1, n, NZ, NX), dtype=torch.float32, device=dev)
    models = np.empty((n, NZ, NX), np.float32)
    d = survey_problem(np.full((NZ, NX), 2000.0, np.float32))
    kw = fwi.problem_kwargs(d)
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev)
    stf, x0, iz, ix = cu(d["stf"]), cu(d["x0"]), cu(d["rec_iz"]), cu(d["rec_ix"])
    torch.cuda.synchronize(dev)
    errors = []

    def work(w):
        try:
            torch.cuda.set_device(dev)
            st = torch.cuda.Stream(dev)
            with torch.cuda.stream(st):
                out = torch.empty((NSHOT, NREC, NT), dtype=torch.float32, device=dev)
                for i in range(w, n, workers):
                    c = random_model(seed * 1000003 + i)
                    models[i] = c
                    ct = cu(c)
                    fwi.forward(ct, stf, x0, iz, ix, out=out, device=device, **kw)
                    X[:, i] = gathers_to_input(out)
                    Y[0, i] = (ct - V_MID) / V_HALF
            st.synchronize()
            fwi.release_context(device)
        except Exception as e:  # re-raised below
            errors.append(e)

    threads = [threading.Thread(target=work, args=(w,)) for w in range(max(1, workers))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    torch.cuda.synchronize(dev)
    return X, Y, models


@dataclass
class TrainLog:
    loss: list = field(default_factory=list)
    seconds: float = 0.0
    samples: int = 0


def train(net: Net, X, Y, epochs=10, batch=32, lr=1e-3, seed=0, log_every=0):
    """Adam on the MSE of the normalised model; returns the per-step loss history."""
    n = X.shape[1]
    rng = np.random.default_rng(seed)
    log = TrainLog()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for ep in range(epochs):
        perm = torch.as_tensor(rng.permutation(n), device=X.device)
        for k in range(0, n - batch + 1, batch):
            idx = perm[k:k + batch]
            xb = X.index_select(1, idx)
            yb = Y.index_select(1, idx)
            out = net.forward(xb)
            loss, dout = mse(net.h, out, yb)
            net.backward(dout)
            net.step(lr * (0.5 ** (ep / max(1, epochs // 3))))
            log.loss.append(loss)
            log.samples += batch
    torch.cuda.synchronize()
    log.seconds = time.perf_counter() - t0
    log.loss = [float(l[0]) for l in log.loss]
    return log


def network_flops_per_sample() -> float:
    """Multiply-add FLOPs of one forward pass (2 per MAC) of the convolutions."""
    H, W, fl = NT, NREC, 0.0
    for c, o, sh, sw in ENCODER:
        H, W = conv_out(H, sh), conv_out(W, sw)
        fl += 2.0 * o * c * 9 * H * W
    for c, o in DECODER:
        H, W = 2 * H, 2 * W
        fl += 2.0 * o * c * 9 * H * W
    fl += 2.0 * 1 * DECODER[-1][1] * 9 * H * W
    return fl


# ---------------------------------------------------------------- FWI from the starts
class _Evaluator:
    """Misfit and gradient of one survey as a recorded graph (fwi.GradGraph):
    each evaluation copies the model into the recorded buffer and replays the
    whole fwi_misfit_grad call, so host launch overhead stays out of the timing."""

    def __init__(self, d: dict, observed: torch.Tensor, c_init: torch.Tensor):
        kw = fwi.problem_kwargs(d)
        dev = c_init.device
        cu = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev)
        self.c = c_init.clone().contiguous()
        self._keep = (cu(d["stf"]), cu(d["x0"]), cu(d["rec_iz"]), cu(d["rec_ix"]), observed.contiguous())
        self.g = fwi.GradGraph(self.c, *self._keep, ckpt_every=d["ckpt_every"], **kw)

    def __call__(self, c: torch.Tensor):
        with torch.no_grad():
            self.c.copy_(c)
        self.g.launch()
        self.g.check()
        return float(self.g.misfit[0]), self.g.grad.clone()

    def close(self):
        self.g.close()


def fwi_run(ev: _Evaluator, c0: torch.Tensor, c_true: torch.Tensor, iters: int = 50, step0: float = 40.0,
            vmin: float = 1400.0, vmax: float = 4600.0):
    """FWI from c0 with the project's L-BFGS (optim.lbfgs: memory 5, box bounds,
    first step at most `step0` m/s per cell), every evaluation one replay of the
    recorded gradient. Returns [(misfit, relative model error, GPU seconds so
    far)] per accepted iterate, the first entry being the start. The seconds
    are wall time of the evaluations (each ends with a device synchronisation),
    so they are the GPU time the run took."""
    from . import optim

    nrm = float(torch.linalg.vector_norm(c_true))
    clock = [0.0]
    evals = []  # (misfit, model error, GPU seconds so far) of every evaluation

    def tracked(c):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J, g = ev(c)
        clock[0] += time.perf_counter() - t0
        evals.append((J, float(torch.linalg.vector_norm(c - c_true)) / nrm, clock[0]))
        return J, g

    _, log = optim.lbfgs(tracked, c0, iters, m=5, step0=step0, lower=vmin, upper=vmax)
    # log.evals[k]: evaluations made when iterate k was accepted
    return [evals[ne - 1] for ne in log.evals]


def compare_fwi(net: Net, n_models: int = 8, seed: int = 777, iters: int = 50, sigma: float = 10.0, device=0,
                mean_model=None):
    """For held-out random models: FWI (L-BFGS) from the Gaussian-smoothed true
    model (sigma cells, the plain start), from the network's prediction, and (if
    given) from `mean_model`, the start available without any survey
    information (the mean of the training models). Returns the per-model
    histories and a summary: mean start / final misfit and model error of each
    start, and the GPU time each start needs to reach the plain start's final
    misfit (None where it does not within `iters` iterations)."""
    from . import synth

    dev = torch.device("cuda", device)
    runs = []
    for i in range(n_models):
        c_np = random_model(seed * 1000003 + i)
        d = survey_problem(c_np)
        kw = fwi.problem_kwargs(d)
        cu = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev)
        c_true = cu(c_np)
        obs = fwi.forward(c_true, cu(d["stf"]), cu(d["x0"]), cu(d["rec_iz"]), cu(d["rec_ix"]), **kw)
        plain0 = cu(synth.smooth(c_np, sigma))
        learned0 = net.predict(gathers_to_input(obs).unsqueeze(1))[0].contiguous()
        ev = _Evaluator(d, obs, plain0)
        hp = fwi_run(ev, plain0, c_true, iters)
        hl = fwi_run(ev, learned0, c_true, iters)
        hm = fwi_run(ev, mean_model.clone(), c_true, iters) if mean_model is not None else None
        ev.close()
        target = hp[-1][0]
        reach = lambda h: next((e[2] for e in h if e[0] <= target), None)
        runs.append(dict(plain=hp, learned=hl, mean=hm, learned_time_to_plain_final=reach(hl),
                         mean_time_to_plain_final=reach(hm) if hm is not None else None, plain_time=hp[-1][2]))
    mean = lambda xs: float(np.mean(xs))
    reached = [r for r in runs if r["learned_time_to_plain_final"] is not None]
    summary = dict(
        models=n_models, iters=iters, smooth_sigma_cells=sigma, optimiser="L-BFGS (optim.lbfgs, m=5)",
        plain_start_model_error=mean([r["plain"][0][1] for r in runs]),
        learned_start_model_error=mean([r["learned"][0][1] for r in runs]),
        plain_final_misfit=mean([r["plain"][-1][0] for r in runs]),
        learned_final_misfit=mean([r["learned"][-1][0] for r in runs]),
        plain_final_model_error=mean([r["plain"][-1][1] for r in runs]),
        learned_final_model_error=mean([r["learned"][-1][1] for r in runs]),
        plain_start_misfit=mean([r["plain"][0][0] for r in runs]),
        learned_start_misfit=mean([r["learned"][0][0] for r in runs]),
        plain_fwi_seconds=mean([r["plain_time"] for r in runs]),
        learned_reaches_plain_final=len(reached),
        learned_seconds_to_plain_final=[r["learned_time_to_plain_final"] for r in runs],
        learned_faster_than_plain=sum(r["learned_time_to_plain_final"] < r["plain_time"] for r in reached),
        learned_over_plain_time_where_reached=(mean([r["learned_time_to_plain_final"] / r["plain_time"]
                                                     for r in reached]) if reached else None),
    )
    if mean_model is not None:
        summary.update(mean_start_model_error=mean([r["mean"][0][1] for r in runs]),
                       mean_start_misfit=mean([r["mean"][0][0] for r in runs]),
                       mean_final_misfit=mean([r["mean"][-1][0] for r in runs]),
                       mean_final_model_error=mean([r["mean"][-1][1] for r in runs]),
                       mean_reaches_plain_final=sum(r["mean_time_to_plain_final"] is not None for r in runs),
                       learned_over_mean_final_misfit=mean([r["learned"][-1][0] / r["mean"][-1][0] for r in runs]))
    return runs, summary


def experiment(n_train=20000, epochs=12, batch=32, n_test=64, iters=50, device=0, seed=5):
    """The whole learned-start experiment: data generation, training, FWI
    comparison. Returns a JSON-able report."""
    torch.cuda.set_device(device)
    t0 = time.perf_counter()
    X, Y, _ = make_dataset(n_train, seed, device)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = Net(device, seed)
    log = train(net, X, Y, epochs=epochs, batch=batch)
    fl = 3.0 * network_flops_per_sample() * log.samples
    mean_model = (V_MID + V_HALF * Y[0].mean(dim=0)).contiguous()
    del X, Y
    _, summary = compare_fwi(net, n_models=n_test, seed=seed + 1000, iters=iters, device=device,
                             mean_model=mean_model)
    return dict(train_samples=n_train, epochs=epochs, params=net.nparams, data_seconds=t_data,
                train_seconds=log.seconds, train_tflops=fl / log.seconds / 1e12,
                loss_first=float(np.mean(log.loss[:20])), loss_last=float(np.mean(log.loss[-20:])), **summary)


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--test", type=int, default=64)
    ap.add_argument("--iters", type=int, default=50)
    a = ap.parse_args()
    print(json.dumps(experiment(a.train, a.epochs, n_test=a.test, iters=a.iters), indent=1))
