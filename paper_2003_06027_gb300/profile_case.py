"""Small cases of the acoustic gradient for Nsight Compute captures.

    python -m paper_2003_06027_gb300.profile_case --case fwi48-nt20

Each case keeps the benchmark's grid and discretisation (201 x 601 + 32 CPML
cells, 8th order) but few time steps, so a `--set full` capture of a handful of
step-kernel launches ends quickly while each launch still touches more data
than the 129 MB L2 (48 shots: ~40 MB per field).
"""

from __future__ import annotations

import argparse

import numpy as np

CASES = {
    # shots, time steps, checkpoint interval
    "fwi48-nt20": (48, 20, 10),
    "fwi16-nt20": (16, 20, 10),
    # the HBM-bound regime: 128 shots, one step's fields (~0.45 GB) far exceed L2 (~3.7 GB arena)
    "fwi128-nt8": (128, 8, 4),
    # the same with the c^2 Laplacian operator
    "lap16-nt20": (16, 20, 10),
    # elastic 300 x 800 discretisation (4th order, 32 CPML cells), 8 shots
    "ela8-nt20": (8, 20, 10),
    # start-model network: training steps on a batch of 32 surveys (shots = batch, steps = Adam steps)
    "cnn32-step4": (32, 4, 0),
}


def main():
    import torch

    from paper_2003_06027_gb300 import fwi, synth

    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="fwi48-nt20", choices=sorted(CASES))
    ap.add_argument("--repeat", type=int, default=2)
    args = ap.parse_args()
    S, nt, K = CASES[args.case]
    if args.case.startswith("cnn"):
        from paper_2003_06027_gb300 import learned as L

        g = torch.Generator(device="cuda").manual_seed(0)
        X = torch.randn((L.NSHOT, S, L.NT, L.NREC), device="cuda", generator=g) * 0.1
        Y = torch.randn((1, S, L.NZ, L.NX), device="cuda", generator=g) * 0.1
        net = L.Net(0, seed=0)
        for _ in range(nt):
            out = net.forward(X)
            loss, dout = L.mse(net.h, out, Y)
            net.backward(dout)
            net.step(1e-4)
        net.h.check()
        print(f"case {args.case}: loss {float(loss[0]):.6e}")
        return
    if args.case.startswith("ela"):
        d = synth.elastic_layered(nshots=S, nt=nt)
        kw = fwi.problem_kwargs(d)
        cu = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
        ea = [cu(d[k]) for k in ("vp", "vs", "rho", "stf", "x0", "mt", "rec_iz", "rec_ix")]
        obs = fwi.forward_elastic(*ea, **kw)
        for _ in range(args.repeat):
            J, g, _, _, _ = fwi.misfit_grad_elastic(*ea, obs, ckpt_every=K, **kw)
        torch.cuda.synchronize()
        t = fwi.last_timing()
        print(f"case {args.case}: J = {float(J[0]):.6e}, fwd {t.fwd_step_ms * 1e3:.1f} us, "
              f"store {t.store_step_ms * 1e3:.1f} us, adj {t.adj_step_ms * 1e3:.1f} us per step")
        return
    d = synth.acoustic_fwi(nshots=S, nt=nt)
    if args.case.startswith("lap"):
        d["op"] = fwi.FWI_OP_LAPLACIAN
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    kw = fwi.problem_kwargs(d)
    c, stf, x0, iz, ix = cu(d["c"]), cu(d["stf"]), cu(d["x0"]), cu(d["rec_iz"]), cu(d["rec_ix"])
    obs = fwi.forward(cu(d["c_true"]), stf, x0, iz, ix, **kw)
    for _ in range(args.repeat):
        J, g, _, _, _ = fwi.misfit_grad(c, stf, x0, iz, ix, obs, ckpt_every=K, **kw)
    torch.cuda.synchronize()
    t = fwi.last_timing()
    print(f"case {args.case}: J = {float(J[0]):.6e}, |grad| = {float(g.norm()):.6e}, "
          f"fwd {t.fwd_step_ms * 1e3:.1f} us, store {t.store_step_ms * 1e3:.1f} us, adj {t.adj_step_ms * 1e3:.1f} us "
          f"per launch, {t.launches} launches")


if __name__ == "__main__":
    main()
