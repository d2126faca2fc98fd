"""Train the learned initial guess of the 2D Sternheimer solves on this library's own solutions.

Usage: python -m paper_1605_08021_gb300.train_cnn [--systems 200] [--held-out 8] [--samples 32]
           [--epochs 30] [--lr 1e-3] [--stern-tol 1e-8] [--out cnn_weights.npy] [--workers 8]

Training set: the seeded lattices of ``acp_workloads.training_lattices`` (closed-shell 2D
lattices of 3 x 3 to 5 x 5 sites at grid spacing ~0.5 bohr).  Their ground states are built on
the host (in spawned worker processes, before this process touches the GPU).  For each system
the library computes the perturbations g_k; a sample is one right-hand side of Alg. 1,
b = Q (psi_i g_k) for a random orbital i and perturbation k, with shift eps_i, solved by the
library's mixed-precision MINRES to stern_tol.  The samples (b, V_eff - eps_i, x*) stay on the
GPU.  One context holds the weights and the Adam state; each step trains on the batch of one
system (``acp_cnn_train_step``), systems in a seeded random order per epoch.

Evaluation: on the held-out systems, fresh right-hand sides are solved from zero and from the
learned start (``learned = 1``); the Lanczos steps of both are reported.  The weights are saved
as FP32 in the packed order of ``acp_cnn_set_weights``, with a JSON file of the run beside them.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import time

import numpy as np


def _ground_state(sysm):
    import acp_workloads as W
    # a converged potential cached for the system (ACP_GS_CACHE) costs one eigensolve
    return W.ground_state(sysm, tol=1e-8)


def _context(P, sysm, gs, **opts):
    import torch
    V = torch.tensor(gs.V, dtype=torch.float64, device="cuda")
    psi = torch.tensor(np.ascontiguousarray(gs.psi.T), dtype=torch.float64, device="cuda")
    o = P.options(occ=float(sysm.occ), precision=P.ACP_PREC_MIXED, **opts)
    return P.Context(sysm.n, sysm.L, sysm.kappa, sysm.scale, V, psi, gs.eps[: gs.n_orb], o)


def _samples(P, sysm, gs, n, rng, stern_tol):
    """n right-hand sides of Alg. 1 and their solutions on the GPU: tensors R, VS, X (n, N), the
    shifts, and the stats of the solve (from zero)."""
    import torch
    ctx = _context(P, sysm, gs, stern_tol=stern_tol)
    G, _, _ = ctx.perturbations(sysm.R, sysm.Z, sysm.sigma)
    psi = torch.tensor(np.ascontiguousarray(gs.psi.T), dtype=torch.float64, device="cuda")
    i = rng.integers(0, gs.n_orb, n)
    k = rng.integers(0, G.shape[0], n)
    b = psi[torch.as_tensor(i, device="cuda")] * G[torch.as_tensor(k, device="cuda")]
    R = ctx.project(b.contiguous())
    shifts = gs.eps[i]
    X, st = ctx.sternheimer_solve(R, shifts)
    V = torch.tensor(gs.V, dtype=torch.float64, device="cuda")
    VS = (V[None, :] - torch.tensor(shifts, dtype=torch.float64, device="cuda")[:, None]).contiguous()
    return R, VS, X, shifts, st


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--systems", type=int, default=200)
    ap.add_argument("--held-out", type=int, default=8)
    ap.add_argument("--samples", type=int, default=32, help="right-hand sides per system")
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--stern-tol", type=float, default=1e-8)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) // 2))
    ap.add_argument("--out", default="cnn_weights.npy")
    args = ap.parse_args(argv)

    import acp_workloads as W
    systems = W.training_lattices(args.systems + args.held_out)
    t0 = time.perf_counter()
    os.environ.setdefault("OMP_NUM_THREADS", "2")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "2")
    with mp.get_context("spawn").Pool(args.workers) as pool:
        gss = pool.map(_ground_state, systems)
    t_gs = time.perf_counter() - t0
    print(f"ground states: {len(systems)} systems in {t_gs:.0f} s", flush=True)

    import torch

    import paper_1605_08021_gb300 as P
    rng = np.random.default_rng(args.seed)
    train = list(zip(systems[: args.systems], gss[: args.systems]))
    held = list(zip(systems[args.systems:], gss[args.systems:]))
    t1 = time.perf_counter()
    data = [(s, _samples(P, s, gs, args.samples, rng, args.stern_tol)[:3]) for s, gs in train]
    torch.cuda.synchronize()
    print(f"training samples: {len(data) * args.samples} solves in {time.perf_counter() - t1:.0f} s", flush=True)

    s0, gs0 = train[0]
    trainer = _context(P, s0, gs0)
    w = W.learned.init_weights(args.seed)
    trainer.cnn_set_weights(w)
    history = []
    for epoch in range(args.epochs):
        order = rng.permutation(len(data))
        losses = [trainer.cnn_train_step(data[j][0].n, *data[j][1], lr=args.lr) for j in order]
        history.append(float(np.mean(losses)))
        print(f"epoch {epoch:3d} mean loss {history[-1]:.4e}", flush=True)
    w = trainer.cnn_get_weights()
    torch.cuda.synchronize()

    report = []
    for s, gs in held:
        R, _, _, shifts, st0 = _samples(P, s, gs, args.samples, rng, args.stern_tol)  # from zero
        ctx = _context(P, s, gs, stern_tol=args.stern_tol, learned=1)
        ctx.cnn_set_weights(w)
        _, st1 = ctx.sternheimer_solve(R, shifts)
        report.append({"system": s.name, "grid": list(s.n), "steps_zero_start": st0["lanczos_steps"],
                       "steps_learned_start": st1["lanczos_steps"]})
        print(report[-1], flush=True)
    np.save(args.out, w)
    meta = {"systems": args.systems, "held_out": args.held_out, "samples_per_system": args.samples,
            "epochs": args.epochs, "lr": args.lr, "stern_tol": args.stern_tol, "seed": args.seed,
            "loss_history": history, "held_out_report": report, "ground_state_seconds": t_gs}
    with open(os.path.splitext(args.out)[0] + ".json", "w") as f:
        json.dump(meta, f, indent=1)


if __name__ == "__main__":
    main()
