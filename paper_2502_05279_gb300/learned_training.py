"""Train and evaluate the learned-interpolation network on the GPU.

Every step runs in the library's kernels (bmg_mlp_loss_grad, bmg_mlp_adam,
bmg_relax); this module only prepares inputs and loops.

Training family: 255 x 255 interior grids, 9-point Q1 stencils of
-div(k grad u), k in {1, 1e6} on 8 x 8 cell blocks (Bernoulli 0.5), one seed
per problem.  Test vectors: uniform[-1,1) vectors after 10 Gauss-Seidel
sweeps of A v = 0 (the loss is invariant to their scale).  Checkpoints are
.npz files holding the parameter vector, the step count and the loss history.

    python -m paper_2502_05279_gb300.learned_training --problems 2000 --epochs 2 --out model.npz
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np
import torch

from . import _lib as B

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
import workloads as w  # noqa: E402

N_VEC = 4
SWEEPS = 10


def init_params(seed: int) -> np.ndarray:
    """He-scaled W1, W2 from SplitMix64 normals; biases and W3 zero, so the
    untrained network gives Dendy's weights."""
    nin, nh, no = 18, 64, 4
    z = w.normal(seed, nin * nh + nh * nh)
    p = np.zeros(B.MLP_PARAMS, dtype=np.float64)
    p[:nin * nh] = z[:nin * nh] * np.sqrt(2.0 / nin)
    o = nin * nh + nh
    p[o:o + nh * nh] = z[nin * nh:] * np.sqrt(2.0 / nh)
    return p.astype(np.float32)


def make_problem(n: int, seed: int, device="cuda"):
    """(coef (5, n+2, n+2), test vectors (K, n+2, n+2)) on the device."""
    planes = w.fe9_from_cells(w.binary_blocks(n, 8, 1.0, 1e6, seed))
    coef = torch.from_numpy(planes).to(device)
    zero = torch.zeros((n + 2, n + 2), dtype=torch.float64, device=device)
    vecs = []
    for k in range(N_VEC):
        v = torch.from_numpy(w.rhs_uniform(n, 50_000_000 + seed * N_VEC + k)).to(device)
        B.relax(9, coef, zero, v, SWEEPS)
        vecs.append(v)
    return coef, torch.stack(vecs)


def train(n_problems: int = 2000, epochs: int = 2, n: int = 255, lr: float = 1e-3, seed: int = 2024,
          first_seed: int = 1000, log=print):
    mlp = B.Mlp(init_params(seed))
    data = []
    t0 = time.perf_counter()
    for s in range(first_seed, first_seed + n_problems):
        coef, vecs = make_problem(n, s)
        _, _, eref = mlp.loss_grad(coef, vecs, want_grad=False)
        data.append((coef, vecs, eref))
    log(f"prepared {n_problems} problems in {time.perf_counter() - t0:.1f} s")
    history = []
    for ep in range(epochs):
        t0 = time.perf_counter()
        losses = []
        for coef, vecs, eref in data:
            L, _, _ = mlp.loss_grad(coef, vecs, eref, want_grad=False)
            losses.append(L)
            mlp.adam(lr)
        history.append(float(np.mean(losses)))
        log(f"epoch {ep}: mean loss {history[-1]:.6f} ({time.perf_counter() - t0:.1f} s)")
    return mlp, history


def evaluate(mlp, n: int = 4095, seed: int = 6, tol: float = 1e-10):
    """Dendy vs learned on one problem of the family: measured V(2,1) factors
    (from bmg_setup's fallback test), setup time and FCG time to tol."""
    kind, planes, f = w.high_contrast_problem(n, seed=seed)
    coef = torch.from_numpy(planes).cuda()
    rhs = torch.from_numpy(f).cuda()
    out = {}
    for name, net in (("dendy", None), ("learned", mlp)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = B.Hierarchy(kind, coef, krylov="fcg", mlp=net)
        torch.cuda.synchronize()
        setup = time.perf_counter() - t0
        x = torch.zeros_like(rhs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, it, rr, ok = h.solve(rhs, x, tol=tol, maxit=1000)
        torch.cuda.synchronize()
        rec = {"setup_s": setup, "solve_s": time.perf_counter() - t0, "iterations": it, "relres": rr,
               "converged": ok}
        if net is not None:
            used, fl, fd = h.interp_info()
            rec.update({"kept": used, "factor_learned": fl, "factor_dendy": fd})
        out[name] = rec
        h.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--problems", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=2)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--eval-n", type=int, default=4095)
    ap.add_argument("--out", default="learned_model.npz")
    args = ap.parse_args()
    mlp, hist = train(args.problems, args.epochs, lr=args.lr)
    np.savez(args.out, params=mlp.params(), loss_history=np.array(hist), problems=args.problems, epochs=args.epochs)
    print(json.dumps({"train_loss": hist, "eval": evaluate(mlp, args.eval_n)}))


if __name__ == "__main__":
    main()
