"""Train and evaluate the learned-interpolation network on the GPU.

Every step runs in the library's kernels (bmg_mlp_twogrid, bmg_mlp_adam,
bmg_setup); this module only prepares inputs and loops.

Training family: 255 x 255 interior grids, 9-point Q1 stencils of
-div(k grad u), k in {1, 1e6} on 8 x 8 cell tiles (Bernoulli 0.5), one seed
per problem.  The loss is the two-grid one: on 31 x 31 Dirichlet crops of the
problems (tile-aligned offsets), the A-energy of the two-grid error
propagation of V(2,1) applied to uniform[-1,1) error vectors, relative to
Dendy's weights (loss 1 = Dendy).  Checkpoints are .npz files holding the
parameter vector, the Adam moments and step count, the epochs run and the loss
history; --resume continues from one (the next epoch draws the permutation it
would have drawn in an uninterrupted run).

    python -m paper_2502_05279_gb300.learned_training --problems 2000 --epochs 8 --out model.npz
    python -m paper_2502_05279_gb300.learned_training --resume model.npz --epochs 4 --out model2.npz
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


def crops_on_device(n_problems: int, crops_per_problem: int = 1, first_seed: int = 1000, vectors: int = N_VEC):
    """(coefs (C, 5, 33, 33), vecs (C, K, 33, 33)) CUDA float64 tensors of the
    training crops (workloads.training_crops)."""
    crops = w.training_crops(n_problems, first_seed=first_seed, crops_per_problem=crops_per_problem,
                             vectors=vectors)
    coefs = torch.from_numpy(np.stack([c[0] for c in crops])).cuda()
    vecs = torch.from_numpy(np.stack([c[1] for c in crops])).cuda()
    return coefs, vecs


def save_checkpoint(path: str, mlp, history, epochs_done: int, problems: int) -> None:
    """Parameters, Adam moments and step, epochs run and loss history."""
    m1, m2, step = mlp.adam_state()
    np.savez(path, params=mlp.params(), adam_m=m1, adam_v=m2, adam_step=step, epochs_done=epochs_done,
             loss_history=np.asarray(history, dtype=np.float64), problems=problems)


def load_checkpoint(path: str):
    """(network with its parameters and Adam state restored, loss history,
    epochs run)."""
    z = np.load(path)
    mlp = B.Mlp(z["params"])
    mlp.set_adam_state(z["adam_m"], z["adam_v"], int(z["adam_step"]))
    return mlp, list(z["loss_history"]), int(z["epochs_done"])


def train(n_problems: int = 2000, epochs: int = 8, batch: int = 152, lr: float = 2e-2, seed: int = 2024,
          first_seed: int = 1000, crops_per_problem: int = 1, log=print, mlp=None, first_epoch: int = 0):
    """Adam on the two-grid loss over mini-batches of crops (a SplitMix64
    permutation per epoch, epoch e drawing stream seed + 1 + e).  mlp: a
    network to continue training (from load_checkpoint) and first_epoch its
    epochs run; else a fresh network.  Returns (network, mean loss per epoch,
    Dendy's energies, seconds spent in training steps)."""
    if mlp is None:
        mlp = B.Mlp(init_params(seed))
    t0 = time.perf_counter()
    coefs, vecs = crops_on_device(n_problems, crops_per_problem, first_seed)
    _, _, eref = mlp.twogrid(coefs, vecs)
    torch.cuda.synchronize()
    log(f"prepared {coefs.shape[0]} crops in {time.perf_counter() - t0:.1f} s")
    C = coefs.shape[0]
    history = []
    train_s = 0.0
    for ep in range(first_epoch, first_epoch + epochs):
        order = torch.from_numpy(np.argsort(w.uniform01(seed + 1 + ep, C), kind="stable")).cuda()
        t0 = time.perf_counter()
        losses = []
        for b0 in range(0, C, batch):
            idx = order[b0:b0 + batch]
            L, _, _ = mlp.twogrid(coefs[idx].contiguous(), vecs[idx].contiguous(), eref[idx].contiguous(),
                                  want_grad=False)
            losses.append(L)
            mlp.adam(lr)
        torch.cuda.synchronize()
        train_s += time.perf_counter() - t0
        history.append(float(np.mean(losses)))
        log(f"epoch {ep}: mean two-grid loss {history[-1]:.6f} ({time.perf_counter() - t0:.2f} s)")
    return mlp, history, eref, train_s


def evaluate(mlp, n: int = 4095, seed: int = 6, tol: float = 1e-10, maxit: int = 300):
    """Dendy vs learned on one problem of the family: the measured V(2,1)
    factors (bmg_setup's fallback test, iterations 5 .. 15), which
    interpolation the setup kept, setup time, and flexible-CG time to tol
    (or the relative residual reached at maxit)."""
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
        h.solve(rhs, x, tol=tol, maxit=2)                 # graph capture, untimed
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, it, rr, ok = h.solve(rhs, x, tol=tol, maxit=maxit)
        torch.cuda.synchronize()
        rec = {"setup_s": round(setup, 4), "solve_s": round(time.perf_counter() - t0, 4), "iterations": it,
               "relres": rr, "converged": ok}
        if net is not None:
            used, fl, fd = h.interp_info()
            rec.update({"kept": used, "factor_learned": fl, "factor_dendy": fd})
        out[name] = rec
        h.close()
    lr_ = out["learned"]
    lr_["gain"] = ("learned weights kept: measured factor %.4f vs Dendy %.4f" % (lr_["factor_learned"],
                                                                              lr_["factor_dendy"])
                   if lr_["kept"] == "learned" and lr_["factor_learned"] < lr_["factor_dendy"]
                   else "no gain: Dendy kept (measured factor learned %.6f, Dendy %.6f)"
                   % (lr_["factor_learned"], lr_["factor_dendy"]))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--problems", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--batch", type=int, default=152)
    ap.add_argument("--lr", type=float, default=2e-2)
    ap.add_argument("--eval-n", type=int, default=4095)
    ap.add_argument("--out", default="learned_model.npz")
    ap.add_argument("--resume", default=None, help="checkpoint to continue from")
    args = ap.parse_args()
    mlp, past, done = (None, [], 0) if args.resume is None else load_checkpoint(args.resume)
    mlp, hist, _, train_s = train(args.problems, args.epochs, args.batch, args.lr, mlp=mlp, first_epoch=done)
    save_checkpoint(args.out, mlp, past + hist, done + args.epochs, args.problems)
    print(json.dumps({"train_loss": past + hist, "train_s": train_s, "eval": evaluate(mlp, args.eval_n)}))


if __name__ == "__main__":
    main()
