"""Data, training and evaluation of the learned initial guess, driven through the C ABI.

Every arithmetic step runs in the library's kernels (operator assembly, SpMM, the Jacobi and
multigrid CG solves, the network's forward/backward/Adam, the residual-judged guess selection,
the Galerkin combination of candidates);
this module only sequences the calls and moves tensors between layouts ([n, k] interleaved
blocks for the solver, contiguous [n] vectors for the network).

The pressure sequences solve A p_t = b_t with A = -L (the negated FVM Laplacian of the grid,
symmetric positive semi-definite, constants in its null space) and b_t = -M u_t for smooth
random face velocities u_t, so that u_t - G p_t is the divergence-free projection of u_t
(the pressure Poisson step of the paper's projection method, Sec. 3).
"""
from __future__ import annotations

import time

import numpy as np

from . import (Guess, Multigrid, Operator, cg_params, cg_solve, cg_workspace_bytes, fvm_assemble, galerkin_guess,
               grid_nodes, guess_cfg, lib, mg_params)
from . import RB_FVM_DIVERGENCE, RB_FVM_LAPLACIAN


def make_problem(torch, grid, k, dev="cuda"):
    """A = -L in FP64 (CSR) and FP32 (matrix-free: the refinement's inner operator), the
    divergence M (FP64) and the multigrid hierarchy of A of a structured grid, for k columns."""
    nodes, per = grid_nodes(grid, dev)
    rp, ci, va, nc = fvm_assemble(nodes, per, RB_FVM_LAPLACIAN, scale=-1.0)
    A64 = Operator(rp, ci, va, nc, dtype="f64", k_max=k)
    A32 = Operator.stencil(nodes, per, scale=-1.0, dtype="f32", k_max=k)
    rp, ci, va, nc = fvm_assemble(nodes, per, RB_FVM_DIVERGENCE)
    M = Operator(rp, ci, va, nc, dtype="f64", k_max=k)
    mg = Multigrid(nodes, per, k_max=k)
    return {"grid": grid, "A64": A64, "A32": A32, "M": M, "mg": mg, "n": A64.n_rows, "k": k, "per": per}


def solve(torch, prob, B, X, mixed=2, rtol=1e-10, work=None):
    """A X = B from the guess in X (overwritten), true relative residual rtol, zero-mean projection."""
    prm = cg_params(rtol=rtol, mixed=mixed, project_mean=True, check_every=50)
    k = B.shape[1]
    if work is None:
        work = torch.empty(cg_workspace_bytes(prob["A64"], k, prm), dtype=torch.uint8, device=B.device)
    return cg_solve(prob["A64"], B, X, A_inner=prob["A32"] if mixed else None, params=prm, work=work)


def generate(torch, prob, spectra, face_fields, dev="cuda"):
    """Pressure sequences: for each step t the k = chains right-hand sides b_t = -M u_t and the
    solutions p_t, solved together (k columns) from the previous step's pressures.
    Returns (Bs, Ps) as [steps, chains, n] FP64 tensors and solver statistics."""
    steps, chains = spectra.shape[0], spectra.shape[1]
    n = prob["n"]
    g = prob["grid"]
    Bs = torch.empty((steps, chains, n), dtype=torch.float64, device=dev)
    Ps = torch.empty((steps, chains, n), dtype=torch.float64, device=dev)
    B = torch.empty((n, chains), dtype=torch.float64, device=dev)
    X = torch.zeros((n, chains), dtype=torch.float64, device=dev)
    prm = mg_params(rtol=1e-10, mixed=True)
    iters = []
    neg = torch.full((chains,), -1.0, dtype=torch.float64, device=dev)  # b = -M u through the SpMM's scale
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for t in range(steps):
        U = face_fields(spectra[t], g.shape, torch, dev)
        prob["M"].spmm(U, B, c=neg)
        r = prob["mg"].solve(B, X, prm)
        iters.append(max(r.iters))
        Bs[t].copy_(B.t())
        Ps[t].copy_(X.t())
    torch.cuda.synchronize()
    return Bs, Ps, {"steps": steps, "chains": chains, "seconds": time.perf_counter() - t0,
                    "median_iters": float(np.median(iters))}


def pairs(steps, chains, holdout):
    """(step, chain) of the training pairs (t >= 2, before the held-out tail) and of the test pairs."""
    train = [(t, c) for t in range(2, steps - holdout) for c in range(chains)]
    test = [(t, c) for t in range(steps - holdout, steps) for c in range(chains)]
    return train, test


def train(torch, net: Guess, Bs, Ps, train_pairs, epochs, batch=4, lr=1e-3, seed=0, lr_final=None):
    """Adam on the mean-squared error of the guess over shuffled minibatches of pairs; the
    learning rate decays geometrically from lr to lr_final over the run.  Returns the
    per-epoch mean loss and the wall time."""
    rng = np.random.default_rng(seed)
    acc = torch.zeros(1, dtype=torch.float64, device=Bs.device)
    history = []
    total = epochs * (len(train_pairs) // batch)
    lr_final = lr if lr_final is None else lr_final
    step = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(epochs):
        order = rng.permutation(len(train_pairs))
        acc.zero_()
        nb = len(order) // batch
        for bi in range(nb):
            for j in range(batch):
                t, c = train_pairs[order[bi * batch + j]]
                net.loss_grad(Bs[t, c], Ps[t - 1, c], Ps[t - 2, c], Ps[t, c], accumulate=j > 0, loss=acc)
            rate = lr * (lr_final / lr) ** (step / max(1, total - 1))
            net.adam_step(lr=rate, grad_scale=1.0 / batch)
            step += 1
        history.append(acc.item() / (nb * batch))
    torch.cuda.synchronize()
    return {"epochs": epochs, "batch": batch, "pairs": len(train_pairs), "seconds": time.perf_counter() - t0,
            "loss_per_epoch": history}


def evaluate(torch, prob, net: Guess, Bs, Ps, test_steps, chains, sweeps=10, omega=2.0 / 3.0):
    """For each held-out step, all chains solved together (k = chains) to 1e-10 from each of
    these initial guesses, the guess's own cost (inference, judging, combination) timed in:
      zero, prev          0 and p_{t-1};
      learned_judged      the network's guess or p_{t-1}, whichever has the smaller residual after
                          `sweeps` damped Jacobi sweeps of both (rb_guess_select);
      galerkin_prev       the A-norm-optimal combination of p_{t-1} and p_{t-2}
                          (rb_galerkin_guess);
      galerkin_learned    the same over p_{t-1}, p_{t-2} and the network's guess;
    with the Jacobi-PCG FP64 CG (zero, prev only), the Jacobi FP32-inner refinement (suffix _ir)
    and the multigrid CG with the FP32 cycle inside FP64 refinement (suffix _mg).  Returns the
    iterations (max over the chains of a step) and milliseconds per step (median, p90), and the
    guesses' accuracy against the stored solution: relative L2 error and energy-norm error."""
    n = prob["n"]
    dev = Bs.device
    A = prob["A64"]
    f64 = dict(dtype=torch.float64, device=dev)
    B = torch.empty((n, chains), **f64)
    X = torch.empty((n, chains), **f64)
    G = torch.empty((chains, n), **f64)
    cand = torch.empty((chains, n), **f64)
    P1, P2, NN = (torch.empty((n, chains), **f64) for _ in range(3))
    gwork = torch.empty(lib().rb_galerkin_workspace_bytes(n, chains, 3), dtype=torch.uint8, device=dev)
    prm = {m: cg_params(rtol=1e-10, mixed=m, project_mean=True, check_every=50) for m in (0, 2)}
    works = {m: torch.empty(cg_workspace_bytes(A, chains, prm[m]), dtype=torch.uint8, device=dev) for m in (0, 2)}
    mgp = mg_params(rtol=1e-10, mixed=True)
    names = ["zero_fp64", "prev_fp64", "prev_ir", "learned_judged_ir", "galerkin_prev_ir", "galerkin_learned_ir",
             "prev_mg", "learned_judged_mg", "galerkin_prev_mg", "galerkin_learned_mg"]
    out = {k: {"iters": [], "ms": []} for k in names}
    picks, res_prev, res_sel, err_prev, err_nn, err_gal, infer_ms = [], [], [], [], [], [], []
    for t in test_steps:
        B.copy_(Bs[t].t())
        for name in names:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if name == "zero_fp64":
                X.zero_()
            elif name.startswith("prev"):
                X.copy_(Ps[t - 1].t())
            elif name.startswith("learned_judged"):
                sel = []
                for c in range(chains):
                    net.predict(Bs[t, c], Ps[t - 1, c], Ps[t - 2, c], out=cand[c])
                    sel.append(net.select(A, Bs[t, c], Ps[t - 1, c], cand[c], G[c], sweeps=sweeps, omega=omega))
                X.copy_(G.t())
                torch.cuda.synchronize()
                if name.endswith("_ir"):
                    infer_ms.append((time.perf_counter() - t0) * 1e3)
            else:
                P1.copy_(Ps[t - 1].t())
                P2.copy_(Ps[t - 2].t())
                cands = [P1, P2]
                if name.startswith("galerkin_learned"):
                    for c in range(chains):
                        net.predict(Bs[t, c], Ps[t - 1, c], Ps[t - 2, c], out=cand[c])
                    NN.copy_(cand.t())
                    cands.append(NN)
                galerkin_guess(A, B, cands, X0=X, work=gwork)
            if name.endswith("_mg"):
                r = prob["mg"].solve(B, X, mgp)
            else:
                mixed = 0 if name.endswith("fp64") else 2
                r = cg_solve(A, B, X, A_inner=prob["A32"] if mixed else None, params=prm[mixed], work=works[mixed])
            torch.cuda.synchronize()
            out[name]["ms"].append((time.perf_counter() - t0) * 1e3)
            out[name]["iters"].append(max(r.iters))
            assert max(r.true_rel_res) <= 1e-10, (name, r.true_rel_res)
        for c, (res, choice) in enumerate(sel):
            ch = int(choice.item())
            picks.append(ch)
            res_prev.append(float(res[0].item()))
            res_sel.append(float(res[ch].item()))
        nrm = Ps[t].norm(dim=1)
        err_prev += ((Ps[t - 1] - Ps[t]).norm(dim=1) / nrm).tolist()
        err_nn += ((cand - Ps[t]).norm(dim=1) / nrm).tolist()
        Xg = galerkin_guess(A, B, [P1, P2, NN], work=gwork)
        err_gal += ((Xg.t() - Ps[t]).norm(dim=1) / nrm).tolist()
    summary = {}
    for name, v in out.items():
        it = np.array(v["iters"], dtype=float)
        ms = np.array(v["ms"], dtype=float)
        summary[name] = {"median_iters": float(np.median(it)), "p90_iters": float(np.percentile(it, 90)),
                         "median_ms_per_step": float(np.median(ms)), "p90_ms_per_step": float(np.percentile(ms, 90)),
                         "ms_per_system": float(np.median(ms)) / chains}
    summary["guess"] = {"sweeps": sweeps, "omega": omega, "learned_picked_fraction": float(np.mean(picks)),
                        "median_rel_res_prev_smoothed": float(np.median(res_prev)),
                        "median_rel_res_selected": float(np.median(res_sel)),
                        "median_rel_err_prev": float(np.median(err_prev)),
                        "median_rel_err_learned": float(np.median(err_nn)),
                        "median_rel_err_galerkin_learned": float(np.median(err_gal)),
                        "inference_and_judge_ms_per_system": float(np.median(infer_ms)) / chains}
    summary["test_steps"] = len(test_steps)
    summary["chains"] = chains
    return summary


def network(grid, channels=(8, 16, 32, 48)):
    """The guess network for a grid periodic in x and y with walls in z."""
    nx, ny, nz = grid.shape
    return Guess(guess_cfg(nx, ny, nz, channels, (1, 1, 0)))
