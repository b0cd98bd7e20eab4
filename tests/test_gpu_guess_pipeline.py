"""The learned-guess pipeline end to end on a small Rayleigh-Benard-shaped grid: solver-made
training pairs, training with the library's kernels, and CG (Jacobi and multigrid) from the
judged guess and from the Galerkin combination of the candidates.

The trained network's predictions are a heuristic (parity unpinned); what is checked is that
every solve reaches the same 1e-10 true residual from any guess, that training lowers the
loss, and what the network gains over the previous-pressure guess on held-out steps."""
import numpy as np
import pytest
import torch

import workloads as W
from paper_2508_06710_gb300 import guess_pipeline as gp

pytestmark = pytest.mark.gpu


def test_pipeline_small_rbc(rb):
    grid = W.rbc_grid(32, 1.4)
    chains, steps, holdout = 8, 44, 4
    prob = gp.make_problem(torch, grid, chains)
    spectra = W.forcing_spectra(steps, chains, seed=5100)
    Bs, Ps, gen = gp.generate(torch, prob, spectra, W.face_fields)
    train_pairs, test_pairs = gp.pairs(steps, chains, holdout)
    net = gp.network(grid, (8, 16, 32))
    net.init_params(torch.as_tensor(W.normal(net.n_params, 5101).astype(np.float32), device="cuda"), head_scale=0.1)
    st = gp.train(torch, net, Bs, Ps, train_pairs, epochs=12, batch=4, lr=2e-3, lr_final=2e-4, seed=5102)
    assert st["loss_per_epoch"][-1] < 0.5 * st["loss_per_epoch"][0], st["loss_per_epoch"]
    ev = gp.evaluate(torch, prob, net, Bs, Ps, range(steps - holdout, steps), chains)
    print(gen, st, ev)
    gs = ev["guess"]
    # what the network gains: a guess closer to the solution than the previous pressure
    assert gs["median_rel_err_learned"] < 0.7 * gs["median_rel_err_prev"], gs
    # the judge never starts from a larger (smoothed) residual than the previous pressure's
    assert gs["median_rel_res_selected"] <= gs["median_rel_res_prev_smoothed"], gs
    # and CG from it reaches the same 1e-10 (asserted inside evaluate) in about as many
    # iterations: at this tolerance the iteration count barely depends on the guess
    assert ev["learned_judged_ir"]["median_iters"] <= 1.05 * ev["prev_ir"]["median_iters"], ev
    # the Galerkin combination of p_{t-1}, p_{t-2} and the network's guess is closer than the
    # previous pressure, and the multigrid solve from it takes no more iterations
    assert gs["median_rel_err_galerkin_learned"] < gs["median_rel_err_prev"], gs
    assert ev["galerkin_learned_mg"]["median_iters"] <= ev["prev_mg"]["median_iters"], ev
