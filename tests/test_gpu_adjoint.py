"""GPU adjoint of the reconstruction MSE w.r.t. the dictionary increments:
against the oracle gradient, central finite differences (h = 1e-6) of the GPU
MSE, and a short Adam refinement through the torch.autograd.Function."""
import numpy as np
import pytest

import oracle
import synth
from _gpu import ctx, params, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    return ctx()


def test_gradient_matches_oracle_and_fd(C):
    import torch
    x_np, off_np, cfg = synth.make("diff", max_series=16)
    g, out, x, off = run_gpu(C, x_np, off_np, cfg)
    r = run_oracle(x_np, off_np, cfg)
    p = params(cfg)
    qlen = torch.from_numpy(g["qlen"]).cuda()
    di = out["dict_inc"].clone()
    grad = C.reconstruct_backward(x, off, out, qlen, di).cpu().numpy()
    k = len(r["dict_inc"])
    gr = oracle.reconstruct_grad(x_np, r["xhat"], r["symbol"], r["qlen"], r["series_piece_off"], off_np, k)
    np.testing.assert_allclose(grad, gr, rtol=1e-9, atol=1e-9 * np.abs(gr).max())
    rng = np.random.default_rng(1)
    for c in rng.choice(k, 8, replace=False):
        h = 1e-6
        dp = di.clone(); dp[c] += h
        dm = di.clone(); dm[c] -= h
        _, xp = C.reconstruct(x, off, out, p, dict_inc=dp)
        _, xm = C.reconstruct(x, off, out, p, dict_inc=dm)
        fd = (C.mse(x, xp).item() - C.mse(x, xm).item()) / (2 * h)
        assert abs(fd - grad[c]) <= 1e-6 * max(abs(grad[c]), 1e-7)


def test_adam_refinement_decreases_mse(C):
    import torch
    import paper_2401_00109_gb300 as jb
    x_np, off_np, cfg = synth.make("diff", max_series=32)
    g, out, x, off = run_gpu(C, x_np, off_np, cfg)
    p = params(cfg)
    qlen = torch.from_numpy(g["qlen"]).cuda()
    di = out["dict_inc"].clone().requires_grad_(True)
    opt = torch.optim.Adam([di], lr=1e-3, betas=(0.9, 0.999))
    F = jb.JabbaMSE()
    losses = []
    for _ in range(50):
        opt.zero_grad()
        loss = F.apply(di, C, x, off, out, qlen, p)
        loss.backward()
        opt.step()
        losses.append(loss.item())
    assert losses[-1] < losses[0]
    assert abs(losses[0] - g["mse"]) <= 1e-12 * g["mse"]
