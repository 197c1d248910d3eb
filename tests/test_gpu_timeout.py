"""Failure detection without a GPU fault: the library's bounded device waits
give up, report JABBA_ERR_TIMEOUT through the status word, and leave the
context usable.

The context's poll limit (jabba_set_spin_limit) is lowered to one poll, so
waits that would have ended give up instead:
  - the compression kernel's waits for its staged series chunks (mbarrier
    phases of the bulk copies), in the plain one-lane-per-launch form;
  - the merge rounds' grid barrier, on a merge of fewer local groups than one
    sort tile (the sort then has no look-back wait, so the barrier is the only
    wait that runs);
  - the merge sort's decoupled look-back, on a merge of millions of groups.
Each call returns, the status reads JABBA_ERR_TIMEOUT, and after the default
limit is restored the same context reproduces the oracle's results.  Nothing
here faults, traps or hangs: every wait is bounded, and after a wait gives up
the later kernels of the call only read in bounds (the compression keeps the
pieces found so far; the merge skips its remaining steps)."""
import numpy as np
import pytest

import synth
from _gpu import assert_parity, ctx, params, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

ERR_TIMEOUT = 5


def _clean_run(C):
    x, off, cfg = synth.make("small")
    g, *_ = run_gpu(C, x, off, cfg)
    assert_parity(g, run_oracle(x, off, cfg))


def _device(x_np, off_np):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x_np)).cuda(), torch.from_numpy(off_np).cuda()


def test_compression_wait_times_out():
    """In the plain form (one launch, one CTA and one active lane per domain)
    the first wait of a launch follows right after its copy was issued; with
    the series out of L2 (a larger buffer written just before) and a limit of
    one poll it gives up before the chunk lands from HBM.  (Later waits find
    their chunk already there: it was issued a chunk of work earlier.  In the
    batched form the issue of a warp's 32 copies takes about as long as they
    take to land.)  Three tries make a miss very unlikely."""
    C = ctx()
    x_np, off_np, cfg = synth.make("small")
    p = params(cfg)
    x, off = _device(x_np, off_np)
    C.set_tuning(dict(C.tuning(), per_domain_launch=1))
    C.compress(x, off, p, series_off_host=off_np)
    assert C.status() == 0
    codes = []
    import torch
    flush = torch.empty(64 << 20, dtype=torch.float64, device=x.device)   # 512 MB: more than L2
    C.set_spin_limit(1)
    try:
        for _ in range(3):
            flush.fill_(1.0)  # the series leave L2, so the first chunk of a launch comes from HBM
            C.compress(x, off, p, series_off_host=off_np)
            codes.append(C.status())
            if codes[-1] == ERR_TIMEOUT:
                break
    finally:
        C.set_spin_limit(0)
        C.set_tuning(dict(C.tuning(), per_domain_launch=0))
    assert ERR_TIMEOUT in codes and set(codes) <= {0, ERR_TIMEOUT}, codes
    _clean_run(C)


@pytest.mark.parametrize("name,max_series", [("small", 4), ("multivar", 8)])
def test_merge_waits_time_out(name, max_series):
    """small x 4: 697 local groups (one sort tile: only the rounds' grid
    barrier waits); multivar x 8: millions of groups (the sort's look-back
    waits first)."""
    C = ctx()
    x_np, off_np, cfg = synth.make(name, max_series=max_series)
    p = params(cfg)
    x, off = _device(x_np, off_np)
    c = C.compress(x, off, p, series_off_host=off_np)
    l = C.digitize_local(c, p)
    C.sync_status(where="digitize")
    m = C.merge_global(l, p)
    assert C.status() == 0
    k_ref = int(m["k"].item())
    C.set_spin_limit(1)
    try:
        C.merge_global(l, p)
        code = C.status()
    finally:
        C.set_spin_limit(0)
    assert code == ERR_TIMEOUT
    m2 = C.merge_global(l, p)
    assert C.status() == 0
    assert int(m2["k"].item()) == k_ref
    for key in ("l2g", "dict_count"):
        n = int(l["n_groups"].item()) if key == "l2g" else k_ref
        assert np.array_equal(m2[key][:n].cpu().numpy(), m[key][:n].cpu().numpy()), key
    _clean_run(C)
