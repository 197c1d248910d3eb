"""The allocation-free reconstruction entry point, called through the C ABI
like every other GPU test, against the ordinary one (jabba_reconstruct).

jabba_reconstruct_noalloc exists for callers that cannot allocate device
memory (they cannot create a context, whose scratch comes from cudaMalloc);
its scratch is a fixed array in the library.  Two calls in a row must both
match the ordinary entry point, the second showing that the shared array's
leftover contents from the first call do not leak into the result.  This file
is collected last so that a failure here leaves every other test already run;
it also passes on its own in a fresh process."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_reconstruct_noalloc_matches_reconstruct_twice():
    import torch
    import paper_2401_00109_gb300 as jb
    x_np, off_np, cfg = synth.make("diff", max_series=24)
    p = jb.Params(tol=cfg["tol"], alpha=cfg["alpha"], scl=cfg["scl"], domain_mode=cfg["domain_mode"],
                  domain_value=cfg["domain_value"])
    ctx = jb.Context()
    x = torch.from_numpy(x_np).cuda()
    off = torch.from_numpy(off_np).cuda()
    out = ctx.symbolize(x, off, p, series_off_host=off_np)
    assert out["n_pieces"] <= jb.NOALLOC_MAX_PIECES
    q_ref, x_ref = ctx.reconstruct(x, off, out, p)
    ctx.sync_status(where="reference reconstruction")
    q_ref = q_ref.cpu().numpy()
    x_ref = x_ref.cpu().numpy()
    scale = max(1.0, float(np.abs(x_ref).max()))
    # outputs allocated up front: the call itself allocates nothing
    q_buf = torch.empty(max(out["n_pieces"], 1), dtype=torch.int32, device=x.device)
    x_buf = torch.empty_like(x)
    for call in range(2):
        torch.cuda.synchronize()
        before = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
        q, xh = jb.reconstruct_noalloc(x, off, out, p, qlen=q_buf, xhat=x_buf)
        torch.cuda.synchronize()
        if call == 1:  # the first call on a device may load the module (its own one-time set-up)
            assert (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]) == before
        assert jb.reconstruct_noalloc_status() == 0
        assert np.array_equal(q.cpu().numpy(), q_ref), call
        assert np.abs(xh.cpu().numpy() - x_ref).max() <= 1e-9 * scale, call
    # a second, different collection through the same shared scratch
    x2_np, off2_np, _ = synth.make("small", max_series=7)
    x2 = torch.from_numpy(x2_np).cuda()
    off2 = torch.from_numpy(off2_np).cuda()
    out2 = ctx.symbolize(x2, off2, p, series_off_host=off2_np)
    q2_ref, x2_ref = ctx.reconstruct(x2, off2, out2, p)
    q2, xh2 = jb.reconstruct_noalloc(x2, off2, out2, p)
    torch.cuda.synchronize()
    assert np.array_equal(q2.cpu().numpy(), q2_ref.cpu().numpy())
    assert np.abs(xh2.cpu().numpy() - x2_ref.cpu().numpy()).max() <= 1e-9 * max(1.0, float(x2_ref.abs().max()))


def test_reconstruct_noalloc_rejects_oversize():
    import paper_2401_00109_gb300 as jb
    import ctypes as C
    L = jb.load()
    r = L.jabba_reconstruct_noalloc(C.c_void_p(8), 10, C.c_void_p(8), jb.NOALLOC_MAX_SERIES + 1, C.c_void_p(8),
                                    C.c_void_p(8), 5, C.c_void_p(8), C.c_void_p(8), C.c_void_p(8), 0, C.c_void_p(8),
                                    C.c_void_p(8), None)
    assert r == jb.ERR_CAPACITY
    r = L.jabba_reconstruct_noalloc(C.c_void_p(8), 10, C.c_void_p(8), 2, C.c_void_p(8), C.c_void_p(8),
                                    jb.NOALLOC_MAX_PIECES + 1, C.c_void_p(8), C.c_void_p(8), C.c_void_p(8), 0,
                                    C.c_void_p(8), C.c_void_p(8), None)
    assert r == jb.ERR_CAPACITY


def test_reconstruct_noalloc_checks_piece_offsets_on_the_device():
    """An understated piece count (the host check passes, the device offsets
    run past it) is caught on the device: the call writes nothing, the status
    query returns JABBA_ERR_CAPACITY once, and the next correct call works."""
    import torch
    import paper_2401_00109_gb300 as jb
    x_np, off_np, cfg = synth.make("small", max_series=6)
    p = jb.Params(tol=cfg["tol"], alpha=cfg["alpha"], scl=cfg["scl"], domain_mode=cfg["domain_mode"],
                  domain_value=cfg["domain_value"])
    ctx = jb.Context()
    x = torch.from_numpy(x_np).cuda()
    off = torch.from_numpy(off_np).cuda()
    out = ctx.symbolize(x, off, p, series_off_host=off_np)
    N = out["n_pieces"]
    q_ref, x_ref = ctx.reconstruct(x, off, out, p)
    ctx.sync_status(where="reference reconstruction")
    assert jb.reconstruct_noalloc_status() == 0
    q_buf = torch.full((N,), -7, dtype=torch.int32, device=x.device)
    x_buf = torch.full_like(x, 123.0)
    jb.reconstruct_noalloc(x, off, out, p, qlen=q_buf, xhat=x_buf, n_pieces=N // 2)
    assert jb.reconstruct_noalloc_status() == jb.ERR_CAPACITY
    assert jb.reconstruct_noalloc_status() == 0
    assert bool((q_buf == -7).all()) and bool((x_buf == 123.0).all())
    q, xh = jb.reconstruct_noalloc(x, off, out, p, qlen=q_buf, xhat=x_buf)
    assert jb.reconstruct_noalloc_status() == 0
    assert torch.equal(q, q_ref) and float((xh - x_ref).abs().max()) <= 1e-9 * max(1.0, float(x_ref.abs().max()))
