"""GPU-vs-oracle parity of the whole forward path (domains, Eq. 1
compression, normalisation, Stage I and II aggregation, label propagation)
and of the inverse symbolization, through the C ABI, on seeded inputs of the
five workloads (bounded samples) and on edge cases."""
import numpy as np
import pytest

import synth
from _gpu import assert_parity, check_flips, ctx, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    return ctx()


@pytest.mark.parametrize("name,max_series", [("small", None), ("uneven", 40), ("multivar", 2), ("diff", 48),
                                             ("scale", 150)])
def test_workload_parity(C, name, max_series):
    x, off, cfg = synth.make(name, max_series=max_series)
    g, *_ = run_gpu(C, x, off, cfg)
    r = run_oracle(x, off, cfg)
    assert len(r["piece_len"]) > 0
    assert_parity(g, r)
    check_flips(f"{name} sample ({max_series or 'all'} series)", x, g["dom_begin"], g["dom_end"], g["piece_len"],
                g["dom_piece_off"], cfg["tol"])


@pytest.mark.parametrize("name,max_series", [("small", None), ("uneven", 40), ("multivar", 2), ("diff", 48),
                                             ("scale", 150)])
def test_pca_key_parity(C, name, max_series):
    """The PCA sort key (Sec. 5 "norm or PCA projection") in Stage I and II:
    the axis, the signed projection order, the key-gap pruning and every
    output equal the oracle's pipeline(key="pca") bit for bit."""
    x, off, cfg = synth.make(name, max_series=max_series)
    cfg = dict(cfg, key_mode=1)
    g, *_ = run_gpu(C, x, off, cfg)
    r = run_oracle(x, off, cfg)
    assert r["axis"] is not None and r["axis"][1] != 0.0   # a tilted axis: negative keys occur
    assert_parity(g, r)


@pytest.mark.parametrize("scl,alpha", [(0.5, 0.1), (2.0, 0.3), (0.0, 0.1)])
def test_pca_key_parity_scl(C, scl, alpha):
    """The PCA key with scl != 1 (an axis off the diagonal) and scl = 0
    (lengths ignored: the axis is (0, 1))."""
    x, off, cfg = synth.make("uneven", max_series=20)
    cfg = dict(cfg, key_mode=1, scl=scl, alpha=alpha)
    g, *_ = run_gpu(C, x, off, cfg, recon=False)
    r = run_oracle(x, off, cfg, recon=False)
    assert_parity(g, r, recon=False)


@pytest.mark.parametrize("round_mode", [0, 1])
def test_round_modes(C, round_mode):
    x, off, cfg = synth.make("small", max_series=5)
    cfg = dict(cfg, round_mode=round_mode)
    g, *_ = run_gpu(C, x, off, cfg)
    r = run_oracle(x, off, cfg)
    assert_parity(g, r)


def test_edge_series_lengths(C):
    """Empty, one-point and two-point series, a constant series and a straight
    line next to ordinary ones."""
    rng = np.random.default_rng(9)
    parts = [np.zeros(0), np.array([1.5]), np.array([0.25, -0.5]), np.full(37, 0.75), 0.01 * np.arange(300.0),
             np.cumsum(rng.standard_normal(1001)) * 0.1, np.zeros(0), rng.standard_normal(65)]
    x = np.concatenate(parts)
    off = np.concatenate([[0], np.cumsum([len(p) for p in parts])]).astype(np.int64)
    for mode, val in [(0, 1), (0, 3), (1, 16), (1, 1)]:
        cfg = dict(tol=0.05, alpha=0.1, scl=1.0, domain_mode=mode, domain_value=val)
        g, *_ = run_gpu(C, x, off, cfg)
        r = run_oracle(x, off, cfg)
        assert_parity(g, r)


def test_tol_zero_exact_path(C):
    """tol = 0 on an integer piecewise-linear series: every admissible piece
    has error exactly 0, which only the exact FP64 path can certify."""
    rng = np.random.default_rng(2)
    x = [0.0]
    while len(x) < 3000:
        slope = float(rng.integers(-4, 5))
        for _ in range(int(rng.integers(1, 40))):
            x.append(x[-1] + slope)
    x = np.array(x)
    off = np.array([0, len(x)], np.int64)
    cfg = dict(tol=0.0, alpha=0.0, scl=1.0, domain_mode=0, domain_value=5)
    g, *_ = run_gpu(C, x, off, cfg)
    r = run_oracle(x, off, cfg)
    assert_parity(g, r)


def test_large_domain_global_scratch(C):
    """A domain with more pieces than the shared-memory tile (white noise,
    small tol: almost every interval is a piece)."""
    rng = np.random.default_rng(4)
    x = rng.standard_normal(9000)
    off = np.array([0, 9000], np.int64)
    cfg = dict(tol=0.01, alpha=0.05, scl=1.0, domain_mode=0, domain_value=1)
    g, *_ = run_gpu(C, x, off, cfg, recon=False)
    r = run_oracle(x, off, cfg, recon=False)
    assert len(r["piece_len"]) > 4096
    assert_parity(g, r, recon=False)


def test_ragged_many_series(C):
    rng = np.random.default_rng(12)
    lens = rng.integers(0, 3000, 400)
    x = np.concatenate([np.cumsum(rng.standard_normal(n)) * 0.05 for n in lens]) if lens.sum() else np.zeros(0)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    cfg = dict(tol=0.1, alpha=0.1, scl=1.0, domain_mode=1, domain_value=257)
    g, *_ = run_gpu(C, x, off, cfg)
    r = run_oracle(x, off, cfg)
    assert_parity(g, r)


def test_nonfinite_and_range_errors(C):
    import paper_2401_00109_gb300 as jb
    import torch
    x = np.cumsum(np.random.default_rng(0).standard_normal(500))
    off = np.array([0, 500], np.int64)
    p = jb.Params(tol=0.1, alpha=0.1)
    for bad, code in [(np.nan, 3), (np.inf, 3), (2.0 ** 40, 7)]:
        y = x.copy()
        y[123] = bad
        c = C.compress(torch.from_numpy(y).cuda(), torch.from_numpy(off).cuda(), p, series_off_host=off)
        with pytest.raises(jb.JabbaError) as e:
            C.sync_status(where="compress")
        assert e.value.code == code
    # the context stays usable
    c = C.compress(torch.from_numpy(x).cuda(), torch.from_numpy(off).cuda(), p, series_off_host=off)
    C.sync_status(where="compress")


def test_duplicate_pieces_and_ties(C):
    """Integer walks with steps in {-1, 0, 1}: many identical pieces and
    centres, so keys tie exactly and the binary64 re-sort of overlapping key
    runs decides the order (ties by position / compact index)."""
    rng = np.random.default_rng(21)
    lens = rng.integers(50, 3000, 60)
    x = np.concatenate([np.cumsum(rng.integers(-1, 2, n)).astype(np.float64) for n in lens])
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    for alpha in (0.05, 0.5):
        cfg = dict(tol=0.5, alpha=alpha, scl=1.0, domain_mode=1, domain_value=128)
        g, *_ = run_gpu(C, x, off, cfg)
        r = run_oracle(x, off, cfg)
        assert_parity(g, r)


def test_merge_sequential_fallback(C):
    """A length weight so large that the merge grid would need too many cells:
    the merge runs its sequential binary64 greedy instead; same result."""
    x, off, cfg = synth.make("small", max_series=6)
    cfg = dict(cfg, scl=1e7)
    g, *_ = run_gpu(C, x, off, cfg)
    r = run_oracle(x, off, cfg)
    assert_parity(g, r)


@pytest.mark.parametrize("M", [1, 8, 64])
def test_noise_partition_parity(C, M):
    """The Gaussian-noise workload of the partition sweep (one series of
    100,000 N(0, 1) draws, tol = 0.01, alpha = 0.05) cut into M equal domains:
    the whole path, reconstruction included, equals the oracle for each M
    (M = 1 puts ~70,000 pieces in one domain: the global-memory arena)."""
    x, off, cfg = synth.make("noise")
    cfg = dict(cfg, domain_value=M)
    g, *_ = run_gpu(C, x, off, cfg)
    r = run_oracle(x, off, cfg)
    assert_parity(g, r)


@pytest.mark.parametrize("name,max_series", [("small", None), ("uneven", 30), ("scale", 120), ("multivar", 1)])
def test_reassign_and_sse_parity(C, name, max_series):
    """Full-reassignment digitization (Alg. 1 Digitize) and the exact SSE of
    both assignments equal the oracle's, bit for bit; the reassignment never
    has a larger SSE than label propagation."""
    import oracle
    x, off, cfg = synth.make(name, max_series=max_series)
    g, out, xg, offg = run_gpu(C, x, off, cfg, recon=False)
    r = run_oracle(x, off, cfg, recon=False)
    assert_parity(g, r, recon=False)
    p = __import__("_gpu").params(cfg)
    sym = C.reassign(out, p)
    ref = oracle.reassign(r["piece_len"], r["piece_inc"], r["sigma_len"], r["sigma_inc"], cfg["scl"],
                          r["dict_len"], r["dict_inc"])
    assert np.array_equal(sym.cpu().numpy(), ref)
    s_re = float(C.sse(out, p, sym).item())
    s_two = float(C.sse(out, p, out["symbol"]).item())
    C.sync_status(where="reassign")
    o_re = oracle.sse(r["piece_len"], r["piece_inc"], r["sigma_len"], r["sigma_inc"], cfg["scl"], r["dict_len"],
                      r["dict_inc"], ref)
    o_two = oracle.sse(r["piece_len"], r["piece_inc"], r["sigma_len"], r["sigma_inc"], cfg["scl"], r["dict_len"],
                       r["dict_inc"], r["symbol"])
    assert s_re == o_re and s_two == o_two
    assert s_re <= s_two


def test_merge_group_capacity_changes(C):
    """Stage II on one context with group capacities that grow and shrink
    between calls (the merge sort's scratch is laid out for each call's
    capacity): the dictionary, the local -> global map and the symbols equal
    the oracle's every time."""
    import torch
    from _gpu import params
    x, off, cfg = synth.make("small")
    r = run_oracle(x, off, cfg, recon=False)
    p = params(cfg)
    c = C.compress(torch.from_numpy(x).cuda(), torch.from_numpy(off).cuda(), p, series_off_host=off)
    C.sync_status(where="compress")
    D = c["n_domains"]
    cnt = c["dom_piece_cnt"][:D].cpu().numpy().astype(np.int64)
    G = len(r["l2g"])
    for mult in (1, 64, 8, 1, 32, 2, 1):
        l = C.digitize_local(c, p, group_capacity=G * mult)
        m = C.merge_global(l, p)
        C.sync_status(where="merge")
        k = int(m["k"].item())
        assert np.array_equal(m["l2g"][:G].cpu().numpy(), r["l2g"]), mult
        assert np.array_equal(m["dict_len"][:k].cpu().numpy(), r["dict_len"]), mult
        assert np.array_equal(m["dict_count"][:k].cpu().numpy(), r["dict_count"]), mult
        N = int(cnt.sum())
        sym = C.symbolize_step(c, l, m, N)
        C.sync_status(where="symbolize")
        assert np.array_equal(sym.cpu().numpy(), r["symbol"]), mult


@pytest.mark.parametrize("form", [0, 1])
def test_merge_forms(form):
    """Both forms of the Stage II rounds (two grid barriers per round with
    coverage marks; one barrier with coverage tested on the fly) give the
    oracle's result, on a dense workload and on one long chain."""
    C2 = ctx()
    C2.set_tuning(dict(merge_form=form))
    for name, ms, extra in (("multivar", 2, {}), ("noise", None, dict(domain_value=8)), ("uneven", 25, {})):
        x, off, cfg = synth.make(name, max_series=ms)
        cfg = dict(cfg, **extra)
        g, *_ = run_gpu(C2, x, off, cfg, recon=False)
        r = run_oracle(x, off, cfg, recon=False)
        assert_parity(g, r, recon=False)


@pytest.mark.parametrize("name,max_series,M", [("small", None, None), ("small", None, 1), ("uneven", 20, None),
                                               ("uneven", 20, 7), ("multivar", 1, None), ("noise", None, 3)])
def test_block_form_parity(C, name, max_series, M):
    """The block form of Sec. 5 (global key sort, contiguous sorted blocks,
    Stage I per block, Stage II over the starting points) equals the oracle's
    block_digitize bit for bit: the key order, the local labels, the map, the
    dictionary and the symbols (M = None: as many blocks as domains)."""
    import oracle
    import torch
    from _gpu import params
    x, off, cfg = synth.make(name, max_series=max_series)
    p = params(cfg)
    out = C.symbolize_blocks(torch.from_numpy(x).cuda(), torch.from_numpy(off).cuda(), p, n_blocks=M,
                             series_off_host=off)
    r0 = run_oracle(x, off, cfg, recon=False)
    Mb = out["n_blocks"]
    r = oracle.block_digitize(r0["piece_len"], r0["piece_inc"], r0["sigma_len"], r0["sigma_inc"], cfg["alpha"],
                              cfg["scl"], Mb)
    N = out["n_pieces"]
    assert np.array_equal(out["blocks"]["order"][:N].cpu().numpy(), r["order"])
    assert np.array_equal(out["blocks"]["dom_slot_off"].cpu().numpy(), r["blk_piece_off"])
    assert np.array_equal(out["local"]["local_label"][:N].cpu().numpy(), r["block_label"])
    assert np.array_equal(out["local"]["dom_group_off"].cpu().numpy(), r["blk_group_off"])
    G = out["n_groups_host"]
    assert np.array_equal(out["l2g"][:G].cpu().numpy(), r["l2g"])
    assert np.array_equal(out["dict_count"].cpu().numpy(), r["dict_count"])
    assert np.array_equal(out["dict_len"].cpu().numpy(), r["dict_len"])
    assert np.array_equal(out["dict_inc"].cpu().numpy(), r["dict_inc"])
    assert np.array_equal(out["symbol"].cpu().numpy(), r["symbol"])
    C.sync_status(where="block form")
