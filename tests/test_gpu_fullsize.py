"""GPU parity at the workloads' full sizes, in the launch configuration the
benchmark times (the graph-capturable Pipeline).  The oracle checks what it
can compute at that size; the greedy merge is checked by the properties that
define it, with an independent spatial index (scipy cKDTree):
  - every piece of every domain (uneven) or of sampled domains (scale)
    equals the oracle's compression bit for bit;
  - sigma equals the oracle's (uneven: from the oracle's own pieces);
  - sampled domains aggregate (Stage I) exactly as the oracle does;
  - Stage II: in binary64 key order, an item is a start iff no earlier start
    lies within alpha, and every other item maps to the earliest start within
    alpha; starts are pairwise farther than alpha;
  - every dictionary entry is the exact mean of its member pieces' sums."""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _pipeline(name, max_series=None):
    import torch
    import paper_2401_00109_gb300 as jb
    x, off, cfg = synth.make(name, max_series=max_series)
    p = jb.Params(tol=cfg["tol"], alpha=cfg["alpha"], scl=cfg["scl"], domain_mode=cfg["domain_mode"],
                  domain_value=cfg["domain_value"])
    ctx = jb.Context()
    cap = max(1 << 16, len(x) // 8)
    pl = jb.Pipeline(ctx, off, len(x), p, group_capacity=cap)
    pl.x.copy_(torch.from_numpy(x))
    pl.enqueue()
    ctx.sync_status(where=name)
    return x, off, cfg, pl


def _host(pl):
    b = pl.b
    D = pl.D
    h = {k: b[k].cpu().numpy() for k in ("dom_begin", "dom_end", "dom_slot_off", "dom_piece_off", "dom_group_off",
                                         "piece_len", "piece_inc", "local_label", "sigma")}
    h["cnt"] = b["dom_piece_cnt"][:D].cpu().numpy().astype(np.int64)
    G = int(b["n_groups"][0].item())
    k = int(b["k"][0].item())
    h["G"], h["k"] = G, k
    h["l2g"] = b["l2g"][:G].cpu().numpy()
    h["dict_len"] = b["dict_len"][:k].cpu().numpy()
    h["dict_inc"] = b["dict_inc"][:k].cpu().numpy()
    h["dict_count"] = b["dict_count"][:k].cpu().numpy()
    raw = b["groups"].cpu().numpy().view(np.uint64).reshape(-1, 6)[:G]
    h["g_inc"] = raw[:, 0:3]
    h["g_lensum"] = raw[:, 3].view(np.int64)
    cd = raw[:, 4].view(np.uint64)
    h["g_count"] = (cd & 0xFFFFFFFF).astype(np.int64)
    h["g_local"] = (cd >> 32).astype(np.int64)
    h["g_domain"] = (raw[:, 5] & 0xFFFFFFFF).astype(np.int64)
    return h


def _compact_pieces(h):
    D = len(h["cnt"])
    idx = np.concatenate([np.arange(h["dom_slot_off"][d], h["dom_slot_off"][d] + h["cnt"][d]) for d in range(D)])
    return h["piece_len"][idx], h["piece_inc"][idx], idx


def _i192(w):
    u = int(w[0]) | (int(w[1]) << 64) | (int(w[2]) << 128)
    return u - (1 << 192) if u >> 191 else u


def _check_merge(h, cfg, n_check=1_000_000):
    """Stage II by its defining properties, with an independent spatial index
    (vectorized; binary64 centres recomputed on the host from the group sums;
    a disagreement is accepted only at a rounding-level tie)."""
    from scipy.spatial import cKDTree
    G = h["G"]
    k = h["k"]
    sl, si = float(h["sigma"][0]), float(h["sigma"][1])
    comp = h["dom_group_off"][h["g_domain"]] + h["g_local"]           # compact index of each record
    assert np.array_equal(np.sort(comp), np.arange(G))
    rec = np.empty(G, np.int64)
    rec[comp] = np.arange(G)
    cnt = h["g_count"][rec].astype(np.float64)
    lensum = h["g_lensum"][rec].astype(np.float64)
    w = h["g_inc"][rec].astype(np.uint64)
    neg = w[:, 2].view(np.int64) < 0
    m = w.copy()
    m[neg] = ~m[neg]                                                  # two's complement magnitude: ~w + 1
    c0 = m[neg, 0] == np.uint64(0xFFFFFFFFFFFFFFFF)
    c1 = c0 & (m[neg, 1] == np.uint64(0xFFFFFFFFFFFFFFFF))
    m[neg, 0] += np.uint64(1)
    m[neg, 1] += c0.astype(np.uint64)
    m[neg, 2] += c1.astype(np.uint64)
    mag = (m[:, 2].astype(np.float64) * 2.0**128 + m[:, 1].astype(np.float64) * 2.0**64
           + m[:, 0].astype(np.float64)) * 2.0**-64
    incsum = np.where(neg, -mag, mag)
    X = (cfg["scl"] * (lensum / cnt)) / sl
    Y = (incsum / cnt) / si
    key = X * X + Y * Y
    order = np.lexsort((np.arange(G), key))
    rank = np.empty(G, np.int64)
    rank[order] = np.arange(G)
    gid = h["l2g"]
    assert gid.min() == 0 and gid.max() == k - 1
    start_of = np.full(k, G, np.int64)
    np.minimum.at(start_of, gid, rank)                                # each global group's earliest member
    assert np.all(np.diff(start_of) > 0)                              # ids follow creation (key) order
    a = cfg["alpha"]
    sp = np.stack([X[order[start_of]], Y[order[start_of]]], 1)
    tree = cKDTree(sp)
    pairs = tree.query_pairs(a * (1 - 1e-9), output_type="ndarray")
    assert len(pairs) == 0                                            # starts pairwise farther than alpha
    rng = np.random.default_rng(3)
    items = rng.choice(G, min(n_check, G), replace=False)
    dist, nb = tree.query(np.stack([X[items], Y[items]], 1), k=8, distance_upper_bound=a * (1 + 1e-9))
    valid = nb < k
    nbc = np.where(valid, nb, 0)
    srank = start_of[nbc]
    ok = valid & (srank <= rank[items][:, None])
    dx = X[order[srank]] - X[items][:, None]
    dy = Y[order[srank]] - Y[items][:, None]
    d2 = dx * dx + dy * dy
    within = ok & (d2 <= a * a)
    best = np.where(within, srank, G).min(1)
    assigned = start_of[gid[items]]
    bad = np.nonzero(best != assigned)[0]
    for i in bad:                                                     # only rounding-level ties may differ
        c = items[i]
        s1, s2 = best[i], assigned[i]
        d_tie = [abs(((X[order[s]] - X[c]) ** 2 + (Y[order[s]] - Y[c]) ** 2) - a * a) <= 1e-12 * a * a
                 for s in (s1, s2) if s < G]
        k_tie = s1 < G and abs(key[order[s1]] - key[order[s2]]) <= 1e-12 * max(key[order[s1]], 1e-300)
        assert any(d_tie) or k_tie, (c, s1, s2)
    assert len(bad) <= 1e-4 * len(items)
    tot_cnt = np.zeros(k, np.int64)
    np.add.at(tot_cnt, gid, h["g_count"][rec])
    assert np.array_equal(tot_cnt, h["dict_count"])
    tot_len = np.zeros(k, np.int64)
    np.add.at(tot_len, gid, h["g_lensum"][rec])
    assert np.array_equal(tot_len.astype(np.float64) / tot_cnt, h["dict_len"])


def test_uneven_full():
    x, off, cfg, pl = _pipeline("uneven")
    h = _host(pl)
    b, e, ds = oracle.domains(off, cfg["domain_mode"], cfg["domain_value"])
    assert np.array_equal(b, h["dom_begin"]) and np.array_equal(e, h["dom_end"])
    ln, inc, po = oracle.compress(x, b, e, cfg["tol"], threads=16)
    gl, gi, _ = _compact_pieces(h)
    assert np.array_equal(po, h["dom_piece_off"])
    assert np.array_equal(ln, gl) and np.array_equal(inc, gi)
    from _gpu import check_flips
    check_flips("uneven full size", x, b, e, gl, h["dom_piece_off"], cfg["tol"])
    sl, si = oracle.sigma(ln, inc)
    assert (sl, si) == (float(h["sigma"][0]), float(h["sigma"][1]))
    # Stage I on sampled domains
    rng = np.random.default_rng(0)
    for d in rng.choice(len(b), 300, replace=False):
        a0, a1 = po[d], po[d + 1]
        lab, go, gc, gls, gii = oracle.local_aggregate(ln[a0:a1], inc[a0:a1], np.array([0, a1 - a0]), sl, si,
                                                       cfg["alpha"], cfg["scl"])
        s0 = h["dom_slot_off"][d]
        assert np.array_equal(lab, h["local_label"][s0:s0 + (a1 - a0)])
        assert h["dom_group_off"][d + 1] - h["dom_group_off"][d] == len(gc)
    _check_merge(h, cfg)


def _records_by_compact(h):
    """Row of each group record, indexed by compact group index."""
    comp = h["dom_group_off"][h["g_domain"]] + h["g_local"]
    rec = np.empty(h["G"], np.int64)
    rec[comp] = np.arange(h["G"])
    return rec


def _device_compact(pl):
    """Compact (domain-order) device views of the slotted per-piece arrays."""
    import torch
    b = pl.b
    D = pl.D
    cnt = b["dom_piece_cnt"][:D].long()
    first = torch.repeat_interleave(b["dom_slot_off"][:D], cnt)
    within = torch.arange(first.numel(), device=first.device) - torch.repeat_interleave(b["dom_piece_off"][:D], cnt)
    idx = first + within
    dom = torch.repeat_interleave(torch.arange(D, device=first.device), cnt)
    return idx, dom


def test_scale_full_labels():
    """The scale-stress workload at full size (100,000 series, 1.44e9 points,
    182 M pieces): compression of sampled domains equals the oracle's; sigma
    equals the oracle's over all pieces; Stage I of sampled domains (the
    GPU's pieces and sigma through the oracle's greedy) gives the same labels
    and group sums; Stage II satisfies its defining properties; every symbol
    is the composition l2g[dom_group_off[d] + local_label] (all pieces); every
    dictionary entry is the exact mean of the pieces carrying its symbol (all
    pieces); breakpoint flips of the sampled domains against the plain-form
    Eq. 1 are logged."""
    import torch
    from _gpu import check_dictionary_exact, check_flips
    x, off, cfg, pl = _pipeline("scale")
    h = _host(pl)
    rng = np.random.default_rng(1)
    D = len(h["cnt"])
    sl, si = float(h["sigma"][0]), float(h["sigma"][1])
    gl, gi, _ = _compact_pieces(h)
    assert oracle.sigma(gl, gi) == (sl, si)
    rec = _records_by_compact(h)
    sample = np.sort(rng.choice(D, 400, replace=False))
    for d in sample:
        ln, inc, _ = oracle.compress(x, h["dom_begin"][d:d + 1], h["dom_end"][d:d + 1], cfg["tol"])
        s0 = h["dom_slot_off"][d]
        n = h["cnt"][d]
        pln, pinc = h["piece_len"][s0:s0 + n], h["piece_inc"][s0:s0 + n]
        assert np.array_equal(ln, pln) and np.array_equal(inc, pinc), d
        lab, go, gc, gls, gii = oracle.local_aggregate(pln, pinc, np.array([0, n]), sl, si, cfg["alpha"], cfg["scl"])
        assert np.array_equal(lab, h["local_label"][s0:s0 + n]), d
        g0, g1 = h["dom_group_off"][d], h["dom_group_off"][d + 1]
        assert g1 - g0 == len(gc), d
        rows = rec[g0:g1]
        assert np.array_equal(h["g_count"][rows], gc) and np.array_equal(h["g_lensum"][rows], gls), d
        for j, r_ in enumerate(rows):
            assert _i192(h["g_inc"][r_]) == oracle.fx_value(gii[j]), (d, j)
    po_s = np.concatenate([[0], np.cumsum(h["cnt"][sample])])
    ln_s = np.concatenate([h["piece_len"][h["dom_slot_off"][d]:h["dom_slot_off"][d] + h["cnt"][d]] for d in sample])
    check_flips("scale full size (400 sampled domains)", x, h["dom_begin"][sample], h["dom_end"][sample], ln_s, po_s,
                cfg["tol"])
    _check_merge(h, cfg)
    del h, gl, gi
    b = pl.b
    N = int(b["dom_piece_off"][-1].item())
    k = int(b["k"][0].item())
    idx, dom = _device_compact(pl)
    lab = b["local_label"][idx].long()
    want = b["l2g"][b["dom_group_off"][dom] + lab]
    assert torch.equal(b["symbol"][:N], want)
    del lab, want, dom
    check_dictionary_exact(b["piece_len"][idx], b["piece_inc"][idx], b["symbol"][:N], b["dict_len"][:k],
                           b["dict_inc"][:k], b["dict_count"][:k])


def test_diff_full_adjoint_and_refinement():
    """The dictionary-refinement workload at full size (1,024 series x 10,000
    points): the whole forward path and the reconstruction equal the oracle's,
    the adjoint equals the oracle's gradient and FP64 central differences
    (h = 1e-6), and 50 Adam steps (lr 1e-3) through the autograd.Function
    end below the starting reconstruction MSE."""
    import torch
    import paper_2401_00109_gb300 as jb
    from _gpu import assert_parity, ctx, params, run_gpu, run_oracle
    x_np, off_np, cfg = synth.make("diff")
    C = ctx()
    g, out, x, off = run_gpu(C, x_np, off_np, cfg)
    r = run_oracle(x_np, off_np, cfg, threads=16)
    assert_parity(g, r)
    from _gpu import check_flips
    check_flips("diff full size", x_np, g["dom_begin"], g["dom_end"], g["piece_len"], g["dom_piece_off"], cfg["tol"])
    p = params(cfg)
    qlen = torch.from_numpy(g["qlen"]).cuda()
    di = out["dict_inc"].clone()
    grad = C.reconstruct_backward(x, off, out, qlen, di).cpu().numpy()
    k = len(r["dict_inc"])
    gr = oracle.reconstruct_grad(x_np, r["xhat"], r["symbol"], r["qlen"], r["series_piece_off"], off_np, k)
    np.testing.assert_allclose(grad, gr, rtol=1e-9, atol=1e-9 * np.abs(gr).max())
    rng = np.random.default_rng(5)
    for c in rng.choice(k, 8, replace=False):
        h = 1e-6
        dp = di.clone()
        dp[c] += h
        dm = di.clone()
        dm[c] -= h
        _, xp = C.reconstruct(x, off, out, p, dict_inc=dp)
        _, xm = C.reconstruct(x, off, out, p, dict_inc=dm)
        fd = (C.mse(x, xp).item() - C.mse(x, xm).item()) / (2 * h)
        assert abs(fd - grad[c]) <= 1e-6 * max(abs(grad[c]), 1e-7), (c, fd, grad[c])
    w = di.clone().requires_grad_(True)
    opt = torch.optim.Adam([w], lr=1e-3, betas=(0.9, 0.999))
    F = jb.JabbaMSE()
    losses = []
    for _ in range(50):
        opt.zero_grad()
        loss = F.apply(w, C, x, off, out, qlen, p)
        loss.backward()
        opt.step()
        losses.append(loss.item())
    assert abs(losses[0] - r["mse"]) <= 1e-9 * r["mse"]
    assert losses[-1] < losses[0]


def test_scale_full_two_in_flight():
    """The benchmark's launch configuration: two pipelines with a batch each
    in flight (front and back halves on two streams, front kernels capped so
    the other batch's merge fits beside them).  After several interleaved
    steps both pipelines hold exactly the result of one pipeline run alone
    with the default configuration, and sampled domains match the oracle."""
    import torch
    import paper_2401_00109_gb300 as jb
    x, off, cfg, pl = _pipeline("scale")
    D = pl.D

    def compact(q, key):
        # the valid slots of every domain, in domain order (slots past a
        # domain's count hold nothing)
        b = q.b
        cnt = b["dom_piece_cnt"][:D].long()
        first = torch.repeat_interleave(b["dom_slot_off"][:D], cnt)
        within = torch.arange(first.numel(), device=first.device) - torch.repeat_interleave(b["dom_piece_off"][:D], cnt)
        return b[key][first + within]

    ref = {k: pl.b[k].clone() for k in ("symbol", "dict_len", "dict_inc", "dict_count", "k", "n_groups",
                                        "dom_piece_off", "dom_piece_cnt")}
    for key in ("piece_len", "piece_inc", "local_label"):
        ref[key] = compact(pl, key)
    ctx2 = jb.Context()
    pl2 = jb.Pipeline(ctx2, off, len(x), pl.p, group_capacity=pl.gcap)
    pl2.x.copy_(torch.from_numpy(x))
    prof = dict(pl.ctx.tuning(), compress_ctas_per_sm=1, local_ctas_cap=3, merge_ctas_per_sm=1)
    for c in (pl.ctx, ctx2):
        c.set_tuning(prof)
    fl = jb.InFlight([pl, pl2])
    for _ in range(5):
        fl.step()
    fl.join()
    torch.cuda.synchronize()
    pl.ctx.sync_status(where="in flight A")
    ctx2.sync_status(where="in flight B")
    N = int(ref["dom_piece_off"][-1].item())
    k = int(ref["k"][0].item())
    for q in (pl, pl2):
        assert int(q.b["k"][0].item()) == k and int(q.b["n_groups"][0].item()) == int(ref["n_groups"][0].item())
        assert torch.equal(q.b["symbol"][:N], ref["symbol"][:N])
        for key in ("dict_len", "dict_inc", "dict_count"):
            assert torch.equal(q.b[key][:k], ref[key][:k]), key
        assert torch.equal(q.b["dom_piece_cnt"][:D], ref["dom_piece_cnt"][:D])
        for key in ("piece_len", "piece_inc", "local_label"):
            assert torch.equal(compact(q, key), ref[key]), key
    h = _host(pl2)
    rng = np.random.default_rng(2)
    for d in rng.choice(len(h["cnt"]), 100, replace=False):
        ln, inc, _ = oracle.compress(x, h["dom_begin"][d:d + 1], h["dom_end"][d:d + 1], cfg["tol"])
        s0 = h["dom_slot_off"][d]
        n = h["cnt"][d]
        assert np.array_equal(ln, h["piece_len"][s0:s0 + n]) and np.array_equal(inc, h["piece_inc"][s0:s0 + n]), d


@pytest.mark.parametrize("name,key_mode", [("multivar", 0), ("uneven", 0), ("multivar", 1)])
def test_full_size_bit_exact(name, key_mode):
    """The multivariate (64 x 2^20) and uneven (10,000 series) workloads at
    full size: every output of the path and the reconstruction equal the
    oracle's (pieces, sigma, local labels, map, dictionary, symbols, quantized
    lengths bit for bit; reconstruction within 1e-9); the multivariate one
    also with the PCA sort key (Sec. 5)."""
    from _gpu import assert_parity, check_flips, ctx, run_gpu, run_oracle
    x, off, cfg = synth.make(name)
    cfg = dict(cfg, key_mode=key_mode)
    g, *_ = run_gpu(ctx(), x, off, cfg)
    r = run_oracle(x, off, cfg, threads=16)
    assert_parity(g, r)
    check_flips(f"{name} full size", x, g["dom_begin"], g["dom_end"], g["piece_len"], g["dom_piece_off"], cfg["tol"])
