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


def _check_merge(h, cfg):
    """Stage II by its defining properties, with an independent spatial index."""
    from scipy.spatial import cKDTree
    G = h["G"]
    sl, si = float(h["sigma"][0]), float(h["sigma"][1])
    comp = h["dom_group_off"][h["g_domain"]] + h["g_local"]           # compact index of each record
    order_rec = np.argsort(comp)
    cnt = h["g_count"][order_rec].astype(np.float64)
    lensum = h["g_lensum"][order_rec].astype(np.float64)
    incsum = np.array([float(np.float64(math.ldexp(1.0, -64)) * 0) for _ in range(0)])  # placeholder
    inc = np.array([_i192(w) for w in h["g_inc"][order_rec]], dtype=object)
    c_inc = np.array([float(v) for v in inc], dtype=np.float64)       # the oracle rounds exactly; see below
    # exact rounding of the 2^-64 fixed point, as the definition does
    c_inc = np.array([oracle.fx_round(np.array([(int(v) % (1 << 256) >> (64 * i)) & (2**64 - 1) for i in range(4)],
                                               np.uint64)) for v in inc])
    c_len = lensum / cnt
    c_inc = c_inc / cnt
    X = (cfg["scl"] * c_len) / sl
    Y = c_inc / si
    key = X * X + Y * Y
    order = np.lexsort((np.arange(G), key))                             # key, then compact index
    rank = np.empty(G, np.int64)
    rank[order] = np.arange(G)
    gid = h["l2g"]
    k = h["k"]
    assert gid.min() == 0 and gid.max() == k - 1
    # the start of each global group = its member of smallest rank
    start_of = np.full(k, G, np.int64)
    np.minimum.at(start_of, gid, rank)
    starts = np.sort(start_of)
    # global ids follow creation order = key order of the starts
    assert np.array_equal(np.argsort(start_of), np.arange(k))
    pts = np.stack([X, Y], 1)
    sp = pts[order[starts]]
    a = cfg["alpha"]
    tree = cKDTree(sp)
    # starts pairwise farther than alpha (exact test on the FP64 coordinates)
    pairs = tree.query_pairs(a * (1 + 1e-9), output_type="ndarray")
    if len(pairs):
        d = sp[pairs[:, 0]] - sp[pairs[:, 1]]
        assert np.all(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] > a * a)
    # every item maps to the earliest start within alpha (starts map to themselves)
    near = tree.query_ball_point(pts, a * (1 + 1e-9))
    a2 = a * a
    for c in range(G):
        best = G
        for j in near[c]:
            s = starts[j]
            if s > rank[c] or s >= best:
                continue
            dx = X[order[s]] - X[c]
            dy = Y[order[s]] - Y[c]
            if dx * dx + dy * dy <= a2:
                best = s
        assert best < G and best == start_of[gid[c]], c
    # dictionary = exact means of the member sums
    tot_cnt = np.zeros(k, np.int64)
    np.add.at(tot_cnt, gid, h["g_count"][order_rec])
    assert np.array_equal(tot_cnt, h["dict_count"])


def test_uneven_full(C=None):
    x, off, cfg, pl = _pipeline("uneven")
    h = _host(pl)
    b, e, ds = oracle.domains(off, cfg["domain_mode"], cfg["domain_value"])
    assert np.array_equal(b, h["dom_begin"]) and np.array_equal(e, h["dom_end"])
    ln, inc, po = oracle.compress(x, b, e, cfg["tol"], threads=16)
    gl, gi, _ = _compact_pieces(h)
    assert np.array_equal(po, h["dom_piece_off"])
    assert np.array_equal(ln, gl) and np.array_equal(inc, gi)
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


def test_scale_full_sampled():
    x, off, cfg, pl = _pipeline("scale")
    h = _host(pl)
    rng = np.random.default_rng(1)
    D = len(h["cnt"])
    for d in rng.choice(D, 400, replace=False):
        ln, inc, _ = oracle.compress(x, h["dom_begin"][d:d + 1], h["dom_end"][d:d + 1], cfg["tol"])
        s0 = h["dom_slot_off"][d]
        n = h["cnt"][d]
        assert np.array_equal(ln, h["piece_len"][s0:s0 + n]) and np.array_equal(inc, h["piece_inc"][s0:s0 + n]), d
    assert h["dict_count"].sum() == h["dom_piece_off"][-1]
