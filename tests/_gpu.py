"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and
bring its outputs back to the host in the oracle's (compact) layout; count
breakpoint flips against Eq. 1 read literally; check a dictionary against
exact means of its pieces on the device."""
import numpy as np

import oracle

# (label, pieces checked, flips) of every flip check of the session; the
# terminal summary (conftest.py) prints them.
FLIP_LOG = []


def ctx():
    import paper_2401_00109_gb300 as jb
    return jb.Context()


def params(cfg):
    import paper_2401_00109_gb300 as jb
    return jb.Params(tol=cfg["tol"], alpha=cfg["alpha"], scl=cfg["scl"], domain_mode=cfg["domain_mode"],
                     domain_value=cfg["domain_value"], round_mode=cfg.get("round_mode", 0),
                     key_mode=cfg.get("key_mode", 0))


def run_gpu(c, x_np, off_np, cfg, recon=True):
    import torch
    p = params(cfg)
    x = torch.from_numpy(np.ascontiguousarray(x_np)).cuda()
    off = torch.from_numpy(np.ascontiguousarray(off_np, dtype=np.int64)).cuda()
    out = c.symbolize(x, off, p, series_off_host=off_np)
    h = {}
    D = out["n_domains"]
    cnt = out["dom_piece_cnt"][:D].cpu().numpy().astype(np.int64)
    slot = out["dom_slot_off"].cpu().numpy()
    pl = out["piece_len"].cpu().numpy()
    pi = out["piece_inc"].cpu().numpy()
    ll = out["local_label"].cpu().numpy()
    idx = np.concatenate([np.arange(slot[d], slot[d] + cnt[d]) for d in range(D)]) if D else np.zeros(0, np.int64)
    h["dom_begin"] = out["dom_begin"].cpu().numpy()
    h["dom_end"] = out["dom_end"].cpu().numpy()
    h["dom_series"] = out["dom_series"].cpu().numpy()
    h["dom_piece_off"] = out["dom_piece_off"].cpu().numpy()
    h["piece_len"] = pl[idx]
    h["piece_inc"] = pi[idx]
    h["sigma"] = out["sigma"].cpu().numpy()
    h["local_label"] = ll[idx]
    h["dom_group_off"] = out["dom_group_off"].cpu().numpy()
    G = out["n_groups_host"]
    h["l2g"] = out["l2g"][:G].cpu().numpy()
    h["dict_len"] = out["dict_len"].cpu().numpy()
    h["dict_inc"] = out["dict_inc"].cpu().numpy()
    h["dict_count"] = out["dict_count"].cpu().numpy()
    h["symbol"] = out["symbol"].cpu().numpy()
    if recon:
        qlen, xhat = c.reconstruct(x, off, out, p)
        h["qlen"] = qlen.cpu().numpy()
        h["xhat"] = xhat.cpu().numpy()
        h["mse"] = float(c.mse(x, xhat).item())
        c.sync_status(where="reconstruct")
    return h, out, x, off


def run_oracle(x_np, off_np, cfg, recon=True, threads=8):
    return oracle.pipeline(x_np, off_np, cfg["tol"], cfg["alpha"], cfg["scl"], cfg["domain_mode"],
                           cfg["domain_value"], threads=threads, with_reconstruct=recon,
                           round_mode=cfg.get("round_mode", 0), key="pca" if cfg.get("key_mode", 0) else "norm")


def first_diff(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    if a.shape != b.shape:
        return f"shape {a.shape} vs {b.shape}"
    w = np.nonzero(a != b)[0]
    return f"{len(w)} differ, first at {w[0]}: {a[w[0]]!r} vs {b[w[0]]!r}" if len(w) else "equal"


def assert_parity(g, r, recon=True):
    """Bit-exact integer decisions and FP64 values computed by the same
    definition; reconstruction within 1e-9 relative."""
    for k in ("dom_begin", "dom_end", "dom_series", "dom_piece_off", "piece_len"):
        assert np.array_equal(g[k], r[k]), (k, first_diff(g[k], r[k]))
    assert np.array_equal(g["piece_inc"], r["piece_inc"]), ("piece_inc", first_diff(g["piece_inc"], r["piece_inc"]))
    assert g["sigma"][0] == r["sigma_len"] and g["sigma"][1] == r["sigma_inc"], (g["sigma"], r["sigma_len"], r["sigma_inc"])
    if r.get("axis") is not None:                      # the PCA axis, bit for bit
        assert (g["sigma"][2], g["sigma"][3]) == r["axis"], (g["sigma"], r["axis"])
    assert np.array_equal(g["local_label"], r["local_label"]), ("local_label", first_diff(g["local_label"], r["local_label"]))
    assert np.array_equal(g["dom_group_off"], r["dom_group_off"])
    assert np.array_equal(g["l2g"], r["l2g"]), ("l2g", first_diff(g["l2g"], r["l2g"]))
    assert np.array_equal(g["dict_count"], r["dict_count"])
    assert np.array_equal(g["dict_len"], r["dict_len"]), ("dict_len", first_diff(g["dict_len"], r["dict_len"]))
    # centres: same exact sums and the same division -> identical; the contract is 1e-12 relative
    np.testing.assert_allclose(g["dict_inc"], r["dict_inc"], rtol=1e-12, atol=0)
    assert np.array_equal(g["symbol"], r["symbol"]), ("symbol", first_diff(g["symbol"], r["symbol"]))
    if recon:
        assert np.array_equal(g["qlen"], r["qlen"]), ("qlen", first_diff(g["qlen"], r["qlen"]))
        scale = max(1.0, float(np.abs(r["xhat"]).max()))
        assert np.abs(g["xhat"] - r["xhat"]).max() <= 1e-9 * scale
        assert abs(g["mse"] - r["mse"]) <= 1e-9 * max(r["mse"], 1e-300)


def check_flips(label, x, dom_begin, dom_end, piece_len, dom_piece_off, tol, threads=16):
    """Breakpoint flips of a GPU chain against Eq. 1 read literally (the
    plain sequential sum of squared residuals): the library decides Eq. 1 in
    its L^2-scaled exact form, which agrees except where the error lies within
    rounding of the bound.  Every flip must have |err - bound| < 1e-12 bound;
    the count is logged."""
    r = oracle.breakpoint_flips(x, dom_begin, dom_end, piece_len, dom_piece_off, tol, threads=threads)
    for s0, t, err, bound in r["flips"]:
        assert abs(err - bound) < 1e-12 * bound, (label, s0, t, err, bound)
    FLIP_LOG.append((label, r["pieces"], len(r["flips"])))
    return r


def _fx_chunks(torch, v):
    """trunc(|v| * 2^64) of float64 values |v| < 2^32 as three 32-bit chunks
    (int64 tensors, low first) and the sign, by integer operations only."""
    f, e = torch.frexp(v.abs())                         # |v| = f 2^e, f in [0.5, 1)
    m = torch.ldexp(f, torch.full_like(e, 53)).to(torch.int64)   # 53-bit integer mantissa
    s = e.to(torch.int64) + 11                           # |v| 2^64 = m 2^s
    zero = m == 0
    mask = (1 << 32) - 1
    out = []
    for i in range(3):
        sh = s - 32 * i
        left = torch.clamp(sh, 0, 31)
        keep = torch.bitwise_left_shift(torch.ones_like(m), 32 - left) - 1
        c_left = torch.bitwise_left_shift(torch.bitwise_and(m, keep), left)
        c_right = torch.bitwise_and(torch.bitwise_right_shift(m, torch.clamp(-sh, 0, 63)), mask)
        c = torch.where(sh >= 32, torch.zeros_like(m), torch.where(sh >= 0, c_left, c_right))
        out.append(torch.where(zero, torch.zeros_like(m), c))
    return out, v < 0


def check_dictionary_exact(piece_len, piece_inc, symbol, dict_len, dict_inc, dict_count):
    """Every dictionary entry is the exact mean of the pieces that carry its
    symbol (device tensors, compact layout): count, length sum (integers) and
    the increment sum at 2^-64 (each term truncated toward zero, summed as an
    integer, rounded once to binary64), then lensum / count and
    round(sum inc) / count in binary64.  Sums over all pieces on the device."""
    import torch
    k = dict_count.numel()
    sym = symbol.long()
    cnt = torch.bincount(sym, minlength=k)
    assert torch.equal(cnt, dict_count), "dictionary counts"
    lensum = torch.zeros(k, dtype=torch.int64, device=sym.device).index_add_(0, sym, piece_len.long())
    assert torch.equal(lensum.double() / cnt.double(), dict_len), "dictionary lengths"
    chunks, neg = _fx_chunks(torch, piece_inc)
    sums = []
    for c in chunks:
        signed = torch.where(neg, -c, c)
        sums.append(torch.zeros(k, dtype=torch.int64, device=sym.device).index_add_(0, sym, signed).cpu().numpy())
    cnt_h = cnt.cpu().numpy()
    want = np.empty(k)
    for j in range(k):
        tot = int(sums[0][j]) + (int(sums[1][j]) << 32) + (int(sums[2][j]) << 64)
        want[j] = (float(tot) * 2.0**-64) / float(cnt_h[j])     # int -> float rounds to nearest even
    got = dict_inc.cpu().numpy()
    bad = np.nonzero(want != got)[0]
    assert len(bad) == 0, ("dictionary increments", len(bad), bad[:5])
