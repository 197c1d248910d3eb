"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and
bring its outputs back to the host in the oracle's (compact) layout."""
import numpy as np

import oracle


def ctx():
    import paper_2401_00109_gb300 as jb
    return jb.Context()


def params(cfg):
    import paper_2401_00109_gb300 as jb
    return jb.Params(tol=cfg["tol"], alpha=cfg["alpha"], scl=cfg["scl"], domain_mode=cfg["domain_mode"],
                     domain_value=cfg["domain_value"], round_mode=cfg.get("round_mode", 0))


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
                           round_mode=cfg.get("round_mode", 0))


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
