"""Pins for the oracle's inverse symbolization (Sec. 3.3): quantization carry,
inverse compression, MSE, and the gradient of the MSE with respect to the
dictionary increments (closed form, finite differences, normal equations)."""
import math

import numpy as np

import oracle
import synth
from _golden import load


def test_quantize_hand():
    g = load("quantize_hand.txt")
    k = len(g["lt"])
    sym = np.arange(k, dtype=np.int32)
    x = np.zeros(7)
    off = np.array([0, 7], np.int64)
    spo = np.array([0, k], np.int64)
    ql, xh = oracle.reconstruct(sym, spo, g["lt"], g["it"], x, off)
    assert ql.tolist() == g["qlen"].astype(int).tolist()
    assert xh.tolist() == g["xhat"].tolist()


def test_quantize_half_even_hand():
    """round_mode 1 (ties to even) on exact ties, with a zero-length piece."""
    g = load("quantize_even_hand.txt")
    k = len(g["lt"])
    sym = np.arange(k, dtype=np.int32)
    n = len(g["xhat"])
    x = np.zeros(n)
    off = np.array([0, n], np.int64)
    spo = np.array([0, k], np.int64)
    ql, xh = oracle.reconstruct(sym, spo, g["lt"], g["it"], x, off, round_mode=1)
    assert ql.tolist() == g["qlen"].astype(int).tolist()
    assert xh.tolist() == g["xhat"].tolist()
    ql0, _ = oracle.reconstruct(sym, spo, g["lt"], g["it"], x, off, round_mode=0)
    assert ql0.tolist() == [2, 1, 1, 3, 3, 2, 1]                      # the two modes differ here


def test_quantize_half_even_dyadic_cumulative_rounding():
    """round_mode 1 with dyadic lengths (exact in binary64): the carry makes
    the value rounded at piece j equal to v_j = (exact cumulative length
    through j) - (quantized lengths before j), so each quantized length is
    v_j rounded to nearest with ties to even, and the cumulative quantized
    length never drifts more than 1/2 from the exact cumulative length.
    (Ties to even do not commute with adding an odd integer, so unlike
    round_mode 0 the cumulative lengths are not simply the rounded exact
    cumulative sums.)"""
    rng = np.random.default_rng(8)
    lt = rng.integers(2, 40, 500) / 2.0                   # multiples of 1/2: many exact ties
    sym = np.arange(500, dtype=np.int32)
    n = int(lt.sum()) + 10
    x = np.zeros(n)
    ql, _ = oracle.reconstruct(sym, np.array([0, 500]), lt, np.zeros(500), x, np.array([0, n]), round_mode=1)
    cum = np.cumsum(lt)
    before = np.concatenate([[0], np.cumsum(ql)[:-1]])
    v = cum - before
    fl = np.floor(v)
    frac = v - fl
    want = np.where(frac > 0.5, fl + 1, np.where(frac < 0.5, fl, fl + (fl % 2)))
    assert np.array_equal(ql, want)
    assert np.any(frac == 0.5) and np.any((frac == 0.5) & (fl % 2 == 1))   # both kinds of tie occur
    assert np.all(np.abs(cum - np.cumsum(ql)) <= 0.5)


def test_quantize_dyadic_cumulative_rounding():
    """With dyadic lengths (exact in FP) the carry makes every cumulative
    length equal to round-half-away of the exact cumulative sum; |e| <= 1/2."""
    rng = np.random.default_rng(7)
    lt = rng.integers(4, 40, 500) / 4.0                   # multiples of 1/4, >= 1
    sym = np.arange(500, dtype=np.int32)
    n = int(lt.sum()) + 10
    x = np.zeros(n)
    ql, _ = oracle.reconstruct(sym, np.array([0, 500]), lt, np.zeros(500), x, np.array([0, n]))
    cum = np.cumsum(lt)
    want = np.floor(cum + 0.5)                             # half away from zero (positive)
    assert np.array_equal(np.cumsum(ql), want)
    assert np.all(np.abs(cum - np.cumsum(ql)) <= 0.5)
    assert ql.min() >= 1


def test_identity_dictionary_reconstructs_chain():
    """With one dictionary entry per piece (exact lengths and increments),
    inverse compression returns the polygonal chain: exact at breakpoints and
    MSE = (1/n) * sum of the Eq. 1 piece errors."""
    x, off, p = synth.make("small", max_series=3)
    b, e, ds = oracle.domains(off, 0, 4)
    ln, inc, po = oracle.compress(x, b, e, p["tol"])
    N = len(ln)
    sym = np.arange(N, dtype=np.int32)
    spo = oracle.series_piece_offsets(off, ds, po)
    ql, xh = oracle.reconstruct(sym, spo, ln.astype(np.float64), inc, x, off)
    assert np.array_equal(ql, ln)
    errs = 0.0
    for d in range(len(b)):
        s = b[d]
        for j in range(po[d], po[d + 1]):
            t = s + ln[j]
            assert abs(xh[t] - x[t]) <= 1e-12
            errs += oracle.piece_error(x, s, t)
            s = t
    assert abs(oracle.mse(x, xh) - errs / len(x)) <= 1e-12 * max(1.0, errs / len(x))


def _setup_small():
    x, off, p = synth.make("small", max_series=4)
    r = oracle.pipeline(x, off, p["tol"], p["alpha"], p["scl"], p["domain_mode"], p["domain_value"])
    return x, off, r


def _jacobian(x, off, r):
    """Dense d xhat / d dict_inc built point by point from the chain definition."""
    k = len(r["dict_inc"])
    A = np.zeros((len(x), k))
    spo = r["series_piece_off"]
    for s in range(len(off) - 1):
        o, n_s = int(off[s]), int(off[s + 1] - off[s])
        pos = 0
        for j in range(spo[s], spo[s + 1]):
            L = int(r["qlen"][j])
            c = int(r["symbol"][j])
            for q in range(1, L + 1):
                if pos + q <= n_s - 1:
                    A[o + pos + q, c] += q / L
            A[o + pos + L + 1:o + n_s, c] += 1.0
            pos += L
    return A


def test_gradient_closed_form_and_fd():
    x, off, r = _setup_small()
    k = len(r["dict_inc"])
    g = oracle.reconstruct_grad(x, r["xhat"], r["symbol"], r["qlen"], r["series_piece_off"], off, k)
    A = _jacobian(x, off, r)
    b = r["xhat"] - A @ r["dict_inc"]                      # affine offset
    assert np.allclose(A @ r["dict_inc"] + b, r["xhat"], atol=1e-12)
    closed = (2.0 / len(x)) * A.T @ (r["xhat"] - x)
    assert np.allclose(g, closed, rtol=1e-9, atol=1e-14)
    # central finite differences, h = 1e-6 (the MSE is quadratic: exact up to rounding)
    rng = np.random.default_rng(0)
    for c in rng.choice(k, 12, replace=False):
        h = 1e-6
        dp = r["dict_inc"].copy(); dp[c] += h
        dm = r["dict_inc"].copy(); dm[c] -= h
        _, xp = oracle.reconstruct(r["symbol"], r["series_piece_off"], r["dict_len"], dp, x, off)
        _, xm = oracle.reconstruct(r["symbol"], r["series_piece_off"], r["dict_len"], dm, x, off)
        fd = (oracle.mse(x, xp) - oracle.mse(x, xm)) / (2 * h)
        assert abs(fd - g[c]) <= 1e-6 * max(abs(g[c]), 1e-6)


def test_gradient_vanishes_at_least_squares_optimum():
    x, off, r = _setup_small()
    k = len(r["dict_inc"])
    A = _jacobian(x, off, r)
    b = r["xhat"] - A @ r["dict_inc"]
    cstar, *_ = np.linalg.lstsq(A, x - b, rcond=None)
    _, xs = oracle.reconstruct(r["symbol"], r["series_piece_off"], r["dict_len"], cstar, x, off)
    gs = oracle.reconstruct_grad(x, xs, r["symbol"], r["qlen"], r["series_piece_off"], off, k)
    g0 = oracle.reconstruct_grad(x, r["xhat"], r["symbol"], r["qlen"], r["series_piece_off"], off, k)
    assert np.abs(gs).max() <= 1e-9 * max(1.0, np.abs(g0).max())
    assert oracle.mse(x, xs) <= r["mse"] + 1e-15
