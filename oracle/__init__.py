"""FP64 CPU oracle of the JABBA symbolization path (arXiv 2401.00109).

TEST INFRASTRUCTURE: only the tests, `__graft_entry__.smoke()` and the CPU
baseline leg of `bench.py` use this package.  The product (the CUDA library and
its binding in `paper_2401_00109_gb300`) never imports it, and it imports
nothing from the product.  The arithmetic lives in `jabba_oracle.c` (plain C,
built without fused multiply-add or fast-math); this module only marshals
numpy arrays through ctypes.

Functions follow the paper's steps (section in brackets):
  domains            Alg. 1 Phase I, Sec. 4.1.1
  compress           Eq. 1, Alg. 1 Phase II, Sec. 4.1.2-4.1.3
  sigma              Eq. 4 (normalisation by the standard deviations)
  greedy             Sec. 3.2 greedy aggregation with the Sec. 5 pruning rule
  local_aggregate    Sec. 5 Stage I, one block per domain
  merge              Sec. 5 Stage II, merge of the local groups
  block_digitize     Sec. 5 two-stage digitization in the block form (global
                     sort, contiguous sorted blocks, merge of starting points)
  pca_axis           Sec. 5 "PCA projection" key: first principal axis
  pipeline(key="pca")  the path with the PCA key in Stage I and II
  symbolize          Sec. 5 label propagation
  reconstruct        Sec. 3.3 inverse digitization, quantization, inverse compression
  mse                Sec. 3.3 reconstruction error
  reconstruct_grad   gradient of the MSE w.r.t. the dictionary increments
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jabba_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libjabba_oracle.so")
_lib = None
_lock = threading.Lock()

I64 = C.POINTER(C.c_int64)
I32 = C.POINTER(C.c_int32)
U64 = C.POINTER(C.c_uint64)
F64 = C.POINTER(C.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=gnu11",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            sig = {
                "jo_count_domains": (C.c_int64, [I64, C.c_int64, C.c_int, C.c_int64]),
                "jo_build_domains": (C.c_int64, [I64, C.c_int64, C.c_int, C.c_int64, I64, I64, I32]),
                "jo_piece_error": (C.c_double, [F64, C.c_int64, C.c_int64]),
                "jo_piece_error_l2": (C.c_double, [F64, C.c_int64, C.c_int64]),
                "jo_piece_admissible": (C.c_int, [F64, C.c_int64, C.c_int64, C.c_double]),
                "jo_piece_error_plain": (C.c_double, [F64, C.c_int64, C.c_int64]),
                "jo_piece_admissible_plain": (C.c_int, [F64, C.c_int64, C.c_int64, C.c_double]),
                "jo_piece_end": (C.c_int64, [F64, C.c_int64, C.c_int64, C.c_double, C.c_int]),
                "jo_piece_ends": (None, [F64, I64, I64, C.c_int64, C.c_double, C.c_int, I64, C.c_int]),
                "jo_compress_domain": (C.c_int64, [F64, C.c_int64, C.c_int64, C.c_double, C.c_int, I32, F64]),
                "jo_compress_all": (None, [F64, I64, I64, C.c_int64, I64, C.c_double, C.c_int, I32, F64, I64,
                                           C.c_int]),
                "jo_sigma": (None, [I32, F64, C.c_int64, F64, F64]),
                "jo_pca_axis": (None, [I32, F64, C.c_int64, C.c_double, F64]),
                "jo_greedy": (C.c_int64, [F64, F64, C.c_int64, C.c_double, C.c_int, I64, I64]),
                "jo_greedy_proj": (C.c_int64, [F64, F64, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_int,
                                               I64, I64]),
                "jo_group_sums": (None, [I32, F64, C.c_int64, I64, C.c_int64, I64, I64, U64]),
                "jo_local_aggregate": (C.c_int64, [I32, F64, C.c_int64, C.c_double, C.c_double, C.c_double,
                                                   C.c_double, I32, I64, I64, U64]),
                "jo_centre": (None, [C.c_int64, C.c_int64, U64, F64, F64]),
                "jo_merge": (C.c_int64, [I64, I64, U64, C.c_int64, C.c_double, C.c_double, C.c_double,
                                         C.c_double, I32, F64, F64, I64]),
                "jo_merge_points": (C.c_int64, [F64, F64, I64, I64, U64, C.c_int64, C.c_double, C.c_int,
                                                C.c_double, C.c_double, I32, F64, F64, I64]),
                "jo_symbolize": (None, [I32, I64, I64, C.c_int64, I32, I32]),
                "jo_reassign": (None, [I32, F64, C.c_int64, C.c_double, C.c_double, C.c_double, F64, F64,
                                       C.c_int64, I32]),
                "jo_sse": (C.c_double, [I32, F64, C.c_int64, C.c_double, C.c_double, C.c_double, F64, F64, I32]),
                "jo_reconstruct_series": (None, [I32, C.c_int64, F64, F64, C.c_double, C.c_int64, C.c_int,
                                                 I32, F64]),
                "jo_mse": (C.c_double, [F64, F64, C.c_int64]),
                "jo_reconstruct_grad_series": (None, [F64, F64, I32, I32, C.c_int64, C.c_int64, C.c_double, F64]),
                "jo_fx_sum": (C.c_double, [F64, C.c_int64]),
                "jo_fx_of": (None, [C.c_double, U64]),
                "jo_fx_round": (C.c_double, [U64]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------- domains
def domains(series_off, mode: int, value: int):
    off = _c(series_off, np.int64)
    S = len(off) - 1
    D = lib().jo_count_domains(_p(off, I64), S, mode, value)
    b = np.empty(D, np.int64)
    e = np.empty(D, np.int64)
    s = np.empty(D, np.int32)
    lib().jo_build_domains(_p(off, I64), S, mode, value, _p(b, I64), _p(e, I64), _p(s, I32))
    return b, e, s


# ---------------------------------------------------------------- compression
def piece_error(x, s: int, e: int) -> float:
    x = _c(x, np.float64)
    return lib().jo_piece_error(_p(x, F64), s, e)


_FORMS = {"l2": 0, "plain": 1}


def admissible(x, s: int, e: int, tol: float, form: str = "l2") -> bool:
    x = _c(x, np.float64)
    f = lib().jo_piece_admissible_plain if _FORMS[form] else lib().jo_piece_admissible
    return bool(f(_p(x, F64), s, e, tol))


def piece_error_plain(x, s: int, e: int) -> float:
    """Eq. 1 error of piece (s, e) in the plain reading: residuals from the
    chord summed sequentially in ascending order (binary64)."""
    x = _c(x, np.float64)
    return lib().jo_piece_error_plain(_p(x, F64), s, e)


def piece_ends(x, starts, dom_ends, tol: float, form: str = "plain", threads: int = 1):
    """End that the greedy of Eq. 1 (in the given reading) reaches from each
    start, inside a domain ending at dom_ends[i]."""
    x = _c(x, np.float64)
    s = _c(starts, np.int64)
    e = _c(dom_ends, np.int64)
    out = np.empty(max(len(s), 1), np.int64)
    lib().jo_piece_ends(_p(x, F64), _p(s, I64), _p(e, I64), len(s), tol, _FORMS[form], _p(out, I64), threads)
    return out[:len(s)].copy()


def breakpoint_flips(x, dom_begin, dom_end, piece_len, dom_piece_off, tol: float, threads: int = 1,
                     form: str = "plain"):
    """Compare a chain of pieces (any implementation's, compact layout) with
    the greedy of Eq. 1 in the given reading, decision by decision: from every
    piece start s, the reading's greedy reaches some end e'; where e' differs
    from the chain's end e, the two disagree on the admissibility of (s, t),
    t = min(e, e') + 1 (a breakpoint flip).  Returns a dict with the number of
    pieces checked, the flips, and for each flip (s, t, err, bound) with err
    the reading's Eq. 1 error of (s, t) and bound = (t - s - 1) tol^2."""
    ln = np.asarray(piece_len, np.int64)
    po = np.asarray(dom_piece_off, np.int64)
    cnt = np.diff(po)
    dom_of = np.repeat(np.arange(len(cnt)), cnt)
    csum = np.concatenate([[0], np.cumsum(ln)])               # csum[i] = total length before piece i
    ends = np.asarray(dom_begin, np.int64)[dom_of] + csum[1:] - csum[po[dom_of]]
    starts = ends - ln
    dend = np.asarray(dom_end, np.int64)[dom_of]
    got = piece_ends(x, starts, dend, tol, form, threads)
    bad = np.nonzero(got != ends)[0]
    t2 = tol * tol
    err_f = piece_error_plain if form == "plain" else piece_error
    flips = []
    for i in bad:
        s0 = int(starts[i])
        t = int(min(got[i], ends[i])) + 1
        flips.append((s0, t, err_f(x, s0, t), float((t - s0 - 1) * t2)))
    return {"pieces": int(len(ln)), "flips": flips}


def compress(x, dom_begin, dom_end, tol: float, threads: int = 1, form: str = "l2"):
    """Pieces of every domain, concatenated in domain order (Sec. 4.1.3).
    form = "l2": Eq. 1 multiplied through by L^2 with an exact sum (default);
    form = "plain": the sequential sum of squared residuals as printed.
    Returns (piece_len int32[N], piece_inc float64[N], dom_piece_off int64[D+1])."""
    x = _c(x, np.float64)
    b = _c(dom_begin, np.int64)
    e = _c(dom_end, np.int64)
    D = len(b)
    cap = e - b
    cap_off = np.zeros(D + 1, np.int64)
    np.cumsum(cap, out=cap_off[1:])
    total = int(cap_off[-1])
    ln = np.empty(max(total, 1), np.int32)
    inc = np.empty(max(total, 1), np.float64)
    cnt = np.zeros(max(D, 1), np.int64)
    lib().jo_compress_all(_p(x, F64), _p(b, I64), _p(e, I64), D, _p(cap_off, I64), tol, _FORMS[form],
                          _p(ln, I32), _p(inc, F64), _p(cnt, I64), threads)
    cnt = cnt[:D]
    off = np.zeros(D + 1, np.int64)
    np.cumsum(cnt, out=off[1:])
    idx = np.concatenate([np.arange(cap_off[d], cap_off[d] + cnt[d]) for d in range(D)]) if D else np.zeros(0, np.int64)
    return ln[idx].copy(), inc[idx].copy(), off


# ---------------------------------------------------------------- digitization
def sigma(piece_len, piece_inc):
    ln = _c(piece_len, np.int32)
    inc = _c(piece_inc, np.float64)
    sl = C.c_double()
    si = C.c_double()
    lib().jo_sigma(_p(ln, I32), _p(inc, F64), len(ln), C.byref(sl), C.byref(si))
    return sl.value, si.value


def greedy(X, Y, alpha: float, prune: bool = True, axis=None):
    """Greedy aggregation (Sec. 3.2) in key order: the squared norm, or with
    axis = (vx, vy) the projection on that unit axis (the PCA key)."""
    X = _c(X, np.float64)
    Y = _c(Y, np.float64)
    n = len(X)
    lab = np.empty(max(n, 1), np.int64)
    st = np.empty(max(n, 1), np.int64)
    if axis is None:
        g = lib().jo_greedy(_p(X, F64), _p(Y, F64), n, alpha, int(prune), _p(lab, I64), _p(st, I64))
    else:
        g = lib().jo_greedy_proj(_p(X, F64), _p(Y, F64), n, alpha, float(axis[0]), float(axis[1]), int(prune),
                                 _p(lab, I64), _p(st, I64))
    return lab[:n], st[:g]


def pca_axis(piece_len, piece_inc, sigma_len=None, sigma_inc=None, scl=1.0, with_r=False):
    """First principal axis of the normalised pieces (the PCA key of Sec. 5),
    from exact order-independent sums (jo_pca_axis): normalisation by the
    standard deviations makes the covariance [[scl^2, scl r], [scl r, 1]]
    with r the correlation of length and increment; its leading eigenvector
    by a closed form in binary64, vx > 0.  (sigma_len, sigma_inc are implied
    by the same sums and accepted for the caller's convenience.)"""
    ln = _c(piece_len, np.int32)
    inc = _c(piece_inc, np.float64)
    out = np.zeros(3, np.float64)
    lib().jo_pca_axis(_p(ln, I32), _p(inc, F64), len(ln), float(scl), _p(out, F64))
    ax = (float(out[0]), float(out[1]))
    return (ax, float(out[2])) if with_r else ax


def group_sums(piece_len, piece_inc, labels, G):
    """Exact sums (count, lensum, incacc) of the groups labels[i] in [0, G)."""
    ln = _c(piece_len, np.int32)
    inc = _c(piece_inc, np.float64)
    lab = _c(labels, np.int64)
    cnt = np.empty(max(G, 1), np.int64)
    ls = np.empty(max(G, 1), np.int64)
    ia = np.zeros((max(G, 1), 4), np.uint64)
    lib().jo_group_sums(_p(ln, I32), _p(inc, F64), len(ln), _p(lab, I64), G, _p(cnt, I64), _p(ls, I64),
                        _p(ia, U64))
    return cnt[:G].copy(), ls[:G].copy(), ia[:G].copy()


def normalised(piece_len, piece_inc, sigma_len, sigma_inc, scl):
    """Eq. 4 coordinates, evaluated as the C oracle does."""
    X = (scl * np.asarray(piece_len, np.float64)) / sigma_len
    Y = np.asarray(piece_inc, np.float64) / sigma_inc
    return X, Y


def local_aggregate(piece_len, piece_inc, dom_piece_off, sigma_len, sigma_inc, alpha, scl):
    """Stage I per domain.  Returns (local_label int32[N], dom_group_off int64[D+1],
    grp_count int64[G], grp_lensum int64[G], grp_incacc uint64[G,4])."""
    ln = _c(piece_len, np.int32)
    inc = _c(piece_inc, np.float64)
    off = _c(dom_piece_off, np.int64)
    D = len(off) - 1
    N = len(ln)
    label = np.empty(max(N, 1), np.int32)
    cnt = np.empty(max(N, 1), np.int64)
    ls = np.empty(max(N, 1), np.int64)
    ia = np.zeros((max(N, 1), 4), np.uint64)
    goff = np.zeros(D + 1, np.int64)
    L = lib()
    g = 0
    for d in range(D):
        a, b = int(off[d]), int(off[d + 1])
        n = b - a
        G = L.jo_local_aggregate(
            C.cast(ln.ctypes.data + 4 * a, I32), C.cast(inc.ctypes.data + 8 * a, F64), n,
            sigma_len, sigma_inc, alpha, scl, C.cast(label.ctypes.data + 4 * a, I32),
            C.cast(cnt.ctypes.data + 8 * g, I64), C.cast(ls.ctypes.data + 8 * g, I64),
            C.cast(ia.ctypes.data + 32 * g, U64))
        g += G
        goff[d + 1] = g
    return label[:N].copy(), goff, cnt[:g].copy(), ls[:g].copy(), ia[:g].copy()


def centre(count: int, lensum: int, incacc):
    ia = _c(incacc, np.uint64)
    cl = C.c_double()
    ci = C.c_double()
    lib().jo_centre(count, lensum, _p(ia, U64), C.byref(cl), C.byref(ci))
    return cl.value, ci.value


def merge(grp_count, grp_lensum, grp_incacc, sigma_len, sigma_inc, alpha, scl):
    """Stage II.  Returns (l2g int32[G], dict_len, dict_inc, dict_count)."""
    cnt = _c(grp_count, np.int64)
    ls = _c(grp_lensum, np.int64)
    ia = _c(grp_incacc, np.uint64).reshape(-1, 4)
    G = len(cnt)
    l2g = np.empty(max(G, 1), np.int32)
    dl = np.empty(max(G, 1), np.float64)
    di = np.empty(max(G, 1), np.float64)
    dc = np.empty(max(G, 1), np.int64)
    k = lib().jo_merge(_p(cnt, I64), _p(ls, I64), _p(ia, U64), G, sigma_len, sigma_inc, alpha, scl,
                       _p(l2g, I32), _p(dl, F64), _p(di, F64), _p(dc, I64))
    return l2g[:G].copy(), dl[:k].copy(), di[:k].copy(), dc[:k].copy()


def merge_points(X, Y, grp_count, grp_lensum, grp_incacc, alpha, axis=None):
    """Stage II over given points of the local groups (their starting points
    in the block form, their centres with the PCA key); axis as in greedy.
    Returns (l2g int32[G], dict_len, dict_inc, dict_count)."""
    X = _c(X, np.float64)
    Y = _c(Y, np.float64)
    cnt = _c(grp_count, np.int64)
    ls = _c(grp_lensum, np.int64)
    ia = _c(grp_incacc, np.uint64).reshape(-1, 4)
    G = len(cnt)
    l2g = np.empty(max(G, 1), np.int32)
    dl = np.empty(max(G, 1), np.float64)
    di = np.empty(max(G, 1), np.float64)
    dc = np.empty(max(G, 1), np.int64)
    mode, vx, vy = (0, 0.0, 0.0) if axis is None else (1, float(axis[0]), float(axis[1]))
    k = lib().jo_merge_points(_p(X, F64), _p(Y, F64), _p(cnt, I64), _p(ls, I64), _p(ia, U64), G, alpha, mode, vx,
                              vy, _p(l2g, I32), _p(dl, F64), _p(di, F64), _p(dc, I64))
    return l2g[:G].copy(), dl[:k].copy(), di[:k].copy(), dc[:k].copy()


def block_digitize(piece_len, piece_inc, sigma_len, sigma_inc, alpha, scl, n_blocks):
    """Two-stage digitization as Sec. 5 states it (the block form): one
    global sort of the normalised pieces by the key rho = X*X + Y*Y (binary64,
    equal keys in compact-piece order); the sorted order cut into n_blocks
    contiguous blocks of ceil(N / n_blocks) pieces (the last ones shorter or
    empty); Stage I aggregates each block by the greedy in its sorted order;
    Stage II merges the local groups' starting points (the first piece of
    each group in key order) by the same greedy; symbols by label
    propagation, returned in compact-piece order.  Returns a dict."""
    ln = _c(piece_len, np.int32)
    inc = _c(piece_inc, np.float64)
    N = len(ln)
    X, Y = normalised(ln, inc, sigma_len, sigma_inc, scl)
    key = X * X + Y * Y
    order = np.lexsort((np.arange(N), key)).astype(np.int64)   # compact index at sorted position
    B = -(-N // n_blocks) if N else 0
    blk_off = np.minimum(np.arange(n_blocks + 1, dtype=np.int64) * B, N)
    lab, goff, cnt, ls, ia = local_aggregate(ln[order], inc[order], blk_off, sigma_len, sigma_inc, alpha, scl)
    G = len(cnt)
    start = np.empty(G, np.int64)       # sorted position of each local group's start
    for b in range(n_blocks):
        a0, a1 = int(blk_off[b]), int(blk_off[b + 1])
        seen = set()
        for i in range(a0, a1):
            g = int(goff[b]) + int(lab[i])
            if g not in seen:
                seen.add(g)
                start[g] = i
    l2g, dl, di, dc = merge_points(X[order[start]], Y[order[start]], cnt, ls, ia, alpha)
    sym_sorted = l2g[goff[np.searchsorted(blk_off, np.arange(N), side="right") - 1] + lab]
    symbol = np.empty(N, np.int32)
    symbol[order] = sym_sorted
    return dict(order=order, blk_piece_off=blk_off, block_label=lab, blk_group_off=goff, grp_count=cnt,
                grp_lensum=ls, grp_incacc=ia, start=start, l2g=l2g, dict_len=dl, dict_inc=di, dict_count=dc,
                symbol=symbol)


def symbolize(local_label, dom_piece_off, dom_group_off, l2g):
    lab = _c(local_label, np.int32)
    po = _c(dom_piece_off, np.int64)
    go = _c(dom_group_off, np.int64)
    m = _c(l2g, np.int32)
    out = np.empty(max(len(lab), 1), np.int32)
    lib().jo_symbolize(_p(lab, I32), _p(po, I64), _p(go, I64), len(po) - 1, _p(m, I32), _p(out, I32))
    return out[:len(lab)].copy()


def reassign(piece_len, piece_inc, sigma_len, sigma_inc, scl, dict_len, dict_inc):
    """Full-reassignment digitization (Alg. 1 Digitize; Sec. 3.2 argmin): the
    index of the nearest dictionary entry of every piece, ties to the smaller
    index."""
    ln = _c(piece_len, np.int32)
    inc = _c(piece_inc, np.float64)
    dl = _c(dict_len, np.float64)
    di = _c(dict_inc, np.float64)
    out = np.empty(max(len(ln), 1), np.int32)
    lib().jo_reassign(_p(ln, I32), _p(inc, F64), len(ln), float(sigma_len), float(sigma_inc), float(scl),
                      _p(dl, F64), _p(di, F64), len(dl), _p(out, I32))
    return out[:len(ln)].copy()


def sse(piece_len, piece_inc, sigma_len, sigma_inc, scl, dict_len, dict_inc, symbol):
    """Sum of squared normalised distances of the pieces to their entries,
    summed exactly (2^-64 fixed point) and rounded once."""
    ln = _c(piece_len, np.int32)
    inc = _c(piece_inc, np.float64)
    dl = _c(dict_len, np.float64)
    di = _c(dict_inc, np.float64)
    sym = _c(symbol, np.int32)
    return lib().jo_sse(_p(ln, I32), _p(inc, F64), len(ln), float(sigma_len), float(sigma_inc), float(scl),
                        _p(dl, F64), _p(di, F64), _p(sym, I32))


# ---------------------------------------------------------------- inverse symbolization
def series_piece_offsets(series_off, dom_series, dom_piece_off):
    """First piece of each series (its domains are consecutive)."""
    S = len(series_off) - 1
    dom_series = np.asarray(dom_series, np.int64)
    first = np.searchsorted(dom_series, np.arange(S + 1), side="left")
    return np.asarray(dom_piece_off, np.int64)[first]


def reconstruct(symbol, series_piece_off, dict_len, dict_inc, x, series_off, round_mode: int = 0):
    """Returns (qlen int32[N], xhat float64[n])."""
    sym = _c(symbol, np.int32)
    spo = _c(series_piece_off, np.int64)
    dl = _c(dict_len, np.float64)
    di = _c(dict_inc, np.float64)
    x = _c(x, np.float64)
    off = _c(series_off, np.int64)
    qlen = np.zeros(max(len(sym), 1), np.int32)
    xhat = np.zeros(max(len(x), 1), np.float64)
    L = lib()
    for s in range(len(off) - 1):
        a, b = int(spo[s]), int(spo[s + 1])
        n_s = int(off[s + 1] - off[s])
        if n_s <= 0:
            continue
        L.jo_reconstruct_series(C.cast(sym.ctypes.data + 4 * a, I32), b - a, _p(dl, F64), _p(di, F64),
                                float(x[off[s]]), n_s, round_mode, C.cast(qlen.ctypes.data + 4 * a, I32),
                                C.cast(xhat.ctypes.data + 8 * int(off[s]), F64))
    return qlen[:len(sym)].copy(), xhat[:len(x)].copy()


def mse(x, xhat) -> float:
    x = _c(x, np.float64)
    xh = _c(xhat, np.float64)
    return lib().jo_mse(_p(x, F64), _p(xh, F64), len(x))


def reconstruct_grad(x, xhat, symbol, qlen, series_piece_off, series_off, k: int):
    """d MSE / d dict_inc (float64[k]) with the quantized lengths held fixed."""
    x = _c(x, np.float64)
    xh = _c(xhat, np.float64)
    sym = _c(symbol, np.int32)
    ql = _c(qlen, np.int32)
    spo = _c(series_piece_off, np.int64)
    off = _c(series_off, np.int64)
    grad = np.zeros(max(k, 1), np.float64)
    L = lib()
    n_total = float(len(x))
    for s in range(len(off) - 1):
        a, b = int(spo[s]), int(spo[s + 1])
        o = int(off[s])
        n_s = int(off[s + 1]) - o
        if n_s <= 0:
            continue
        L.jo_reconstruct_grad_series(C.cast(x.ctypes.data + 8 * o, F64), C.cast(xh.ctypes.data + 8 * o, F64),
                                     C.cast(sym.ctypes.data + 4 * a, I32), C.cast(ql.ctypes.data + 4 * a, I32),
                                     b - a, n_s, n_total, _p(grad, F64))
    return grad[:k].copy()


# ---------------------------------------------------------------- fixed point (tests)
def fx_sum(values) -> float:
    v = _c(values, np.float64)
    return lib().jo_fx_sum(_p(v, F64), len(v))


def fx_of(value: float) -> int:
    limbs = np.zeros(4, np.uint64)
    lib().jo_fx_of(float(value), _p(limbs, U64))
    u = sum(int(limbs[i]) << (64 * i) for i in range(4))
    return u - (1 << 256) if u >> 255 else u


def fx_round(limbs) -> float:
    lm = _c(limbs, np.uint64)
    return lib().jo_fx_round(_p(lm, U64))


def fx_value(limbs) -> int:
    """Signed integer value (in units of 2^-64) of 4 little-endian limbs."""
    u = sum(int(limbs[i]) << (64 * i) for i in range(4))
    return u - (1 << 256) if u >> 255 else u


# ---------------------------------------------------------------- whole path
def local_aggregate_pca(piece_len, piece_inc, dom_piece_off, sigma_len, sigma_inc, alpha, scl, axis):
    """Stage I per domain with the PCA key (projection on `axis`); outputs as
    local_aggregate."""
    ln = _c(piece_len, np.int32)
    inc = _c(piece_inc, np.float64)
    off = _c(dom_piece_off, np.int64)
    X, Y = normalised(ln, inc, sigma_len, sigma_inc, scl)
    label = np.empty(len(ln), np.int32)
    goff = np.zeros(len(off), np.int64)
    sums = []
    for d in range(len(off) - 1):
        a, b = int(off[d]), int(off[d + 1])
        lab, st = greedy(X[a:b], Y[a:b], alpha, True, axis)
        label[a:b] = lab
        sums.append(group_sums(ln[a:b], inc[a:b], lab, len(st)))
        goff[d + 1] = goff[d] + len(st)
    cnt = np.concatenate([s_[0] for s_ in sums]) if sums else np.zeros(0, np.int64)
    ls = np.concatenate([s_[1] for s_ in sums]) if sums else np.zeros(0, np.int64)
    ia = np.concatenate([s_[2] for s_ in sums]) if sums else np.zeros((0, 4), np.uint64)
    return label, goff, cnt, ls, ia


def pipeline(x, series_off, tol, alpha, scl=1.0, domain_mode=0, domain_value=4, threads=1,
             with_reconstruct=True, round_mode=0, key="norm"):
    """The whole forward path on one collection; returns a dict of every
    stage.  key = "pca": Stage I and II sort by the projection on the first
    principal axis of the normalised pieces (pca_axis) instead of the norm."""
    b, e, ds = domains(series_off, domain_mode, domain_value)
    ln, inc, po = compress(x, b, e, tol, threads)
    sl, si = sigma(ln, inc)
    axis = None
    if key == "pca":
        axis = pca_axis(ln, inc, sl, si, scl)
        lab, go, gc, gl, gi = local_aggregate_pca(ln, inc, po, sl, si, alpha, scl, axis)
        # local centres, normalised (Eq. 4) as in jo_merge
        cX, cY = np.empty(len(gc)), np.empty(len(gc))
        for g in range(len(gc)):
            cl, ci = centre(int(gc[g]), int(gl[g]), gi[g])
            cX[g] = (scl * cl) / sl
            cY[g] = ci / si
        l2g, dl, di, dc = merge_points(cX, cY, gc, gl, gi, alpha, axis)
    else:
        lab, go, gc, gl, gi = local_aggregate(ln, inc, po, sl, si, alpha, scl)
        l2g, dl, di, dc = merge(gc, gl, gi, sl, si, alpha, scl)
    sym = symbolize(lab, po, go, l2g)
    out = dict(dom_begin=b, dom_end=e, dom_series=ds, piece_len=ln, piece_inc=inc, dom_piece_off=po,
               sigma_len=sl, sigma_inc=si, axis=axis, local_label=lab, dom_group_off=go, grp_count=gc,
               grp_lensum=gl, grp_incacc=gi, l2g=l2g, dict_len=dl, dict_inc=di, dict_count=dc, symbol=sym)
    if with_reconstruct:
        spo = series_piece_offsets(series_off, ds, po)
        ql, xh = reconstruct(sym, spo, dl, di, x, series_off, round_mode)
        out.update(series_piece_off=spo, qlen=ql, xhat=xh, mse=mse(x, xh))
    return out
