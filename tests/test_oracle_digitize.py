"""Pins for the oracle's normalisation, greedy aggregation, two-stage merge and
label propagation (Sec. 3.2 Eqs. 4-9, Sec. 5).  Checks use exact sums
(math.fsum / Fraction), numpy's own std, hand fixtures, brute force and the
invariants that characterize the greedy."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from _golden import load


def test_fixed_point_exact():
    rng = np.random.default_rng(0)
    for v in list(rng.standard_normal(200) * 10.0 ** rng.integers(-20, 15, 200)) + [0.0, -0.0, 1.5, -2.75, 2.0**-64, -(2.0**-65)]:
        got = oracle.fx_of(v)
        f = Fraction(v) * 2**64
        want = math.floor(f) if f >= 0 else -math.floor(-f)            # truncate toward zero
        assert got == want
    # multiples of 2^-40: no bits below the 2^-64 resolution, so the fixed-point
    # total is the exact sum, and its rounding must equal math.fsum's
    vals = np.round(rng.standard_normal(10000) * 3.0 * 2**40) / 2**40
    assert oracle.fx_sum(vals) == math.fsum(vals)                    # correctly rounded exact sum
    vals = np.concatenate([vals, -vals[:5000], [1e10, -1e10, 0.125]])
    assert oracle.fx_sum(vals) == math.fsum(vals)
    assert oracle.fx_sum(np.array([1.0, 2.0**-60, 2.0**-60])) == 1.0 + 2.0**-59


def test_fixed_point_rounding_ties_even():
    # 2^53 + 1 (in units of 2^-64) is a tie between 2^53 and 2^53 + 2
    u = (2**53 + 1)
    limbs = np.array([u & (2**64 - 1), u >> 64, 0, 0], np.uint64)
    assert oracle.fx_round(limbs) == float(2**53) * 2.0**-64
    u = (2**53 + 3)
    limbs = np.array([u, 0, 0, 0], np.uint64)
    assert oracle.fx_round(limbs) == float(2**53 + 4) * 2.0**-64
    neg = (1 << 256) - (2**54 + 1)                                   # -(2^54 + 1): rounds to -2^54
    limbs = np.array([(neg >> (64 * i)) & (2**64 - 1) for i in range(4)], np.uint64)
    assert oracle.fx_round(limbs) == -float(2**54) * 2.0**-64
    big = (2**70 + 2**17 + 1) << 3                                   # above-half remainder rounds up
    limbs = np.array([(big >> (64 * i)) & (2**64 - 1) for i in range(4)], np.uint64)
    assert oracle.fx_round(limbs) == float(Fraction(big, 2**64))


def test_sigma_population_std():
    x, off, p = synth.make("small")
    b, e, _ = oracle.domains(off, 0, 4)
    ln, inc, po = oracle.compress(x, b, e, p["tol"])
    sl, si = oracle.sigma(ln, inc)
    assert abs(sl - np.std(ln.astype(np.float64))) <= 1e-12 * sl
    assert abs(si - np.std(inc)) <= 1e-12 * si
    # exact definition: mean-of-squares minus squared mean from exact sums of
    # inc and of the exact squares, each term truncated at 2^-64
    n = len(ln)

    def trunc64(f):
        f = f * 2**64
        return (math.floor(f) if f >= 0 else -math.floor(-f))

    s1 = float(Fraction(sum(trunc64(Fraction(v)) for v in inc), 2**64))
    s2 = float(Fraction(sum(trunc64(Fraction(v) ** 2) for v in inc), 2**64))
    m = s1 / n
    v = s2 / n - m * m
    assert si == math.sqrt(v)
    assert sl == math.sqrt(float(int((ln.astype(np.int64) ** 2).sum())) / n - (float(int(ln.sum())) / n) ** 2)
    # degenerate: all lengths equal -> sigma_len = 1 (divisor 1)
    assert oracle.sigma(np.full(7, 3, np.int32), np.arange(7.0))[0] == 1.0


def test_greedy_hand():
    g = load("aggregate_hand.txt")
    lab, st = oracle.greedy(g["X"], g["Y"], float(g["alpha"][0]))
    assert lab.tolist() == g["labels"].astype(int).tolist()


def brute_labels(X, Y, alpha):
    """Characterization of the greedy by its invariants, computed by brute
    force in exact rational arithmetic on the FP64 coordinates: in key order,
    a point joins the earliest start before it within alpha, else starts."""
    n = len(X)
    key = [Fraction(X[i]) ** 2 + Fraction(Y[i]) ** 2 for i in range(n)]
    order = sorted(range(n), key=lambda i: (key[i], i))
    a2 = Fraction(alpha) ** 2
    lab = [-1] * n
    starts = []
    for i in order:
        for g, s in enumerate(starts):
            if (Fraction(X[i]) - Fraction(X[s])) ** 2 + (Fraction(Y[i]) - Fraction(Y[s])) ** 2 <= a2:
                lab[i] = g
                break
        else:
            lab[i] = len(starts)
            starts.append(i)
    return np.array(lab)


@pytest.mark.parametrize("seed", range(6))
def test_greedy_matches_bruteforce_and_unpruned(seed):
    rng = np.random.default_rng(seed)
    n = 120
    if seed % 2:
        # points on a dyadic grid with a dyadic alpha: every FP64 operation is
        # exact, so ties at distance exactly alpha occur and must agree
        X = np.round(rng.uniform(0, 1, n) * 64) / 64
        Y = np.round(rng.normal(0, 0.5, n) * 64) / 64
        alpha = [0.0625, 0.125, 0.25][seed % 3]
    else:
        X = rng.uniform(0, 1, n)
        Y = rng.normal(0, 0.5, n)
        alpha = [0.05, 0.1, 0.2][seed % 3]
    lab, st = oracle.greedy(X, Y, alpha, prune=True)
    lab0, _ = oracle.greedy(X, Y, alpha, prune=False)
    assert np.array_equal(lab, lab0)                      # Sec. 5 pruning is lossless
    ref = brute_labels(X, Y, alpha)
    # exact-arithmetic decisions can differ from FP64 only for distances within
    # a few ulp of alpha; these fixtures have none
    assert np.array_equal(lab, ref)


def test_greedy_invariants_and_sse_bound():
    rng = np.random.default_rng(11)
    X = rng.uniform(0, 3, 2000)
    Y = rng.normal(0, 1, 2000)
    alpha = 0.1
    lab, st = oracle.greedy(X, Y, alpha)
    k = len(st)
    P = np.stack([X, Y], 1)
    S = P[st]
    d2 = ((P - S[lab]) ** 2).sum(1)
    assert np.all(d2 <= alpha * alpha * (1 + 1e-12))             # members within alpha of start
    dd = ((S[:, None, :] - S[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(dd, np.inf)
    assert np.all(dd > alpha * alpha)                              # starts pairwise > alpha apart
    sse = 0.0
    for g in range(k):
        m = P[lab == g]
        c = m.mean(0)
        var = ((m - c) ** 2).sum(1).mean()
        assert var <= alpha * alpha * (1 + 1e-12)                  # Eq. 9: Var <= alpha^2
        sse += ((m - c) ** 2).sum()
    assert sse <= alpha * alpha * (len(X) - k) * (1 + 1e-12)       # SSE <= alpha^2 (N - k)


def test_greedy_degenerate():
    X = np.array([0.0, 1.0, 1.0, 0.0, 2.0])
    Y = np.array([0.0, 1.0, 1.0, 0.0, 2.0])
    lab, st = oracle.greedy(X, Y, 0.0)                            # alpha = 0: exact duplicates only
    assert lab.tolist() == [0, 1, 1, 0, 2]
    # scl = 0 ignores lengths (Eq. 4)
    X0, Y0 = oracle.normalised(np.array([1, 50, 3]), np.array([0.1, 0.1, 0.5]), 2.0, 1.0, 0.0)
    assert np.all(X0 == 0.0)
    lab, _ = oracle.greedy(X0, Y0, 0.01)
    assert lab[0] == lab[1] != lab[2]


def test_exhaustive_optimal_grouping_tiny():
    """On <= 7 points, no partition into groups of radius alpha (around one of
    their points) uses fewer groups than... the greedy is a cover: k_opt <= k_greedy
    and the greedy SSE is no better than the optimum over all alpha-partitions."""
    rng = np.random.default_rng(2)
    for trial in range(8):
        n = 6
        X = rng.uniform(0, 0.3, n)
        Y = rng.uniform(0, 0.3, n)
        alpha = 0.12
        lab, st = oracle.greedy(X, Y, alpha)
        P = np.stack([X, Y], 1)

        def partitions(items):
            if not items:
                yield []
                return
            first, rest = items[0], items[1:]
            for p in partitions(rest):
                for i in range(len(p)):
                    yield p[:i] + [[first] + p[i]] + p[i + 1:]
                yield [[first]] + p

        best_k, best_sse = n + 1, math.inf
        for part in partitions(list(range(n))):
            ok = all(any(all(((P[m] - P[c]) ** 2).sum() <= alpha ** 2 for m in grp) for c in grp) for grp in part)
            if not ok:
                continue
            sse = sum(((P[grp] - P[grp].mean(0)) ** 2).sum() for grp in part)
            if len(part) < best_k or (len(part) == best_k and sse < best_sse):
                best_k, best_sse = len(part), sse
        assert best_k <= len(st)
        g_sse = sum(((P[lab == g] - P[lab == g].mean(0)) ** 2).sum() for g in range(len(st)))
        if best_k == len(st):
            assert best_sse <= g_sse + 1e-15


def test_two_stage_small_config():
    x, off, p = synth.make("small")
    r = oracle.pipeline(x, off, p["tol"], p["alpha"], p["scl"], p["domain_mode"], p["domain_value"])
    po, go = r["dom_piece_off"], r["dom_group_off"]
    N = len(r["piece_len"])
    # label propagation = composition (Sec. 5)
    for d in range(len(po) - 1):
        for q in range(po[d], po[d + 1]):
            assert r["symbol"][q] == r["l2g"][go[d] + r["local_label"][q]]
    # every dictionary entry is the exact mean of its member pieces
    k = len(r["dict_len"])
    assert r["dict_count"].sum() == N
    for c in range(k):
        m = r["symbol"] == c
        assert r["dict_count"][c] == m.sum()
        assert r["dict_len"][c] == float(Fraction(int(r["piece_len"][m].sum()), int(m.sum())))
        assert r["dict_inc"][c] == math.fsum(r["piece_inc"][m]) / float(m.sum())
    # local groups: exact sums of their pieces
    for d in range(0, len(po) - 1, 7):
        for g in range(go[d], go[d + 1]):
            m = np.zeros(N, bool)
            m[po[d]:po[d + 1]] = r["local_label"][po[d]:po[d + 1]] == g - go[d]
            assert r["grp_count"][g] == m.sum()
            assert r["grp_lensum"][g] == r["piece_len"][m].sum()
            assert oracle.fx_value(r["grp_incacc"][g]) == sum(oracle.fx_of(v) for v in r["piece_inc"][m])


def test_merge_singletons_equal_local():
    """One domain with alpha below every pairwise distance: every local group is
    a singleton and the merge reproduces the single-stage greedy."""
    rng = np.random.default_rng(4)
    ln = rng.integers(1, 40, 200).astype(np.int32)
    inc = rng.standard_normal(200)
    sl, si = oracle.sigma(ln, inc)
    po = np.array([0, 200], np.int64)
    lab, go, gc, gl, gi = oracle.local_aggregate(ln, inc, po, sl, si, 0.0, 1.0)
    l2g, dl, di, dc = oracle.merge(gc, gl, gi, sl, si, 0.0, 1.0)
    X, Y = oracle.normalised(ln, inc, sl, si, 1.0)
    ref, _ = oracle.greedy(X, Y, 0.0)
    sym = oracle.symbolize(lab, po, go, l2g)
    # identical points (same len, inc) are merged either way; partitions must agree
    assert np.array_equal(sym, ref)


def test_merge_alpha0_merges_identical_only():
    gc = np.array([1, 2, 1, 3], np.int64)
    gl = np.array([5, 10, 5, 9], np.int64)
    def limbs(v):
        u = oracle.fx_of(v) % (1 << 256)
        return np.array([(u >> (64 * i)) & (2**64 - 1) for i in range(4)], np.uint64)
    gi = np.stack([limbs(v) for v in [1.0, 2.0, 1.0, 0.5]])
    l2g, dl, di, dc = oracle.merge(gc, gl, gi, 1.0, 1.0, 0.0, 1.0)
    assert l2g[0] == l2g[1] == l2g[2] != l2g[3]          # centres (5, 1) x3 identical; (3, 1/6) differs
    # the centre (3, 1/6) has the smaller norm, so its global group is created first
    assert l2g[3] == 0 and dc.tolist() == [3, 4]


def test_reassign_hand():
    """Full reassignment on the hand-derived fixture (nearest entry, ties to
    the smaller index) and its exact SSE."""
    from _golden import load
    g = load("reassign_hand.txt")
    ln = g["len"].astype(np.int32)
    lab = oracle.reassign(ln, g["inc"], 1.0, 1.0, 1.0, g["dict_len"], g["dict_inc"])
    assert np.array_equal(lab, g["labels"].astype(np.int32))
    assert oracle.sse(ln, g["inc"], 1.0, 1.0, 1.0, g["dict_len"], g["dict_inc"], lab) == g["sse"][0]


@pytest.mark.parametrize("seed", [0, 1])
def test_reassign_matches_vectorized_argmin_and_beats_two_stage(seed):
    """The reassignment equals a vectorised argmin over all entries (same
    binary64 operations; numpy's argmin keeps the first minimum); every piece
    is at least as close to its reassigned entry as to its two-stage entry,
    so the SSE cannot grow; the exact SSE is within n 2^-64 of math.fsum."""
    import math
    import synth
    x, off, cfg = synth.make("small", max_series=6 + seed)
    r = oracle.pipeline(x, off, cfg["tol"], cfg["alpha"], cfg["scl"], cfg["domain_mode"], cfg["domain_value"],
                        with_reconstruct=False)
    sl, si, scl = r["sigma_len"], r["sigma_inc"], cfg["scl"]
    ln, inc = r["piece_len"], r["piece_inc"]
    dl, di = r["dict_len"], r["dict_inc"]
    lab = oracle.reassign(ln, inc, sl, si, scl, dl, di)
    X = (scl * ln.astype(np.float64)) / sl
    Y = inc / si
    Xc = (scl * dl) / sl
    Yc = di / si
    dx = X[:, None] - Xc[None, :]
    dy = Y[:, None] - Yc[None, :]
    d2 = dx * dx + dy * dy
    assert np.array_equal(lab, np.argmin(d2, axis=1).astype(np.int32))
    rows = np.arange(len(ln))
    assert np.all(d2[rows, lab] <= d2[rows, r["symbol"]])
    s_re = oracle.sse(ln, inc, sl, si, scl, dl, di, lab)
    s_two = oracle.sse(ln, inc, sl, si, scl, dl, di, r["symbol"])
    assert s_re <= s_two
    ref = math.fsum(d2[rows, lab])
    assert abs(s_re - ref) <= len(ln) * 2.0**-64 + 2 * math.ulp(ref)


# ---------------------------------------------------------------- block form (Sec. 5 as stated)
def _block_inputs(name="small", max_series=6):
    x, off, cfg = synth.make(name, max_series=max_series)
    b, e, _ = oracle.domains(off, cfg["domain_mode"], cfg["domain_value"])
    ln, inc, po = oracle.compress(x, b, e, cfg["tol"], 4)
    sl, si = oracle.sigma(ln, inc)
    return ln, inc, po, sl, si, cfg


def _exact_means(ln, inc, symbol, k):
    """Dictionary by the definition: per symbol the binary64 mean length and
    the exactly summed, once-rounded increment divided by the count."""
    dl = np.empty(k)
    di = np.empty(k)
    dc = np.zeros(k, np.int64)
    for c in range(k):
        m = symbol == c
        n = int(m.sum())
        dc[c] = n
        dl[c] = float(int(ln[m].astype(np.int64).sum())) / n
        di[c] = float(sum(Fraction(v) for v in inc[m])) / n
    return dl, di, dc


@pytest.mark.parametrize("which", ["one block", "one piece per block"])
def test_block_form_reduces_to_the_plain_greedy(which):
    """With one block, Stage I is the greedy over all pieces and its starts
    are pairwise farther than alpha, so Stage II keeps every one; with one
    piece per block, Stage II is the greedy over all pieces.  Either way the
    block form is the plain greedy of Sec. 3.2 (unpruned here), with the
    exact means as the dictionary."""
    ln, inc, po, sl, si, cfg = _block_inputs()
    N = len(ln)
    M = 1 if which == "one block" else N
    r = oracle.block_digitize(ln, inc, sl, si, cfg["alpha"], cfg["scl"], M)
    X, Y = oracle.normalised(ln, inc, sl, si, cfg["scl"])
    lab, _ = oracle.greedy(X, Y, cfg["alpha"], prune=False)
    assert np.array_equal(r["symbol"], lab.astype(np.int32))
    k = int(lab.max()) + 1
    dl, di, dc = _exact_means(ln, inc, lab, k)
    assert np.array_equal(r["dict_count"], dc)
    assert np.array_equal(r["dict_len"], dl) and np.array_equal(r["dict_inc"], di)


@pytest.mark.parametrize("M", [3, 17, 200])
def test_block_form_invariants(M):
    """Blocks are contiguous ranges of the global key order; in each block
    the members lie within alpha of their local start and the local starts
    are pairwise farther apart; the global starts are pairwise farther than
    alpha and every local start lies within alpha of its global start; the
    dictionary holds the exact means of the pieces of each symbol."""
    ln, inc, po, sl, si, cfg = _block_inputs("uneven", 3)
    a = cfg["alpha"]
    a2 = a * a
    r = oracle.block_digitize(ln, inc, sl, si, a, cfg["scl"], M)
    X, Y = oracle.normalised(ln, inc, sl, si, cfg["scl"])
    key = X * X + Y * Y
    o = r["order"]
    N = len(ln)
    assert np.array_equal(np.sort(o), np.arange(N))
    ks = key[o]
    assert np.all(ks[1:] >= ks[:-1])
    tie = ks[1:] == ks[:-1]
    assert np.all(o[1:][tie] > o[:-1][tie])
    bo, go, lab, st = r["blk_piece_off"], r["blk_group_off"], r["block_label"], r["start"]
    Xs, Ys = X[o], Y[o]
    d2 = lambda i, j: (Xs[j] - Xs[i]) * (Xs[j] - Xs[i]) + (Ys[j] - Ys[i]) * (Ys[j] - Ys[i])
    for b in range(M):
        for i in range(bo[b], bo[b + 1]):
            g = go[b] + lab[i]
            assert bo[b] <= st[g] <= i and d2(st[g], i) <= a2
        starts = [st[g] for g in range(go[b], go[b + 1])]
        for u in range(len(starts)):
            for v in range(u + 1, len(starts)):
                assert d2(starts[u], starts[v]) > a2
    l2g = r["l2g"]
    k = len(r["dict_len"])
    gstart = {}
    for g in np.argsort(ks[st], kind="stable"):
        gstart.setdefault(int(l2g[g]), st[g])
    assert sorted(gstart) == list(range(k))
    gs = [gstart[c] for c in range(k)]
    for g in range(len(st)):
        assert d2(gstart[int(l2g[g])], st[g]) <= a2
    for u in range(k):
        for v in range(u + 1, k):
            assert d2(gs[u], gs[v]) > a2
    dl, di, dc = _exact_means(ln, inc, r["symbol"], k)
    assert np.array_equal(r["dict_count"], dc)
    assert np.array_equal(r["dict_len"], dl) and np.array_equal(r["dict_inc"], di)


# ---------------------------------------------------------------- PCA key (Sec. 5 "norm or PCA projection")
@pytest.mark.parametrize("name,scl", [("small", 1.0), ("uneven", 1.0), ("small", 3.0), ("multivar", 0.25)])
def test_pca_axis_is_the_leading_eigenvector(name, scl):
    """pca_axis against numpy's symmetric eigensolver on the covariance of
    the normalised points; with scl = 1 both variances are 1 and the axis is
    the diagonal (1, sign(r)) / sqrt(2) whatever the correlation r."""
    ln, inc, po, sl, si, cfg = _block_inputs(name, 4)
    ax = np.array(oracle.pca_axis(ln, inc, sl, si, scl))
    X, Y = oracle.normalised(ln, inc, sl, si, scl)
    w, V = np.linalg.eigh(np.cov(np.vstack([X, Y]), bias=True))
    v = V[:, -1] * (1 if V[0, -1] > 0 else -1)
    assert abs(np.hypot(*ax) - 1.0) < 1e-15
    assert np.max(np.abs(ax - v)) < 1e-9
    if scl == 1.0:
        r = np.corrcoef(X, Y)[0, 1]
        assert np.max(np.abs(ax - np.array([1.0, np.sign(r)]) / np.sqrt(2.0))) < 1e-9


@pytest.mark.parametrize("scl", [1.0, 0.5])
def test_pca_correlation_from_exact_sums(scl):
    """The correlation r behind the PCA axis equals the population
    correlation of (len, inc) in exact rational arithmetic (up to the 2^-64
    truncation of the sums and binary64 rounding), and the axis is the
    leading eigenvector of [[scl^2, scl r], [scl r, 1]] (checked against the
    closed form evaluated in exact-enough floating point)."""
    from fractions import Fraction
    rng = np.random.default_rng(12)
    ln = rng.integers(1, 60, 500).astype(np.int32)
    inc = 0.3 * ln * rng.normal(0, 1, 500) + rng.normal(0, 2, 500)
    (vx, vy), r = oracle.pca_axis(ln, inc, scl=scl, with_r=True)
    n = len(ln)
    fl = [Fraction(int(v)) for v in ln]
    fi = [Fraction(float(v)) for v in inc]
    ml, mi = sum(fl) / n, sum(fi) / n
    cov = sum((a - ml) * (b - mi) for a, b in zip(fl, fi)) / n
    vl = sum((a - ml) ** 2 for a in fl) / n
    vi = sum((b - mi) ** 2 for b in fi) / n
    r_exact = float(cov) / (math.sqrt(float(vl)) * math.sqrt(float(vi)))
    assert abs(r - r_exact) <= 1e-12 * abs(r_exact)
    M = np.array([[scl * scl, scl * r], [scl * r, 1.0]])
    w, V = np.linalg.eigh(M)
    v = V[:, -1] * (1 if V[0, -1] > 0 else -1)
    assert np.max(np.abs(np.array([vx, vy]) - v)) < 1e-12
    assert abs(math.hypot(vx, vy) - 1.0) < 1e-15


def test_pca_axis_degenerate():
    ln = np.full(10, 3, np.int32)
    inc = np.full(10, 0.5)
    assert oracle.pca_axis(ln, inc, 1.0, 1.0, 1.0) == (1.0, 0.0)
    assert oracle.pca_axis(ln[:0], inc[:0], 1.0, 1.0, 1.0) == (1.0, 0.0)


@pytest.mark.parametrize("seed", [3, 4])
def test_pca_greedy_order_pruning_and_invariants(seed):
    """The greedy with the projection key: pruning loses nothing (the key
    gap bounds the distance), every start is the first item in key order
    (ties by position) among those no earlier group covers, members lie
    within alpha of their start and the starts are pairwise farther apart."""
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 1, 600)
    Y = 0.5 * X + rng.normal(0, 0.3, 600)
    alpha = 0.3
    th = rng.uniform(0, np.pi)
    ax = (float(np.cos(th)), float(np.sin(th)))
    lab, st = oracle.greedy(X, Y, alpha, True, ax)
    lab0, st0 = oracle.greedy(X, Y, alpha, False, ax)
    assert np.array_equal(lab, lab0) and np.array_equal(st, st0)
    key = ax[0] * X + ax[1] * Y
    order = np.lexsort((np.arange(len(X)), key))
    rank = np.empty(len(X), np.int64)
    rank[order] = np.arange(len(X))
    for g, s in enumerate(st):
        free = np.nonzero(lab >= g)[0]
        assert s == free[np.argmin(rank[free])]
        m = np.nonzero(lab == g)[0]
        assert np.all((X[m] - X[s]) ** 2 + (Y[m] - Y[s]) ** 2 <= alpha * alpha)
    for u in range(len(st)):
        d = (X[st[u + 1:]] - X[st[u]]) ** 2 + (Y[st[u + 1:]] - Y[st[u]]) ** 2
        assert np.all(d > alpha * alpha)


def test_pca_pipeline_exact_means_and_composition():
    """The two-stage path with the PCA key: the symbols are the composition
    of the local labels and the map, and every dictionary entry is the exact
    mean of the pieces of its symbol."""
    x, off, cfg = synth.make("small", max_series=6)
    r = oracle.pipeline(x, off, cfg["tol"], cfg["alpha"], cfg["scl"], cfg["domain_mode"], cfg["domain_value"],
                        key="pca", with_reconstruct=False)
    po, go = r["dom_piece_off"], r["dom_group_off"]
    for d in range(len(po) - 1):
        for p in range(po[d], po[d + 1]):
            assert r["symbol"][p] == r["l2g"][go[d] + r["local_label"][p]]
    k = len(r["dict_len"])
    dl, di, dc = _exact_means(r["piece_len"], r["piece_inc"], r["symbol"], k)
    assert np.array_equal(r["dict_count"], dc)
    assert np.array_equal(r["dict_len"], dl) and np.array_equal(r["dict_inc"], di)


def test_block_form_hand_starts_not_centres():
    """Hand-derived block form (Sec. 5 as stated: the STARTING points are
    merged).  scl = 0 puts every piece at X = 0, sigma_inc = 1 makes Y = inc;
    alpha = 0.1, six pieces in two blocks of three.
      block 0 (keys ascend: 0, .30, .39): start 0 alone; start .30 takes .39
        (gap .09)                               -> groups {0}, {.30, .39}
      block 1 (.42, .60, .65): start .42 alone (.18 to .60); start .60 takes
        .65                                     -> groups {.42}, {.60, .65}
      Stage II over the starts 0, .30, .42, .60: consecutive gaps .30, .12,
        .18 all exceed alpha                    -> four symbols.
    Merging the centres instead would join {.30, .39} (centre .345) with
    {.42} (gap .075 <= alpha): three symbols."""
    inc = np.array([0.0, 0.30, 0.39, 0.42, 0.60, 0.65])
    ln = np.ones(6, np.int32)
    r = oracle.block_digitize(ln, inc, 1.0, 1.0, 0.1, 0.0, 2)
    assert list(r["order"]) == [0, 1, 2, 3, 4, 5]
    assert list(r["symbol"]) == [0, 1, 1, 2, 3, 3]
    assert list(r["dict_count"]) == [1, 2, 1, 2]
    exp = [float(sum(Fraction(v) for v in inc[r["symbol"] == c])) / float((r["symbol"] == c).sum()) for c in range(4)]
    assert list(r["dict_inc"]) == exp and list(r["dict_len"]) == [1.0] * 4
    # the per-domain reading (one domain = one block of all six, centres merged) differs
    lab, goff, cnt, ls, ia = oracle.local_aggregate(ln, inc, np.array([0, 3, 6]), 1.0, 1.0, 0.1, 0.0)
    l2g, dl, di, dc = oracle.merge(cnt, ls, ia, 1.0, 1.0, 0.1, 0.0)
    assert len(dl) == 3 and list(dc) == [1, 3, 2]
