"""Pins for the oracle's domain construction and compression (Alg. 1 Phases
I-II, Sec. 3.1 Eq. 1, Sec. 4.1).  Checks use exact rational arithmetic,
hand-derived fixtures and invariants, never the oracle's own formula."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from _golden import load


def exact_err(x, s, e):
    """Eq. 1 sum over the interior points in exact rational arithmetic."""
    L = e - s
    xs, xe = Fraction(x[s]), Fraction(x[e])
    tot = Fraction(0)
    for k in range(1, L):
        r = xs + (xe - xs) * Fraction(k, L) - Fraction(x[s + k])
        tot += r * r
    return tot


def breakpoints(b, lens):
    return b + np.concatenate([[0], np.cumsum(lens)])


def test_domains_hand():
    g = load("domains_hand.txt")
    off = g["series_off"].astype(np.int64)
    b, e, s = oracle.domains(off, 0, 4)
    assert b.tolist() == g["equal4_begin"].astype(int).tolist()
    assert e.tolist() == g["equal4_end"].astype(int).tolist()
    assert s.tolist() == g["equal4_series"].astype(int).tolist()
    b, e, s = oracle.domains(off, 1, 4)
    assert b.tolist() == g["fixed4_begin"].astype(int).tolist()
    assert e.tolist() == g["fixed4_end"].astype(int).tolist()
    assert s.tolist() == g["fixed4_series"].astype(int).tolist()


@pytest.mark.parametrize("mode,value", [(0, 1), (0, 3), (0, 1000), (1, 1), (1, 7), (1, 4096)])
def test_domains_cover_and_share_endpoints(mode, value):
    rng = np.random.default_rng(5)
    lens = rng.integers(0, 60, 40)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    b, e, s = oracle.domains(off, mode, value)
    for si in range(len(lens)):
        idx = np.where(s == si)[0]
        n = lens[si]
        if n < 2:
            assert len(idx) == 0
            continue
        assert b[idx[0]] == off[si] and e[idx[-1]] == off[si] + n - 1
        assert np.all(b[idx[1:]] == e[idx[:-1]])          # s_{k+1} = e_k
        assert np.all(e[idx] > b[idx])
        if mode == 1:
            assert np.all(e[idx] - b[idx] <= value)


@pytest.mark.parametrize("form", ["l2", "plain"])
def test_compress_hand(form):
    g = load("compress_hand.txt")
    x = g["x"]
    ln, inc, off = oracle.compress(x, np.array([0]), np.array([len(x) - 1]), float(g["tol"][0]), form=form)
    assert ln.tolist() == g["len"].astype(int).tolist()
    assert inc.tolist() == g["inc"].tolist()


@pytest.mark.parametrize("form", ["l2", "plain"])
def test_tol0_kinks_are_breakpoints(form):
    """Integer-valued piecewise-linear series with integer slopes: residuals
    are exactly zero on each segment, so with tol = 0 the breakpoints are the
    kinks plus the domain boundaries, nothing else."""
    rng = np.random.default_rng(1)
    kinks = [0]
    x = [0.0]
    while len(x) < 400:
        seg = int(rng.integers(1, 30))
        slope = int(rng.integers(-5, 6))
        if seg and slope == 0 and len(kinks) > 1:
            slope = 1
        for _ in range(seg):
            x.append(x[-1] + slope)
        kinks.append(len(x) - 1)
    x = np.array(x)
    # drop "kinks" where the slope did not change
    d = np.diff(x)
    true = [0] + [i for i in range(1, len(x) - 1) if d[i - 1] != d[i]] + [len(x) - 1]
    off = np.array([0, len(x)], np.int64)
    for M in (1, 3, 7):
        b, e, _ = oracle.domains(off, 0, M)
        ln, inc, po = oracle.compress(x, b, e, 0.0, form=form)
        bp = set()
        for dd in range(len(b)):
            lens = ln[po[dd]:po[dd + 1]]
            bp |= set(breakpoints(b[dd], lens).tolist())
        expect = set(true) | set(b.tolist()) | set(e.tolist())
        assert bp == expect


@pytest.mark.parametrize("form", ["l2", "plain"])
@pytest.mark.parametrize("M", [1, 4])
def test_straight_line_one_piece_per_domain(M, form):
    x = 0.25 * np.arange(1000) - 3.0
    off = np.array([0, 1000], np.int64)
    b, e, _ = oracle.domains(off, 0, M)
    ln, inc, po = oracle.compress(x, b, e, 0.01, form=form)
    assert np.all(np.diff(po) == 1)
    assert ln.tolist() == (e - b).tolist()


@pytest.mark.parametrize("form", ["l2", "plain"])
@pytest.mark.parametrize("tol", [0.05, 0.3, 1.0])
def test_pieces_admissible_maximal_exact(tol, form):
    """Every piece satisfies Eq. 1 and (unless it ends at the domain end) the
    next end violates it; both checked in exact rational arithmetic.  Together
    with tiling this characterizes the greedy output."""
    rng = np.random.default_rng(int(tol * 100))
    x = np.cumsum(rng.standard_normal(300)) * 0.3 + np.sin(np.arange(300) / 7.0)
    off = np.array([0, 300], np.int64)
    b, e, _ = oracle.domains(off, 0, 3)
    ln, inc, po = oracle.compress(x, b, e, tol, form=form)
    t2 = Fraction(tol) * Fraction(tol)
    slack = Fraction(1, 10**9)
    for d in range(len(b)):
        lens = ln[po[d]:po[d + 1]]
        bp = breakpoints(b[d], lens)
        assert bp[-1] == e[d]
        for j in range(len(lens)):
            s, t = int(bp[j]), int(bp[j + 1])
            bound = (t - s - 1) * t2
            assert exact_err(x, s, t) <= bound * (1 + slack)
            for tt in range(s + 1, t):                       # every prefix end admissible
                assert exact_err(x, s, tt) <= (tt - s - 1) * t2 * (1 + slack)
            if t < e[d]:
                assert exact_err(x, s, t + 1) >= (t - s) * t2 * (1 - slack)
            assert inc[po[d] + j] == x[t] - x[s]


def test_endpoint_recovery():
    """The chain through the breakpoints is recovered from t_0 and the
    increments (Sec. 3.1): x[s] + cumulative inc matches x at each breakpoint."""
    x, off, p = synth.make("small", max_series=2)
    b, e, _ = oracle.domains(off, 0, 4)
    ln, inc, po = oracle.compress(x, b, e, p["tol"])
    for d in range(len(b)):
        lens = ln[po[d]:po[d + 1]]
        bp = breakpoints(b[d], lens)
        rec = x[b[d]] + np.cumsum(inc[po[d]:po[d + 1]])
        j = np.arange(1, len(lens) + 1)
        assert np.all(np.abs(rec - x[bp[1:]]) <= j * 2.3e-16 * np.abs(x).max() * 4)


def test_piece_error_matches_exact():
    rng = np.random.default_rng(3)
    x = rng.standard_normal(50)
    for s, t in [(0, 5), (3, 40), (10, 11), (0, 49)]:
        ex = float(exact_err(x, s, t))
        for a in (oracle.piece_error(x, s, t), oracle.piece_error_plain(x, s, t)):
            assert abs(a - ex) <= 1e-13 * max(1.0, ex)


def test_forms_agree_away_from_the_bound():
    """The two readings of Eq. 1 (L^2-scaled exact sum, plain sequential sum)
    give the same chain on seeded walks; any breakpoint where they could
    differ must have its error within rounding of the bound."""
    x, off, p = synth.make("small")
    b, e, _ = oracle.domains(off, 0, 4)
    a = oracle.compress(x, b, e, p["tol"], form="l2")
    c = oracle.compress(x, b, e, p["tol"], form="plain")
    for u, v in zip(a, c):
        assert np.array_equal(u, v)
    r = oracle.breakpoint_flips(x, b, e, a[0], a[2], p["tol"], threads=2)
    assert r["pieces"] == len(a[0]) and r["flips"] == []


def test_breakpoint_flips_reports_a_wrong_breakpoint():
    """The flip checker against a planted mistake: a chain whose first piece
    is cut one interval early (every later piece kept, so the chain still
    tiles the domain) is reported at that piece, with an error far from the
    bound."""
    rng = np.random.default_rng(11)
    x = np.cumsum(rng.standard_normal(400)) * 0.3
    off = np.array([0, 400], np.int64)
    b, e, _ = oracle.domains(off, 0, 1)
    ln, inc, po = oracle.compress(x, b, e, 0.5, form="plain")
    assert ln[0] >= 3
    bad = np.concatenate([[ln[0] - 1, 1], ln[1:]]).astype(np.int32)
    r = oracle.breakpoint_flips(x, b, e, bad, np.array([0, len(bad)]), 0.5)
    assert r["pieces"] == len(bad)
    s0, t, err, bound = r["flips"][0]
    assert (s0, t) == (0, int(ln[0]))                   # the cut end: admissible, yet the chain stopped
    assert err <= bound and abs(err - bound) > 1e-12 * bound


def test_compress_threads_identical():
    x, off, p = synth.make("small")
    b, e, _ = oracle.domains(off, 0, 4)
    r1 = oracle.compress(x, b, e, p["tol"], threads=1)
    r4 = oracle.compress(x, b, e, p["tol"], threads=4)
    for a, c in zip(r1, r4):
        assert np.array_equal(a, c)
