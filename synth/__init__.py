"""Seeded synthetic time-series collections shaped like the paper's workloads.

This module only draws random numbers and lays the series out in memory; it
holds none of the symbolization method's arithmetic, so both the CPU oracle
(`oracle/`) and the CUDA path (`paper_2401_00109_gb300/`) take their inputs from
here without sharing any method code.

Layout returned by every generator (CSR over series):
  x          float64[n_total]  all series concatenated
  series_off int64[S + 1]      series s occupies x[series_off[s]:series_off[s+1]]

Every series is z-normalised, (x - mean) / std with the population std, the
preprocessing the paper's experiments assume for symbolic representations.

Workloads (sizes, generators and parameters; paper section in brackets):
  small     16 x 2,000: cumulative N(0,1) walk + 2 sin(2 pi t / 200);
            4 equal domains per series; tol = alpha = 0.1, scl = 1; seed 0.
  uneven    10,000 series, lengths uniform in [500, 50,000]: N(0, 0.5) walk plus
            piecewise-constant level shifts (Poisson(1/1000) jumps per point,
            each N(0, 3)); domains of 1,000 intervals; tol = alpha = 0.05.
  multivar  64 channels x 2^20: 3 sinusoids (period U(50, 5000), amplitude
            U(0.5, 2), phase U(0, 2 pi)) plus stationary AR(1) noise (phi = 0.9,
            innovation std 0.2); 1,024 equal domains per channel; tol = 0.1,
            alpha = 0.2.  Stands in for the UEA multivariate archive [Sec. 7.2].
  diff      1,024 x 10,000, generator as `small`; 4 equal domains per series;
            tol = alpha = 0.1 (dictionary refinement workload).
  scale     100,000 series, lengths log-uniform in [100, 100,000] (rounded);
            each series drawn uniformly from {walk, multivar channel, uneven
            level-shift walk}; domains of 4,096 intervals; tol = alpha = 0.1.
  noise     one series of 100,000 N(0, 1) draws; tol = 0.01, alpha = 0.05;
            the number of equal domains M is the variable of the partition
            sweep [Sec. 7.3] (default 1).
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

EQUAL_COUNT = 0
FIXED_LEN = 1

CONFIGS = {
    "small":    dict(index=0, tol=0.1,  alpha=0.1,  scl=1.0, domain_mode=EQUAL_COUNT, domain_value=4,    seed=0),
    "uneven":   dict(index=1, tol=0.05, alpha=0.05, scl=1.0, domain_mode=FIXED_LEN,   domain_value=1000, seed=1),
    "multivar": dict(index=2, tol=0.1,  alpha=0.2,  scl=1.0, domain_mode=EQUAL_COUNT, domain_value=1024, seed=2),
    "diff":     dict(index=3, tol=0.1,  alpha=0.1,  scl=1.0, domain_mode=EQUAL_COUNT, domain_value=4,    seed=3),
    "scale":    dict(index=4, tol=0.1,  alpha=0.1,  scl=1.0, domain_mode=FIXED_LEN,   domain_value=4096, seed=4),
    "noise":    dict(index=5, tol=0.01, alpha=0.05, scl=1.0, domain_mode=EQUAL_COUNT, domain_value=1,    seed=5),
}


def _znorm(v: np.ndarray) -> np.ndarray:
    v = v - v.mean()
    sd = v.std()
    if sd > 0:
        v /= sd
    return v


def walk_sine(rng: np.random.Generator, n: int) -> np.ndarray:
    """Cumulative N(0,1) walk plus 2 sin(2 pi t / 200), t = 0..n-1."""
    t = np.arange(n, dtype=np.float64)
    return np.cumsum(rng.standard_normal(n)) + 2.0 * np.sin(2.0 * np.pi * t / 200.0)


def walk(rng: np.random.Generator, n: int) -> np.ndarray:
    """Cumulative N(0,1) walk."""
    return np.cumsum(rng.standard_normal(n))


def level_shift_walk(rng: np.random.Generator, n: int) -> np.ndarray:
    """N(0, 0.5) walk plus cumulative level shifts: per point a Poisson(1/1000)
    number of jumps, each N(0, 3)."""
    steps = rng.normal(0.0, 0.5, n)
    counts = rng.poisson(1.0 / 1000.0, n)
    jumps = np.zeros(n)
    hit = counts > 0
    jumps[hit] = rng.standard_normal(int(hit.sum())) * 3.0 * np.sqrt(counts[hit])
    return np.cumsum(steps) + np.cumsum(jumps)


def sines_ar1(rng: np.random.Generator, n: int) -> np.ndarray:
    """Sum of 3 sinusoids (period U(50,5000), amplitude U(0.5,2), phase
    U(0,2 pi)) plus AR(1) noise, phi = 0.9, innovation std 0.2, started from its
    stationary distribution."""
    t = np.arange(n, dtype=np.float64)
    per = rng.uniform(50.0, 5000.0, 3)
    amp = rng.uniform(0.5, 2.0, 3)
    ph = rng.uniform(0.0, 2.0 * np.pi, 3)
    s = np.zeros(n)
    for k in range(3):
        s += amp[k] * np.sin(2.0 * np.pi * t / per[k] + ph[k])
    phi, sd = 0.9, 0.2
    innov = rng.normal(0.0, sd, n)
    innov[0] = rng.normal(0.0, sd / math.sqrt(1.0 - phi * phi))
    try:
        from scipy.signal import lfilter
        ar = lfilter([1.0], [1.0, -phi], innov)
    except ImportError:  # pragma: no cover - scipy is present on both machines
        ar = np.empty(n)
        acc = 0.0
        for i in range(n):
            acc = phi * acc + innov[i]
            ar[i] = acc
    return s + ar


def _lengths(name: str, rng: np.random.Generator) -> np.ndarray:
    if name == "small":
        return np.full(16, 2000, dtype=np.int64)
    if name == "uneven":
        return rng.integers(500, 50000, size=10000, endpoint=True).astype(np.int64)
    if name == "multivar":
        return np.full(64, 1 << 20, dtype=np.int64)
    if name == "diff":
        return np.full(1024, 10000, dtype=np.int64)
    if name == "scale":
        u = rng.uniform(math.log(100.0), math.log(100000.0), size=100000)
        return np.rint(np.exp(u)).astype(np.int64)
    if name == "noise":
        return np.full(1, 100000, dtype=np.int64)
    raise KeyError(name)


def _kind(name: str, rng: np.random.Generator, S: int) -> np.ndarray:
    if name == "scale":
        return rng.integers(0, 3, size=S)
    return np.zeros(S, dtype=np.int64)


def _series(name: str, kind: int, rng: np.random.Generator, n: int) -> np.ndarray:
    if name in ("small", "diff"):
        return walk_sine(rng, n)
    if name == "uneven":
        return level_shift_walk(rng, n)
    if name == "multivar":
        return sines_ar1(rng, n)
    if name == "scale":
        return (walk, sines_ar1, level_shift_walk)[kind](rng, n)
    if name == "noise":
        return rng.standard_normal(n)
    raise KeyError(name)


def make(name: str, max_series: int | None = None, seed: int | None = None,
         threads: int | None = None, out: np.ndarray | None = None):
    """Generate workload `name`; returns (x, series_off, params).

    The series of a workload are independent streams spawned from one
    SeedSequence, so `max_series=k` yields exactly the first k series of the
    full workload (a bounded sample of the same data).  `out`, if given, is a
    float64 buffer (e.g. pinned host memory) of at least n_total elements that
    receives x.
    """
    cfg = dict(CONFIGS[name])
    if seed is None:
        seed = cfg["seed"]
    root = np.random.SeedSequence([seed, cfg["index"]])
    len_ss, kind_ss, ser_ss = root.spawn(3)
    lengths = _lengths(name, np.random.default_rng(len_ss))
    kinds = _kind(name, np.random.default_rng(kind_ss), len(lengths))
    S = len(lengths) if max_series is None else min(max_series, len(lengths))
    lengths = lengths[:S]
    kinds = kinds[:S]
    off = np.zeros(S + 1, dtype=np.int64)
    np.cumsum(lengths, out=off[1:])
    n = int(off[-1])
    x = np.empty(n, dtype=np.float64) if out is None else out[:n]
    children = ser_ss.spawn(S)

    def one(s: int) -> None:
        rng = np.random.default_rng(children[s])
        x[off[s]:off[s + 1]] = _znorm(_series(name, int(kinds[s]), rng, int(lengths[s])))

    if threads is None:
        threads = min(32, os.cpu_count() or 1)
    if threads > 1 and S > 1:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(one, range(S)))
    else:
        for s in range(S):
            one(s)
    cfg.pop("seed")
    cfg.pop("index")
    return x, off, cfg


def sizes(name: str, max_series: int | None = None, seed: int | None = None):
    """(n_series, n_points) of workload `name` (or of its first max_series
    series) without generating the data."""
    cfg = CONFIGS[name]
    if seed is None:
        seed = cfg["seed"]
    root = np.random.SeedSequence([seed, cfg["index"]])
    len_ss, _, _ = root.spawn(3)
    lengths = _lengths(name, np.random.default_rng(len_ss))
    if max_series is not None:
        lengths = lengths[:max_series]
    return len(lengths), int(lengths.sum())


def series_kinds(name: str, seed: int | None = None) -> np.ndarray:
    """Generator index per series (scale workload: 0 walk, 1 sinusoids, 2 level shifts)."""
    cfg = CONFIGS[name]
    if seed is None:
        seed = cfg["seed"]
    root = np.random.SeedSequence([seed, cfg["index"]])
    len_ss, kind_ss, _ = root.spawn(3)
    lengths = _lengths(name, np.random.default_rng(len_ss))
    return _kind(name, np.random.default_rng(kind_ss), len(lengths))
