"""CPU-only checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point that include/jabba.h declares; argument errors are
reported synchronously without a GPU."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "jabba.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(jabba_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    import paper_2401_00109_gb300 as jb
    path = jb.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (jabba_\w+)", out))
    names = declared()
    assert len(names) >= 12
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    lib = C.CDLL(path)
    for n in names:
        assert getattr(lib, n)


def test_status_strings_and_plan_on_host():
    import paper_2401_00109_gb300 as jb
    L = jb.load()
    assert L.jabba_status_string(0) == b"ok"
    assert b"capacity" in L.jabba_status_string(2)
    assert b"sm_103a" in L.jabba_version()
    off = np.array([0, 10, 11, 13, 20], np.int64)
    D, slots = jb.Context.plan(off, jb.Params(domain_mode=0, domain_value=4))
    assert (D, slots) == (9, 9 + 0 + 1 + 6)
    D, slots = jb.Context.plan(off, jb.Params(domain_mode=1, domain_value=4))
    assert (D, slots) == (6, 16)
    with pytest.raises(jb.JabbaError):
        jb.Context.plan(off, jb.Params(tol=-1.0))
    with pytest.raises(jb.JabbaError):
        jb.Context.plan(off, jb.Params(domain_value=0))
    with pytest.raises(jb.JabbaError):
        jb.Context.plan(np.array([0, 5, 3], np.int64), jb.Params())


def test_plan_matches_oracle_domains():
    import oracle
    import paper_2401_00109_gb300 as jb
    rng = np.random.default_rng(0)
    lens = rng.integers(0, 500, 300)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    for mode, val in [(0, 1), (0, 7), (1, 33), (1, 4096)]:
        D, slots = jb.Context.plan(off, jb.Params(domain_mode=mode, domain_value=val))
        b, e, s = oracle.domains(off, mode, val)
        assert D == len(b) and slots == int((e - b).sum())


def test_create_without_gpu_fails_loudly():
    import torch
    import paper_2401_00109_gb300 as jb
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        jb.Context()
    h = C.c_void_p()
    assert jb.load().jabba_create(C.byref(h), 0) != 0


def header_params():
    """Parameter counts of the functions that include/jabba.h declares."""
    src = open(os.path.join(ROOT, "include", "jabba.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(jabba_[a-z_]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
        args = m.group(2).strip()
        out[m.group(1)] = 0 if args in ("", "void") else len([a for a in args.split(",") if a.strip()])
    return out


def test_binding_signatures_match_the_header():
    """Every entry point the Python binding declares with ctypes takes as
    many arguments as include/jabba.h says (a binding that drifts from the
    header would pass wrong pointers)."""
    import paper_2401_00109_gb300 as jb
    L = jb.load()
    counts = header_params()
    assert len(counts) >= 20
    checked = 0
    for name, n in counts.items():
        f = getattr(L, name)
        if f.argtypes is None:
            continue
        assert len(f.argtypes) == n, (name, len(f.argtypes), n)
        checked += 1
    assert checked >= 20


def test_noalloc_limits_match_the_header():
    """The Python-side limits of the allocation-free reconstruction are the
    header's #defines (the binding rejects nothing the library would accept
    and the other way round)."""
    import paper_2401_00109_gb300 as jb
    src = open(os.path.join(ROOT, "include", "jabba.h")).read()
    vals = {}
    for name in ("JABBA_NOALLOC_MAX_PIECES", "JABBA_NOALLOC_MAX_SERIES"):
        m = re.search(r"#define\s+" + name + r"\s+\(?\s*1\s*<<\s*(\d+)\s*\)?", src)
        assert m, name
        vals[name] = 1 << int(m.group(1))
    assert jb.NOALLOC_MAX_PIECES == vals["JABBA_NOALLOC_MAX_PIECES"]
    assert jb.NOALLOC_MAX_SERIES == vals["JABBA_NOALLOC_MAX_SERIES"]
