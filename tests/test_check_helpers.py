"""The device-side check helpers of the GPU tests, run on CPU tensors against
the oracle: the 2^-64 fixed-point chunks of an increment equal the oracle's
fixed-point image, the exact-mean dictionary check accepts the oracle's
dictionary and rejects one increment moved by one ulp, and the flip log
records a clean chain."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")


def test_fx_chunks_match_oracle():
    from _gpu import _fx_chunks
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.standard_normal(600) * 10.0 ** rng.integers(-20, 9, 600),
                        [0.0, -0.0, 5e-324, 2.0**31 - 1, -3.0, 2.0**-64, 2.0**-65, 1.5 * 2.0**-64]])
    ch, neg = _fx_chunks(torch, torch.from_numpy(v))
    for i in range(len(v)):
        mag = int(ch[0][i]) + (int(ch[1][i]) << 32) + (int(ch[2][i]) << 64)
        assert (-mag if bool(neg[i]) else mag) == oracle.fx_of(v[i]), v[i]


def test_dictionary_check_on_oracle_output():
    from _gpu import check_dictionary_exact
    x, off, cfg = synth.make("small")
    r = oracle.pipeline(x, off, cfg["tol"], cfg["alpha"], cfg["scl"], cfg["domain_mode"], cfg["domain_value"],
                        with_reconstruct=False)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a))
    check_dictionary_exact(t(r["piece_len"]), t(r["piece_inc"]), t(r["symbol"]), t(r["dict_len"]), t(r["dict_inc"]),
                           t(r["dict_count"]))
    bad = r["dict_inc"].copy()
    bad[3] = np.nextafter(bad[3], 1.0)
    with pytest.raises(AssertionError):
        check_dictionary_exact(t(r["piece_len"]), t(r["piece_inc"]), t(r["symbol"]), t(r["dict_len"]), t(bad),
                               t(r["dict_count"]))


def test_flip_check_logs_clean_chain():
    from _gpu import FLIP_LOG, check_flips
    x, off, cfg = synth.make("small", max_series=3)
    b, e, _ = oracle.domains(off, cfg["domain_mode"], cfg["domain_value"])
    ln, _, po = oracle.compress(x, b, e, cfg["tol"])
    n0 = len(FLIP_LOG)
    r = check_flips("oracle chain", x, b, e, ln, po, cfg["tol"], threads=2)
    assert r["flips"] == [] and FLIP_LOG[n0:] == [("oracle chain", len(ln), 0)]
    FLIP_LOG.pop()
