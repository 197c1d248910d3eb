"""Launch tuning: every launch configuration of the batched kernels computes
the same result bit for bit (checked against the oracle), the autotuner
leaves a valid configuration, and invalid configurations are refused."""
import numpy as np
import pytest

import synth
from _gpu import assert_parity, ctx, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    return ctx()


@pytest.fixture(scope="module")
def sample():
    # the scale-stress mix (walk / sinusoid + AR(1) / level shifts, 4,096-interval
    # domains): domains land in every tile size
    x, off, cfg = synth.make("scale", max_series=120)
    return x, off, cfg, run_oracle(x, off, cfg, recon=False)


CONFIGS = [
    dict(compress_ctas_per_sm=1, compress_pack=0, local_mid_warps=2, local_big_warps=4, merge_ctas_per_sm=1,
         per_domain_launch=0, local_k_warps=4, local_ctas_cap=1, merge_form=0, merge_warps=8),
    dict(compress_ctas_per_sm=2, compress_pack=1, local_mid_warps=8, local_big_warps=8, merge_ctas_per_sm=2,
         per_domain_launch=0, local_k_warps=1, local_ctas_cap=3, merge_form=1, merge_warps=4),
    dict(compress_ctas_per_sm=3, compress_pack=1, local_mid_warps=1, local_big_warps=4, merge_ctas_per_sm=4,
         per_domain_launch=0, local_k_warps=1, local_ctas_cap=0, merge_form=0, merge_warps=4),
    dict(compress_ctas_per_sm=3, compress_pack=1, local_mid_warps=4, local_big_warps=4, merge_ctas_per_sm=4,
         per_domain_launch=0, local_k_warps=4, local_ctas_cap=0, merge_form=1, merge_warps=8),
    # the plain form: one launch per domain for compression and Stage I
    dict(compress_ctas_per_sm=3, compress_pack=1, local_mid_warps=4, local_big_warps=4, merge_ctas_per_sm=4,
         per_domain_launch=1, local_k_warps=1, local_ctas_cap=0, merge_form=1, merge_warps=4),
]


@pytest.mark.parametrize("cfg_t", CONFIGS)
def test_every_configuration_matches_oracle(C, sample, cfg_t):
    x, off, cfg, r = sample
    C.set_tuning(cfg_t)
    assert C.tuning() == cfg_t
    g, *_ = run_gpu(C, x, off, cfg, recon=False)
    assert_parity(g, r, recon=False)


def test_autotune_picks_valid_configuration(C, sample):
    import paper_2401_00109_gb300 as jb
    x, off, cfg, r = sample
    C.set_tuning(dict(per_domain_launch=0))
    C.autotune(True)
    try:
        g, *_ = run_gpu(C, x, off, cfg, recon=False)
    finally:
        C.autotune(False)
    assert_parity(g, r, recon=False)
    t = C.tuning()
    assert t["compress_ctas_per_sm"] in (1, 2, 3) and t["compress_pack"] in (0, 1)
    assert t["local_mid_warps"] in (1, 2, 4, 8) and t["local_big_warps"] in (4, 8)
    assert t["local_k_warps"] in (1, 4)
    assert t["merge_ctas_per_sm"] in (1, 2, 4) and t["per_domain_launch"] == 0 and t["merge_warps"] in (4, 8)
    # the configuration chosen keeps producing the oracle's result
    g, *_ = run_gpu(C, x, off, cfg, recon=False)
    assert_parity(g, r, recon=False)
    for bad in (dict(compress_ctas_per_sm=4), dict(local_mid_warps=3), dict(merge_ctas_per_sm=0),
                dict(per_domain_launch=2), dict(local_k_warps=2), dict(local_ctas_cap=17), dict(merge_form=2),
                dict(merge_warps=6)):
        with pytest.raises(jb.JabbaError):
            C.set_tuning(bad)
    assert C.tuning() == t


def test_plain_form_refused_while_tuning(C, sample):
    import paper_2401_00109_gb300 as jb
    x, off, cfg, r = sample
    C.set_tuning(dict(per_domain_launch=1))
    C.autotune(True)
    try:
        with pytest.raises(jb.JabbaError):
            run_gpu(C, x, off, cfg, recon=False)
    finally:
        C.autotune(False)
        C.set_tuning(dict(per_domain_launch=0))
