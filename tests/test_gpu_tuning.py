"""Launch-shape tuning table (gbsh_set_lhaf_tuning_ex, gbsh_set_batch_tuning_ex) and the
autotuner on the GPU: every entry evaluates the same subsets; single evaluations agree with
the library default to the compensated sum's rounding and are bit-reproducible under one
entry; batched results are bit-identical under any entry."""
import numpy as np
import pytest

from oracle import lhaf as L
from paper_2010_15595_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _dev(A):
    import torch
    return torch.from_numpy(np.ascontiguousarray(A)).to("cuda")


@pytest.mark.parametrize("prec_name", ["PREC_FP64", "PREC_TF"])
def test_tuned_single_plans_agree(gbsh, prec_name):
    prec = getattr(gbsh, prec_name)
    N = 30
    A = W.single_lhaf_mid(N, seed=5)
    dA = _dev(A)
    ref, _, sq = L.lhaf_subset_stats(A)
    tol = max(1e-9, 512 * 2.0 ** -53 * sq ** 0.5 / abs(ref))  # FP64 gate of the parity tests
    base = gbsh.lhaf(dA, precision=prec)
    vals = []
    try:
        for cfg in [(8, gbsh.LADDER_FINE, 18), (16, gbsh.LADDER_FINE, 12), (10, gbsh.LADDER_COARSE, 9)]:
            gbsh.set_lhaf_tuning(prec, N, *cfg)
            p = gbsh.plan(N, precision=prec)
            assert p["nchunks"] == 2 ** min(cfg[2], N // 2)
            assert p["warps"] <= cfg[0]
            a, b = gbsh.lhaf(dA, precision=prec), gbsh.lhaf(dA, precision=prec)
            assert a == b  # one entry: bit-reproducible
            vals.append(a)
    finally:
        gbsh.set_lhaf_tuning(prec, N)
    assert gbsh.lhaf(dA, precision=prec) == base
    for v in vals:  # regrouped compensated sum: agreement far below the FP64 term error
        assert abs(v - base) <= 1e-13 * abs(base), (v, base)
        assert abs(v - ref) <= tol * abs(ref)


def test_fine_ladder_uses_more_warps(gbsh):
    """The fine ladder gives the mid popcounts more warps per CTA than the coarse one, in
    more classes; both cover every subset once."""
    N = 40
    try:
        gbsh.set_lhaf_tuning(gbsh.PREC_TF, N, 16, gbsh.LADDER_COARSE, 18)
        coarse = gbsh.plan(N, precision=gbsh.PREC_TF)
        gbsh.set_lhaf_tuning(gbsh.PREC_TF, N, 16, gbsh.LADDER_FINE, 18)
        fine = gbsh.plan(N, precision=gbsh.PREC_TF)
    finally:
        gbsh.set_lhaf_tuning(gbsh.PREC_TF, N)
    assert fine["nclass"] >= coarse["nclass"]
    assert fine["kcap"] == coarse["kcap"]  # same first class (16 warps)


def test_visit_once_under_fine_ladder(gbsh):
    try:
        gbsh.set_lhaf_tuning(gbsh.PREC_FP64, 31, 16, gbsh.LADDER_FINE, 7)
        c = gbsh.visit_counts(31).cpu().numpy()
    finally:
        gbsh.set_lhaf_tuning(gbsh.PREC_FP64, 31)
    assert c[0] == 0 and (c[1:] == 1).all()


def test_batch_small_class_warps_bit_identical(gbsh):
    from paper_2010_15595_gb300 import autotune
    mats = autotune.synthetic_batch(13, count=96, seed=11)
    base = gbsh.lhaf_batch(mats)
    try:
        for w0, w1 in [(8, 4), (12, 6), (16, 12)]:
            gbsh.set_batch_tuning(gbsh.PREC_FP64, 13, w1, warps_small=w0)
            assert gbsh.get_batch_tuning(gbsh.PREC_FP64, 13) == (w0, w1)
            assert np.array_equal(gbsh.lhaf_batch(mats), base)
    finally:
        gbsh.set_batch_tuning(gbsh.PREC_FP64, 13, 0, warps_small=0)


def test_autotuner_single_size(gbsh, tmp_path, monkeypatch):
    """A restricted search at N = 24 picks a candidate, applies it, records it, and the cache
    re-applies it in a fresh table state."""
    from paper_2010_15595_gb300 import autotune
    monkeypatch.setenv("GBSH_TUNE_CACHE", str(tmp_path / "tune.json"))
    try:
        r = autotune.tune_lhaf(24, gbsh.PREC_FP64, warps_caps=(8, 12), log2_chunks=(10, 12), reps=1)
        assert gbsh.get_lhaf_tuning(gbsh.PREC_FP64, 24) == tuple(r["best"])
        gbsh.set_lhaf_tuning(gbsh.PREC_FP64, 24)
        assert autotune.apply_cache() == 1
        assert gbsh.get_lhaf_tuning(gbsh.PREC_FP64, 24) == tuple(r["best"])
    finally:
        gbsh.set_lhaf_tuning(gbsh.PREC_FP64, 24)
