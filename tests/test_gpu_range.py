"""Subset-range evaluation (gbsh_lhaf_range_async + gbsh_combine_partials): ranges of the
enumeration that partition [0, 2^n) give partials whose combined sum is the full loop
hafnian -- the split that lets one evaluation run on several GPUs with a single exchange
of 5 doubles per range."""
import numpy as np
import pytest

from oracle import lhaf as L
from paper_2010_15595_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _dev(A):
    import torch
    return torch.from_numpy(np.ascontiguousarray(A)).to("cuda")


@pytest.mark.parametrize("N,prec", [(32, 0), (32, 4), (40, 4), (27, 0)])
def test_ranges_combine_to_full(gbsh, N, prec):
    A = W.single_lhaf_mid(N)
    dA = _dev(A)
    full = gbsh.lhaf(dA, precision=prec)
    n = (N + 1) // 2
    total = 1 << n
    for cuts in ([0, total // 2, total],                     # two halves (chunk-aligned)
                 sorted({0, total // 5 + 3, total // 3 + 7, total - 1, total})):  # uneven, unaligned
        parts = [gbsh.lhaf_range(dA, a, b, precision=prec) for a, b in zip(cuts[:-1], cuts[1:])]
        got = gbsh.partial_value(gbsh.combine_partials(np.array(parts)))
        assert abs(got - full) <= 1e-12 * abs(full), (N, prec, cuts, got, full)
    if N <= 32 and prec == gbsh.PREC_TF:  # the accurate path at the stated tolerance
        ref = L.lhaf_subset_ld(A)
        assert abs(full - ref) <= 1e-9 * abs(ref)


def test_empty_and_bad_ranges(gbsh):
    dA = _dev(W.single_lhaf_mid(20))
    p = gbsh.lhaf_range(dA, 100, 100)
    assert np.all(p == 0)
    with pytest.raises(gbsh.GbshError):
        gbsh.lhaf_range(dA, 10, 5)
    with pytest.raises(gbsh.GbshError):
        gbsh.lhaf_range(dA, 0, (1 << 10) + 1)


def test_rank_split_matches_single_launch(gbsh):
    """The bounds a world of 3 ranks would use, evaluated one after the other on this GPU."""
    A = W.large_lhaf(36)
    dA = _dev(A)
    full = gbsh.lhaf(dA, precision=gbsh.PREC_TF)
    parts = [gbsh.lhaf_range(dA, *gbsh.range_bounds(36, r, 3), precision=gbsh.PREC_TF)
             for r in range(3)]
    got = gbsh.partial_value(gbsh.combine_partials(np.array(parts)))
    assert abs(got - full) <= 1e-12 * abs(full)
