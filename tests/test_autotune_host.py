"""Autotuner host logic (no GPU): the candidate sets by batch shape and the
signature's bucketing."""
from paper_2004_02484_gb300 import autotune as AT
from paper_2004_02484_gb300 import workloads as wl


def test_large_2d_batches_are_tuned_over_strip_shapes():
    big = wl.heat2d_large_batch(n=2, m=256, horizon=4)
    c = AT.candidates(big, quick=True)
    assert c and all(x["strips"] == 1 for x in c)
    assert {x["strip_rows"] for x in c} == {0, 64}
    assert all(set(AT.solver_opts(dict(x, s_per_solve=1.0))) == set(x) for x in c)


def test_small_batches_are_tuned_over_cluster_shapes():
    small = [wl.heat2d_single()]
    c = AT.candidates(small, quick=True)
    assert c and all("strips" not in x for x in c)
    assert {x["cluster"] for x in c} == {0, 2, 4, 8}
    oned = wl.heat1d_ragged_batch(8)
    assert {x["cluster"] for x in AT.candidates(oned)} == {0, 1}


def test_signature_buckets_sizes_and_separates_precisions():
    a = wl.heat1d_ragged_batch(16)
    b = wl.heat1d_ragged_batch(17)
    assert AT.signature(a, 1) == AT.signature(b, 1)  # same log2 buckets
    assert AT.signature(a, 1) != AT.signature(a, 0)
