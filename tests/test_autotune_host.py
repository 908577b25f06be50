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


def test_mixed_1d_batches_are_tuned_over_line_inner_counts():
    oned = wl.heat1d_ragged_batch(8)
    c = AT.candidates(oned, quick=True, precision=1)
    assert [x["lines"] for x in c] == [0, 0, 0, 2]
    assert {(x["n_lo"], x["n_u_it"]) for x in c[:3]} == {(2, 1), (2, 2), (1, 1)}
    assert all(set(AT.solver_opts(dict(x, s_per_solve=1.0))) == set(x) for x in c)
    # FP64 batches, and batches with a stage beyond the line path, keep the
    # cluster candidates
    assert all("lines" not in x for x in AT.candidates(oned, quick=True, precision=0))
    wide = oned + [wl.heat1d(300, 5, 2, 0.01, seed=5)]
    assert all("lines" not in x for x in AT.candidates(wide, quick=True, precision=1))


def test_signature_buckets_sizes_and_separates_precisions():
    a = wl.heat1d_ragged_batch(16)
    b = wl.heat1d_ragged_batch(17)
    assert AT.signature(a, 1) == AT.signature(b, 1)  # same log2 buckets
    assert AT.signature(a, 1) != AT.signature(a, 0)
