"""Host checks of the seeded input generators (no method arithmetic is involved)."""
import numpy as np

from paper_1503_03004_gb300 import synth


def test_affinity_is_symmetric_and_follows_the_recipe():
    n, k = 2500, 20
    p = synth.affinity(n=n, k=k, seed=1003, dtype="f64")
    A = p.M
    assert np.array_equal(A, A.T)
    labels = synth.affinity_labels(n, k, 1003)
    sizes = np.bincount(labels, minlength=k)
    assert sizes.max() - sizes.min() <= 1 and sizes.sum() == n
    same = labels[:, None] == labels[None, :]
    clean = ~p.S0_mask
    assert not np.diag(p.S0_mask).any() and np.array_equal(p.S0_mask, p.S0_mask.T)
    assert abs(p.S0_mask[np.triu_indices(n, 1)].mean() - 0.03) < 0.002
    assert abs(A[same & clean].mean() - 0.8) < 2e-3 and abs(A[same & clean].std() - 0.05) < 2e-3
    assert abs(A[~same & clean].mean() - 0.05) < 1e-3 and abs(A[~same & clean].std() - 0.02) < 1e-3


def test_affinity_row_blocks_match_the_whole_matrix():
    n = 5000   # three 2048-row tiles, the last one ragged
    full = synth.affinity(n=n, k=20, seed=7, dtype="f64").M
    for i0, i1 in ((0, 100), (2000, 2100), (4096, 5000), (1, 4999)):
        A, _ = synth.affinity_rows(n, 20, i0, i1, seed=7)
        assert np.array_equal(A, full[i0:i1])


def test_generators_are_deterministic():
    a = synth.affinity(n=3000, k=20, seed=5, dtype="bf16").M
    b = synth.affinity(n=3000, k=20, seed=5, dtype="bf16").M
    assert np.array_equal(a, b)
    assert np.array_equal(synth.planted(50, 40, 3, p=0.1, amp=1.0, seed=9).M,
                          synth.planted(50, 40, 3, p=0.1, amp=1.0, seed=9).M)
