"""Seeded input generator (no GPU): determinism, sizes, the id bijection, RMAT
quadrant statistics (Sec. VI-A.3: a,b,c,d = .57,.19,.19,.05, edge factor 16),
Erdos-Renyi uniformity and source sampling."""
import numpy as np
import pytest

import graphgen


def test_rmat_sizes_and_determinism():
    s1, d1 = graphgen.rmat_host(12, seed=3)
    s2, d2 = graphgen.rmat_host(12, seed=3)
    s3, _ = graphgen.rmat_host(12, seed=4)
    assert s1.size == 16 * 2**12 and d1.size == s1.size
    assert (s1 == s2).all() and (d1 == d2).all()
    assert not (s1 == s3).all()
    assert s1.min() >= 0 and s1.max() < 2**12 and d1.min() >= 0 and d1.max() < 2**12


def test_rmat_thread_count_does_not_change_output(monkeypatch):
    a = graphgen.rmat_host(15, seed=9)
    monkeypatch.setattr(graphgen, "_threads", lambda: 1)
    b = graphgen.rmat_host(15, seed=9)
    assert (a[0] == b[0]).all() and (a[1] == b[1]).all()


@pytest.mark.parametrize("scale", [0, 1, 2, 5, 8, 13, 16])
def test_permutation_is_bijection(scale):
    n = 1 << scale
    img = np.array([graphgen.perm(scale, 77, x) for x in range(n)])
    assert sorted(img.tolist()) == list(range(n))


def test_permutation_relabels_raw_edges():
    scale = 10
    rs, rd = graphgen.rmat_host(scale, seed=5, permute=False)
    ps, pd = graphgen.rmat_host(scale, seed=5, permute=True)
    table = np.array([graphgen.perm(scale, 5, x) for x in range(1 << scale)])
    assert (table[rs] == ps).all() and (table[rd] == pd).all()


def test_rmat_quadrant_frequencies():
    """Every level of the raw recursion picks quadrant (0,0),(0,1),(1,0),(1,1)
    with probabilities a,b,c,d; 6-sigma binomial bounds per level."""
    scale = 14
    src, dst = graphgen.rmat_host(scale, seed=21, permute=False)
    m = src.size
    probs = np.array(graphgen.RMAT_ABCD)
    for level in range(scale):
        bu = (src >> (scale - 1 - level)) & 1
        bv = (dst >> (scale - 1 - level)) & 1
        q = 2 * bu + bv
        counts = np.bincount(q, minlength=4)
        sigma = np.sqrt(m * probs * (1 - probs))
        assert (np.abs(counts - m * probs) < 6 * sigma).all(), (level, counts)


def test_er_uniform():
    n, m = 1024, 200000
    src, dst = graphgen.er_host(n, m, seed=2)
    assert src.min() >= 0 and src.max() < n
    for x in (src, dst):
        c = np.bincount(x, minlength=n)
        chi2 = ((c - m / n) ** 2 / (m / n)).sum()
        assert chi2 < n + 8 * np.sqrt(2 * n)  # chi-square with n-1 dof, generous bound
    assert abs(np.corrcoef(src, dst)[0, 1]) < 0.02


def test_er_non_power_of_two():
    src, dst = graphgen.er_host(1000, 50000, seed=1)
    assert src.max() < 1000 and dst.max() < 1000 and src.max() > 990


def test_sample_sources():
    src, dst = graphgen.rmat_host(10, seed=1)
    mask = graphgen.nonisolated_mask_host(1 << 10, src, dst)
    want = np.zeros(1 << 10, np.uint8)
    loops = src == dst
    want[src[~loops]] = 1
    want[dst[~loops]] = 1
    assert (mask == want).all()
    s = graphgen.sample_sources(mask, 64, seed=11)
    assert s.size == 64 and np.unique(s).size == 64 and mask[s].all()
    assert (s == graphgen.sample_sources(mask, 64, seed=11)).all()
    small = np.zeros(100, np.uint8)
    small[[3, 50, 99]] = 1
    assert sorted(graphgen.sample_sources(small, 64, seed=1).tolist()) == [3, 50, 99]
