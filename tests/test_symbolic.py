"""Host logic of the symbolic factorization (no GPU): sizes of the block factor and of the dense
supernode on structures whose fill is known in closed form.

Natural ordering of a graph whose edges join every pair j < k with k - j <= b (a band) keeps the
factor inside the band: column j holds c_j = min(b, N - 1 - j) off-diagonal blocks, its parent is
j + 1, so the elimination tree is one path and the whole factor is the top chain.  A
left-looking block Cholesky then takes sum_j c_j (c_j + 1) / 2 block products (c_j of them into
diagonal blocks).  The top chain becomes a dense supernode when it has at least 32 block
columns and at least half of its lower-triangle blocks; the stored blocks then number
N + N (N - 1) / 2 (explicit zeros outside the band), while the algorithmic counts stay those of
the band.  Sec. 4.2 / App. E: symbolic analysis once per structure, supernodal numeric factor.
"""
import types

import numpy as np
import pytest

from paper_2207_09442_b300 import layer, synth

D3 = 6  # SE(3) block size


def _band_graph(n, b, kind=3):
    ei, ej = [], []
    for j in range(n):
        for k in range(j + 1, min(n, j + b + 1)):
            ei.append(j)
            ej.append(k)
    ei.append(0)
    ej.append(-1)  # gauge prior on pose 0
    return types.SimpleNamespace(kind=kind, pose_offsets=np.array([0, n], np.int64),
                                 edge_offsets=np.array([0, len(ei)], np.int64),
                                 edge_i=np.array(ei, np.int32), edge_j=np.array(ej, np.int32))


def _flops(D, n, c):
    """FP64 flops the block factorization counts for column counts c (diagonal-block updates at
    their lower triangle, off-diagonal blocks by substitution, diagonal blocks factored)."""
    c = np.asarray(c, np.int64)
    n_upd = int((c * (c + 1) // 2).sum())
    n_diag = int(c.sum())
    return (2.0 * (n_upd - n_diag) * D ** 3 + n_diag * D * D * (D + 1) + n_diag * D * D * (D + 1)
            + n * 2.0 * D ** 3 / 3.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2207_09442_b300 import build
    build.build()


@pytest.mark.parametrize("n,b", [(64, 40), (40, 39), (48, 30)])
def test_band_graph_dense_supernode(n, b):
    st = layer.analyze(_band_graph(n, b), ordering="natural")
    c = [min(b, n - 1 - j) for j in range(n)]
    have, full = sum(c), n * (n - 1) // 2
    assert 2 * have >= full  # dense enough to amalgamate
    assert st["supernode_cols_max"] == n and st["n_supernodes"] == 1
    assert st["n_levels_max"] == n
    assert st["n_blocks_L"] == n + full  # explicit zeros stored
    assert st["n_block_updates"] == sum(x * (x + 1) // 2 for x in c)  # algorithmic, band only
    assert st["factor_flops"] == pytest.approx(_flops(D3, n, c), rel=1e-15)


def test_sparse_chain_is_not_amalgamated():
    """An odometry chain (band 1): 64 one-column levels but 63 of 2016 blocks, far too sparse."""
    n = 64
    st = layer.analyze(_band_graph(n, 1), ordering="natural")
    assert st["supernode_cols_max"] == 0 and st["n_supernodes"] == 0
    assert st["n_blocks_L"] == n + n - 1
    assert st["n_block_updates"] == n - 1
    assert st["factor_flops"] == pytest.approx(_flops(D3, n, [1] * (n - 1) + [0]), rel=1e-15)


def test_short_chain_is_not_amalgamated():
    """A complete graph on 31 poses is one dense chain of 31 columns: below the 32-column
    threshold, so it keeps the level schedule (nothing to add: it is dense already)."""
    n = 31
    st = layer.analyze(_band_graph(n, n), ordering="natural")
    assert st["supernode_cols_max"] == 0
    assert st["n_blocks_L"] == n + n * (n - 1) // 2
    st2 = layer.analyze(_band_graph(32, 32), ordering="natural")
    assert st2["supernode_cols_max"] == 32


def test_se2_band_counts():
    n, b = 50, 36
    st = layer.analyze(_band_graph(n, b, kind=2), ordering="natural")
    c = [min(b, n - 1 - j) for j in range(n)]
    assert st["supernode_cols_max"] == n
    assert st["factor_flops"] == pytest.approx(_flops(3, n, c), rel=1e-15)


def test_benchmark_graphs():
    """The 128-pose benchmark graphs keep the level schedule (top chains of ~14 columns); the
    2048-pose graphs of the scalability workload get one dense supernode each, of well over 100
    block columns (the separator the random loop closures fill in)."""
    small = layer.analyze(synth.pgo_se3(batch=4, n_poses=128, n_lc=32, config_id=2))
    assert small["n_supernodes"] == 0
    big = layer.analyze(synth.pgo_se3(batch=2, n_poses=2048, n_lc=512, config_id=2))
    assert big["n_supernodes"] == 2 and big["supernode_cols_max"] > 100
    # amalgamation adds storage, not algorithmic work: the flops are the sparse structure's,
    # far below the dense n^3/3 count of the same batch
    assert big["factor_flops"] < big["dense_flops"] / 100


def test_analyze_rejects_bad_structure():
    g = _band_graph(8, 2)
    g.edge_j = g.edge_j.copy()
    g.edge_j[0] = 8  # pose index out of range
    from paper_2207_09442_b300 import dnls
    with pytest.raises(dnls.DnlsError):
        layer.analyze(g)
