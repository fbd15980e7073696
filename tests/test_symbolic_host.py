"""The symbolic analysis on the host (no GPU): a small C++ driver compiled with g++ runs
build_graph_host on seeded graphs of the benchmark shapes and checks the invariants the CUDA
factorization and solves rely on (level schedule, top chain and its row partition, lane counts,
gather lists with their early/late split and ordering, the dense supernode's storage and source
lists, assembly maps).  It then runs the device factorization's steps as plain host loops on a
seeded SPD matrix with the graph's pattern, through the same structure and the same block-row
mapping of the supernode's trailing updates, and checks L L^T against the matrix."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2207_09442_b300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("symbolic") / "check")
    src = [os.path.join(HERE, "host_symbolic_check.cpp"),
           os.path.join(ROOT, "paper_2207_09442_b300", "csrc", "dnls_symbolic.cpp")]
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-o", out] + src,
                   check=True)
    return out


def _run(checker, batch):
    lines = [str(batch.batch)]
    for k in range(batch.batch):
        p0, p1 = int(batch.pose_offsets[k]), int(batch.pose_offsets[k + 1])
        e0, e1 = int(batch.edge_offsets[k]), int(batch.edge_offsets[k + 1])
        lines.append(f"{p1 - p0} {e1 - e0}")
        lines += [f"{int(batch.edge_i[e])} {int(batch.edge_j[e])}" for e in range(e0, e1)]
    res = subprocess.run([checker], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         check=True)
    return res.stdout.split("\n")[:-1]


@pytest.mark.parametrize("make", [
    lambda: synth.pgo_se3(batch=4, n_poses=128, config_id=2),             # benchmark shape
    lambda: synth.pgo_se3(batch=6, n_poses_range=(16, 256), config_id=4),  # uneven sizes
    lambda: synth.pgo_se3(batch=2, n_poses=24, n_lc=0, config_id=153),     # pure chains
    lambda: synth.pgo_se3(batch=3, n_poses=8, n_lc=6, config_id=154),      # dense small graphs
    lambda: synth.pgo_se3(batch=2, n_poses=48, n_lc=400, config_id=160),   # supernode: most of L
    lambda: synth.pgo_se3(batch=1, n_poses=600, n_lc=150, config_id=162),  # supernode on sparse levels
])
def test_symbolic_invariants(checker, make):
    b = make()
    out = _run(checker, b)
    assert len(out) == b.batch
    for line in out:
        assert line.startswith("ok"), line
        assert float(line.split()[5]) < 1e-12  # emulated factorization: L L^T = A


def test_supernode_is_emulated(checker):
    """The 600-pose graph gets a dense supernode (its first level below the number of levels),
    and the emulation goes through it."""
    b = synth.pgo_se3(batch=1, n_poses=600, n_lc=150, config_id=162)
    _, nlev, chain_lev, _, dense_lev, resid = _run(checker, b)[0].split()
    assert int(dense_lev) == int(chain_lev) < int(nlev) and float(resid) < 1e-12


def test_pure_chain_is_all_top_chain(checker):
    """An odometry chain eliminates as a path: one column per level, the top chain starts at
    level 0."""
    b = synth.pgo_se3(batch=1, n_poses=24, n_lc=0, config_id=153)
    _, nlev, chain_lev, _, dense_lev, _ = _run(checker, b)[0].split()
    assert int(nlev) == 24 and int(chain_lev) == 0 and int(dense_lev) == 24  # sparse: no supernode


def test_flop_count_matches_block_structure(checker):
    """The algorithmic flop count: 2 D^3 per update into an off-diagonal block, D^2 (D+1) into a
    diagonal block (its lower triangle), D^2 (D+1) per off-diagonal block's panel and 2 D^3 / 3
    per diagonal factorization.  For a path of n poses (no fill, every column one block below
    the diagonal) that is (n-1) updates into diagonal blocks, n-1 panels and n factors."""
    n, D = 24, 6
    b = synth.pgo_se3(batch=1, n_poses=n, n_lc=0, config_id=153)
    flops = float(_run(checker, b)[0].split()[3])
    expect = (n - 1) * D * D * (D + 1) + (n - 1) * D * D * (D + 1) + n * 2.0 * D ** 3 / 3.0
    assert flops == pytest.approx(expect, rel=1e-12)
