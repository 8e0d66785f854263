"""Access-pattern analysis on the GPU against the oracle: the stride
distribution of Sect. 4.2 (Fig. 4a) and the sectors per warp-wide gather.
Integer counts, so bit-exact."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import adversarial_matrices, crs, dev
from paper_0910_4836_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import paper_0910_4836_gb300 as g
    g.build()


def matrices():
    yield "laplace", S.laplace2d(64, 64)
    yield "hh_like_50k", S.hh_like(50_000, 1)
    yield "zipf_20k", S.zipf_rows(20_000, 2, lmax=3000)
    yield "random_rect", S.small_random(3000, 5000, 3, density=0.004)
    for i, A in enumerate(adversarial_matrices()):
        yield f"adv{i}_{A.name}", A


MATS = list(matrices())


@pytest.mark.parametrize("name,A", MATS, ids=[m[0] for m in MATS])
def test_stride_hist_matches_oracle(name, A):
    from paper_0910_4836_gb300.analysis import stride_hist
    f, b = stride_hist(dev(A.col, torch.int32))
    fo, bo = O.stride_hist(A.col)
    assert np.array_equal(f, fo) and np.array_equal(b, bo), name
    assert f.sum() + b.sum() == max(A.nnz - 1, 0)


@pytest.mark.parametrize("name,A", MATS, ids=[m[0] for m in MATS])
def test_warp_sectors_crs_matches_oracle(name, A):
    from paper_0910_4836_gb300.analysis import warp_sectors
    M = crs(A)
    for lanes in (1, 4, 32):
        for eb in (4, 8):
            assert np.array_equal(warp_sectors(M, lanes, eb), O.warp_sectors_crs(A, lanes, eb)), (name, lanes, eb)


@pytest.mark.parametrize("name,A", [m for m in MATS if m[1].n_rows == m[1].n_cols],
                         ids=[m[0] for m in MATS if m[1].n_rows == m[1].n_cols])
def test_warp_sectors_jds_and_sell_match_oracle(name, A):
    from paper_0910_4836_gb300.analysis import stride_hist, warp_sectors
    M = crs(A)
    for perm in ("symmetric", "row_only"):
        sym = perm == "symmetric"
        J = M.to_jds("NUJDS", perm, unroll=2)
        Jo = O.jds_build(A, sym)
        assert np.array_equal(warp_sectors(J), O.warp_sectors_jds(Jo)), (name, perm)
        f, b = stride_hist(J.col)
        assert np.array_equal(f, O.stride_hist(Jo.col)[0]) and np.array_equal(b, O.stride_hist(Jo.col)[1])
        for w in (32, 128):
            G = M.to_jds("SELL", perm, window=w)
            assert np.array_equal(warp_sectors(G), O.warp_sectors_sell(O.sell_build(A, w, sym))), (name, perm, w)


def test_warp_sectors_rbjds_unsupported():
    from paper_0910_4836_gb300 import GbspError
    from paper_0910_4836_gb300.analysis import warp_sectors
    R = crs(S.laplace2d(16, 16)).to_jds("RBJDS", "symmetric", block=64)
    with pytest.raises(GbspError):
        warp_sectors(R)


def test_warp_sectors_bad_lanes():
    from paper_0910_4836_gb300 import GbspError
    from paper_0910_4836_gb300.analysis import warp_sectors
    M = crs(S.laplace2d(16, 16))
    for lanes in (0, 3, 64):
        with pytest.raises(GbspError):
            warp_sectors(M, lanes)
