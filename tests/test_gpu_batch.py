"""Batched persistent launch, CUDA-graph replay, bounded ready-flag wait and
the autotuner."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import assert_close64, crs, dev, host
from paper_0910_4836_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import paper_0910_4836_gb300 as g
    g.build()


def small_batch(count=24, seed=3):
    return S.batch_set(count, seed, lo=500, hi=20000)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batch_matches_single_launches(dtype):
    from paper_0910_4836_gb300 import Batch
    mats = small_batch()
    ks = S.batch_k(len(mats), "mixed")
    items, singles = [], []
    for b, (A, k) in enumerate(zip(mats, ks)):
        M = crs(A, dtype=dtype)
        M.set_kernel("vector", lanes=(4, 8, 16)[b % 3], rows_per_warp=2, rhs_tile=(4, 8, 16)[b % 3])
        if b % 4 == 1 and A.n_rows == A.n_cols:
            M = M.to_jds(("JDS", "NUJDS", "RBJDS", "SOJDS")[(b // 4) % 4], "symmetric", block=256)
        elif b % 4 == 3:
            M = M.to_jds("SELL", "row_only", window=(32, 128, 1024)[(b // 4) % 3], unroll=(1, 2, 4)[b % 3])
        shape = (A.n_cols,) if k == 1 else (A.n_cols, k)
        X = torch.as_tensor(np.stack([S.vector(A.n_cols, 10 * b + c) for c in range(k)], axis=1)
                            .reshape(shape)).to(dtype).cuda()
        Y = torch.full((A.n_rows,) if k == 1 else (A.n_rows, k), 7.0, dtype=dtype, device="cuda")
        items.append((M, X, Y))
        singles.append(M.spmm(X))
    bt = Batch(items, chunk=2048)
    nw, grid = bt.info()
    assert nw >= len(mats) and grid >= 1
    bt.run()
    torch.cuda.synchronize()
    for (M, X, Y), ref in zip(items, singles):
        assert torch.equal(Y, ref)
    # graph replay gives the same bits again
    for _, _, Y in items:
        Y.fill_(-1.0)
    g = bt.graph()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for (M, X, Y), ref in zip(items, singles):
        assert torch.equal(Y, ref)


def test_batch_against_oracle():
    from paper_0910_4836_gb300 import Batch
    mats = small_batch(12, 5)
    items, refs = [], []
    for b, A in enumerate(mats):
        M = crs(A)
        x = S.vector(A.n_cols, b)
        items.append((M, dev(x), torch.empty(A.n_rows, dtype=torch.float64, device="cuda")))
        refs.append(O.crs_spmv_exact(A, x))
    bt = Batch(items)
    bt.run()
    for (M, X, Y), (ref, s) in zip(items, refs):
        assert_close64(host(Y), ref, s, "batched")


def test_ready_flag_bounded_wait():
    """A flag that nothing sets: the persistent kernel gives up after its
    limit, reports GBSP_ERR_TIMEOUT and leaves the context usable."""
    from paper_0910_4836_gb300 import Batch
    A = S.laplace2d(32, 32)
    M = crs(A)
    x = dev(S.vector(A.n_cols, 1))
    Y = torch.full((A.n_rows,), 5.0, dtype=torch.float64, device="cuda")
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    bt = Batch([(M, x, Y)], ready=flag)
    bt.run(status)
    torch.cuda.synchronize()
    assert int(status.item()) == -6  # GBSP_ERR_TIMEOUT
    assert torch.all(Y == 5.0)       # no work done
    # set the flag (work finished earlier on the stream) and run again
    flag.fill_(1)
    status.zero_()
    bt.run(status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert torch.equal(Y, M.spmv(x))


def test_autotune_keeps_a_valid_fast_choice():
    A = S.hh_like(200_000, 7)
    x = S.vector(A.n_cols, 7)
    ref, s = O.crs_spmv_exact(A, x)
    M = crs(A)
    M.prepare_tiled(1024)
    opts, ms = M.autotune(1)
    assert ms > 0 and opts["kernel"] in (1, 2, 3)  # VECTOR, TILED or RUNS
    assert_close64(host(M.spmv(dev(x))), ref, s, f"tuned {opts}")
    J = M.to_jds("JDS", "symmetric")
    jopts, jms = J.autotune(1)
    assert jopts["format"] in (1, 2, 4) and jms > 0
    Oj = O.jds_build(A, True)
    yp = host(J.spmv(dev(O.permute(Oj.perm, x))))
    assert_close64(yp, O.permute(Oj.perm, ref), O.permute(Oj.perm, s), f"tuned JDS {jopts}")
    # a second handle with the same signature reuses the cached choice
    M2 = crs(A)
    M2.prepare_tiled(1024)
    o2, ms2 = M2.autotune(1)
    assert o2["kernel"] == opts["kernel"] and ms2 == ms


def test_autotuned_batch_builder():
    from paper_0910_4836_gb300 import Batch
    mats = small_batch(10, 9)
    ks = [1, 4, 16] * 3 + [1]
    bt, handles, Xs, Ys = Batch.autotuned(mats, ks)
    for b, (A, k, H, X) in enumerate(zip(mats, ks, handles, Xs)):
        X.copy_(torch.as_tensor(np.stack([S.vector(A.n_cols, 40 + b + c) for c in range(k)], axis=1)
                                .reshape(X.shape)))
    bt.run()
    torch.cuda.synchronize()
    for H, X, Y in zip(handles, Xs, Ys):
        assert torch.equal(Y, H.spmm(X))


def test_autotuned_batch_with_sell_items():
    """The autotuner may pick SELL per matrix; the batch still reproduces
    each chosen handle's own product bit for bit."""
    from paper_0910_4836_gb300 import Batch, JDSMatrix
    mats = small_batch(16, 7)
    ks = S.batch_k(len(mats), "mixed")
    bt, handles, Xs, Ys = Batch.autotuned(mats, ks, torch.float64, device="cuda")
    for b, X in enumerate(Xs):
        X.copy_(torch.as_tensor(np.stack([S.vector(X.shape[0], 100 * b + c) for c in range(ks[b])], axis=1)
                                .reshape(X.shape)))
    refs = [H.spmm(X) for H, X in zip(handles, Xs)]
    bt.run()
    torch.cuda.synchronize()
    for Y, ref in zip(Ys, refs):
        assert torch.equal(Y, ref)
    assert all(isinstance(h, JDSMatrix) or h.__class__.__name__ == "CRSMatrix" for h in handles)


def test_all_sell_one_vector_batch():
    """A batch of one-vector FP64 SELL items (the plain batched SELL walk):
    each result equals the handle's own product bit for bit, also when one
    item reads and writes a strided column."""
    from paper_0910_4836_gb300 import Batch
    mats = small_batch(20, 11)
    items, refs = [], []
    for b, A in enumerate(mats):
        H = crs(A).to_jds("SELL", "row_only", window=(128, 1024)[b % 2], unroll=(2, 4)[b % 2])
        X = dev(S.vector(A.n_cols, 200 + b))
        Y = torch.full((A.n_rows,), 3.0, dtype=torch.float64, device="cuda")
        items.append((H, X, Y))
        refs.append(H.spmv(X))
    bt = Batch(items, chunk=2048)
    bt.run()
    torch.cuda.synchronize()
    for (_, _, Y), ref in zip(items, refs):
        assert torch.equal(Y, ref)
    # one item reading and writing a strided column: same bits
    A0 = mats[0]
    X2 = dev(np.stack([S.vector(A0.n_cols, 200), S.vector(A0.n_cols, 201)], axis=1))
    Y2 = torch.zeros((A0.n_rows, 2), dtype=torch.float64, device="cuda")
    items2 = [(items[0][0], X2[:, :1], Y2[:, :1])] + items[1:]
    for _, _, Y in items2[1:]:
        Y.fill_(-1.0)
    Batch(items2, chunk=2048).run()
    torch.cuda.synchronize()
    assert torch.equal(Y2[:, 0], refs[0])
    for (_, _, Y), ref in zip(items2[1:], refs[1:]):
        assert torch.equal(Y, ref)
