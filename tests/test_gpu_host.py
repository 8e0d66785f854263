"""Products with host vectors (gbsp_spmv_host): copy in, product, copy out
on one stream.  The result must be the device path's, bit for bit."""
import ctypes

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


def handles(A):
    M = crs(A)
    yield "CRS", M, 1
    yield "SELL row_only", M.to_jds("SELL", "row_only", window=128, unroll=4), 0
    yield "NUJDS symmetric", M.to_jds("NUJDS", "symmetric", unroll=2), 1


@pytest.mark.parametrize("pinned", [True, False])
def test_host_product_equals_device_product(pinned):
    A = S.hh_like(200_000, 41)
    x = S.vector(A.n_cols, 41)
    ref, s = O.crs_spmv_exact(A, x)
    xh = torch.as_tensor(x)
    if pinned:
        xh = xh.pin_memory()
    for name, H, basis in handles(A):
        yd = H.spmv(dev(x), basis=basis)
        yh = H.spmv_host(xh, basis=basis)
        torch.cuda.synchronize()
        assert torch.equal(yh, yd.cpu()), name
        if basis == 1:
            assert_close64(yh.numpy(), ref, s, name)
        # accumulate: y_host += A x
        y0 = torch.as_tensor(S.vector(A.n_rows, 42))
        yacc = y0.clone()
        H.spmv_host(xh, out=yacc, accumulate=True, basis=basis)
        torch.cuda.synchronize()
        ydev = dev(y0.numpy())
        H.spmv(dev(x), out=ydev, accumulate=True, basis=basis)
        assert torch.equal(yacc, ydev.cpu()), name


def test_host_product_transpose_and_streams():
    A = S.small_random(3000, 2000, 43, density=0.01)
    M = crs(A)
    M.transpose()
    g = S.vector(A.n_rows, 44)
    gh = torch.as_tensor(g).pin_memory()
    zt = M.spmv_host(gh, transpose=True, basis=1)
    torch.cuda.synchronize()
    assert torch.equal(zt, M.spmv(dev(g), transpose=True, basis=1).cpu())
    # alternating streams, each with its own stage and output: all correct
    xs = [torch.as_tensor(S.vector(A.n_cols, 50 + i)).pin_memory() for i in range(6)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    stages = [M.host_stage(), M.host_stage()]
    outs = [torch.empty(A.n_rows, dtype=torch.float64).pin_memory() for _ in range(6)]
    for i, xi in enumerate(xs):
        M.spmv_host(xi, out=outs[i], stage=stages[i & 1], stream=streams[i & 1], basis=1)
    torch.cuda.synchronize()
    for i, xi in enumerate(xs):
        assert np.array_equal(outs[i].numpy(), host(M.spmv(dev(xi.numpy()), basis=1))), i


def test_host_product_rejections():
    from paper_0910_4836_gb300 import GbspError, _lib
    A = S.laplace2d(16, 16)
    M = crs(A)
    with pytest.raises(ValueError):
        M.spmv_host(torch.ones(A.n_cols, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        M.spmv_host(torch.ones(A.n_cols + 1, dtype=torch.float64))
    with pytest.raises(ValueError):
        M.spmv_host(torch.ones(A.n_cols, dtype=torch.float32))
    with pytest.raises(ValueError):
        small = torch.empty(5, dtype=torch.float64, device="cuda")
        M.spmv_host(torch.ones(A.n_cols, dtype=torch.float64), stage=(small, small))
    with pytest.raises(GbspError):
        M.spmv_host(torch.ones(A.n_cols, dtype=torch.float64), transpose=True, basis=1)  # no transpose attached
    # NULL stage through the ABI
    L = _lib.load()
    xh = torch.ones(A.n_cols, dtype=torch.float64)
    yh = torch.empty(A.n_rows, dtype=torch.float64)
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    assert L.gbsp_spmv_host(M.handle, 0, 1, 0, vp(xh), vp(yh), None, None, None) == -1
