"""The documented Python usage, end to end on a small HH-like matrix: CRS,
SELL in the original basis, NUJDS in the permuted basis, SpMM, the adjoint,
dval, host vectors and the checkpointed autograd power iteration, each
result checked against the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import assert_close64, host

pytestmark = pytest.mark.gpu


def test_documented_usage():
    from paper_0910_4836_gb300 import CRSMatrix, build, synth as S
    from paper_0910_4836_gb300.autograd import Pattern, power_apply
    build()
    A = S.hh_like(200_000, seed=1)
    M = CRSMatrix.from_host(A)
    xh = S.vector(A.n_cols, 1)
    x = torch.as_tensor(xh).cuda()
    ref, s = O.crs_spmv_exact(A, xh)

    assert_close64(host(M.spmv(x)), ref, s, "CRS")
    G = M.to_jds("SELL", "row_only", window=128, unroll=4)
    assert_close64(host(G.spmv_original(x)), ref, s, "SELL original basis")
    J = M.to_jds("NUJDS", "symmetric", unroll=2)
    y_p = J.spmv(J.permute(x))
    assert_close64(host(J.permute(y_p, back=True)), ref, s, "NUJDS permuted basis")

    Xh = np.stack([S.vector(A.n_cols, 30 + c) for c in range(16)], axis=1)
    Y = G.spmm(torch.as_tensor(Xh).cuda(), basis=1)
    for c in (0, 7, 15):
        r, sc = O.crs_spmv_exact(A, np.ascontiguousarray(Xh[:, c]))
        assert_close64(host(Y[:, c]), r, sc, f"SELL SpMM column {c}")

    M.transpose()
    g = M.spmv(torch.as_tensor(ref).cuda(), transpose=True)
    rt, st = O.crs_spmv_t_exact(A, ref)
    assert_close64(host(g), rt, st, "adjoint")
    d = host(M.dval(torch.as_tensor(ref).cuda(), x))
    assert np.array_equal(d, O.dval(A, ref, xh))  # one rounded product per entry

    yh = M.spmv_host(torch.as_tensor(xh).pin_memory())
    torch.cuda.synchronize()
    assert_close64(yh.numpy(), ref, s, "host vectors")

    p = Pattern.from_host(A, forward="auto", adjoint="auto")
    val = torch.as_tensor(A.val, device="cuda").requires_grad_(True)
    xx = x.clone().requires_grad_(True)
    loss = (power_apply(p, val, xx, m=4, checkpoint=2) ** 2).sum()
    loss.backward()
    L_ref, dv_ref, dx_ref = O.power_loss_grad(A, xh, 4)
    assert abs(loss.item() - L_ref) <= 1e-12 * abs(L_ref)
    for got, want in ((val.grad, dv_ref), (xx.grad, dx_ref)):
        err = np.abs(host(got) - want)
        assert np.all(err <= 1e-11 * np.abs(want) + 1e-14 * np.abs(want).max())
