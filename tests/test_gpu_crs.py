"""CRS products on the GPU against the oracle (Sect. 2 CRS kernel)."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import (TOL64, adversarial_matrices, assert_close64, crs, dev, dot2_bound,
                      full_config, host)
from paper_0910_4836_gb300 import synth as S

pytestmark = pytest.mark.gpu

VECTOR_OPTS = [(l, r) for l in (1, 2, 4, 8, 16, 32) for r in (1, 2, 4)]
RUNS_OPTS = [(1, 4), (1, 8), (2, 4), (2, 8), (4, 4), (4, 8), (8, 8)]
TILES = (1024, 2048)


@pytest.fixture(scope="module", autouse=True)
def _build():
    import paper_0910_4836_gb300 as g
    g.build()


def kernels(M):
    """Yield (name, configure) for every CRS kernel option."""
    for l, r in VECTOR_OPTS:
        yield f"vector_l{l}_r{r}", lambda M=M, l=l, r=r: M.set_kernel("vector", lanes=l, rows_per_warp=r)
    for l, r in RUNS_OPTS:
        yield f"runs_l{l}_r{r}", lambda M=M, l=l, r=r: M.set_kernel("runs", lanes=l, rows_per_warp=r)
    for t in TILES:
        yield f"tiled_{t}", lambda M=M, t=t: M.prepare_tiled(t)


def test_laplace_config0_all_kernels():
    A = S.laplace2d()
    x = S.vector(A.n_cols, 0)
    ref, s = O.crs_spmv_exact(A, x)
    dense = A.to_dense() @ x
    M = crs(A)
    xd = dev(x)
    for name, conf in kernels(M):
        conf()
        y = host(M.spmv(xd))
        assert_close64(y, ref, s, name)
        assert np.all(np.abs(y - dense) <= 2 * TOL64 * s)


@pytest.mark.parametrize("idx", range(9))
def test_adversarial_all_kernels(idx):
    A = adversarial_matrices()[idx]
    x = S.vector(A.n_cols, 10 + idx)
    ref, s = O.crs_spmv_exact(A, x)
    M = crs(A)
    xd = dev(x)
    for name, conf in kernels(M):
        conf()
        y = host(M.spmv(xd))
        assert_close64(y, ref, s, f"{A.name} {name}")


@pytest.mark.parametrize("maker", [lambda: S.hh_like(300_000, 3), lambda: S.zipf_rows(200_000, 4),
                                   lambda: S.stencil27(30, 4)])
def test_integer_inputs_bit_exact(maker):
    A = S.integer_values(maker(), 5, 1024)
    x = S.int_vector(A.n_cols, 5, 1024)
    ref = O.crs_spmv(A, x)
    M = crs(A)
    xd = dev(x)
    for name, conf in kernels(M):
        conf()
        y = host(M.spmv(xd))
        assert np.array_equal(y, ref), name


def test_accumulate_and_determinism():
    A = S.zipf_rows(50_000, 12, lmax=4000)
    x = S.vector(A.n_cols, 12)
    y0 = S.vector(A.n_rows, 13)
    ref, s = O.crs_spmv_exact(A, x, y0, accumulate=True)
    s = s + np.abs(y0)
    M = crs(A)
    xd = dev(x)
    for name, conf in kernels(M):
        conf()
        y = dev(y0)
        M.spmv(xd, out=y, accumulate=True)
        assert_close64(host(y), ref, s, name)
        a = host(M.spmv(xd))
        b = host(M.spmv(xd))
        assert np.array_equal(a.view(np.int64), b.view(np.int64)), f"{name} not deterministic"


def test_strided_vectors_and_spmm():
    A = S.hh_like(50_000, 14)
    X = np.stack([S.vector(A.n_cols, 20 + c) for c in range(16)], axis=1)
    M = crs(A)
    Xd = dev(X)
    # one strided column through the k = 1 path
    for name, conf in kernels(M):
        conf()
        Y = torch.zeros((A.n_rows, 3), dtype=torch.float64, device="cuda")
        M.spmm(Xd[:, 5:6], out=Y[:, 1:2])
        ref, s = O.crs_spmv_exact(A, X[:, 5])
        assert_close64(host(Y[:, 1]), ref, s, name + " strided")
        assert np.all(host(Y[:, 0]) == 0) and np.all(host(Y[:, 2]) == 0)
    Yref, Sref = O.crs_spmm_exact(A, X)
    for k in (2, 4, 5, 16):
        for tile in (2, 4, 16):
            M.set_kernel("vector", rhs_tile=tile)
            Y = host(M.spmm(dev(X[:, :k].copy())))
            for c in range(k):
                assert_close64(Y[:, c], Yref[:, c], Sref[:, c], f"spmm k={k} tile={tile} col={c}")


def test_spmm_integer_bit_exact():
    A = S.integer_values(S.zipf_rows(30_000, 15, lmax=2000), 15, 512)
    X = np.stack([S.int_vector(A.n_cols, 30 + c, 512) for c in range(16)], axis=1)
    ref = O.crs_spmm(A, X)
    M = crs(A)
    for k in (4, 16):
        assert np.array_equal(host(M.spmm(dev(X[:, :k].copy()))), ref[:, :k])


def configure(M, name, compensated=None):
    if name.startswith("tiled"):
        if M._tile_table is None or M.kernel_opts()["tile"] != int(name.split("_")[1]):
            M.prepare_tiled(int(name.split("_")[1]))
        M.set_kernel("tiled", compensated=compensated)
    else:
        kind, l, r = name.split("_")
        M.set_kernel(kind, lanes=int(l[1:]), rows_per_warp=int(r[1:]), compensated=compensated)


KERNEL_NAMES = ([f"vector_l{l}_r{r}" for l, r in VECTOR_OPTS] + [f"runs_l{l}_r{r}" for l, r in RUNS_OPTS]
                + [f"tiled_{t}" for t in TILES])


def test_fp32_plain_and_compensated():
    A = S.zipf_rows(100_000, 16, lmax=5000)
    x = S.vector(A.n_cols, 16)
    A32 = A.astype(np.float32)
    x32 = x.astype(np.float32)
    # the reference is the exact product of the float32-rounded data
    ref, s = O.crs_spmv_exact(S.CRS(A.n_rows, A.n_cols, A.row_ptr, A.col,
                                    A32.val.astype(np.float64)), x32.astype(np.float64))
    lens = A.row_lengths()
    M = crs(A32, dtype=torch.float32)
    xd = dev(x32)
    bound = dot2_bound(ref, s, lens)
    n = lens.astype(np.float64) + 6
    plain_bound = (n * 2.0 ** -24 / (1 - n * 2.0 ** -24)) * s + 2.0 ** -24 * np.abs(ref)
    for name in KERNEL_NAMES:
        configure(M, name, compensated=True)
        y = host(M.spmv(xd)).astype(np.float64)
        assert np.all(np.abs(y - ref) <= bound), f"{name}: compensated error above the Dot2 bound"
        configure(M, name, compensated=False)
        yp = host(M.spmv(xd)).astype(np.float64)
        assert np.all(np.abs(yp - ref) <= plain_bound), f"{name}: plain float error above gamma_n"


def test_fp32_integer_bit_exact():
    A = S.integer_values(S.hh_like(100_000, 17), 17, 8)
    x = S.int_vector(A.n_cols, 17, 8)
    ref = O.crs_spmv(A, x).astype(np.float32)
    M = crs(A, dtype=torch.float32)
    xd = dev(x.astype(np.float32))
    for comp in (False, True):
        for name in KERNEL_NAMES:
            configure(M, name, compensated=comp)
            assert np.array_equal(host(M.spmv(xd)), ref), (name, comp)


def test_validation_status():
    A = S.small_random(100, 80, 3, density=0.1)
    M = crs(A)
    assert M.validate() == 0
    bad_col = A.col.copy()
    bad_col[3] = 80
    from paper_0910_4836_gb300 import CRSMatrix
    B = CRSMatrix(dev(A.row_ptr), dev(bad_col), dev(A.val), A.n_cols)
    assert B.validate() == -2
    bad_rp = A.row_ptr.copy()
    bad_rp[10], bad_rp[11] = bad_rp[11], bad_rp[10] - 1
    C = CRSMatrix(dev(bad_rp), dev(A.col), dev(A.val), A.n_cols)
    assert C.validate() == -2


def test_argument_errors():
    from paper_0910_4836_gb300 import CRSMatrix, GbspError
    A = S.small_random(50, 40, 3, density=0.1)
    M = crs(A)
    x = dev(S.vector(40, 1))
    with pytest.raises(GbspError):
        M.set_kernel("vector", lanes=3)
    for l, r in ((16, 8), (8, 4), (2, 2), (4, 1)):
        with pytest.raises(GbspError):
            M.set_kernel("runs", lanes=l, rows_per_warp=r)
    with pytest.raises(GbspError):
        M.set_kernel("vector", rows_per_warp=8)  # a RUNS shape only
    M.set_kernel("vector", lanes=16, rows_per_warp=2)
    M.set_kernel("runs")  # the pair is RUNS's own default, not VECTOR's leftover
    assert (M.kernel_opts()["lanes"], M.kernel_opts()["rows_per_warp"]) == (4, 4)
    with pytest.raises(GbspError):
        M.spmv(dev(S.vector(50, 1)), transpose=True)  # no transpose attached
    with pytest.raises(ValueError):
        M.spmv(dev(S.vector(41, 1)))
    # overlapping x and y
    buf = torch.zeros(100, dtype=torch.float64, device="cuda")
    with pytest.raises(GbspError):
        M.spmv(buf[:40], out=buf[20:70])
    with pytest.raises(GbspError):
        M.set_kernel("tiled")  # not prepared yet
    M.prepare_tiled(1024)
    M.spmv(x)
    # the bulk copies of TILED need 16-byte aligned arrays
    val_buf = torch.zeros(A.nnz + 1, dtype=torch.float64, device="cuda")
    val_buf[1:] = dev(A.val)
    B = CRSMatrix(dev(A.row_ptr), dev(A.col), val_buf[1:], A.n_cols)
    with pytest.raises(GbspError):
        B.prepare_tiled(1024)


def test_unaligned_arrays():
    """Arrays aligned only to their element size (val 8-byte, col 4-byte
    aligned: borrowed slices of larger buffers) give the same products."""
    from paper_0910_4836_gb300 import CRSMatrix
    A = S.zipf_rows(60_000, 21, lmax=3000)
    x = S.vector(A.n_cols, 21)
    ref, s = O.crs_spmv_exact(A, x)
    val_buf = torch.zeros(A.nnz + 1, dtype=torch.float64, device="cuda")
    val_buf[1:] = dev(A.val)
    col_buf = torch.zeros(A.nnz + 1, dtype=torch.int32, device="cuda")
    col_buf[1:] = dev(A.col, torch.int32)
    xd = dev(x)
    for vb, cb in ((val_buf[1:], dev(A.col, torch.int32)), (dev(A.val), col_buf[1:]), (val_buf[1:], col_buf[1:])):
        B = CRSMatrix(dev(A.row_ptr, torch.int32), cb, vb, A.n_cols)
        for l, r in VECTOR_OPTS:
            B.set_kernel("vector", lanes=l, rows_per_warp=r)
            assert_close64(host(B.spmv(xd)), ref, s, f"unaligned vector l{l} r{r}")


@pytest.mark.slow
@pytest.mark.parametrize("cfg", [1, 2, 4])
def test_full_size_configs(cfg):
    """Full-size workloads in the benchmark's launch configuration: every
    output entry against the accurate oracle."""
    A = full_config(cfg)
    x = S.vector(A.n_cols, cfg)
    ref, s = O.crs_spmv_exact(A, x)
    M = crs(A)
    xd = dev(x)
    for name in ("tiled", "vector", "vector l4 r4", "runs l2 r8", "runs l4 r4"):
        if name == "tiled":
            M.prepare_tiled(2048)
        elif name == "vector":
            M.set_kernel("vector", lanes=8 if cfg != 4 else 16, rows_per_warp=2)
        else:
            kind, l, r = name.split()
            M.set_kernel(kind, lanes=int(l[1:]), rows_per_warp=int(r[1:]))
        y = host(M.spmv(xd))
        assert_close64(y, ref, s, f"config {cfg} {name}")
