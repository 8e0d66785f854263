"""The basic gather sums of Sect. 4.1 (ADD / SCP over PD, CS, IS, IR and
Gaussian strides) on the GPU against the oracle."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import dev, host
from paper_0910_4836_gb300 import synth as S

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _build():
    import paper_0910_4836_gb300 as g
    g.build()


def bound(n, n_partials, abs_sum):
    """Error bound of the kernel's summation: a chain of ceil(n/T) terms per
    thread (T = 256 threads x CTAs), a 5-level shuffle tree, a chain over 8
    warps, then the partials (a chain of ceil(P/256) per thread and the same
    trees), plus the SCP product rounding: gamma_m sum|t|."""
    T = 256 * n_partials
    m = math.ceil(n / T) + 5 + 8 + math.ceil(n_partials / 256) + 5 + 8 + 1
    return m * U64 / (1 - m * U64) * abs_sum


def run(op, access, n, b, a=None, k=1, ind=None, status=None):
    from paper_0910_4836_gb300.gather import GatherSum
    g = GatherSum(op, access, n, dev(b), a=None if a is None else dev(a), k=k,
                  ind=None if ind is None else dev(ind, torch.int32), status=status)
    return float(host(g())[0]), g.n_partials


def cases():
    """(name, access, n, k, ind, len_b): sizes span many CTAs and end in a
    ragged tail."""
    n = 300_001
    yield "PD", "PD", n, 1, None, n
    for k in (8, 530):
        m = 20_011 if k == 530 else n
        yield f"CS k={k}", "CS", m, k, None, k * (m - 1) + 1
        yield f"IS k={k}", "IND", m, 1, S.stride_indices(m, k), k * (m - 1) + 1
    for k in (1, 8, 530):
        ind = S.geometric_indices(n if k < 530 else 20_011, 1.0 / k, 31 + k)
        yield f"IR k={k}", "IND", len(ind), 1, ind, int(ind[-1]) + 1
    ind = S.gaussian_indices(n, 16.0, 256.0, 16 * n, 41)
    yield "Gauss mean=16 var=256", "IND", n, 1, ind, 16 * n


@pytest.mark.parametrize("op", ["ADD", "SCP"])
@pytest.mark.parametrize("case", list(cases()), ids=lambda c: c[0])
def test_gather_random_within_bound(op, case):
    name, access, n, k, ind, len_b = case
    b = S.vector(len_b, 51)
    a = S.vector(n, 52) if op == "SCP" else None
    s, npart = run(op, access, n, b, a, k, ind)
    ref, abs_sum = O.gather_sum_exact(op, access, n, b, a=a, k=k, ind=ind)
    assert abs(s - ref) <= bound(n, npart, abs_sum), (name, s, ref)


@pytest.mark.parametrize("op", ["ADD", "SCP"])
@pytest.mark.parametrize("case", list(cases()), ids=lambda c: c[0])
def test_gather_integers_bit_exact(op, case):
    """Integer inputs with every partial sum below 2^53: any summation
    order is exact, so the GPU sum equals the oracle's bit for bit."""
    name, access, n, k, ind, len_b = case
    b = S.int_vector(len_b, 61, 1000)
    a = S.int_vector(n, 62, 1000) if op == "SCP" else None
    s, _ = run(op, access, n, b, a, k, ind)
    assert s == O.gather_sum(op, access, n, b, a=a, k=k, ind=ind), name


def test_gather_is_deterministic():
    n = 1_000_003
    b = S.vector(4 * n, 71)
    a = S.vector(n, 72)
    ind = S.geometric_indices(n, 0.25, 73)
    first, _ = run("SCP", "IND", n, b[: int(ind[-1]) + 1], a, 1, ind)
    for _ in range(3):
        assert run("SCP", "IND", n, b[: int(ind[-1]) + 1], a, 1, ind)[0] == first


@pytest.mark.parametrize("n", [0, 1, 2, 255, 256, 2047, 2049])
def test_gather_small_and_empty(n):
    b = S.int_vector(max(n, 1), 81, 1000)
    a = S.int_vector(max(n, 1), 82, 1000)
    s, _ = run("SCP", "PD", n, b, a)
    assert s == (O.gather_sum("SCP", "PD", n, b, a=a) if n else 0.0)


def test_gather_bad_index_is_skipped_and_reported():
    """Entries of ind outside [0, len_b) add nothing and set the status
    word (the kernel's own bounds check; nothing is read out of range)."""
    n = 10_000
    b = S.int_vector(n, 91, 1000)
    ind = np.arange(n, dtype=np.int32)
    ind[17] = -5
    ind[9_000] = n
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    s, _ = run("ADD", "IND", n, b, ind=ind, status=status)
    keep = np.ones(n, bool)
    keep[[17, 9_000]] = False
    assert s == float(b[keep].sum())
    assert int(host(status)[0]) == -1  # GBSP_ERR_ARG


def test_gather_argument_errors():
    from paper_0910_4836_gb300 import GbspError
    from paper_0910_4836_gb300.gather import GatherSum
    b = torch.zeros(100, dtype=torch.float64, device="cuda")
    with pytest.raises(GbspError):
        GatherSum("ADD", "CS", 11, b, k=10)()   # (n-1)*k = 100 >= len_b
    with pytest.raises(GbspError):
        GatherSum("ADD", "PD", 101, b)()
    with pytest.raises(GbspError):
        GatherSum("ADD", "CS", 5, b, k=0)()


def test_fma_chain_closed_form():
    """The FP64 issue-rate launch computes what it claims: with x0 = 1,
    a = 1/2, b = 1, chain j after k steps is 2 + (j - 1) 2^-k exactly, so a
    thread's sum of its 8 chains is 16 + 20 / 2^k; idle lanes write 0."""
    from paper_0910_4836_gb300 import build
    from paper_0910_4836_gb300.gather import FmaChain
    build()
    for n, active, k in ((1000, 32, 3), (4096, 5, 3), (257, 32, 0), (2048, 16, 40)):
        f = FmaChain(n, active_lanes=active, iters=k)
        out = f().cpu().numpy()
        lanes = np.arange(n) % 32
        want = np.where(lanes < active, 16.0 + 20.0 / 2.0 ** k, 0.0)
        assert np.array_equal(out, want), (n, active, k)
        assert f.flops == 16.0 * k * np.count_nonzero(lanes < active)


def _uniform_indices(n, length, seed):
    ind = np.minimum((S.uniform01(seed, 233, np.arange(n)) * length).astype(np.int64), length - 1)
    ind[min(5, n - 1)] = length - 1  # the last element (an odd tail is read directly)
    return ind.astype(np.int32)


@pytest.mark.parametrize("op", ["ADD", "SCP"])
@pytest.mark.parametrize("len_b", [4_000_001, 4_000_000, 3, 2])
def test_gather_tma_within_bound_and_bit_exact(op, len_b):
    """IND through TMA gather4 copies: random indices over the whole vector,
    a ragged number of them, odd and even lengths; within the summation
    bound on random data and bit-exact on integers."""
    n = 300_007
    ind = _uniform_indices(n, len_b, 101 + len_b % 7)
    b = S.vector(len_b, 102)
    a = S.vector(n, 103) if op == "SCP" else None
    s, npart = run(op, "IND_TMA", n, b, a, 1, ind)
    ref, abs_sum = O.gather_sum_exact(op, "IND", n, b, a=a, ind=ind)
    assert abs(s - ref) <= bound(n, npart, abs_sum), (s, ref)
    bi = S.int_vector(len_b, 104, 1000)
    ai = S.int_vector(n, 105, 1000) if op == "SCP" else None
    assert run(op, "IND_TMA", n, bi, ai, 1, ind)[0] == O.gather_sum(op, "IND", n, bi, a=ai, ind=ind)


def test_gather_tma_bad_index_is_skipped_and_reported():
    n = 10_000
    b = S.int_vector(n + 1, 111, 1000)
    ind = np.arange(n, dtype=np.int32)
    ind[17] = -5
    ind[9_000] = n + 1
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    s, _ = run("ADD", "IND_TMA", n, b, ind=ind, status=status)
    keep = np.ones(n, bool)
    keep[[17, 9_000]] = False
    assert s == float(b[:n][keep].sum())
    assert int(host(status)[0]) == -1  # GBSP_ERR_ARG


def test_stage_sweep_closed_form():
    """Every CTA streams the vector's whole 16-byte blocks through shared
    memory in 32 KB chunks and adds the first double of each: the sum of
    b[4096 c] over the chunks; all CTAs agree and no wait gives up."""
    from paper_0910_4836_gb300.gather import stage_sweep
    for len_b in (1, 2, 4097, 1_000_001):
        b = S.int_vector(len_b, 121, 1000)
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        out = host(stage_sweep(dev(b), status=status))
        whole = (len_b * 8) // 16 * 16
        want = float(sum(b[4096 * c] for c in range((whole + 32767) // 32768)))
        assert np.all(out == want), (len_b, out[:3], want)
        assert int(host(status)[0]) == 0
