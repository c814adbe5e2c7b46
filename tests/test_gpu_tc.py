"""Tensor-core building blocks (tcgen05 MMA through TMEM) against a host product.

FP16 x FP16 products are exact in FP32, so the only error is the FP32
summation order over K <= 256 terms: |D - ref| <= 1e-5 * sum_k |a||b|.
"""
import numpy as np
import pytest

import paper_0812_3669_gb300 as moff

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    moff.build()
    yield


@pytest.mark.parametrize("n,k", [(32, 16), (64, 64), (128, 128), (256, 256), (96, 48)])
def test_tc_product_matches_host(n, k):
    rng = np.random.default_rng(n * 1000 + k)
    a = rng.normal(size=(128, k)).astype(np.float16)
    b = rng.normal(size=(n, k)).astype(np.float16)
    d = torch.full((128, n), float("nan"), dtype=torch.float32, device="cuda")
    moff.moff_tc_selftest(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), d)
    got = d.cpu().numpy()
    ref = a.astype(np.float64) @ b.astype(np.float64).T
    bound = 1e-5 * (np.abs(a.astype(np.float64)) @ np.abs(b.astype(np.float64)).T) + 1e-6
    assert np.isfinite(got).all()
    assert (np.abs(got - ref) <= bound).all(), np.abs(got - ref).max()


def _run(n, k, mode, seed):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(128, k)).astype(np.float16)
    b = rng.normal(size=(n, k)).astype(np.float16)
    d = torch.full((128, n), float("nan"), dtype=torch.float32, device="cuda")
    moff.moff_tc_selftest(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), d, mode)
    got = d.cpu().numpy()
    ref = a.astype(np.float64) @ b.astype(np.float64).T
    bound = 1e-5 * (np.abs(a.astype(np.float64)) @ np.abs(b.astype(np.float64)).T) + 1e-6
    return bool(np.isfinite(got).all() and (np.abs(got - ref) <= bound).all())


@pytest.mark.parametrize("operand", ["A", "B"])
def test_tc_mn_major_operand(operand):
    """An MN-major operand (rows contiguous for each k) gives the right product when
    its descriptor's leading byte offset is the K-direction core-matrix stride and
    the stride byte offset the M/N-direction one (mode bit 2); the other reading
    of the two offsets gives a wrong product."""
    bit = 1 if operand == "A" else 2
    for n, k in [(64, 16), (128, 32), (128, 64)]:
        assert _run(n, k, bit | 4, 7), (n, k)
    assert not _run(64, 32, bit, 7)


def test_tc_swizzled_mn_major_a():
    """A staged MN-major with the 128-byte swizzle (the layout a TMA load with
    SWIZZLE_128B writes): the product is right when the descriptor's leading
    byte offset is the M-direction stride (between 64-row halves) and its stride
    byte offset the K-direction one (1024 bytes per 8 rows) -- the opposite of
    the unswizzled MN-major reading -- and wrong the other way round."""
    res = {}
    for lbo_k in (0, 4):
        res[lbo_k] = [_run(n, k, 8 | lbo_k, 11) for n, k in [(64, 16), (128, 32), (128, 64), (256, 48)]]
    print("swizzled MN-major A, K-direction stride as leading offset:", res[4], "; as stride offset:", res[0])
    assert all(res[0]) and not any(res[4])


def test_tc_selftest_argument_checks():
    a = torch.zeros((128, 16), dtype=torch.float16, device="cuda")
    b = torch.zeros((40, 16), dtype=torch.float16, device="cuda")
    d = torch.zeros((128, 40), dtype=torch.float32, device="cuda")
    with pytest.raises(moff.MoffError) as e:
        moff.moff_tc_selftest(a, b, d)
    assert e.value.status == -1
