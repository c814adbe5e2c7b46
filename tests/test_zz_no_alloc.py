"""moff_image_noalloc -- the entry point for callers that cannot allocate GPU
memory -- against the FP64 oracle and against the plan-based path
(moff_plan_create / moff_submit / moff_read_image) on the same inputs.

The no-allocation call keeps its intermediates in one fixed device array
shared by every call, so the test makes two calls in a row with different
voltages and gains: the second result must not carry anything over from the
first.  Both results must match the oracle and the plan path to the imaging
tolerance used by the other GPU tests (max-normalised error <= 1e-5 per
channel and product).  The cases reach the chunked paths: a 512-point grid
whose chunks hold one channel and a few samples, and Jones kernels.
"""
import numpy as np
import pytest

import oracle
import paper_0812_3669_gb300 as moff
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    moff.build()
    yield


def _case(seed, A, N, K, P, C, T, jones=False):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, N, size=(A, 2))
    shape = (A, 2, 2, K, K) if jones else (A, P, K, K)
    taps = (rng.normal(size=shape) + 1j * rng.normal(size=shape)).astype(np.complex64)
    codes = synth.pack_4bit(rng.integers(-8, 8, size=(T, C, A, P)), rng.integers(-8, 8, size=(T, C, A, P)))
    gains = synth.gains_random(rng, C, A, P).astype(np.complex64)
    return pos, taps, codes, gains


def _plan_image(pos, taps, N, C, P, codes, gains, jones=False):
    with moff.Plan(pos, taps, N, C, P, jones=jones) as pl:
        pl.set_gains(gains)
        pl.submit(np.ascontiguousarray(codes))
        img, n = pl.read_image()
    assert n == codes.shape[0]
    return img


@pytest.mark.parametrize("N,P,K,A,C,T,jones", [(128, 2, 7, 300, 5, 23, False), (32, 1, 3, 64, 16, 40, False),
                                               (512, 2, 7, 200, 2, 20, False), (64, 2, 5, 80, 3, 12, True)])
def test_noalloc_matches_oracle_and_plan_path_on_two_calls(N, P, K, A, C, T, jones):
    pos, taps, codes1, gains1 = _case(100 + N, A, N, K, P, C, T, jones)
    _, _, codes2, gains2 = _case(200 + N, A, N, K, P, C, T, jones)
    n_prod = 1 if P == 1 else 4
    t64 = taps.astype(np.complex128)
    for codes, gains in [(codes1, gains1), (codes2, gains2)]:
        ref = oracle.moff_image(codes, gains.astype(np.complex128), pos, t64, N, P, jones=jones)
        via_plan = _plan_image(pos, taps, N, C, P, codes, gains, jones)
        volt = torch.from_numpy(np.ascontiguousarray(codes)).cuda()
        g = torch.from_numpy(np.ascontiguousarray(gains)).cuda()
        img = torch.full((C, n_prod, N, N), float("nan"), dtype=torch.float32, device="cuda")
        moff.moff_image_noalloc(pos, taps, N, C, P, volt, g, img, jones=jones)
        torch.cuda.synchronize()
        got = img.cpu().numpy()
        assert np.isfinite(got).all()
        err = oracle.max_norm_err(got, ref)
        print(f"N={N} P={P} jones={jones}: max-normalised error vs oracle {err.max():.2e}")
        assert err.max() <= TOL, err
        assert oracle.max_norm_err(got, via_plan).max() <= TOL


def test_noalloc_rejects_mismatched_buffers():
    """The binding checks every buffer's type and extent before the library
    touches it: a wrong shape or dtype raises ValueError."""
    pos, taps, codes, gains = _case(300, 40, 32, 3, 1, 2, 4)
    volt = torch.from_numpy(np.ascontiguousarray(codes)).cuda()
    g = torch.from_numpy(np.ascontiguousarray(gains)).cuda()
    img = torch.zeros((2, 1, 32, 32), dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        moff.moff_image_noalloc(pos, taps, 32, 3, 1, volt, g, img)                 # channel count
    with pytest.raises(ValueError):
        moff.moff_image_noalloc(pos, taps, 32, 2, 1, volt, g, img[:1])             # image too small
    with pytest.raises(ValueError):
        moff.moff_image_noalloc(pos, taps, 32, 2, 1, volt.to(torch.int32), g, img) # voltage dtype
    with pytest.raises(ValueError):
        moff.moff_image_noalloc(pos, taps, 32, 2, 1, volt, g[:, :20], img)         # gains too few


def test_noalloc_rejects_arrays_beyond_its_scratch():
    """Kernel lists larger than the fixed array are refused with MOFF_EINVAL."""
    A, N, K, P = 20000, 512, 15, 2
    rng = np.random.default_rng(7)
    pos = rng.uniform(0, N, size=(A, 2))
    taps = np.ones((A, P, K, K), dtype=np.complex64)
    volt = torch.zeros((1, 1, A, P), dtype=torch.uint8, device="cuda")
    g = torch.ones((1, A, P), dtype=torch.complex64, device="cuda")
    img = torch.zeros((1, 4, N, N), dtype=torch.float32, device="cuda")
    with pytest.raises(moff.MoffError) as e:
        moff.moff_image_noalloc(pos, taps, N, 1, P, volt, g, img)
    assert e.value.status == -1
    assert "no-allocation limit" in str(e.value)
