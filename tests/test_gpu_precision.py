"""FP16 tensor-core path (MOFF_PREC_FP16TC) vs the FP64 oracle.

Bar: max-normalised error <= 3e-3 per (channel, product), the reduced-
precision tolerance.  The error budget: weighted voltages and kernel-row
spectra are rounded once to FP16 (relative 2^-11 each) under exact power-of-
two scales, products accumulate in FP32 on the tensor cores, the column
transform and squaring are FP32; an emulation of this arithmetic on the
1024-antenna array gives ~2e-4.  Each test prints its per-image errors.
"""
import numpy as np
import pytest

import oracle
import paper_0812_3669_gb300 as moff
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL16 = 3e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    moff.build()
    yield


def c64(x):
    return np.asarray(x).astype(np.complex64).astype(np.complex128)


def case(seed, A, N, K, P, C, T, jones=False, spread=None, sigma=2.5):
    rng = np.random.default_rng(seed)
    spread = N if spread is None else spread
    pos = rng.uniform(0, spread, size=(A, 2)) + (N - spread) / 2
    shape = (A, 2, 2, K, K) if jones else (A, P, K, K)
    taps = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    re = np.clip(np.rint(rng.normal(0, sigma, size=(T, C, A, P))), -8, 7).astype(int)
    im = np.clip(np.rint(rng.normal(0, sigma, size=(T, C, A, P))), -8, 7).astype(int)
    return pos, c64(taps), synth.pack_4bit(re, im), c64(synth.gains_random(rng, C, A, P))


def tc_image(pos, taps, N, C, P, codes, gains, jones=False):
    with moff.Plan(pos, taps, N, C, P, jones=jones, fp16tc=True) as pl:
        pl.set_gains(gains)
        pl.submit(np.ascontiguousarray(codes))
        img, n = pl.read_image()
    assert n == codes.shape[0]
    return img


def check(img, ref, label):
    err = oracle.max_norm_err(img, ref)
    print(f"{label}: max-normalised error per image " + " ".join(f"{e:.2e}" for e in err.max(axis=1)))
    assert np.isfinite(img).all()
    assert err.max() <= TOL16, err
    return err


@pytest.mark.parametrize("N,P,K,A,T", [(32, 1, 3, 60, 150), (64, 2, 5, 120, 40), (128, 2, 7, 300, 200),
                                        (256, 1, 7, 300, 20), (512, 2, 5, 200, 9)])
def test_fp16tc_every_grid_size(N, P, K, A, T):
    pos, taps, codes, gains = case(300 + N + P, A, N, K, P, C=2, T=T)
    img = tc_image(pos, taps, N, 2, P, codes, gains)
    check(img, oracle.moff_image(codes, gains, pos, taps, N, P), f"N={N} P={P}")


def test_fp16tc_jones():
    pos, taps, codes, gains = case(330, 60, 64, 5, 2, C=2, T=70, jones=True)
    img = tc_image(pos, taps, 64, 2, 2, codes, gains, jones=True)
    check(img, oracle.moff_image(codes, gains, pos, taps, 64, 2, jones=True), "Jones N=64")


def test_fp16tc_tiny_workload():
    cfg = synth.config_tiny()
    taps, gains = c64(cfg["taps"]), c64(cfg["gains"])
    img = tc_image(cfg["pos"], taps, 32, 16, 1, cfg["codes"], gains)
    check(img, oracle.moff_image(cfg["codes"], gains, cfg["pos"], taps, 32, 1), "tiny workload")


def test_fp16tc_full_size_dualpol_sampled_channels():
    """1024-antenna hex core, 128x128 grid, 1024 channels, 1000 samples (8 blocks of
    128, the last one ragged), three sampled channels against the oracle."""
    cfg = synth.config_dualpol()
    T, C, A, P, N = 1000, cfg["n_chan"], cfg["pos"].shape[0], 2, cfg["grid_n"]
    taps, gains = c64(cfg["taps"]), c64(cfg["gains"])
    codes_d = synth.device_codes(8123669 + 101, T, C, A, P)
    with moff.Plan(cfg["pos"], taps, N, C, P, fp16tc=True) as pl:
        pl.set_gains(gains)
        pl.submit(codes_d)
        img, n = pl.read_image()
    assert n == T
    chans = [0, 517, 1023]
    ref = oracle.moff_image(codes_d[:, chans].cpu().numpy(), gains[chans], cfg["pos"], taps, N, P)
    check(img[chans], ref, "1024-antenna dual-pol, full size")


def test_fp16tc_deterministic_and_gain_rescale():
    pos, taps, codes, gains = case(340, 150, 128, 7, 2, C=2, T=130)
    a = tc_image(pos, taps, 128, 2, 2, codes, gains)
    b = tc_image(pos, taps, 128, 2, 2, codes, gains)
    assert np.array_equal(a, b)
    # gains scaled by 2^10: the per-channel voltage scale follows, the image scales by 2^20
    c = tc_image(pos, taps, 128, 2, 2, codes, gains * 1024.0)
    np.testing.assert_allclose(c, a * 2.0 ** 20, rtol=0, atol=1e-6 * np.abs(a).max() * 2.0 ** 20)


def test_fp16tc_rejects_too_many_rows_per_grid_row():
    rng = np.random.default_rng(5)
    A, N, K = 4000, 64, 9
    pos = rng.uniform(0, N, size=(A, 2))
    taps = np.ones((A, 1, K, K))
    with pytest.raises(moff.MoffError) as e:
        moff.Plan(pos, taps, N, 1, 1, fp16tc=True)
    assert e.value.status == -1 and "tensor-core" in str(e.value)
