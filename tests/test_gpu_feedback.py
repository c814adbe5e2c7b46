"""Feedback calibration (Sec. 6, Eqs. FBeq1-FBeq3) on the GPU vs the FP64 oracle.

The sums R (image pixel towards the calibrator times each antenna's conjugated
calibrated signal) and S (the pixel's power) are held to the imaging path's
bars: 1e-5 max-normalised per (channel, pol) on the FP32 path and 3e-3 on the
FP16 tensor-core path; the gain-error estimate follows from them.  A simulated
point source with gain errors must converge under repeated updates.
"""
import numpy as np
import pytest

import oracle
import paper_0812_3669_gb300 as moff
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    moff.build()
    yield


def c64(x):
    return np.asarray(x).astype(np.complex64).astype(np.complex128)


def case(seed, A, N, K, P, C, T, spread=None):
    rng = np.random.default_rng(seed)
    spread = N * 0.8 if spread is None else spread
    pos = rng.uniform(0, spread, size=(A, 2)) + (N - spread) / 2
    taps = c64(rng.normal(size=(A, P, K, K)) + 1j * rng.normal(size=(A, P, K, K)))
    re = np.clip(np.rint(rng.normal(0, 2.5, size=(T, C, A, P))), -8, 7).astype(int)
    im = np.clip(np.rint(rng.normal(0, 2.5, size=(T, C, A, P))), -8, 7).astype(int)
    return pos, taps, synth.pack_4bit(re, im), c64(synth.gains_random(rng, C, A, P))


def max_norm(a, b, axis):
    return np.abs(a - b).max(axis=axis) / np.abs(b).max(axis=axis)


@pytest.mark.parametrize("fp16tc,N,P,K,A,k,tol", [(False, 64, 2, 5, 120, (11, 37), 1e-5),
                                                 (False, 32, 1, 3, 60, (0, 31), 1e-5),
                                                 (True, 128, 2, 7, 300, (70, 5), 3e-3)])
def test_feedback_sums_match_oracle(fp16tc, N, P, K, A, k, tol):
    C, T = 3, 150          # three time chunks on the FP32 path, two on the tensor-core path
    pos, taps, codes, gains = case(600 + N, A, N, K, P, C, T)
    with moff.Plan(pos, taps, N, C, P, fp16tc=fp16tc) as pl:
        pl.set_gains(gains)
        pl.submit(codes[:40])                 # before the calibrator: not in the sums
        pl.set_calibrator(*k)
        pl.submit(codes[40:])
        R, S, n = pl.read_feedback()
        img, ni = pl.read_image()
        delta = pl.feedback_gains()
    assert n == T - 40 and ni == T
    Ro, So = oracle.feedback_sums(codes[40:], gains, pos, taps, N, k)
    eS = np.abs(S - So) / So
    eR = max_norm(R, Ro, axis=1)                      # per (channel, pol)
    print(f"fp16tc={fp16tc} N={N}: S rel err {eS.max():.2e}, R max-normalised err {eR.max():.2e}")
    assert eS.max() <= tol and eR.max() <= tol
    assert np.allclose(R.sum(axis=1), S, rtol=10 * tol, atol=0)   # FBeq1 = sum of FBeq2
    do = oracle.feedback_delta(Ro, So, gains, A)
    assert np.abs(delta - do).max() <= 50 * tol * np.abs(gains).max()
    # the image is untouched by the taps (same blocks without a calibrator)
    with moff.Plan(pos, taps, N, C, P, fp16tc=fp16tc) as pl2:
        pl2.set_gains(gains)
        pl2.submit(codes[:40])
        pl2.submit(codes[40:])
        img2, _ = pl2.read_image()
    assert np.array_equal(img, img2)


def test_feedback_converges_on_a_simulated_point_source():
    """Delta kernels at integer anchors, one source at pixel theta_s, instrument
    gains h (amplitude 0.8-1.2, random phase), calibration g = (1 + eps) / h with
    10 % complex errors; 4-bit quantised voltages with receiver noise.  Three
    rounds of (integrate, apply the estimate) must shrink the residual spread
    of g h around its mean at least threefold."""
    N, A, T, C = 64, 40, 400, 2
    rng = np.random.default_rng(7)
    cells = rng.choice(N * N, size=A, replace=False)
    pos = np.stack([cells % N, cells // N], axis=1).astype(float)
    th = (10, 20)
    geo = np.exp(-2j * np.pi * (pos[:, 0] * th[0] + pos[:, 1] * th[1]) / N)
    h = (0.8 + 0.4 * rng.random((C, A))) * np.exp(2j * np.pi * rng.random((C, A)))
    s = 2.5 * (rng.normal(size=(T, C)) + 1j * rng.normal(size=(T, C))) / np.sqrt(2)
    noise = 0.5 * (rng.normal(size=(T, C, A)) + 1j * rng.normal(size=(T, C, A))) / np.sqrt(2)
    x = s[:, :, None] * h[None] * geo[None, None] + noise
    codes = synth.pack_4bit(np.clip(np.rint(x.real), -7, 7).astype(int),
                            np.clip(np.rint(x.imag), -7, 7).astype(int))[..., None]     # [T, C, A, 1]
    eps = 0.1 * (rng.normal(size=(C, A)) + 1j * rng.normal(size=(C, A))) / np.sqrt(2)
    g = ((1 + eps) / h)[..., None]
    spread = lambda gg: np.abs((gg[..., 0] * h) / (gg[..., 0] * h).mean(axis=1, keepdims=True) - 1).max()
    taps = np.ones((A, 1, 1, 1), complex)
    history = [spread(g)]
    dev = torch.from_numpy(np.ascontiguousarray(codes)).cuda()
    with moff.Plan(pos, taps, N, C, 1) as pl:
        pl.set_calibrator(*th)
        for _ in range(3):
            pl.set_gains(g)
            pl.read_feedback(reset=True)
            pl.submit(dev)
            g = g + pl.feedback_gains().astype(np.complex128)
            history.append(spread(g))
    print("residual spread of g h per round:", " ".join(f"{v:.4f}" for v in history))
    assert history[-1] < history[0] / 3


def test_feedback_device_updates_follow_the_oracle():
    """One device update (apply=1) equals the oracle's update of the gains: the
    next block's sums, computed with the updated gains, match the oracle run
    with g + delta_g."""
    N, P, K, A, C, T = 64, 2, 5, 80, 2, 50
    pos, taps, codes, gains = case(640, A, N, K, P, C, T)
    k = (9, 50)
    with moff.Plan(pos, taps, N, C, P) as pl:
        pl.set_gains(gains)
        pl.set_calibrator(*k)
        pl.submit(codes)
        d = pl.feedback_gains(apply=True)
        pl.read_feedback(reset=True)
        pl.submit(codes)
        R2, S2, _ = pl.read_feedback()
    Ro, So = oracle.feedback_sums(codes, gains, pos, taps, N, k)
    g1 = gains + oracle.feedback_delta(Ro, So, gains, A)
    assert np.abs(d - (g1 - gains)).max() <= 1e-3 * np.abs(gains).max()
    g1_dev = c64(gains + d.astype(np.complex128))          # the gains the device now holds
    Ro2, So2 = oracle.feedback_sums(codes, g1_dev, pos, taps, N, k)
    assert max_norm(R2, Ro2, axis=1).max() <= 1e-5
    assert (np.abs(S2 - So2) / So2).max() <= 1e-5


def test_feedback_argument_and_state_errors():
    pos, taps, codes, gains = case(650, 20, 32, 3, 2, 1, 5)
    with moff.Plan(pos, taps, 32, 1, 2) as pl:
        with pytest.raises(moff.MoffError) as e:
            pl.read_feedback()
        assert e.value.status == -4
        with pytest.raises(moff.MoffError) as e:
            pl.set_calibrator(32, 0)
        assert e.value.status == -1
        pl.set_calibrator(3, 4)
        pl.submit(codes)
        R, S, n = pl.read_feedback()
        assert n == 5 and np.isfinite(R).all()
        pl.reset()
        R, S, n = pl.read_feedback()
        assert n == 0 and np.abs(R).max() == 0 and np.abs(S).max() == 0
        pl.set_calibrator(-1, -1)
        with pytest.raises(moff.MoffError):
            pl.read_feedback()
    jt = np.ones((20, 2, 2, 3, 3), complex)
    with moff.Plan(pos, jt, 32, 1, 2, jones=True) as pj:
        with pytest.raises(moff.MoffError) as e:
            pj.set_calibrator(1, 1)
        assert e.value.status == -1
