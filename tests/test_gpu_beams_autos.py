"""The electric-field image tapped as tied-array beams, and the autocorrelation
part of the image subtracted to leave the baselines-only image, vs the oracle.

Beams are the image path's field E_t,p(k) at chosen pixels, before squaring:
1e-5 of the largest |E| per (channel, beam, pol) on the FP32 path, 3e-3 on
the FP16 tensor-core path.  The baselines-only image is held to 1e-5 of the
full image's largest pixel per (channel, product).
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


def case(seed, A, N, K, P, C, T):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, N * 0.8, size=(A, 2)) + N * 0.1
    taps = c64(rng.normal(size=(A, P, K, K)) + 1j * rng.normal(size=(A, P, K, K)))
    re = np.clip(np.rint(rng.normal(0, 2.5, size=(T, C, A, P))), -8, 7).astype(int)
    im = np.clip(np.rint(rng.normal(0, 2.5, size=(T, C, A, P))), -8, 7).astype(int)
    return pos, taps, synth.pack_4bit(re, im), c64(synth.gains_random(rng, C, A, P))


def oracle_field(codes, gains, pos, taps, N, P, pix):
    """E_t,p at the pixels: [T, C, n, P] from the oracle's grid + transform."""
    W = oracle.grid_matrix(pos, taps, N, P)
    out = []
    for c in range(codes.shape[1]):
        y = oracle.calibrate(oracle.unpack_4bit(codes[:, c]), gains[c])
        E = oracle.sky_transform(oracle.grid(y, W, N, P))            # [T, P, N, N]
        out.append(np.stack([E[:, :, ky, kx] for kx, ky in pix], axis=1))
    return np.stack(out, axis=1)


@pytest.mark.parametrize("fp16tc,graph,N,P,K,A,tol", [(False, False, 64, 2, 5, 120, 1e-5),
                                                     (False, True, 32, 1, 3, 50, 1e-5),
                                                     (True, False, 128, 2, 7, 300, 3e-3)])
def test_beams_match_the_oracle_field(fp16tc, graph, N, P, K, A, tol):
    C, T = 3, 150
    pos, taps, codes, gains = case(700 + N, A, N, K, P, C, T)
    pix = [(0, 0), (N - 1, N - 1), (N // 3, N // 2 + 1), (5, N - 2), (N // 2, 7)]
    with moff.Plan(pos, taps, N, C, P, fp16tc=fp16tc, graph=graph) as pl:
        pl.set_gains(gains)
        pl.set_beams([p[0] for p in pix], [p[1] for p in pix])
        pl.submit(codes[:40])
        b1 = pl.read_beams()
        pl.submit(codes[40:])
        b2 = pl.read_beams()
        pl.submit(codes[40:])                   # a replay (graph) of the same block
        b3 = pl.read_beams()
    assert b1.shape == (40, C, len(pix), P) and b2.shape == (T - 40, C, len(pix), P)
    ref = oracle_field(codes, gains, pos, taps, N, P, pix)
    for got, want in [(b1, ref[:40]), (b2, ref[40:]), (b3, ref[40:])]:
        err = np.abs(got - want).max(axis=0) / np.abs(want).max(axis=0)    # per (c, beam, pol)
        assert err.max() <= tol, err.max()
    print(f"fp16tc={fp16tc} graph={graph}: beam max error {err.max():.2e}")


@pytest.mark.parametrize("P,K,A", [(2, 5, 90), (1, 3, 60)])
def test_baselines_only_image_matches_oracle(P, K, A):
    N, C, T = 64, 2, 130
    pos, taps, codes, gains = case(720 + P, A, N, K, P, C, T)
    with moff.Plan(pos, taps, N, C, P) as pl:
        pl.set_gains(gains)
        pl.set_autocorr(True)
        pl.submit(codes[:70])
        pl.submit(codes[70:])
        cross, n = pl.read_image_cross()
        full, _ = pl.read_image()
    assert n == T
    ref_full = oracle.moff_image(codes, gains, pos, taps, N, P)
    ref_auto = np.stack([oracle.auto_image(codes, gains, pos, taps, N, P, channel=c) for c in range(C)])
    ref_cross = ref_full - ref_auto
    den = np.abs(ref_full).reshape(C, -1, N * N).max(axis=-1)
    err = np.abs(cross - ref_cross).reshape(C, -1, N * N).max(axis=-1) / den
    print(f"P={P}: baselines-only image error / full-image max {err.max():.2e}; "
          f"autos share of the full image {np.abs(ref_auto).max() / np.abs(ref_full).max():.2f}")
    assert err.max() <= 1e-5
    assert np.abs(full - ref_full).max() <= 1e-5 * np.abs(ref_full).max()


def test_baselines_only_equals_the_fx_route_on_a_tiny_array():
    """Against the oracle's FX route without autocorrelations (software
    holography of the baselines, Sec. 3)."""
    N, P, K, A, C, T = 32, 2, 3, 9, 1, 12
    pos, taps, codes, gains = case(740, A, N, K, P, C, T)
    with moff.Plan(pos, taps, N, C, P) as pl:
        pl.set_gains(gains)
        pl.set_autocorr(True)
        pl.submit(codes)
        cross, _ = pl.read_image_cross()
    fx = oracle.fx_image(codes, gains, pos, taps, N, P, autos=False)
    full = oracle.moff_image(codes, gains, pos, taps, N, P)[0]
    assert np.abs(cross[0] - fx).max() <= 1e-5 * np.abs(full).max()


def test_states_and_errors():
    pos, taps, codes, gains = case(750, 20, 32, 3, 2, 1, 10)
    with moff.Plan(pos, taps, 32, 1, 2) as pl:
        pl.set_gains(gains)
        with pytest.raises(moff.MoffError) as e:
            pl.read_image_cross()
        assert e.value.status == -4
        pl.submit(codes)
        pl.set_autocorr(True)                 # switched on mid-integration
        pl.submit(codes)
        with pytest.raises(moff.MoffError) as e:
            pl.read_image_cross()
        assert e.value.status == -4
        pl.reset()
        pl.submit(codes)
        img, n = pl.read_image_cross(reset=True)
        assert n == 10 and np.isfinite(img).all()
        with pytest.raises(moff.MoffError) as e:
            pl.read_beams()
        assert e.value.status == -4
        with pytest.raises(moff.MoffError) as e:
            pl.set_beams([32], [0])
        assert e.value.status == -1
        with pytest.raises(moff.MoffError):
            pl.set_beams(list(range(17)), list(range(17)))
        pl.set_beams([1, 2], [3, 4])
        assert pl.read_beams().shape == (0, 1, 2, 2)
        pl.set_beams([], [])
    jt = np.ones((20, 2, 2, 3, 3), complex)
    with moff.Plan(pos, jt, 32, 1, 2, jones=True) as pj:
        with pytest.raises(moff.MoffError) as e:
            pj.set_autocorr(True)
        assert e.value.status == -1
