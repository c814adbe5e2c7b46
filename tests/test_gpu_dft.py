"""Factored-DFT tensor-core route of the FP16 path (both transform axes as
tcgen05 contractions, N = 16 x N/16) against the FP64 oracle, with the
gridding on the tensor cores (cell tiles, the default) and as the FP32 gather
fused with the row transform (MOFF_TC_GRID=0).

Bar: max-normalised error <= 3e-3 per (channel, product), the reduced-precision
tolerance.  Error budget: the gridded field, the stage-1 results and the
row-transformed field are each rounded once to FP16 (relative 2^-11) under
exact power-of-two scales, the DFT and twiddle tables once (built in FP64),
products accumulate in FP32 in TMEM, sums over a chunk in FP32 and across
chunks in FP64.  Each test prints its per-image errors.
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


ROUTES = ("fp16_dft", "fp16_tcgrid")


@pytest.fixture(params=["tcgrid", "gather"])
def grid_kind(request, monkeypatch):
    """Both gridding variants of the route: on the tensor cores, or the FP32 gather."""
    if request.param == "gather":
        monkeypatch.setenv("MOFF_TC_GRID", "0")
    return "fp16_tcgrid" if request.param == "tcgrid" else "fp16_dft"


def dft_image(pos, taps, N, C, P, codes, gains, jones=False, autotune=False, route=None):
    with moff.Plan(pos, taps, N, C, P, jones=jones, fp16tc=True, autotune=autotune) as pl:
        assert pl.route() in ROUTES and (route is None or pl.route() == route), pl.route()
        pl.set_gains(gains)
        pl.submit(np.ascontiguousarray(codes))
        img, n = pl.read_image()
    assert n == codes.shape[0]
    return img


def check(img, ref, label, tol=TOL16):
    err = oracle.max_norm_err(img, ref)
    print(f"{label}: max-normalised error per image " + " ".join(f"{e:.2e}" for e in err.max(axis=1)))
    assert np.isfinite(img).all()
    assert err.max() <= tol, err
    return err


@pytest.mark.parametrize("N,P,K,A,T,jones,scratch_mb", [
    (256, 1, 7, 300, 37, False, None),
    (256, 2, 5, 200, 21, False, 6),       # 3 samples per chunk: chunks of 3, ragged last one
    (512, 2, 7, 300, 13, False, None),
    (512, 1, 3, 100, 10, False, 5),       # 5 samples per chunk, channel chunks of 1
    (512, 2, 5, 150, 9, True, None),      # Jones kernels
])
def test_dft_route_shapes(monkeypatch, grid_kind, N, P, K, A, T, jones, scratch_mb):
    monkeypatch.setenv("MOFF_TC_DFT", "1")
    if scratch_mb:
        monkeypatch.setenv("MOFF_SCRATCH_MB", str(scratch_mb))
    C = 3
    pos, taps, codes, gains = case(700 + N + 10 * P + K, A, N, K, P, C, T, jones=jones)
    img = dft_image(pos, taps, N, C, P, codes, gains, jones=jones, route=grid_kind)
    check(img, oracle.moff_image(codes, gains, pos, taps, N, P, jones=jones),
          f"{grid_kind} N={N} P={P} K={K} jones={jones}")


def test_dft_route_dense_array_is_automatic(grid_kind):
    """A filled lattice too dense for the row-spectrum contraction takes the
    factored-DFT route on its own (no environment override), at N = 256."""
    rng = np.random.default_rng(71)
    side, N, K, P, C, T = 48, 256, 7, 2, 2, 12
    pos = synth.positions_lattice(rng, side, side, 1.0, 0.05, (N / 2 - side, N / 2 - side))
    taps = c64(synth.taps_gaussian(rng, pos, K, 1.2, n_pol=P))
    gains = c64(synth.gains_random(rng, C, pos.shape[0], P))
    re = np.clip(np.rint(rng.normal(0, 2, size=(T, C, pos.shape[0], P))), -7, 7).astype(int)
    im = np.clip(np.rint(rng.normal(0, 2, size=(T, C, pos.shape[0], P))), -7, 7).astype(int)
    codes = synth.pack_4bit(re, im)
    img = dft_image(pos, taps, N, C, P, codes, gains, route=grid_kind)
    check(img, oracle.moff_image(codes, gains, pos, taps, N, P), f"{grid_kind} dense 48x48 lattice, N=256")


@pytest.mark.parametrize("rows8", ["1", "0"])
@pytest.mark.parametrize("P,jones", [(1, False), (2, False), (2, True)])
def test_row_transform_kernels_on_the_512_grid(monkeypatch, rows8, P, jones):
    """Both row transforms of the tensor-core gridding route on the 512 grid -- 8 x 64 with the second
    stage transposed (the default) and 16 x 32 (MOFF_ROWS8=0) -- against the oracle, both pol counts and
    Jones kernels, ragged samples, channel chunks of one (several launches per block)."""
    monkeypatch.setenv("MOFF_TC_DFT", "1")
    monkeypatch.setenv("MOFF_ROWS8", rows8)
    monkeypatch.setenv("MOFF_SCRATCH_MB", "200")
    C, T, K, A = 2, 19, 5, 220
    pos, taps, codes, gains = case(880 + P + 3 * int(jones), A, 512, K, P, C, T, jones=jones)
    img = dft_image(pos, taps, 512, C, P, codes, gains, jones=jones, route="fp16_tcgrid")
    check(img, oracle.moff_image(codes, gains, pos, taps, 512, P, jones=jones),
          f"rows8={rows8} P={P} jones={jones}")


def test_plane_store_paths_agree(monkeypatch):
    """The row plane kernel's two store paths -- TMA boxes of 32 rows x 32 samples for warps whose rows
    lie inside the channel's plane rows, 16-byte stores from registers otherwise (MOFF_VP_TMA=0: all
    rows) -- write the same FP16 planes, so the images are bit-identical: a lattice large enough for the
    row plane kernel, whose plane rows per channel are no multiple of 32 (the last warp of each
    channel stores directly), ragged samples, three channels."""
    monkeypatch.setenv("MOFF_TC_DFT", "1")
    rng = np.random.default_rng(612)
    side, N, K, P, C, T = 80, 256, 5, 2, 3, 45
    pos = synth.positions_lattice(rng, side, side, 1.0, 0.05, (N / 2 - side, N / 2 - side))
    A = len(pos)
    taps = c64(synth.taps_gaussian(rng, pos, K, 1.2, n_pol=P))
    gains = c64(synth.gains_random(rng, C, A, P))
    codes = synth.pack_4bit(rng.integers(-8, 8, size=(T, C, A, P)), rng.integers(-8, 8, size=(T, C, A, P)))
    monkeypatch.delenv("MOFF_VP_TMA", raising=False)
    boxed = dft_image(pos, taps, N, C, P, codes, gains, route="fp16_tcgrid")
    monkeypatch.setenv("MOFF_VP_TMA", "0")
    direct = dft_image(pos, taps, N, C, P, codes, gains, route="fp16_tcgrid")
    assert np.array_equal(boxed, direct)
    check(boxed, oracle.moff_image(codes, gains, pos, taps, N, P), "plane store paths")


def test_dft_route_deterministic_and_gain_rescale(monkeypatch, grid_kind):
    monkeypatch.setenv("MOFF_TC_DFT", "1")
    pos, taps, codes, gains = case(760, 120, 256, 5, 2, C=2, T=11)
    a = dft_image(pos, taps, 256, 2, 2, codes, gains)
    b = dft_image(pos, taps, 256, 2, 2, codes, gains)
    assert np.array_equal(a, b)
    # gains x 2^10: the per-channel voltage scale follows exactly, the image scales by 2^20
    c = dft_image(pos, taps, 256, 2, 2, codes, gains * 1024.0)
    np.testing.assert_allclose(c, a * 2.0 ** 20, rtol=0, atol=1e-6 * np.abs(a).max() * 2.0 ** 20)


def test_dft_route_refuses_pixel_taps(monkeypatch):
    monkeypatch.setenv("MOFF_TC_DFT", "1")
    pos, taps, codes, gains = case(770, 50, 256, 3, 1, C=1, T=2)
    with moff.Plan(pos, taps, 256, 1, 1, fp16tc=True) as pl:
        with pytest.raises(moff.MoffError) as e:
            pl.set_calibrator(3, 4)
        assert e.value.status == -1
        with pytest.raises(moff.MoffError) as e:
            pl.set_beams([1], [2])
        assert e.value.status == -1
        # the plan still images after the refusals
        pl.submit(np.ascontiguousarray(codes))
        img, n = pl.read_image()
    assert n == 2 and np.isfinite(img).all()


def test_dft_route_autotuned_shape(monkeypatch):
    """MOFF_AUTOTUNE times the gridding shapes of the tensor-core row transform;
    whichever it picks, the image stays within the tolerance."""
    monkeypatch.setenv("MOFF_TC_DFT", "1")
    pos, taps, codes, gains = case(780, 250, 512, 5, 2, C=2, T=8)
    monkeypatch.setenv("MOFF_TC_GRID", "0")          # the autotuner times the gather's shapes
    with moff.Plan(pos, taps, 512, 2, 2, fp16tc=True, autotune=True) as pl:
        assert pl.route() == "fp16_dft"
        t = pl.tuning()
        assert t["source"] in (1, 2) and t["staged"] == 0
        pl.set_gains(gains)
        pl.submit(np.ascontiguousarray(codes))
        img, _ = pl.read_image()
    check(img, oracle.moff_image(codes, gains, pos, taps, 512, 2), "autotuned N=512")


def test_autotuner_picks_the_column_kernel_width(monkeypatch):
    """MOFF_AUTOTUNE times the column kernel at 8 and 16 columns per CTA on the plan's
    chunk and keeps the faster; the image is within the tolerance either way, and the
    two widths give the same image up to the order of FP32 sums (bit-identical here:
    each pixel's sums run in the same order at both widths)."""
    monkeypatch.setenv("MOFF_TC_DFT", "1")
    monkeypatch.delenv("MOFF_COLS_W", raising=False)
    pos, taps, codes, gains = case(790, 220, 256, 5, 2, C=3, T=20)
    with moff.Plan(pos, taps, 256, 3, 2, fp16tc=True, autotune=True) as pl:
        assert pl.route() in ROUTES
        t = pl.dft_tuning()
        assert t["source"] == 1 and t["cols_width"] in (8, 16) and t["ms_w8"] > 0 and t["ms_w16"] > 0, t
        assert t["cols_width"] == (16 if t["ms_w16"] < t["ms_w8"] else 8)
        pl.set_gains(gains)
        pl.submit(np.ascontiguousarray(codes))
        img, n = pl.read_image()
    check(img, oracle.moff_image(codes, gains, pos, taps, 256, 2), f"autotuned column width {t['cols_width']}")
    imgs = {}
    for w in (8, 16):
        monkeypatch.setenv("MOFF_COLS_W", str(w))
        with moff.Plan(pos, taps, 256, 3, 2, fp16tc=True) as pl:
            assert pl.dft_tuning()["cols_width"] == w
            pl.set_gains(gains)
            pl.submit(np.ascontiguousarray(codes))
            imgs[w], _ = pl.read_image()
    assert np.array_equal(imgs[8], imgs[16])
